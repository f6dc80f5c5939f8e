"""The multi-rank host logic of bench.py on two CPU ranks (gloo): every rank
takes its own reference view of the same scene (no collective on the data
path), the job time is the slowest rank's, and the rate counts every rank's
pixels.  The GPU work itself needs no exchange, so nothing else crosses
ranks."""
import json
import os
import socket
import sys

import pytest

REPO = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    sys.path.insert(0, REPO)
    os.environ.update(WORLD_SIZE=str(world), RANK=str(rank), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import bench
    from paper_1805_07920_gb300 import synth
    r, w, _, dist = bench.dist_setup(False)
    assert (r, w) == (rank, world) and dist is not None
    sc = bench.assign_reference(synth.make_scene("tiny"), r)
    ms = 100.0 + 50.0 * r                         # rank 1 is the slower one
    job_ms = bench.max_over_ranks(ms, dist, "cpu")
    rate = bench.job_rate(sc.width * sc.height, 6, 3, w, job_ms)
    with open(os.path.join(out_dir, f"rank{r}.json"), "w") as f:
        json.dump({"ref": sc.ref, "src": list(sc.src), "job_ms": job_ms, "rate": rate,
                   "px": sc.width * sc.height}, f)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    assert res[0]["ref"] != res[1]["ref"]                         # one reference per rank
    for r in res:
        assert r["ref"] not in r["src"] and len(set(r["src"])) == len(r["src"]) >= 1
        assert r["job_ms"] == 150.0                               # max over ranks
    expect = res[0]["px"] * 6 * 3 * world / 0.150 / 1e6
    assert abs(res[0]["rate"] - expect) < 1e-9 * expect and res[0]["rate"] == res[1]["rate"]


def test_single_rank_needs_no_group():
    sys.path.insert(0, REPO)
    import bench
    assert bench.max_over_ranks(42.0, None, "cpu") == 42.0
    assert bench.job_rate(1000, 6, 2, 1, 1000.0) == pytest.approx(0.012)
