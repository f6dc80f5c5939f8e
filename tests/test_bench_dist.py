"""The multi-rank host logic of bench.py on two CPU ranks (gloo): every rank
takes its own reference view of the same scene (no collective on the data
path), the job time is the slowest rank's, and the rate counts every rank's
pixels.  The GPU work itself needs no exchange, so nothing else crosses
ranks.  A rank that leaves between steps turns the survivors' next
collective into an error within the group's timeout, not a hang."""
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


def _rank_leaves(rank, world, port, out_dir):
    """Rank 1 joins the group and leaves before the timing exchange (between
    steps, nothing in flight); rank 0 must get an error from it, in time."""
    import time
    sys.path.insert(0, REPO)
    os.environ.update(WORLD_SIZE=str(world), RANK=str(rank), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port), AMH_DIST_TIMEOUT_S="10")
    import bench
    r, w, _, dist = bench.dist_setup(False)
    if r == 1:
        return                                   # leaves without the exchange
    t0 = time.time()
    try:
        bench.max_over_ranks(100.0, dist, "cpu")
        outcome = "completed"
    except Exception as e:                       # the survivor sees the failure
        outcome = f"error: {type(e).__name__}"
    with open(os.path.join(out_dir, "rank0.json"), "w") as f:
        json.dump({"outcome": outcome, "seconds": time.time() - t0}, f)


def test_a_rank_that_leaves_is_detected(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    mp.start_processes(_rank_leaves, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    res = json.load(open(tmp_path / "rank0.json"))
    assert res["outcome"].startswith("error"), res
    assert res["seconds"] < 60, res



def _stub_device(args, sc, rank, world, local, barrier):
    """Stands in for measure_device: no GPU work, a fixed time per rank
    (rank 1 slower) and the end-to-end leg with its own times."""
    barrier()
    return {"ms": 200.0 + 100.0 * rank, "form": "fp32_blend",
            "e2e": {"ms": 900.0 + 10.0 * rank, "h2d_bytes_per_step": 1, "d2h_bytes_per_step": 2, "steps": 3},
            "roofline": {"frac": 0.5}, "clocks": {"sm_mhz": 2070.0}, "gpu_launches": 13 * args.steps,
            "pairs_per_step": 7}


def _run_ours_rank(rank, world, port, out_dir):
    sys.path.insert(0, REPO)
    os.environ.update(WORLD_SIZE=str(world), RANK=str(rank), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    out = open(os.path.join(out_dir, f"out{rank}.txt"), "w")
    sys.stdout = out
    import bench
    from paper_1805_07920_gb300 import synth
    args = bench.parse_args(["--gpus", str(world), "--steps", "4", "--warmup", "3"])
    rc = bench.run_ours(args, measure=_stub_device, scene=synth.make_scene("tiny"), want_cuda=False)
    out.close()
    with open(os.path.join(out_dir, f"rc{rank}.txt"), "w") as f:
        f.write(str(rc))


def test_run_ours_on_two_gloo_ranks(tmp_path):
    """bench.run_ours itself on two CPU ranks, the device work stubbed: one
    JSON line from rank 0 with n_gpus 2, a distinct reference per rank, and
    the job rate taken at the slowest rank's time."""
    mp = pytest.importorskip("torch.multiprocessing")
    sys.path.insert(0, REPO)
    import bench
    from paper_1805_07920_gb300 import synth
    world = 2
    mp.start_processes(_run_ours_rank, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    assert [open(tmp_path / f"rc{r}.txt").read() for r in range(world)] == ["0", "0"]
    assert open(tmp_path / "out1.txt").read().strip() == ""             # rank 1 prints nothing
    lines = [ln for ln in open(tmp_path / "out0.txt").read().splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    sc = synth.make_scene("tiny")
    assert d["n_gpus"] == world and d["steps"] == 4
    refs = d["config"]["reference_per_rank"]
    assert len(refs) == world and len(set(refs)) == world and refs[0] == sc.ref
    px = sc.width * sc.height
    assert d["value"] == pytest.approx(round(bench.job_rate(px, bench.ITERS, 4, world, 300.0), 3))
    assert d["ms_per_step"] == pytest.approx(300.0 / 4, abs=1e-3)
    assert d["e2e"]["value"] == pytest.approx(round(bench.job_rate(px, bench.ITERS, 3, world, 910.0), 3))


def test_world_size_must_match_gpus(monkeypatch):
    """A launcher whose world size differs from --gpus is refused before any
    device work."""
    sys.path.insert(0, REPO)
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    assert bench.check_world(8) is not None and bench.check_world(2) is None
    called = []
    rc = bench.run_ours(bench.parse_args(["--gpus", "8"]), measure=lambda *a: called.append(a), want_cuda=False)
    assert rc != 0 and not called


def test_spawn_ranks_sets_each_ranks_environment(tmp_path):
    """Without a launcher, --gpus N starts N processes with their rank
    variables; the first failing rank's exit code is returned."""
    sys.path.insert(0, REPO)
    import bench
    code = ("import os, sys; r = os.environ['RANK']; "
            f"open(os.path.join({str(tmp_path)!r}, 'r' + r), 'w').write("
            "','.join(os.environ[k] for k in ('RANK', 'LOCAL_RANK', 'WORLD_SIZE', 'MASTER_ADDR')))")
    assert bench.spawn_ranks(3, [sys.executable, "-c", code]) == 0
    for r in range(3):
        assert open(tmp_path / f"r{r}").read() == f"{r},{r},3,127.0.0.1"
    assert bench.spawn_ranks(2, [sys.executable, "-c", "import os, sys; sys.exit(int(os.environ['RANK']) * 5)"]) == 5
