#!/usr/bin/env python3
"""Throughput of the AMHMVS checkerboard update on GB300.

One step = one whole depth map of the 3200x2112 reference with 10 source
views: random initialisation + 6 iterations (12 colour phases: ACP, the 8 x N
bilateral-NCC cost matrix, joint view selection, weighted choice and
refinement), all in this repository's CUDA kernels through the C-ABI.

Metric: Mpixel-iterations/s = W * H * 6 * steps * ranks / (max over ranks of
the device time of the timed steps).  Multi-GPU runs give every rank its own
reference view of the same 11-camera scene (independent depth maps, weak
scaling, no collective on the data path).

Printed: one JSON line with the value, the end-to-end figure through the
C-ABI with host buffers (host->device image upload and device->host map
read-back inside the timed region), the roofline of the dominant kernel
(FP32 ALU bound), the FP64 oracle timed on the host cores as a reported CPU
baseline, and the SM clocks sampled during the timed region.

``--impl reference`` times the FP64 oracle (the reference arm of this
project: the paper ships no code) on a bounded crop of the same workload on
the host cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

REPO = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, REPO)

METRIC = "Mpixel-iterations/s (3200x2112, 10 src)"
UNIT = "Mpx-iter/s"
SCENE = "large"
ITERS = 6
SEED = 11
# Algorithmic FP32 work of one (hypothesis, view) cost evaluation: 36 window
# samples x 22 flop (3 homography, 2 perspective-divide multiplies, 11
# bilinear, 6 moment flops) + 80 flop per pair (homography set-up, validity,
# NCC from the moments).
FLOP_PER_SAMPLE = 22
SAMPLES_PER_PAIR = 36
FLOP_PER_PAIR_SETUP = 80
FLOP_PER_PAIR = SAMPLES_PER_PAIR * FLOP_PER_SAMPLE + FLOP_PER_PAIR_SETUP
FP32_LANES_PER_SM = 128
# dram__bytes_read.sum + dram__bytes_write.sum per phase launch from an ncu
# capture, keyed by the hash of the phase kernel's sources it was taken on
# and the interpolation form (null whenever the sources changed since).
KNOWN_TRAFFIC: dict[str, float] = {
    "443431915a570157/fp32_blend": 212933120.0 + 145355264.0,         # profiles/phase_kernel_large.md
    "443431915a570157/texture_bilinear": 213670656.0 + 146705664.0,   # profiles/phase_kernel_texture_large.md
}


PHASE_KERNEL_SOURCES = ("amh_device.cuh", "amh_kernels.cu", "amh_kernels.h", "amh_update.cuh")
# the batched form's variants (AMH_BATCH_VARIANTS): block tile / warp pixel layout
VARIANT_NAMES = ["16x16/warp 16x4", "32x8/warp 32x2", "64x4/warp 64x1", "16x16/warp 8x8", "32x8/warp 16x4"]


def kernel_source_hash() -> str:
    """Hash of the sources the phase kernel is compiled from."""
    h = hashlib.sha256()
    csrc = os.path.join(REPO, "paper_1805_07920_gb300", "csrc")
    for f in PHASE_KERNEL_SOURCES:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


def parse(argv=None):
    return parse_args(argv)


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the batched-form and learned-proposal measurements (run only at N = 1)")
    ap.add_argument("--texture-bilinear", action="store_true",
                    help="time the texture-filter precision form (AMH_FLAG_TEXTURE_BILINEAR) instead of the "
                         "default FP32-blend form")
    ap.add_argument("--staged-fetch", action="store_true",
                    help="time the shared-memory staged matrix sweep (AMH_FLAG_STAGED_FETCH) instead of the "
                         "default texture-only fetch path")
    return ap.parse_args(argv)


def dist_setup(want_cuda: bool):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import datetime

        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        # a rank that dies or never arrives turns the others' next collective
        # into an error after this long instead of a hang
        timeout = datetime.timedelta(seconds=float(os.environ.get("AMH_DIST_TIMEOUT_S", "600")))
        dist.init_process_group("nccl" if want_cuda else "gloo", timeout=timeout)
        pg = dist
    return rank, world, local, pg


def spawn_ranks(n: int, cmd: list[str], port: int | None = None) -> int:
    """Launch `cmd` as n local ranks, one process per GPU (RANK = LOCAL_RANK =
    r, WORLD_SIZE = n, rendezvous on 127.0.0.1), wait for all of them and
    return the first non-zero exit code (0 when every rank succeeded)."""
    import socket
    if port is None:
        with socket.socket() as sk:
            sk.bind(("127.0.0.1", 0))
            port = sk.getsockname()[1]
    procs = []
    for r in range(n):
        env = dict(os.environ, RANK=str(r), LOCAL_RANK=str(r), WORLD_SIZE=str(n), LOCAL_WORLD_SIZE=str(n),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        procs.append(subprocess.Popen(cmd, env=env))
    rcs = [p.wait() for p in procs]
    return next((rc for rc in rcs if rc), 0)


def check_world(gpus: int) -> str | None:
    """None when the launcher's world size (WORLD_SIZE, 1 without one) is the
    --gpus the run was asked for, else the reason it is not."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if world != gpus:
        return f"--gpus {gpus} but the launcher started {world} rank(s)"
    return None


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")
    NAMES = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, mx, reasons, n = [], [], set(), 0
        for ln in out.splitlines():
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            n += 1
            for name, val in zip(self.NAMES, parts[3:7]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": n}


# ---------------------------------------------------------------------------
# workload
# ---------------------------------------------------------------------------
def assign_reference(sc, rank: int):
    """The work of rank r: view (ref + r) mod n of the same scene as the
    reference, its sources the other views by camera distance along the arc
    (rank 0 keeps the scene's own reference and sources)."""
    from paper_1805_07920_gb300 import synth
    if not rank:
        return sc
    n = len(sc.cams)
    ref = (sc.ref + rank) % n
    src = sorted([v for v in range(n) if v != ref], key=lambda v: (abs(v - ref), v))[:len(sc.src)]
    return synth.Scene(sc.name, sc.seed, sc.cams, sc.images, ref, src, sc.depth_min, sc.depth_max, {}, {})


def rank_scene(rank: int):
    from paper_1805_07920_gb300 import synth
    return assign_reference(synth.make_scene(SCENE), rank)


def max_over_ranks(ms: float, dist, device: str) -> float:
    """The slowest rank's time (the whole job's time); ms itself without a
    process group."""
    if not dist:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(pixels: int, iters: int, steps: int, world: int, ms: float) -> float:
    """Mpixel-iterations/s of the whole job: every rank updates `pixels`
    pixels `iters` times per step."""
    return pixels * iters * steps * world / (ms / 1e3) / 1e6


def cpu_oracle_rate(sc, seconds: float, crop=(320, 212), threads: int = 1):
    """FP64 oracle on a centred crop of the reference with all sources: init +
    iterations until `seconds` have passed; `threads` > 1 splits the rows of
    each phase over host threads (same results)."""
    import oracle
    from paper_1805_07920_gb300 import synth
    oracle.build() if not os.path.exists(oracle.LIB_PATH) else None
    oracle.set_threads(threads)
    w, h = crop
    x0, y0 = (sc.width - w) // 2, (sc.height - h) // 2
    c = synth.crop_scene(sc, x0, y0, w, h)
    o = oracle.Oracle.from_scene(c, seed=SEED)
    t0 = time.perf_counter()
    o.init_random()
    its = 0
    while its < ITERS:
        o.iterate(1)
        its += 1
        if time.perf_counter() - t0 >= seconds:
            break
    dt = time.perf_counter() - t0
    oracle.set_threads(1)
    return w * h * its / dt / 1e6, dict(crop=f"{w}x{h}", iterations=its, seconds=round(dt, 2))


def run_reference(args):
    rank, world, _, pg = dist_setup(False)
    if rank != 0:
        return 0
    sc = rank_scene(0)
    crop = (160, 106)
    vals = []
    for i in range(args.warmup + args.steps):
        v, info = cpu_oracle_rate(sc, 0.0, crop=crop)   # init + 1 iteration
        if i >= args.warmup:
            vals.append(v)
    val = float(np.mean(vals))
    ms = crop[0] * crop[1] * 1 / (val * 1e6) * 1e3
    line = {
        "impl": "reference", "metric": METRIC, "value": round(val, 6), "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 2), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(sc),
        "cpu_baseline": {"value": round(val, 6), "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"each step: oracle init + 1 iteration on a {crop[0]}x{crop[1]} centred "
                                   f"crop of the reference with all {len(sc.src)} full-size sources"},
        "e2e": {"value": round(val, 6), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def workload_config(sc):
    return {"workload": f"{SCENE}: {sc.width}x{sc.height} reference + {len(sc.src)} source views, "
                        f"random init + {ITERS} checkerboard iterations",
            "width": sc.width, "height": sc.height, "n_src": len(sc.src), "iterations": ITERS,
            "window": "11x11 stride 2 (36 samples)",
            "l2": "inputs larger than L2: ~280 MB resident per context (textures + state) vs 129 MB L2"}


def run_ours(args, measure=None, scene=None, want_cuda: bool = True):
    """This project's arm: every rank times its own reference view (device
    work in `measure`, by default measure_device); the job's time is the
    slowest rank's and rank 0 prints the JSON line.  `measure`, `scene` and
    `want_cuda` exist for the multi-rank host test, which runs this on CPU
    ranks with a stub in place of the device work."""
    bad = check_world(args.gpus)
    if bad:
        print(f"bench.py: {bad}", file=sys.stderr)
        return 2
    rank, world, local, dist = dist_setup(want_cuda)
    dev = "cuda" if want_cuda else "cpu"
    pg = (dist.get_backend() if dist else "none")
    print(f"bench rank {rank}: device {dev}:{local}, process group {pg}, world size {world}", file=sys.stderr,
          flush=True)
    if scene is None:
        from paper_1805_07920_gb300 import synth
        scene = synth.make_scene(SCENE)
    sc = assign_reference(scene, rank)

    def barrier():
        if dist:
            dist.barrier()

    m = (measure or measure_device)(args, sc, rank, world, local, barrier)
    ms = max_over_ranks(m["ms"], dist, dev)
    value = job_rate(sc.width * sc.height, ITERS, args.steps, world, ms)
    e2e = m.get("e2e")
    if e2e is not None:
        e_ms = max_over_ranks(e2e.pop("ms"), dist, dev)
        e2e = {"value": round(job_rate(sc.width * sc.height, ITERS, e2e["steps"], world, e_ms), 3), "unit": UNIT,
               **e2e}
    refs = [sc.ref]
    if dist:
        refs = [None] * world
        dist.all_gather_object(refs, sc.ref)

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded ray-cast scene)",
            "config": workload_config(sc) | {"parallelism": f"replicas{world}: one reference view per GPU",
                                             "interpolation": m.get("form", "fp32_blend"),
                                             "reference_per_rank": refs},
            "roofline": m.get("roofline"), "cpu_baseline": m.get("cpu_baseline"),
            "cpu_baseline_all_cores": m.get("cpu_baseline_all_cores"), "e2e": e2e,
            "extras": m.get("extras", {}),
            "clocks": m.get("clocks"), "gpu_launches": m.get("gpu_launches"),
            "pairs_per_step": m.get("pairs_per_step"),
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def measure_device(args, sc, rank, world, local, barrier):
    """The device work of one rank: init + 6 iterations of its reference view
    per step, timed with CUDA events on the launching stream after a barrier;
    then the roofline of the phase kernel, the end-to-end run through the
    C-ABI with host buffers, the other forms and the oracle on the host
    (rank 0 of a one-rank job only)."""
    import torch
    torch.cuda.set_device(local)
    from paper_1805_07920_gb300 import amh
    amh.lib()
    W, H = sc.width, sc.height
    form_flags = (amh.AMH_FLAG_TEXTURE_BILINEAR if args.texture_bilinear else 0) | \
        (amh.AMH_FLAG_STAGED_FETCH if args.staged_fetch else 0)
    form = "texture_bilinear" if args.texture_bilinear else "fp32_blend"
    if args.staged_fetch:
        form += "+staged"
    ctx = amh.Context.from_scene(sc, seed=SEED, flags=form_flags)
    stream = torch.cuda.current_stream()

    def step():
        ctx.init_random()
        ctx.iterate(ITERS)

    for _ in range(max(args.warmup, 1)):
        step()
    ctx.synchronize()
    # deterministic work per step: count the (hypothesis, view) evaluations once
    ctx.pair_count(reset=True)
    ctx.init_random()
    pairs_init = ctx.pair_count(reset=True)
    ctx.iterate(ITERS)
    pairs_phase, staged_phase = ctx.pair_counts(reset=True)

    clock = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    clock.start()
    time.sleep(0.3)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ph = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps * 2 * ITERS)]
    ev0.record(stream)
    k = 0
    for _ in range(args.steps):
        ctx.init_random()
        for _it in range(ITERS):
            for color in (0, 1):
                ph[k][0].record(stream)
                ctx.step_phase(color)
                ph[k][1].record(stream)
                k += 1
    ev1.record(stream)
    ev1.synchronize()
    torch.cuda.synchronize()
    clocks = clock.stop()
    ms = ev0.elapsed_time(ev1)
    phase_ms = float(np.mean([a.elapsed_time(b) for a, b in ph]))
    barrier()

    # roofline of the dominant kernel (the colour-phase kernel)
    props = torch.cuda.get_device_properties(local)
    sm_max = clocks["sm_max_mhz"] or 2070.0
    peak = props.multi_processor_count * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    flop_per_launch = pairs_phase / (2 * ITERS) * FLOP_PER_PAIR
    achieved = flop_per_launch / (phase_ms / 1e3) / 1e12
    khash = kernel_source_hash()
    roofline = {"bound": "alu", "achieved": round(achieved, 3), "peak": round(peak, 2), "unit": "TFLOP/s",
                "frac": round(achieved / peak, 4), "traffic": KNOWN_TRAFFIC.get(f"{khash}/{form}"),
                "kernel": "phase_kernel", "launch_ms": round(phase_ms, 3),
                "flop_per_launch": flop_per_launch, "pairs_per_launch": pairs_phase / (2 * ITERS),
                "peak_basis": f"{props.multi_processor_count} SMs x 128 FP32 lanes x 2 flop x {sm_max:.0f} MHz "
                              f"(max SM clock)", "kernel_hash": khash}
    # the second ceiling: one 2x2 texture gather per window sample, against the
    # gather rate of this GPU measured in this run by a gather-only loop
    gpeak = amh.gather_peak()
    samples_per_s = pairs_phase / (2 * ITERS) * SAMPLES_PER_PAIR / (phase_ms * 1e-3)
    tex_per_s = (pairs_phase - staged_phase) / (2 * ITERS) * SAMPLES_PER_PAIR / (phase_ms * 1e-3)
    roofline["staged_pair_fraction"] = round(staged_phase / max(1, pairs_phase), 4)
    roofline["fetch"] = {"bound": "texture gather", "achieved": round(tex_per_s / 1e12, 4),
                         "peak": round(gpeak / 1e12, 4), "unit": "T samples/s",
                         "frac": round(tex_per_s / gpeak, 4),
                         "all_samples_per_s": round(samples_per_s / 1e12, 4),
                         "note": "achieved counts the samples fetched through the texture unit; the staged "
                                 "fraction of the evaluations reads shared-memory boxes instead",
                         "peak_basis": "amh_gather_peak: gather-only loop over update-like windows, measured live"}

    # end to end through the C-ABI with host buffers
    e2e = None
    if args.e2e_steps > 0:
        pinned = [torch.from_numpy(im).pin_memory() for im in sc.images]
        host_imgs = [p.numpy() for p in pinned]
        outs = {k2: torch.empty(s, dtype=torch.float32).pin_memory() for k2, s in
                (("depth", (H, W)), ("normal", (H, W, 3)), ("cost", (H, W)))}
        sel_out = torch.empty((H, W), dtype=torch.int32).pin_memory()
        h2d = int(sum(sc.images[v].nbytes for v in [sc.ref] + list(sc.src)))
        d2h = int(sum(t.numel() * 4 for t in outs.values()) + sel_out.numel() * 4)

        def e2e_step():
            c = amh.Context(sc.cams, host_imgs, sc.ref, sc.src,
                            amh.default_params(depth_min=sc.depth_min, depth_max=sc.depth_max, seed=SEED,
                                               flags=form_flags))
            c.init_random()
            c.iterate(ITERS)
            amh.lib().amh_read_maps(c.ctx, amh._ptr(outs["depth"].numpy()), amh._ptr(outs["normal"].numpy()),
                                    amh._ptr(outs["cost"].numpy()), amh._ptr(sel_out.numpy()),
                                    amh.AMH_MEM_HOST)
            c.close()
        e2e_step()
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            e2e_step()
        torch.cuda.synchronize()
        e_ms = (time.perf_counter() - t0) * 1e3
        e2e = {"ms": e_ms, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "steps": args.e2e_steps,
               "path": "amh_create from pinned host images + init + 6 iterations + amh_read_maps to pinned "
                       "host + amh_destroy"}

    extras = {}
    if not args.no_extras and world == 1:     # one-GPU measurements of the other forms
        if not args.texture_bilinear and not args.staged_fetch:
            extras["staged_fetch_3200x2112"] = bench_form(sc, args.steps, phase_ms, ctx, "staged")
            extras["texture_bilinear_3200x2112"] = bench_form(sc, args.steps, phase_ms, ctx, "texture")
            extras["images_f16_3200x2112"] = bench_form(sc, args.steps, phase_ms, ctx, "f16")
        extras["batched_ring20"] = bench_batch(args, None)
        extras["learned_proposal_1600x1056"] = bench_learned()

    cpu = cpu_all = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, info = cpu_oracle_rate(sc, args.cpu_seconds)
        cpu = {"value": round(v, 6), "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"FP64 oracle, one thread: init + {info['iterations']} iteration(s) on a {info['crop']} "
                         f"centred crop of the reference with all {len(sc.src)} full-size sources "
                         f"({info['seconds']} s)"}
        ncores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
        va, ia = cpu_oracle_rate(sc, args.cpu_seconds / 2, crop=(640, 424), threads=ncores)
        cpu_all = {"value": round(va, 6), "unit": UNIT, "cores": ncores, "kind": "oracle",
                   "sample": f"the same oracle with the rows of each phase split over {ncores} host threads: init + "
                             f"{ia['iterations']} iteration(s) on a {ia['crop']} centred crop ({ia['seconds']} s)"}
    return {"ms": ms, "form": form, "roofline": roofline, "e2e": e2e, "extras": extras, "clocks": clocks,
            "cpu_baseline": cpu, "cpu_baseline_all_cores": cpu_all,
            "gpu_launches": args.steps * (1 + 2 * ITERS), "pairs_per_step": pairs_init + pairs_phase}


def bench_form(sc, steps, default_phase_ms, default_ctx, form):
    """The same workload in another form -- "texture": the texture unit's
    filter interpolates (AMH_FLAG_TEXTURE_BILINEAR); "f16": the images stored
    as FP16 (AMH_FLAG_IMAGES_F16); "staged": the matrix sampled from
    shared-memory boxes where the windows fit (AMH_FLAG_STAGED_FETCH) -- :
    throughput, phase-launch time, and the fraction of pixels
    within 1 % of the ground truth next to the default form's (both after the
    last timed step)."""
    import torch
    from paper_1805_07920_gb300 import amh
    if form == "texture":
        ctx = amh.Context.from_scene(sc, seed=SEED, flags=amh.AMH_FLAG_TEXTURE_BILINEAR)
        what = "texture-unit linear filter (fractions and their product rounded to 1/256)"
    elif form == "staged":
        ctx = amh.Context.from_scene(sc, seed=SEED, flags=amh.AMH_FLAG_STAGED_FETCH)
        what = ("the 8 x N matrix sampled from shared-memory boxes of bilinear cells where a warp's windows fit "
                "(t >= 1), the rest through the texture unit")
    else:
        ctx = amh.Context.from_scene(sc, seed=SEED, images=[im.astype(np.float16) for im in sc.images])
        what = "images stored as FP16 textures, FP32 interpolation and moments"
    stream = torch.cuda.current_stream()
    for _ in range(2):
        ctx.init_random()
        ctx.iterate(ITERS)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ph = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps * 2 * ITERS)]
    ev0.record(stream)
    k = 0
    for _ in range(steps):
        ctx.init_random()
        for _it in range(ITERS):
            for color in (0, 1):
                ph[k][0].record(stream)
                ctx.step_phase(color)
                ph[k][1].record(stream)
                k += 1
    ev1.record(stream)
    ev1.synchronize()
    ms = ev0.elapsed_time(ev1)
    phase_ms = float(np.mean([a.elapsed_time(b) for a, b in ph]))
    gt = sc.gt_depth[sc.ref].astype(np.float64)
    m = gt > 0
    m[:5] = m[-5:] = False
    m[:, :5] = m[:, -5:] = False

    def acc(c):
        d = c.read_maps()["depth"].astype(np.float64)
        return round(float((np.abs(d - gt)[m] <= 0.01 * gt[m]).mean()), 4)
    out = {"metric": METRIC, "unit": UNIT, "value": round(job_rate(sc.width * sc.height, ITERS, steps, 1, ms), 3),
           "ms_per_step": round(ms / steps, 3), "launch_ms": round(phase_ms, 3),
           "launch_ms_default_form": round(default_phase_ms, 3),
           "accuracy_1pct": acc(ctx), "accuracy_1pct_default_form": acc(default_ctx), "form": what}
    ctx.close()
    return out


def bench_batch(args, dist):
    """Batched form: the 20-camera ring, every view the reference with its 10
    nearest views as sources (8 x 1920x1080, 6 x 2560x1440, 6 x 3200x2112), one
    persistent launch per colour phase, init + 6 iterations replayed from a
    CUDA graph, tile variant picked by the autotuner."""
    import torch
    from paper_1805_07920_gb300 import amh, synth
    sc = synth.make_scene("ring20")
    n = len(sc.cams)
    refs = list(range(n))
    srcs = [synth.ring_sources(r, n, 10) for r in refs]
    p = amh.default_params(depth_min=sc.depth_min, depth_max=sc.depth_max, seed=SEED)
    b = amh.Batch(sc.cams, sc.images, refs, srcs, p)
    chosen, tune_ms = b.autotune(iters=1)
    for _ in range(max(1, args.warmup)):
        b.run(ITERS)
    b.synchronize()
    b.pair_count(reset=True)
    b.run(ITERS)
    pairs = b.pair_count(reset=True)
    steps = max(1, min(args.steps, 3))
    if dist:
        dist.barrier()
    b.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        b.run(ITERS)
    b.synchronize()
    ms = (time.perf_counter() - t0) * 1e3
    px = sum(w * h for (w, h, _) in b.sizes)
    post = postprocess(b, sc, refs)
    b.close()
    # the same batch in the texture-filter precision form, same tile variant
    pt = amh.default_params(depth_min=sc.depth_min, depth_max=sc.depth_max, seed=SEED,
                            flags=amh.AMH_FLAG_TEXTURE_BILINEAR)
    bt = amh.Batch(sc.cams, sc.images, refs, srcs, pt)
    bt.set_variant(chosen)
    bt.run(ITERS)
    bt.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        bt.run(ITERS)
    bt.synchronize()
    ms_t = (time.perf_counter() - t0) * 1e3
    bt.close()
    texture = {"value": round(px * ITERS * steps / (ms_t / 1e3) / 1e6, 3), "ms_per_batch": round(ms_t / steps, 3),
               "flags": "AMH_FLAG_TEXTURE_BILINEAR"}
    return {"metric": "Mpixel-iterations/s over all 20 references", "unit": UNIT, "postprocess": post,
            "texture_bilinear": texture,
            "value": round(px * ITERS * steps / (ms / 1e3) / 1e6, 3), "ms_per_batch": round(ms / steps, 3),
            "pixels_per_iteration": px, "pairs_per_batch": pairs, "launches_per_batch": 1 + 2 * ITERS,
            "tile_variant": VARIANT_NAMES[chosen], "variants": VARIANT_NAMES,
            "autotune_ms": [round(float(m), 3) for m in tune_ms], "timing": "host wall clock around graph launches"}


def postprocess(b, sc, refs):
    """The post-processing of Sec. 3.3 on the batch's 20 depth maps: the 4x4
    median of every map, then the consistency fusion of all of them (f_eps
    0.3, f_ang 30 degrees, f_con 2), timed with CUDA events."""
    import torch
    from paper_1805_07920_gb300 import amh
    D, N = [], []
    for r in range(len(refs)):
        st = b.get_state(r)
        D.append(torch.from_numpy(np.ascontiguousarray(st["plane"][..., 3])).cuda())
        N.append(torch.from_numpy(np.ascontiguousarray(st["plane"][..., :3])).cuda())
    stream = torch.cuda.current_stream()
    cams = [sc.cams[r] for r in refs]
    # one untimed pass first: the output tensors come from the caching
    # allocator afterwards, so the events time the kernels, not cudaMalloc
    del_ = amh.fuse(cams, [amh.median4(d) for d in D], N)
    del del_
    torch.cuda.synchronize()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    e[0].record(stream)
    Dm = [amh.median4(d) for d in D]
    e[1].record(stream)
    pts, cnt = amh.fuse(cams, Dm, N)
    e[2].record(stream)
    e[2].synchronize()
    fused = int(sum(int(((c >= 2) & (d > 0)).sum().item()) for c, d in zip(cnt, Dm)))
    return {"median4_ms": round(e[0].elapsed_time(e[1]), 3), "fuse_ms": round(e[1].elapsed_time(e[2]), 3),
            "fused_points": fused, "pixels": int(sum(d.numel() for d in Dm)),
            "params": "f_eps 0.3, f_ang 30 deg, f_con 2"}


def bench_learned():
    """Learned-proposal form on the held-out 1600x1056 scenes (seeds 2003,
    2004; 10 sources): device time of the plain method's init + 6 iterations
    against the time the proposal schedule (network on the state after 2
    iterations) needs to reach the same accuracy (pixels within 1 % of the
    ground-truth depth)."""
    from paper_1805_07920_gb300 import amh, learned, synth
    out = {}
    net = None
    for seed in (2003, 2004):
        sc = synth.make_scene("learned", seed=seed)
        if net is None:
            net = amh.Net(*amh.net_size_for(sc.width, sc.height))
            net.load(learned.WEIGHTS)
        r = learned.evaluate_scene(sc, net, seed, schedules={"net@2": learned.SCHEDULES["net@2"]},
                                   log=lambda s: None)
        s = r["schedules"]["net@2"]
        out[f"seed_{seed}"] = {
            "plain_ms_6_iterations": round(r["ms_plain_final"], 3), "plain_accuracy_1pct": round(r["acc_plain"][-1], 4),
            "learned_iterations_to_plain_accuracy": s["iters_to_plain_final"],
            "learned_ms_to_plain_accuracy": None if s["ms_to_plain_final"] is None else round(s["ms_to_plain_final"], 3),
            "network_ms": [round(m, 3) for m in s["ms_net"]],
            "accuracy_per_iteration": {"plain": [round(a, 4) for a in r["acc_plain"]],
                                       "learned": [round(a, 4) for a in s["acc"]]}}
    net.close()
    out["scenes"] = "learned family, 1600x1056, 10 sources, held out of training and of the schedule choice"
    out["timing"] = "CUDA events per iteration on the launching stream (accuracy read-back excluded)"
    return out


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        # no launcher: one process per GPU, started here
        return spawn_ranks(args.gpus, [sys.executable, os.path.abspath(__file__), *sys.argv[1:]])
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
