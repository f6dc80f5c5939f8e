"""The ablations of Sec. 4 on synthetic scenes with ground truth: the method
with asymmetric checkerboard propagation and multi-hypothesis joint view
selection against each of them replaced (symmetric propagation, heuristic
per-hypothesis k-best view selection) and against both replaced.  Reports,
after every iteration, the fraction of valid pixels with depth within 1 % of
the ground truth, and the device time of each iteration (the counterpart of
the paper's convergence comparison of its two propagation schemes).

    python -m paper_1805_07920_gb300.ablation [--scene large] [--iters 6]
"""
from __future__ import annotations

import argparse
import json
import sys

import numpy as np

from . import amh, synth

MODES = {
    "full": 0,
    "symmetric_propagation": amh.AMH_FLAG_SYMMETRIC_PROPAGATION,
    "heuristic_views": amh.AMH_FLAG_HEURISTIC_VIEWS,
    "both": amh.AMH_FLAG_SYMMETRIC_PROPAGATION | amh.AMH_FLAG_HEURISTIC_VIEWS,
}


def accuracy(depth, scene, margin=5, rel=0.01):
    """Fraction of pixels with ground truth (and >= margin px from the border)
    whose depth is within rel of it."""
    gt = scene.gt_depth[scene.ref]
    v = gt > 0
    v[:margin] = v[-margin:] = False
    v[:, :margin] = v[:, -margin:] = False
    return float((np.abs(depth[v] - gt[v]) <= rel * gt[v]).mean())


def convergence(scene, seed=5, iters=6, modes=MODES):
    import torch
    stream = torch.cuda.current_stream()
    out = {}
    for name, flags in modes.items():
        p = amh.default_params(depth_min=scene.depth_min, depth_max=scene.depth_max, seed=seed, flags=flags)
        ctx = amh.Context.from_scene(scene, p)
        ctx.init_random()
        acc, ms = [], []
        for _ in range(iters):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            ctx.iterate(1)
            b.record(stream)
            b.synchronize()
            ms.append(a.elapsed_time(b))
            acc.append(accuracy(ctx.get_state()["plane"][..., 3], scene))
        ctx.close()
        out[name] = {"accuracy_1pct": [round(x, 4) for x in acc], "ms_per_iteration": [round(x, 3) for x in ms]}
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(prog="python -m paper_1805_07920_gb300.ablation")
    ap.add_argument("--scene", default="large")
    ap.add_argument("--seed", type=int, default=None, help="scene seed (default: the scene's own)")
    ap.add_argument("--iters", type=int, default=6)
    a = ap.parse_args(argv)
    sc = synth.make_scene(a.scene, seed=a.seed)
    res = convergence(sc, iters=a.iters)
    print(json.dumps({"scene": f"{a.scene} {sc.width}x{sc.height}, {len(sc.src)} sources", "modes": res}, indent=1))


if __name__ == "__main__":
    sys.exit(main())
