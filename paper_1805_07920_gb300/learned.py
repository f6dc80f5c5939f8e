"""Training and evaluation of the learned proposal network (``amh_net_*``).

The network is this project's extension of the method: it reads the state the
checkerboard update has reached after ``T_IN`` iterations (on the
half-resolution grid) and predicts the residuals towards the state the plain
method reaches after its full ``T_FINAL`` iterations (Sec. 4 runs 6).  Its
proposal joins one following iteration as an extra candidate that the
unchanged matching cost scores, so the plain method stays the arbiter.

Training data is the plain method's own output on seeded synthetic scenes (no
ground truth is used for training); the forward pass, every gradient and the
Adam step run in the library's kernels.  Evaluation compares, on held-out
scenes, the fraction of pixels within 1 % of the ground-truth depth after each
iteration with and without the proposal, and the device time to reach the
plain method's final accuracy.

    python -m paper_1805_07920_gb300.learned train --out DIR [--scenes 200]
    python -m paper_1805_07920_gb300.learned evaluate --weights FILE [--seeds 2000 2001]
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

from . import amh, synth

T_IN = (1, 2)       # iteration counts after which the network may read the state
T_FINAL = 6         # the plain method's iteration count
COST_MAX = 0.5      # targets only where the plain method's final cost is below this
TRAIN_SEED0 = 1000
VAL_SEED0 = 1900
EVAL_SEEDS = (2000, 2001, 2002)
WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights", "proposal_net.npz")


# ---------------------------------------------------------------------------
# host-side example preparation (same definitions as the feature / target
# kernels: intensity / 255 - 0.5, log depth scaled to [-1, 1] over the depth
# range, normal, cost / 2, read at full-resolution pixel (2X, 2Y))
# ---------------------------------------------------------------------------
def _grid(W, H, w2, h2):
    X, Y = np.meshgrid(np.arange(w2), np.arange(h2))
    return np.minimum(2 * X, W - 1), np.minimum(2 * Y, H - 1)


def features(image, state, depth_min, depth_max, w2, h2):
    H, W = image.shape
    x, y = _grid(W, H, w2, h2)
    pl = state["plane"][y, x].astype(np.float32)
    lmid = 0.5 * (np.log(depth_min) + np.log(depth_max))
    lscale = 2.0 / np.log(depth_max / depth_min)
    f = np.zeros((h2, w2, 6), np.float32)
    f[..., 0] = image[y, x] / 255.0 - 0.5
    f[..., 1] = (np.log(np.maximum(pl[..., 3], 1e-6)) - lmid) * lscale
    f[..., 2:5] = pl[..., :3]
    f[..., 5] = state["cost"][y, x] * 0.5
    return f, pl


def targets(state_in_planes, state_final, w2, h2, cost_max=COST_MAX):
    H, W = state_final["cost"].shape
    x, y = _grid(W, H, w2, h2)
    pf = state_final["plane"][y, x].astype(np.float64)
    pi = state_in_planes.astype(np.float64)
    ok = (state_final["cost"][y, x] < cost_max) & (pf[..., 3] > 0) & (pi[..., 3] > 0)
    t = np.zeros((h2, w2, 4), np.float32)
    t[..., 0] = np.where(ok, np.log(np.maximum(pf[..., 3], 1e-30)) - np.log(np.maximum(pi[..., 3], 1e-30)), 0)
    t[..., 1:] = np.where(ok[..., None], pf[..., :3] - pi[..., :3], 0)
    return t, ok


def _to_device(examples):
    """Examples as CUDA tensors (features float32, targets float32, mask
    uint8), uploaded once; amh_net_set_example mirrors them on the device."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    out = [tuple(torch.from_numpy(np.ascontiguousarray(a, dt)).to(dev) for a, dt in
                 ((f, np.float32), (t, np.float32), (m, np.uint8))) for f, t, m in examples]
    torch.cuda.synchronize()
    return out


def plain_example(scene, seed):
    """Run the plain method on a scene; return its states after each of T_IN
    iterations and after T_FINAL."""
    p = amh.default_params(depth_min=scene.depth_min, depth_max=scene.depth_max, seed=seed)
    ctx = amh.Context.from_scene(scene, p)
    ctx.init_random()
    states = {}
    for t in range(1, T_FINAL + 1):
        ctx.iterate(1)
        if t in T_IN:
            states[t] = ctx.get_state()
    s_fin = ctx.get_state()
    ctx.close()
    return states, s_fin


def make_examples(seeds, width, height, log=print):
    """One example per scene and T_IN entry: features of that state, targets
    towards the final state."""
    w2, h2 = amh.net_size_for(width, height)
    ex = []
    t0 = time.time()
    for i, s in enumerate(seeds):
        sc = synth.scene_learned(int(s), width=width, height=height)
        states, s_fin = plain_example(sc, int(s))
        for t, st in states.items():
            f, pin = features(sc.images[sc.ref], st, sc.depth_min, sc.depth_max, w2, h2)
            tg, m = targets(pin, s_fin, w2, h2)
            ex.append((f.astype(np.float16), tg, m.astype(np.uint8)))
        if (i + 1) % 20 == 0:
            log(f"  scenes {i + 1}/{len(seeds)}  {time.time() - t0:.0f} s")
    return ex, (w2, h2)


def train(out_dir, n_scenes=200, width=1600, height=1056, steps=8000, lr=1e-3, seed=0, log=print):
    os.makedirs(out_dir, exist_ok=True)
    log(f"rendering {n_scenes} training scenes at {width}x{height}, plain method states after {T_IN} -> {T_FINAL}")
    train_ex, (w2, h2) = make_examples(range(TRAIN_SEED0, TRAIN_SEED0 + n_scenes), width, height, log)
    val_ex, _ = make_examples(range(VAL_SEED0, VAL_SEED0 + 6), width, height, log)
    net = amh.Net(w2, h2, seed=seed)
    rng = np.random.default_rng(seed)
    hist, val_hist = [], []
    train_dev, val_dev = _to_device(train_ex), _to_device(val_ex)

    def val_loss():
        tot = 0.0
        for x, t, m in val_dev:
            net.set_example(x, t, m)
            net.forward()
            tot += net.backward()
        return tot / len(val_dev)

    v0 = val_loss()
    val_hist.append((0, v0))
    log(f"val loss at start {v0:.4f} (zero-residual loss {np.mean([np.abs(t).sum(-1)[m > 0].mean() for _, t, m in val_ex]):.4f})")
    t0 = time.time()
    for it in range(1, steps + 1):
        x, t, m = train_dev[int(rng.integers(len(train_dev)))]
        mirror_x, mirror_y = rng.random() < 0.5, rng.random() < 0.5     # random x / y mirroring
        net.set_example(x, t, m, mirror_x, mirror_y)
        net.forward()
        loss = net.backward()
        cur = lr * 0.5 * (1 + np.cos(np.pi * (it - 1) / steps))     # cosine decay
        net.adam(cur)
        hist.append(loss)
        if it % 500 == 0 or it == steps:
            v = val_loss()
            val_hist.append((it, v))
            log(f"step {it}: train {np.mean(hist[-500:]):.4f}  val {v:.4f}  lr {cur:.2e}  {time.time() - t0:.0f} s")
    path = os.path.join(out_dir, "proposal_net.npz")
    net.save(path)
    rep = dict(n_scenes=n_scenes, width=width, height=height, steps=steps, lr=lr, t_in=list(T_IN), t_final=T_FINAL,
               cost_max=COST_MAX, train_seconds=time.time() - t0,
               train_loss=[float(np.mean(hist[i:i + 100])) for i in range(0, len(hist), 100)],
               val_loss=val_hist, weights=path)
    with open(os.path.join(out_dir, "train_report.json"), "w") as fh:
        json.dump(rep, fh, indent=1)
    return path, rep


# ---------------------------------------------------------------------------
# evaluation
# ---------------------------------------------------------------------------
def accuracy(depth, scene, margin=5, rel=0.01):
    gt = scene.gt_depth[scene.ref]
    v = gt > 0
    v[:margin] = v[-margin:] = False
    v[:, :margin] = v[:, -margin:] = False
    return float((np.abs(depth[v] - gt[v]) <= rel * gt[v]).mean())


def _timed(fn, stream):
    import torch
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    fn()
    b.record(stream)
    b.synchronize()
    return a.elapsed_time(b)


# proposal schedules: the iterations (0-based) before which the network runs
# on the current state, and for how many iterations each proposal is scored
SCHEDULES = {"net@1": ((1,), 1), "net@1+2": ((1, 2), 1), "net@1 keep 2": ((1,), 2), "net@2": ((2,), 1)}


def _run(ctx, net, scene, iters, at, keep, stream):
    acc, ms_it, ms_net = [], [], []
    active = 0
    for it in range(iters):
        if it in at:
            ms_net.append(_timed(lambda: (net.features(ctx), net.forward(), net.propose(ctx)), stream))
            active = keep
        ms_it.append(_timed(lambda: ctx.iterate(1), stream))
        if active:
            active -= 1
            if not active:
                amh.clear_proposal(ctx)
        acc.append(accuracy(ctx.get_state()["plane"][..., 3], scene))
    return acc, ms_it, ms_net


def evaluate_scene(scene, net, seed, iters=T_FINAL, schedules=SCHEDULES, log=print):
    """Accuracy after each iteration, plain and under each proposal schedule,
    and the device time to reach the plain method's final accuracy."""
    import torch
    stream = torch.cuda.current_stream()
    p = amh.default_params(depth_min=scene.depth_min, depth_max=scene.depth_max, seed=seed)
    ctx = amh.Context.from_scene(scene, p)
    ms_init = _timed(ctx.init_random, stream)
    acc_plain, ms_plain, _ = _run(ctx, net, scene, iters, (), 0, stream)
    target = acc_plain[-1]
    r = dict(seed=int(seed), width=scene.width, height=scene.height, acc_plain=acc_plain, ms_init=ms_init,
             ms_iter_plain=ms_plain, ms_plain_final=ms_init + sum(ms_plain), schedules={})
    for name, (at, keep) in schedules.items():
        ctx.init_random()
        acc, ms_it, ms_net = _run(ctx, net, scene, iters, at, keep, stream)
        k = next((i + 1 for i, a in enumerate(acc) if a >= target), None)
        ms_to = None
        if k:
            ms_to = ms_init + sum(ms_it[:k]) + sum(m for a_, m in zip(at, ms_net) if a_ < k)
        r["schedules"][name] = dict(acc=acc, ms_iter=ms_it, ms_net=ms_net, iters_to_plain_final=k,
                                    ms_to_plain_final=ms_to)
    ctx.close()
    log(json.dumps(r, default=lambda v: round(v, 4) if isinstance(v, float) else v))
    return r


def evaluate(weights=WEIGHTS, seeds=EVAL_SEEDS, width=1600, height=1056, log=print):
    w2, h2 = amh.net_size_for(width, height)
    net = amh.Net(w2, h2)
    net.load(weights)
    out = []
    for s in seeds:
        sc = synth.make_scene("learned", seed=int(s)) if (width, height) == (1600, 1056) else \
            synth.scene_learned(int(s), width=width, height=height)
        out.append(evaluate_scene(sc, net, int(s), log=log))
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(prog="python -m paper_1805_07920_gb300.learned")
    sub = ap.add_subparsers(dest="cmd", required=True)
    t = sub.add_parser("train")
    t.add_argument("--out", required=True)
    t.add_argument("--scenes", type=int, default=200)
    t.add_argument("--width", type=int, default=1600)
    t.add_argument("--height", type=int, default=1056)
    t.add_argument("--steps", type=int, default=8000)
    t.add_argument("--lr", type=float, default=1e-3)
    t.add_argument("--eval", action="store_true", help="evaluate on the held-out scenes afterwards")
    e = sub.add_parser("evaluate")
    e.add_argument("--weights", default=WEIGHTS)
    e.add_argument("--seeds", type=int, nargs="*", default=list(EVAL_SEEDS))
    e.add_argument("--width", type=int, default=1600)
    e.add_argument("--height", type=int, default=1056)
    e.add_argument("--out", default=None)
    a = ap.parse_args(argv)
    log = lambda s: print(s, flush=True)
    if a.cmd == "train":
        path, _ = train(a.out, a.scenes, a.width, a.height, a.steps, a.lr, log=log)
        if a.eval:
            res = evaluate(path, log=log)
            with open(os.path.join(a.out, "eval_report.json"), "w") as fh:
                json.dump(res, fh, indent=1)
    else:
        res = evaluate(a.weights, a.seeds, a.width, a.height, log=log)
        if a.out:
            with open(a.out, "w") as fh:
                json.dump(res, fh, indent=1)


if __name__ == "__main__":
    sys.exit(main())
