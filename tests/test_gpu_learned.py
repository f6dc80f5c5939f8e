"""The learned proposal network through the C-ABI: forward outputs, loss and
every weight / bias gradient of the BF16 tensor-core kernels against the FP64
oracle (oracle/learned.py, BF16 rounding emulated at the same points), Adam
against PyTorch's CPU Adam, the feature / target / head conversions, and the
injection of the proposal into the checkerboard update (a candidate scored by
the unchanged cost, leaving every other pixel as the plain method has it).

Tolerances: the kernels accumulate in FP32 where the oracle uses FP64, so a
value that lands near a BF16 rounding boundary can be stored one BF16 ulp
(2^-8 relative) apart; that touches a small fraction of the activations, and
the outputs and gradients are compared by relative L2 error (<= 3e-3) and
largest element error (<= 3e-2 of the tensor's largest magnitude).  The loss
targets sit 0.5..1.5 away from the outputs so no sign of the L1 gradient is
decided by rounding.

End to end, a value of FP32 accumulation landing on the other side of a BF16
rounding boundary from the FP64 one moves that stored activation by one BF16
ulp, and the network carries such moves on to every later layer and gradient
(an FP32-accumulation emulation of the oracle already differs from it by up
to 3e-4 in the first layer's weight gradient), so the whole-network
comparison is a coarse check (relative L2 <= 3e-3 forward, <= 3e-2 for
gradients).  The exact check is per operation: every stored tensor of the
kernels is read back and each operation recomputed by the oracle from the
kernels' own inputs, where the only differences left are the FP32
accumulation (bounded by 2e-5 of the sum of the absolute terms) and, for
BF16-stored results, the rounding of a near-tie (at most one BF16 ulp, on
< 1 % of the elements)."""
import numpy as np
import pytest

from oracle import learned as OL
from parity_utils import COST_TOL, color_mask, fp32_state, same_plane

pytestmark = pytest.mark.gpu

H2, W2 = 40, 72            # levels 40x72, 20x36, 10x18, 5x9: several 64-pixel tiles and ragged tails


@pytest.fixture(scope="module")
def amh():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_07920_gb300 import amh as m
    m.lib()
    return m


def _params(seed):
    r = np.random.default_rng(seed)
    return {k: (w.astype(np.float32), r.normal(0, 0.05, b.shape).astype(np.float32))
            for k, (w, b) in OL.init_params(seed).items()}


def _close(a, b, what, rel=3e-3, mx=3e-2):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    err = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)
    big = np.abs(a - b).max() / max(np.abs(b).max(), 1e-30)
    assert err <= rel and big <= mx, f"{what}: rel L2 {err:.2e}, max {big:.2e}"


def _setup(amh, seed=1):
    r = np.random.default_rng(seed)
    net = amh.Net(W2, H2, seed=3)
    params = _params(seed)
    net.set_params(params)
    x0 = r.normal(0, 0.5, (H2, W2, 16)).astype(np.float32)
    net.set_input(x0)
    return net, params, x0, r


def test_forward_matches_oracle(amh):
    net, params, x0, _ = _setup(amh, 1)
    out = net.forward(want_output=True)
    ref16, _ = OL.forward(params, x0.astype(np.float64), bf16=True)
    _close(out, ref16, "forward vs BF16-emulating oracle")
    ref64, _ = OL.forward(params, x0.astype(np.float64), bf16=False)
    _close(out, ref64, "forward vs FP64 oracle", rel=3e-2, mx=1e-1)     # the BF16 storage error itself


def test_loss_and_gradients_match_oracle(amh):
    net, params, x0, r = _setup(amh, 2)
    out = net.forward(want_output=True)
    sign = np.where(r.random((H2, W2, 4)) < 0.5, -1.0, 1.0)
    target = (out[..., :4] + sign * r.uniform(0.5, 1.5, (H2, W2, 4))).astype(np.float32)
    mask = r.random((H2, W2)) < 0.7
    net.set_targets(target, mask.astype(np.uint8))
    loss = net.backward()
    ref_out, cache = OL.forward(params, x0.astype(np.float64), bf16=True)
    ref_loss, dout = OL.l1_loss(ref_out, target.astype(np.float64), mask)
    assert abs(loss - ref_loss) <= 1e-4 * ref_loss
    g = net.get_grads()
    ref = OL.backward(cache, dout, bf16=True)
    errs = []
    for name, _, _ in amh.NET_LAYERS:
        for i, what in ((0, "dW"), (1, "db")):
            a, b = np.asarray(g[name][i], np.float64), ref[name][i]
            errs.append((f"{what} {name}", np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)))
    print("whole-network gradient rel L2:", ", ".join(f"{k} {v:.1e}" for k, v in errs))
    bad = [(k, v) for k, v in errs if v > 3e-2]
    assert not bad, bad


def _ulp_bf16(v):
    a = np.maximum(np.abs(np.asarray(v, np.float64)), 2.0 ** -126)
    return 2.0 ** (np.floor(np.log2(a)) - 7)


def _check_bf16(got, ref, scale, what):
    """got: a BF16-stored kernel result; ref: the FP64 value before rounding;
    scale: the sum of the absolute terms behind ref (FP32 accumulation can
    move a value near zero across the ReLU by up to 2e-5 of it)."""
    r = OL.bf16_round(ref)
    same = got == r
    assert (same | (np.abs(got - ref) <= _ulp_bf16(ref) + 2e-5 * scale)).all(), f"{what}: beyond one BF16 ulp"
    assert same.mean() >= 0.99, f"{what}: {1 - same.mean():.3%} rounded differently"


def _check_acc(got, ref, scale, what, k=2e-5):
    """FP32-accumulated result against FP64: |got - ref| <= k * sum |terms|."""
    err = np.abs(np.asarray(got, np.float64) - ref)
    assert (err <= k * scale + 1e-30).all(), f"{what}: worst {np.max(err / (scale + 1e-30)):.1e} of the term sum"


def test_every_operation_elementwise(amh):
    """Each forward and backward operation, recomputed by the oracle from the
    kernels' own stored inputs, element by element."""
    net, params, x0, r = _setup(amh, 4)
    net.forward()
    G = {k: net.read(k).astype(np.float64) for k in net.NET_TENSORS}
    Pw = {k: OL.bf16_round(w) for k, (w, b) in params.items()}
    Pb = {k: np.asarray(b, np.float64) for k, (w, b) in params.items()}
    absw = {k: np.abs(v) for k, v in Pw.items()}
    np.testing.assert_array_equal(G["x0"], OL.bf16_round(x0))
    relu = lambda v: np.maximum(v, 0.0)
    conv = lambda x, L: OL.conv3x3(x, Pw[L], Pb[L])
    # encoder: conv + ReLU (<= 1 ulp), pooling (exact: the mean of four BF16 values is exact in FP32)
    for L, xin, y, pooled in (("e1", "x0", "e1", "in_e2"), ("e2", "in_e2", "e2", "in_e3"),
                              ("e3", "in_e3", "e3", "in_e4"), ("e4", "in_e4", "e4", None)):
        _check_bf16(G[y], relu(conv(G[xin], L)), OL.conv3x3(np.abs(G[xin]), absw[L], np.abs(Pb[L])), f"forward {L}")
        if pooled:
            np.testing.assert_array_equal(G[pooled], OL.bf16_round(OL.pool2(G[y])), err_msg=pooled)
    # decoder: upsampling (a copy), conv + ReLU, then the skip sum rounded once
    for L, up_src, xin, rr, skip, y in (("d3", "e4", "in_d3", "r3", "e3", "d3"), ("d2", "d3", "in_d2", "r2", "e2", "d2"),
                                        ("d1", "d2", "in_d1", "r1", "e1", "d1")):
        np.testing.assert_array_equal(G[xin], OL.up2(G[up_src]), err_msg=xin)
        _check_bf16(G[rr], relu(conv(G[xin], L)), OL.conv3x3(np.abs(G[xin]), absw[L], np.abs(Pb[L])), f"forward {L}")
        s_ = G[rr] + G[skip]
        assert (np.abs(G[y] - OL.bf16_round(s_)) <= _ulp_bf16(s_)).all() and (G[y] == OL.bf16_round(s_)).mean() > 0.9999
    _check_acc(G["out"], conv(G["d1"], "out"),
               OL.conv3x3(np.abs(G["d1"]), absw["out"], np.abs(Pb["out"])), "forward out")

    # backward from a loss with well-separated targets
    target = (G["out"][..., :4] + np.where(r.random((H2, W2, 4)) < 0.5, -1.0, 1.0) * r.uniform(0.5, 1.5, (H2, W2, 4)))
    mask = r.random((H2, W2)) < 0.7
    net.set_targets(target.astype(np.float32), mask.astype(np.uint8))
    net.backward()
    D = {L: net.read("dy:" + L).astype(np.float64) for L, _, _ in amh.NET_LAYERS}
    _, dout = OL.l1_loss(G["out"], target.astype(np.float32).astype(np.float64), mask)
    np.testing.assert_allclose(D["out"], dout, rtol=1e-6, atol=0, err_msg="loss gradient")
    # weight and bias gradients from each layer's stored input and output gradient
    g = net.get_grads()
    inputs = {"e1": "x0", "e2": "in_e2", "e3": "in_e3", "e4": "in_e4", "d3": "in_d3", "d2": "in_d2",
              "d1": "in_d1", "out": "d1"}
    b16 = OL.bf16_round
    for L, xin in inputs.items():
        dw = OL.conv3x3_wgrad(G[xin], b16(D[L]))[0]          # tensor cores: BF16 dy
        db = OL.conv3x3_wgrad(G[xin], D[L])[1]               # FP32 bias sums
        sw = OL.conv3x3_wgrad(np.abs(G[xin]), np.abs(b16(D[L])))[0]
        sb = OL.conv3x3_wgrad(np.abs(G[xin]), np.abs(D[L]))[1]
        _check_acc(g[L][0], dw, sw, f"dW {L}", k=1e-4)
        _check_acc(g[L][1], db, sb, f"db {L}", k=1e-4)
    # data gradients: each layer's masked output gradient from the next one's

    def dg(L):   # d (input of L) from L's stored output gradient, and its term-sum scale
        return OL.conv3x3_dgrad(b16(D[L]), Pw[L]), OL.conv3x3_dgrad(np.abs(b16(D[L])), absw[L])

    gd1, sd1 = dg("out")
    _check_acc(D["d1"], gd1 * (G["r1"] > 0), sd1, "dy d1")
    t, st_ = dg("d1")
    gd2, sd2 = OL.up2_bwd(t), OL.up2_bwd(st_)
    _check_acc(D["d2"], gd2 * (G["r2"] > 0), sd2, "dy d2")
    t, st_ = dg("d2")
    gd3, sd3 = OL.up2_bwd(t), OL.up2_bwd(st_)
    _check_acc(D["d3"], gd3 * (G["r3"] > 0), sd3, "dy d3")
    t, st_ = dg("d3")
    _check_acc(D["e4"], OL.up2_bwd(t) * (G["e4"] > 0), OL.up2_bwd(st_), "dy e4")
    t, st_ = dg("e4")
    _check_acc(D["e3"], (gd3 + OL.pool2_bwd(t)) * (G["e3"] > 0), sd3 + OL.pool2_bwd(st_), "dy e3")
    t, st_ = dg("e3")
    _check_acc(D["e2"], (gd2 + OL.pool2_bwd(t)) * (G["e2"] > 0), sd2 + OL.pool2_bwd(st_), "dy e2")
    t, st_ = dg("e2")
    _check_acc(D["e1"], (gd1 + OL.pool2_bwd(t)) * (G["e1"] > 0), sd1 + OL.pool2_bwd(st_), "dy e1")


def test_adam_matches_torch(amh):
    torch = pytest.importorskip("torch")
    net, params, x0, r = _setup(amh, 3)
    out = net.forward(want_output=True)
    net.set_targets((out[..., :4] + 1.0).astype(np.float32), np.ones((H2, W2), np.uint8))
    net.backward()
    g = net.get_grads()
    tp = []
    for name, _, _ in amh.NET_LAYERS:
        for i in (0, 1):
            p = torch.tensor(params[name][i].astype(np.float32), requires_grad=True)
            p.grad = torch.tensor(g[name][i])
            tp.append(p)
    opt = torch.optim.Adam(tp, lr=1e-3, betas=(0.9, 0.999), eps=1e-8)
    opt.step()
    net.adam(1e-3)
    got = net.get_params()
    k = 0
    for name, _, _ in amh.NET_LAYERS:
        for i in (0, 1):
            np.testing.assert_allclose(got[name][i], tp[k].detach().numpy(), rtol=1e-5, atol=1e-7, err_msg=name)
            k += 1


def _features_host(scene, st, w2, h2, p):
    W, H = st["plane"].shape[1], st["plane"].shape[0]
    X, Y = np.meshgrid(np.arange(w2), np.arange(h2))
    x, y = np.minimum(2 * X, W - 1), np.minimum(2 * Y, H - 1)
    pl = st["plane"][y, x].astype(np.float64)
    lmid = 0.5 * (np.log(p.depth_min) + np.log(p.depth_max))
    lscale = 2.0 / np.log(p.depth_max / p.depth_min)
    f = np.zeros((h2, w2, 16))
    f[..., 0] = scene.images[scene.ref][y, x] / 255.0 - 0.5
    f[..., 1] = (np.log(np.maximum(pl[..., 3], 1e-6)) - lmid) * lscale
    f[..., 2:5] = pl[..., :3]
    f[..., 5] = st["cost"][y, x] * 0.5
    return f, pl


def _proposal_host(scene, out, pin, W, H):
    """The head's plane (n, d) per half-resolution pixel, as the header defines it."""
    h2, w2 = out.shape[:2]
    K = np.asarray(scene.cams[scene.ref].K, np.float64).reshape(3, 3)
    Ki = np.linalg.inv(K)
    X, Y = np.meshgrid(np.arange(w2), np.arange(h2))
    ray = np.stack([np.minimum(2 * X, W - 1), np.minimum(2 * Y, H - 1), np.ones_like(X)], -1) @ Ki.T
    D = pin[..., 3] * np.exp(np.clip(out[..., 0], -3, 3))
    n = pin[..., :3] + out[..., 1:4]
    n = n / np.linalg.norm(n, axis=-1, keepdims=True)
    n = np.where(((n * ray).sum(-1) < 0)[..., None], n, -n)
    d = -D * (n * ray).sum(-1)
    return n, d, Ki


def test_features_targets_and_injection(amh, tiny_scene, oracle_mod):
    scene = tiny_scene
    H, W = scene.images[scene.ref].shape
    p = amh.default_params(depth_min=scene.depth_min, depth_max=scene.depth_max, seed=11)
    ctx = amh.Context.from_scene(scene, p)
    ctx.init_random()
    ctx.iterate(1)
    st = ctx.get_state()
    w2, h2 = amh.net_size_for(W, H)
    net = amh.Net(w2, h2, seed=5)
    # features from the context == features from the host
    net.features(ctx)
    out = net.forward(want_output=True)
    f, pin = _features_host(scene, st, w2, h2, p)
    net2 = amh.Net(w2, h2, seed=5)
    net2.set_input(f.astype(np.float32))
    _close(out, net2.forward(want_output=True), "features from the state", rel=1e-3, mx=1e-2)
    # targets: the loss against the context's later state, with the host's mask and residuals
    ctx2 = amh.Context.from_scene(scene, p)
    ctx2.set_state(**{k: st[k] for k in ("plane", "cost", "sel", "vbest", "wmask", "choice")}, t=st["t"])
    ctx2.iterate(2)
    st2 = ctx2.get_state()
    net.targets(ctx2, cost_max=0.5)
    loss = net.backward()
    X, Y = np.meshgrid(np.arange(w2), np.arange(h2))
    x, y = np.minimum(2 * X, W - 1), np.minimum(2 * Y, H - 1)
    pf = st2["plane"][y, x].astype(np.float64)
    ok = (st2["cost"][y, x] < 0.5) & (pf[..., 3] > 0) & (pin[..., 3] > 0)
    tgt = np.concatenate([np.log(pf[..., 3:4]) - np.log(pin[..., 3:4]), pf[..., :3] - pin[..., :3]], -1)
    ref_loss = np.abs(out[..., :4] - tgt)[ok].sum() / max(1, ok.sum())
    assert ok.sum() > 0 and abs(loss - ref_loss) <= 1e-4 * max(ref_loss, 1e-3)

    # injection: one phase with the proposal against one without, from the same state
    net.propose(ctx)
    ctx_plain = amh.Context.from_scene(scene, p)
    ctx_plain.set_state(**{k: st[k] for k in ("plane", "cost", "sel", "vbest", "wmask", "choice")}, t=st["t"])
    ctx.step_phase(0)
    ctx_plain.step_phase(0)
    a, b = ctx.get_state(), ctx_plain.get_state()
    mask = color_mask(H, W, 0)
    won = mask & (a["choice"] == 15)
    assert won.sum() > 0, "no proposal was ever preferred"
    for k in ("plane", "cost", "sel", "vbest", "wmask", "choice"):
        np.testing.assert_array_equal(a[k][~won], b[k][~won], err_msg=f"{k} changed where the proposal lost")
    assert (a["cost"][won] < b["cost"][won]).all()
    # the winning plane is the head's proposal at that pixel ...
    n, d, Ki = _proposal_host(scene, out, pin, W, H)
    ys, xs = np.nonzero(won)
    ray = np.stack([xs, ys, np.ones_like(xs)], -1) @ Ki.T
    nb, db = n[np.minimum(ys // 2, h2 - 1), np.minimum(xs // 2, w2 - 1)], d[np.minimum(ys // 2, h2 - 1), np.minimum(xs // 2, w2 - 1)]
    Dx = -db / (nb * ray).sum(-1)
    exp_plane = np.concatenate([nb, Dx[:, None]], -1)
    assert same_plane(a["plane"][won].astype(np.float64), exp_plane, rel_d=1e-4, ang=1e-6).mean() >= 0.999
    # ... and its cost is the oracle's unified cost of that plane under the pixel's weights
    orc = oracle_mod.Oracle.from_scene(scene, oracle_mod.default_params(depth_min=scene.depth_min,
                                                                         depth_max=scene.depth_max, seed=11))
    s = fp32_state(dict(plane=st["plane"].astype(np.float64), cost=st["cost"].astype(np.float64),
                        sel=st["sel"], vprev=np.where(st["vbest"] == 255, -1, st["vbest"].astype(np.int32)),
                        t=st["t"]))
    orc.set_state(plane=s["plane"], cost=s["cost"], sel=s["sel"], vprev=s["vprev"], t=s["t"])
    sample = np.random.default_rng(0).permutation(len(ys))[:200]
    dc = [abs(orc.score_plane(int(xs[i]), int(ys[i]), a["plane"][ys[i], xs[i]].astype(np.float64))
              - a["cost"][ys[i], xs[i]]) for i in sample]
    assert np.mean(np.array(dc) <= COST_TOL) >= 0.99, np.max(dc)
    # clearing the proposal restores the plain update exactly
    amh.clear_proposal(ctx)
    ctx_plain.set_state(**{k: a[k] for k in ("plane", "cost", "sel", "vbest", "wmask", "choice")}, t=a["t"])
    ctx.step_phase(1)
    ctx_plain.step_phase(1)
    a2, b2 = ctx.get_state(), ctx_plain.get_state()
    for k in ("plane", "cost", "choice"):
        np.testing.assert_array_equal(a2[k], b2[k])


def test_net_rejects_bad_arguments(amh):
    with pytest.raises(amh.AmhError):
        amh.Net(60, 40)            # not a multiple of 8
    with pytest.raises(amh.AmhError):
        amh.Net(0, 8)


@pytest.mark.parametrize("device", [False, True])
def test_set_example_mirrors_on_the_device(amh, device):
    """amh_net_set_example against the host-side reference of the training
    augmentation: columns (rows) reversed for an x (y) mirror, the normal's x
    (y) negated in feature 2 (3) and target 1 (2), features padded to 16
    channels and stored as BF16 (round to nearest even); targets and mask
    exactly."""
    import torch
    r = np.random.default_rng(11)
    net = amh.Net(W2, H2, seed=3)
    f = r.normal(0, 1, (H2, W2, 6)).astype(np.float32)
    t = r.normal(0, 1, (H2, W2, 4)).astype(np.float32)
    m = (r.random((H2, W2)) < 0.6).astype(np.uint8)
    for mx in (False, True):
        for my in (False, True):
            ef, et, em = f.copy(), t.copy(), m.copy()
            if mx:
                ef, et, em = ef[:, ::-1].copy(), et[:, ::-1].copy(), em[:, ::-1].copy()
                ef[..., 2] *= -1
                et[..., 1] *= -1
            if my:
                ef, et, em = ef[::-1].copy(), et[::-1].copy(), em[::-1].copy()
                ef[..., 3] *= -1
                et[..., 2] *= -1
            x0 = np.zeros((H2, W2, 16), np.float32)
            x0[..., :6] = ef
            x0 = torch.from_numpy(x0).to(torch.bfloat16).float().numpy()
            if device:
                dev = [torch.from_numpy(a).cuda() for a in (f, t, m)]
                net.set_example(*dev, mirror_x=mx, mirror_y=my)
                net.synchronize()
            else:
                net.set_example(f, t, m, mirror_x=mx, mirror_y=my)
            assert np.array_equal(net.read("x0"), x0), (mx, my)
            assert np.array_equal(net.read("target"), et), (mx, my)
            assert np.array_equal(net.read("mask")[..., 0], em.astype(np.float32)), (mx, my)
    net.close()

