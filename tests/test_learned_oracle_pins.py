"""Pins of the learned-proposal network's CPU oracle (oracle/learned.py).

The network is this project's own extension, so what fixes its oracle is
mathematics, not the paper: a 3x3 convolution written out as a brute-force
five-fold loop; the adjoint identities that tie the data and weight
gradients to the forward convolution (and pooling to upsampling); the whole
network and its gradients rebuilt from PyTorch library operators (NCHW
conv2d, avg_pool2d, nearest interpolate, autograd) in float64; central finite
differences; BF16 rounding against PyTorch's own conversion.  A transposed
operand, a flipped tap, a skip wired to the wrong level or a dropped ReLU mask
fails at least one of them.
"""
import numpy as np
import pytest

from oracle import learned as L


def _rng(seed=0):
    return np.random.default_rng(seed)


def test_conv3x3_brute_force():
    r = _rng(1)
    H, W, Ci, Co = 4, 5, 3, 2
    x, w, b = r.normal(size=(H, W, Ci)), r.normal(size=(9, Co, Ci)), r.normal(size=Co)
    y = L.conv3x3(x, w, b)
    ref = np.zeros((H, W, Co))
    for i in range(H):
        for j in range(W):
            for co in range(Co):
                s = b[co]
                for dy in (-1, 0, 1):
                    for dx in (-1, 0, 1):
                        ii, jj = i + dy, j + dx
                        if 0 <= ii < H and 0 <= jj < W:
                            for ci in range(Ci):
                                s += w[3 * (dy + 1) + (dx + 1), co, ci] * x[ii, jj, ci]
                ref[i, j, co] = s
    np.testing.assert_allclose(y, ref, rtol=1e-13, atol=1e-13)


def test_conv_gradients_are_adjoints():
    r = _rng(2)
    H, W, Ci, Co = 6, 7, 4, 5
    x, w = r.normal(size=(H, W, Ci)), r.normal(size=(9, Co, Ci))
    dy = r.normal(size=(H, W, Co))
    zero = np.zeros(Co)
    # <conv(x), dy> = <x, dgrad(dy)>
    lhs = (L.conv3x3(x, w, zero) * dy).sum()
    assert abs(lhs - (x * L.conv3x3_dgrad(dy, w)).sum()) < 1e-10 * max(1.0, abs(lhs))
    # <conv_w(x), dy> is linear in w with gradient wgrad
    dw, db = L.conv3x3_wgrad(x, dy)
    w2 = r.normal(size=w.shape)
    assert abs((L.conv3x3(x, w2, zero) * dy).sum() - (w2 * dw).sum()) < 1e-10 * max(1.0, abs(lhs))
    np.testing.assert_allclose(db, dy.reshape(-1, Co).sum(0), rtol=1e-13)


def test_pool_and_upsample_adjoints():
    r = _rng(3)
    x, d = r.normal(size=(8, 6, 3)), r.normal(size=(4, 3, 3))
    assert abs((L.pool2(x) * d).sum() - (x * L.pool2_bwd(d)).sum()) < 1e-12
    z, e = r.normal(size=(4, 3, 3)), r.normal(size=(8, 6, 3))
    assert abs((L.up2(z) * e).sum() - (z * L.up2_bwd(e)).sum()) < 1e-12
    # pooling a constant keeps it; upsampling then pooling is the identity
    np.testing.assert_allclose(L.pool2(np.full((4, 4, 2), 3.5)), 3.5)
    np.testing.assert_allclose(L.pool2(L.up2(z)), z, rtol=1e-15)


def _torch_net(params, x0):
    torch = pytest.importorskip("torch")
    F = torch.nn.functional
    P = {k: (torch.tensor(np.asarray(w).reshape(3, 3, w.shape[1], w.shape[2])).permute(2, 3, 0, 1).contiguous()
             .requires_grad_(), torch.tensor(np.asarray(b)).requires_grad_()) for k, (w, b) in params.items()}
    x = torch.tensor(x0).permute(2, 0, 1)[None]

    def conv(name, v, relu=True):
        y = F.conv2d(v, P[name][0], P[name][1], padding=1)
        return F.relu(y) if relu else y

    e1 = conv("e1", x)
    e2 = conv("e2", F.avg_pool2d(e1, 2))
    e3 = conv("e3", F.avg_pool2d(e2, 2))
    e4 = conv("e4", F.avg_pool2d(e3, 2))
    d3 = conv("d3", F.interpolate(e4, scale_factor=2, mode="nearest")) + e3
    d2 = conv("d2", F.interpolate(d3, scale_factor=2, mode="nearest")) + e2
    d1 = conv("d1", F.interpolate(d2, scale_factor=2, mode="nearest")) + e1
    out = conv("out", d1, relu=False)
    return out[0].permute(1, 2, 0), P


def test_network_against_torch_library_ops():
    torch = pytest.importorskip("torch")
    r = _rng(4)
    params = {k: (w, r.normal(0, 0.1, size=b.shape)) for k, (w, b) in L.init_params(5).items()}
    x0 = r.normal(size=(16, 24, 16))
    out, cache = L.forward(params, x0)
    tout, P = _torch_net(params, x0)
    np.testing.assert_allclose(out, tout.detach().numpy(), rtol=1e-10, atol=1e-10)
    # gradients of the L1 loss through autograd
    target = r.normal(size=(16, 24, 4))
    mask = r.random((16, 24)) < 0.7
    loss, dout = L.l1_loss(out, target, mask)
    g = L.backward(cache, dout)
    tl = (torch.abs(tout[..., :4] - torch.tensor(target)).sum(-1) * torch.tensor(mask)).sum() / mask.sum()
    assert abs(tl.item() - loss) < 1e-12
    tl.backward()
    for name, (tw, tb) in P.items():
        gw = tw.grad.permute(2, 3, 0, 1).reshape(9, tw.shape[0], tw.shape[1]).numpy()
        np.testing.assert_allclose(g[name][0], gw, rtol=1e-9, atol=1e-12, err_msg=name)
        np.testing.assert_allclose(g[name][1], tb.grad.numpy(), rtol=1e-9, atol=1e-12, err_msg=name)


def test_backward_by_finite_differences():
    r = _rng(6)
    params = {k: (w, r.normal(0, 0.05, size=b.shape)) for k, (w, b) in L.init_params(7).items()}
    x0 = r.normal(size=(8, 16, 16))
    G = r.normal(size=(8, 16, 16))           # loss = <out, G>, smooth in the weights
    out, cache = L.forward(params, x0)
    g = L.backward(cache, G)
    eps = 1e-6
    for name in ("e1", "e3", "d3", "d1", "out"):
        w, b = params[name]
        for _ in range(3):
            idx = tuple(int(r.integers(0, s)) for s in w.shape)
            wp, wm = w.copy(), w.copy()
            wp[idx] += eps
            wm[idx] -= eps
            fp = (L.forward({**params, name: (wp, b)}, x0)[0] * G).sum()
            fm = (L.forward({**params, name: (wm, b)}, x0)[0] * G).sum()
            fd = (fp - fm) / (2 * eps)
            assert abs(fd - g[name][0][idx]) < 1e-5 * max(1.0, abs(fd)), (name, idx, fd, g[name][0][idx])
        j = int(r.integers(0, b.shape[0]))
        bp, bm = b.copy(), b.copy()
        bp[j] += eps
        bm[j] -= eps
        fd = ((L.forward({**params, name: (w, bp)}, x0)[0] * G).sum()
              - (L.forward({**params, name: (w, bm)}, x0)[0] * G).sum()) / (2 * eps)
        assert abs(fd - g[name][1][j]) < 1e-5 * max(1.0, abs(fd)), (name, j)


def test_l1_loss_definition():
    out = np.zeros((2, 2, 16))
    out[..., 0] = [[1.0, -2.0], [0.5, 0.0]]
    tgt = np.zeros((2, 2, 4))
    mask = np.array([[True, True], [False, True]])
    loss, g = L.l1_loss(out, tgt, mask)
    assert loss == pytest.approx((1.0 + 2.0 + 0.0) / 3)
    assert g[0, 0, 0] == pytest.approx(1 / 3) and g[0, 1, 0] == pytest.approx(-1 / 3)
    assert g[1, 0, 0] == 0.0 and g[1, 1, 0] == 0.0 and not g[..., 4:].any()


def test_bf16_round_matches_torch_and_ties_to_even():
    torch = pytest.importorskip("torch")
    assert L.bf16_round(1.0 + 2.0 ** -8) == 1.0                     # tie, even below
    assert L.bf16_round(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6     # tie, even above
    assert L.bf16_round(1.0 + 2.0 ** -8 + 2.0 ** -20) == 1.0 + 2.0 ** -7
    x = _rng(8).normal(size=4096) * np.exp(_rng(9).uniform(-20, 20, 4096))
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(L.bf16_round(x), ref)


def test_bf16_forward_rounds_stored_activations_only():
    r = _rng(10)
    params = L.init_params(11)
    x0 = r.normal(size=(8, 8, 16))
    o64, _ = L.forward(params, x0)
    o16, c16 = L.forward(params, x0, bf16=True)
    for k in ("e1", "e2", "d3", "in_e2"):
        np.testing.assert_array_equal(c16[k], L.bf16_round(c16[k]))
    rel = np.linalg.norm(o16 - o64) / np.linalg.norm(o64)
    assert 1e-5 < rel < 5e-2
