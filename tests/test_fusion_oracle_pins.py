"""Pins of the post-processing oracle (oracle/fusion.py): the 4x4 median
against a brute-force loop and against closed forms (a constant stays, a
ramp moves by half a pixel), and the consistency fusion against ground truth
(depth maps rendered for every view fuse into points on the true surface with
the true normals; a view whose depth is scaled by 10 % stops agreeing with
the others; a stricter f_con keeps a subset)."""
import numpy as np
import pytest

from oracle import fusion as F


def test_median4_brute_force():
    d = np.random.default_rng(1).uniform(1, 9, (7, 9))
    m = F.median4(d)
    H, W = d.shape
    for y in range(H):
        for x in range(W):
            v = sorted(d[min(max(y + dy, 0), H - 1), min(max(x + dx, 0), W - 1)]
                       for dy in (-2, -1, 0, 1) for dx in (-2, -1, 0, 1))
            assert m[y, x] == pytest.approx(0.5 * (v[7] + v[8]), rel=1e-15)


def test_median4_closed_forms():
    np.testing.assert_array_equal(F.median4(np.full((6, 8), 3.25)), 3.25)
    ramp = np.tile(np.arange(12, dtype=np.float64), (6, 1))
    m = F.median4(ramp)
    np.testing.assert_allclose(m[:, 2:11], ramp[:, 2:11] - 0.5, rtol=0, atol=1e-15)


@pytest.fixture(scope="module")
def fusion_scene(synth_mod):
    return synth_mod.make_scene("fusion")


def _maps(sc):
    V = len(sc.cams)
    return [sc.gt_depth[v].astype(np.float64) for v in range(V)], [sc.gt_normal[v].astype(np.float64) for v in range(V)]


def test_ground_truth_fuses_onto_the_surface(fusion_scene):
    sc = fusion_scene
    D, N = _maps(sc)
    pts, valid, cnt, _ = F.fuse(sc.cams, D, N)
    for v, c in enumerate(sc.cams):
        assert valid[v].mean() >= 0.85
        K, R, t = (np.asarray(a, np.float64).reshape(s) for a, s in ((c.K, (3, 3)), (c.R, (3, 3)), (c.t, 3)))
        H, W = D[v].shape
        ys, xs = np.mgrid[0:H, 0:W]
        X = (D[v][..., None] * (np.stack([xs, ys, np.ones_like(xs)], -1) @ np.linalg.inv(K).T) - t) @ R
        m = valid[v]
        err = np.linalg.norm(pts[v][..., :3] - X, axis=-1)[m] / D[v][m]
        assert np.median(err) < 2e-3 and np.quantile(err, 0.99) < 1e-2
        ang = np.degrees(np.arccos(np.clip((pts[v][..., 3:] * (N[v] @ R)).sum(-1), -1, 1)))[m]
        assert np.quantile(ang, 0.99) < 5.0


def test_inconsistent_view_is_rejected(fusion_scene):
    sc = fusion_scene
    D, N = _maps(sc)
    _, v0, c0, _ = F.fuse(sc.cams, D, N)
    D2 = [d.copy() for d in D]
    D2[1] *= 1.1
    _, v1, c1, _ = F.fuse(sc.cams, D2, N)
    assert v1[1].mean() < 0.05                          # view 1 agrees with nobody
    for v in (0, 2, 3, 4):
        assert c1[v].mean() < c0[v].mean() - 0.5        # everybody loses view 1
        assert (c1[v] <= c0[v]).all()


def test_stricter_consensus_keeps_a_subset(fusion_scene):
    sc = fusion_scene
    D, N = _maps(sc)
    va = F.fuse(sc.cams, D, N, f_con=1)[1]
    vb = F.fuse(sc.cams, D, N, f_con=2)[1]
    vc = F.fuse(sc.cams, D, N, f_con=4)[1]
    for a, b, c in zip(va, vb, vc):
        assert (b <= a).all() and (c <= b).all() and c.sum() < a.sum()


def _pair_cams(synth_mod, b, W=64, H=48, f=100.0):
    K = np.array([[f, 0.0, (W - 1) / 2], [0.0, f, (H - 1) / 2], [0.0, 0.0, 1.0]])
    R = np.eye(3)
    return [synth_mod.Camera(K, R, np.zeros(3), W, H),
            synth_mod.Camera(K, R, np.array([-b, 0.0, 0.0]), W, H)]   # centre (b, 0, 0)


def test_fronto_parallel_pair_closed_form(synth_mod):
    """Two cameras with the same orientation, centres b apart along x, a
    fronto-parallel plane: view 0 sees it at depth 5, view 1 (slightly off) at
    5.05.  View 0's pixel x lands on view 1's pixel x - 20 b exactly (f = 100),
    where the disparity difference is f b |1/5 - 1/5.05| = 0.198 b: one
    agreeing view for b = 1 (a fused point halfway, at depth 5.025), none for
    b = 2 (0.396 > f_eps = 0.3)."""
    W, H = 64, 48
    D = [np.full((H, W), 5.0), np.full((H, W), 5.05)]
    N = [np.tile(np.array([0.0, 0.0, -1.0]), (H, W, 1))] * 2
    pts, valid, cnt, amb = F.fuse(_pair_cams(synth_mod, 1.0), D, N, f_eps=0.3, f_ang_deg=30.0, f_con=1)
    xs = np.arange(W)
    seen = np.broadcast_to(xs >= 20, (H, W))               # x - 20 inside view 1
    assert not amb[0].any()
    np.testing.assert_array_equal(cnt[0], seen.astype(cnt[0].dtype))
    np.testing.assert_array_equal(valid[0], seen)
    np.testing.assert_allclose(pts[0][..., 2][seen], 5.025, rtol=0, atol=1e-12)
    X0 = 5.0 * (xs - (W - 1) / 2) / 100.0                    # view 0's point
    X1 = 5.05 * (xs - 20 - (W - 1) / 2) / 100.0 + 1.0        # view 1's point at x - 20
    np.testing.assert_allclose(pts[0][..., 0][seen], np.broadcast_to(0.5 * (X0 + X1), (H, W))[seen], atol=1e-12)
    # twice the baseline: the same depth offset is twice the disparity, rejected
    _, valid2, cnt2, _ = F.fuse(_pair_cams(synth_mod, 2.0), D, N, f_eps=0.3, f_ang_deg=30.0, f_con=1)
    assert not valid2[0].any() and not cnt2[0].any()
