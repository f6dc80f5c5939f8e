"""Post-processing on the GPU through the C-ABI against the FP64 oracle
(oracle/fusion.py): the 4x4 median exactly (the FP32 result is the exact
median rounded once), the consistency fusion on the ground-truth maps of a
5-view scene and on the method's own depth maps: the same agreeing-view count
on every pixel the oracle does not flag as a near-tie (a projection within
1e-3 px of a rounding boundary, a test within 1e-3 of its threshold), and the
fused points and normals within FP32 rounding."""
import numpy as np
import pytest

from oracle import fusion as F

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def amh():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_07920_gb300 import amh as m
    m.lib()
    return m


@pytest.mark.parametrize("shape", [(120, 160), (23, 37), (1, 9), (5, 1)])
def test_median4_exact(amh, shape):
    import torch
    d = np.random.default_rng(shape[0] * 7 + shape[1]).uniform(1, 9, shape).astype(np.float32)
    d[0, 0] = d[-1, -1]                                   # a repeated value
    got = amh.median4(torch.from_numpy(d).cuda()).cpu().numpy()
    np.testing.assert_array_equal(got, F.median4(d).astype(np.float32))


def _fuse_both(amh, sc, D, N, **kw):
    import torch
    pts_g, cnt_g = amh.fuse(sc.cams, [torch.from_numpy(d).cuda() for d in D], [torch.from_numpy(n).cuda() for n in N], **kw)
    pts_o, val_o, cnt_o, amb = F.fuse(sc.cams, D, N, **kw)
    return [p.cpu().numpy() for p in pts_g], [c.cpu().numpy() for c in cnt_g], pts_o, val_o, cnt_o, amb


def _check(res, D):
    pts_g, cnt_g, pts_o, val_o, cnt_o, amb = res
    for v in range(len(D)):
        clear = ~amb[v]
        assert clear.mean() > 0.95
        np.testing.assert_array_equal(cnt_g[v][clear], cnt_o[v][clear], err_msg=f"view {v}")
        both = clear & val_o[v]
        dx = np.linalg.norm(pts_g[v][..., :3] - pts_o[v][..., :3], axis=-1)[both] / D[v][both]
        assert dx.max() < 1e-4, dx.max()
        dn = np.abs(pts_g[v][..., 3:] - pts_o[v][..., 3:]).max(-1)[both]
        assert dn.max() < 1e-4
        assert not pts_g[v][clear & ~val_o[v]].any()


def test_fusion_ground_truth(amh, synth_mod):
    sc = synth_mod.make_scene("fusion")
    V = len(sc.cams)
    D = [sc.gt_depth[v].astype(np.float32) for v in range(V)]
    N = [sc.gt_normal[v].astype(np.float32) for v in range(V)]
    _check(_fuse_both(amh, sc, D, N), D)
    _check(_fuse_both(amh, sc, D, N, f_eps=1.0, f_ang_deg=10.0, f_con=3), D)


def test_fusion_of_estimated_maps(amh, synth_mod):
    """Every view of the 5-view scene in turn the reference (the others its
    sources), 4 iterations, 4x4 median, then fusion."""
    import torch
    sc = synth_mod.make_scene("fusion")
    V = len(sc.cams)
    D, N = [], []
    for r in range(V):
        src = [v for v in range(V) if v != r]
        p = amh.default_params(depth_min=sc.depth_min, depth_max=sc.depth_max, seed=80 + r)
        g = amh.Context(sc.cams, sc.images, r, src, p)
        g.init_random()
        g.iterate(4)
        st = g.get_state()
        D.append(amh.median4(torch.from_numpy(np.ascontiguousarray(st["plane"][..., 3])).cuda()).cpu().numpy())
        N.append(np.ascontiguousarray(st["plane"][..., :3]))
    res = _fuse_both(amh, sc, D, N)
    _check(res, D)
    assert np.mean([v.mean() for v in res[3]]) > 0.5      # most pixels fuse


@pytest.mark.parametrize("baseline,agree", [(1.0, True), (2.0, False)])
def test_fusion_fronto_parallel_pair(amh, synth_mod, baseline, agree):
    """The closed-form pair of the oracle's pins (same orientation, centres
    `baseline` apart, depths 5 and 5.05 on a fronto-parallel plane): one
    agreeing view and fused points at depth 5.025 for baseline 1, none for 2."""
    import torch
    W, H, f = 64, 48, 100.0
    K = np.array([[f, 0.0, (W - 1) / 2], [0.0, f, (H - 1) / 2], [0.0, 0.0, 1.0]])
    cams = [synth_mod.Camera(K, np.eye(3), np.zeros(3), W, H),
            synth_mod.Camera(K, np.eye(3), np.array([-baseline, 0.0, 0.0]), W, H)]
    D = [np.full((H, W), 5.0, np.float32), np.full((H, W), 5.05, np.float32)]
    N = [np.tile(np.array([0.0, 0.0, -1.0], np.float32), (H, W, 1))] * 2
    pts, cnt = amh.fuse(cams, [torch.from_numpy(d).cuda() for d in D], [torch.from_numpy(n).cuda() for n in N],
                        f_con=1)
    c0 = cnt[0].cpu().numpy()
    seen = np.broadcast_to(np.arange(W) >= 20 * baseline, (H, W)) if agree else np.zeros((H, W), bool)
    np.testing.assert_array_equal(c0, seen.astype(np.uint8))
    if agree:
        np.testing.assert_allclose(pts[0].cpu().numpy()[..., 2][seen], 5.025, rtol=1e-6)
