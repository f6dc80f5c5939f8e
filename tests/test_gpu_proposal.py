"""Caller-supplied plane proposals (amh_set_proposal): one plane per 2 x 2
block, scored at each pixel as one more refinement candidate under the
pixel's view weights (choice code 15), so the method stays the arbiter.

With the ground-truth planes of the scene as the proposal: every pixel where
the proposal loses is bit-identical to the plain update, winners exist, a
winner's plane is the proposal's plane met at that pixel's ray, and its cost
is the oracle's unified cost of that plane; host and device copies of the
proposal give the same result; a proposal with no valid plane changes
nothing."""
import numpy as np
import pytest

from parity_utils import COST_TOL, color_mask, fp32_state, same_plane

pytestmark = pytest.mark.gpu
KEYS = ("plane", "cost", "sel", "vbest", "wmask", "choice")


@pytest.fixture(scope="module")
def amh():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_07920_gb300 import amh as m
    m.lib()
    return m


def _gt_proposal(scene):
    """(h2, w2, 4) planes (n, d), n . X + d = 0 in reference-camera
    coordinates, from the ground truth at pixel (2X, 2Y)."""
    H, W = scene.images[scene.ref].shape
    w2, h2 = (W + 1) // 2, (H + 1) // 2
    Y, X = np.mgrid[0:h2, 0:w2]
    x, y = np.minimum(2 * X, W - 1), np.minimum(2 * Y, H - 1)
    D = scene.gt_depth[scene.ref][y, x].astype(np.float64)
    n = scene.gt_normal[scene.ref][y, x].astype(np.float64)
    Ki = np.linalg.inv(np.asarray(scene.cams[scene.ref].K, np.float64))
    P = D[..., None] * (np.stack([x, y, np.ones_like(x)], -1) @ Ki.T)
    d = -(n * P).sum(-1)
    d = np.where((D > 0) & np.isfinite(d), d, 0.0)
    return np.concatenate([n, d[..., None]], -1).astype(np.float32), Ki


def _pair_from(amh, scene, st, p):
    c = amh.Context.from_scene(scene, p)
    c.set_state(**{k: st[k] for k in KEYS}, t=st["t"])
    return c


def test_ground_truth_proposal(amh, tiny_scene, oracle_mod):
    sc = tiny_scene
    H, W = sc.images[sc.ref].shape
    p = amh.default_params(depth_min=sc.depth_min, depth_max=sc.depth_max, seed=17)
    base = amh.Context.from_scene(sc, p)
    base.init_random()
    base.iterate(1)
    st = base.get_state()
    prop, Ki = _gt_proposal(sc)
    a_ctx, b_ctx = _pair_from(amh, sc, st, p), _pair_from(amh, sc, st, p)
    amh.set_proposal(a_ctx, prop)
    a_ctx.step_phase(0)
    b_ctx.step_phase(0)
    a, b = a_ctx.get_state(), b_ctx.get_state()
    won = color_mask(H, W, 0) & (a["choice"] == 15)
    assert won.sum() > 0.02 * color_mask(H, W, 0).sum(), won.sum()
    for k in KEYS:
        np.testing.assert_array_equal(a[k][~won], b[k][~won], err_msg=f"{k} changed where the proposal lost")
    assert (a["cost"][won] < b["cost"][won]).all()
    ys, xs = np.nonzero(won)
    cell = prop[np.minimum(ys // 2, prop.shape[0] - 1), np.minimum(xs // 2, prop.shape[1] - 1)].astype(np.float64)
    ray = np.stack([xs, ys, np.ones_like(xs)], -1) @ Ki.T
    Dx = -cell[:, 3] / (cell[:, :3] * ray).sum(-1)
    exp = np.concatenate([cell[:, :3], Dx[:, None]], -1)
    assert same_plane(a["plane"][won].astype(np.float64), exp, rel_d=1e-4, ang=1e-6).mean() >= 0.999
    orc = oracle_mod.Oracle.from_scene(sc, oracle_mod.default_params(depth_min=sc.depth_min,
                                                                      depth_max=sc.depth_max, seed=17))
    s = fp32_state(dict(plane=st["plane"].astype(np.float64), cost=st["cost"].astype(np.float64), sel=st["sel"],
                        vprev=np.where(st["vbest"] == 255, -1, st["vbest"].astype(np.int32)), t=st["t"]))
    orc.set_state(plane=s["plane"], cost=s["cost"], sel=s["sel"], vprev=s["vprev"], t=s["t"])
    pick = np.random.default_rng(1).permutation(len(ys))[:200]
    dc = np.array([abs(orc.score_plane(int(xs[i]), int(ys[i]), a["plane"][ys[i], xs[i]].astype(np.float64))
                       - a["cost"][ys[i], xs[i]]) for i in pick])
    assert (dc <= COST_TOL).mean() >= 0.99, dc.max()


def test_device_and_host_proposals_agree(amh, tiny_scene):
    import torch
    sc = tiny_scene
    p = amh.default_params(depth_min=sc.depth_min, depth_max=sc.depth_max, seed=18)
    base = amh.Context.from_scene(sc, p)
    base.init_random()
    base.iterate(1)
    st = base.get_state()
    prop, _ = _gt_proposal(sc)
    a_ctx, b_ctx = _pair_from(amh, sc, st, p), _pair_from(amh, sc, st, p)
    amh.set_proposal(a_ctx, prop)
    amh.set_proposal(b_ctx, torch.from_numpy(prop).cuda())
    a_ctx.iterate(1)
    b_ctx.iterate(1)
    a, b = a_ctx.get_state(), b_ctx.get_state()
    for k in KEYS:
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)


def test_proposal_without_valid_planes_changes_nothing(amh, tiny_scene):
    sc = tiny_scene
    p = amh.default_params(depth_min=sc.depth_min, depth_max=sc.depth_max, seed=19)
    base = amh.Context.from_scene(sc, p)
    base.init_random()
    base.iterate(1)
    st = base.get_state()
    prop, _ = _gt_proposal(sc)
    prop[..., 3] = 0.0                      # d <= 0: no plane
    a_ctx, b_ctx = _pair_from(amh, sc, st, p), _pair_from(amh, sc, st, p)
    amh.set_proposal(a_ctx, prop[:3, :5])   # a smaller grid repeats its edge cells
    a_ctx.iterate(1)
    b_ctx.iterate(1)
    a, b = a_ctx.get_state(), b_ctx.get_state()
    for k in KEYS:
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)
    with pytest.raises(amh.AmhError):
        amh.set_proposal(a_ctx, np.zeros((0, 4, 4), np.float32))
