"""Pins of the FP64 oracle against what the paper and mathematics fix.

The oracle is the yardstick of every GPU parity test, so it is checked here
against things other than itself: an independent library run (cuRAND's host
Philox), textbook routines (numpy's weighted covariance / Pearson
correlation), closed forms (point transfer through a plane, integer-shift
warps on a rectified pair, identical and affinely related patches), the
paper's printed constants, hand-built view-selection cases whose outcome
follows from counting alone, and brute force on a tiny scene.
"""
import ctypes
import json
import math
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


# --------------------------------------------------------------------------
# Philox4x32-10 against cuRAND's host generator (run, not read)
# --------------------------------------------------------------------------
def _curand_host_philox(seed, n):
    for path in ("/usr/local/cuda/lib64/libcurand.so", "libcurand.so", "libcurand.so.10"):
        try:
            L = ctypes.CDLL(path)
            break
        except OSError:
            L = None
    if L is None:
        pytest.skip("libcurand not available")
    g = ctypes.c_void_p()
    assert L.curandCreateGeneratorHost(ctypes.byref(g), 161) == 0  # PHILOX4_32_10
    try:
        assert L.curandSetPseudoRandomGeneratorSeed(g, ctypes.c_ulonglong(seed)) == 0
        out = np.zeros(n, np.uint32)
        assert L.curandGenerate(g, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(n)) == 0
    finally:
        L.curandDestroyGenerator(g)
    return out


@pytest.mark.parametrize("seed", [0, 1, 0x123456789ABCDEF0, 0xFFFFFFFFFFFFFFFF])
def test_philox_matches_curand_host(oracle_mod, seed):
    ref = _curand_host_philox(seed, 4 * 64)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    # the host generator's block i is the counter (0, 0, i, 0) under key = seed
    ours = np.concatenate([oracle_mod.philox4x32_10([0, 0, i, 0], key) for i in range(64)])
    np.testing.assert_array_equal(ours, ref)


def test_philox_counter_words_all_matter(oracle_mod):
    base = oracle_mod.philox4x32_10([5, 6, 7, 8], [9, 10])
    for i in range(4):
        c = [5, 6, 7, 8]
        c[i] ^= 1
        assert not np.array_equal(oracle_mod.philox4x32_10(c, [9, 10]), base)
    assert not np.array_equal(oracle_mod.philox4x32_10([5, 6, 7, 8], [9, 11]), base)


def test_u01_is_exact_24_bit(oracle_mod):
    assert oracle_mod.u01(0) == 0.0
    assert oracle_mod.u01(0xFFFFFFFF) == 1.0 - 2.0 ** -24
    assert oracle_mod.u01(0x100) == 2.0 ** -24
    assert oracle_mod.u01(0x80000000) == 0.5
    assert oracle_mod.u01(0x800000FF) == 0.5   # the low 8 bits are dropped


# --------------------------------------------------------------------------
# parameters and the closed forms of Eqs. (2), (3)
# --------------------------------------------------------------------------
def test_default_params_are_the_papers(oracle_mod):
    g = _golden("params_sec4.json")
    p = oracle_mod.default_params()
    for k, v in g.items():
        if k.startswith("_"):
            continue
        assert getattr(p, k) == v, k


def test_tau_schedule(oracle_mod):
    # Eq. (2) with tau_mc_init = 0.8, alpha = 90 (Sec. 4): starts at 0.8 and
    # decays as a Gaussian in t: log(tau(t)/0.8) * 90 = -t^2
    assert oracle_mod.tau_mc(0) == 0.8
    for t in range(1, 7):
        assert math.log(oracle_mod.tau_mc(t) / 0.8) * 90.0 == pytest.approx(-t * t, rel=1e-12)
    vals = [oracle_mod.tau_mc(t) for t in range(7)]
    assert all(a > b for a, b in zip(vals, vals[1:]))
    # values at the six iterations, to five decimals
    np.testing.assert_allclose(vals, [0.80000, 0.79116, 0.76522, 0.72387, 0.66970, 0.60597, 0.53626],
                               atol=6e-6)


def test_confidence_closed_form(oracle_mod):
    # Eq. (3) with beta = 0.3: C(0) = 1, C(beta) = e^{-1/2}, even in m
    assert oracle_mod.confidence(0.0) == 1.0
    assert oracle_mod.confidence(0.3) == pytest.approx(math.exp(-0.5), rel=1e-14)
    assert oracle_mod.confidence(-0.7) == oracle_mod.confidence(0.7)
    assert oracle_mod.confidence(0.6) == pytest.approx(math.exp(-2.0), rel=1e-14)


# --------------------------------------------------------------------------
# bilinear sampling
# --------------------------------------------------------------------------
def test_bilinear_exact_at_texels_and_on_affine_ramps(oracle_mod):
    rng = np.random.default_rng(0)
    img = rng.integers(0, 256, (9, 13)).astype(np.float64)
    for y in range(9):
        for x in range(13):
            assert oracle_mod.bilinear(img, x, y) == img[y, x]
    yy, xx = np.mgrid[0:9, 0:13]
    ramp = 3.0 + 1.25 * xx - 0.5 * yy
    for _ in range(200):
        x, y = rng.uniform(0, 12), rng.uniform(0, 8)
        assert oracle_mod.bilinear(ramp, x, y) == pytest.approx(3.0 + 1.25 * x - 0.5 * y, abs=1e-12)
    # centre of a texel quad is the mean of its four texels
    assert oracle_mod.bilinear(img, 2.5, 3.5) == pytest.approx(img[3:5, 2:4].mean(), abs=1e-12)


def test_bilinear_clamps_to_edge(oracle_mod):
    img = np.arange(20, dtype=np.float64).reshape(4, 5)
    assert oracle_mod.bilinear(img, -3.0, -7.0) == img[0, 0]
    assert oracle_mod.bilinear(img, 9.0, 1.0) == img[1, 4]
    assert oracle_mod.bilinear(img, 4.0, 3.0) == img[3, 4]
    assert oracle_mod.bilinear(img, 1.5, 10.0) == pytest.approx(0.5 * (img[3, 1] + img[3, 2]))


def _textbook(img, x, y):
    """Bilinear value from the four product weights (a different form of the
    interpolation than the oracle's lerps)."""
    x0, y0 = int(np.floor(x)), int(np.floor(y))
    fx, fy = x - x0, y - y0
    return ((1 - fx) * (1 - fy) * img[y0, x0] + fx * (1 - fy) * img[y0, x0 + 1]
            + (1 - fx) * fy * img[y0 + 1, x0] + fx * fy * img[y0 + 1, x0 + 1])


def test_texture_bilinear_on_the_weight_grid(oracle_mod):
    """Fractions k/16 put alpha, beta and alpha * beta on the 1/256 grid: the
    texture form is then the plain bilinear value."""
    rng = np.random.default_rng(3)
    img = rng.integers(0, 256, (6, 7)).astype(np.float64)
    for _ in range(300):
        x = rng.integers(0, 5) + rng.integers(0, 16) / 16.0
        y = rng.integers(0, 4) + rng.integers(0, 16) / 16.0
        assert oracle_mod.bilinear_texture(img, x, y) == pytest.approx(_textbook(img, x, y), abs=1e-12)
        assert oracle_mod.bilinear_texture(img, x, y) == pytest.approx(oracle_mod.bilinear(img, x, y), abs=1e-12)


def test_texture_bilinear_rounding_rules(oracle_mod):
    row = np.array([[0.0, 256.0], [0.0, 256.0]])
    # fractions rounded half up to 1/256
    assert oracle_mod.bilinear_texture(row, 0.5 / 256, 0.0) == 1.0
    assert oracle_mod.bilinear_texture(row, 0.49 / 256, 0.0) == 0.0
    assert oracle_mod.bilinear_texture(row, 1.49 / 256, 0.0) == 1.0
    assert oracle_mod.bilinear_texture(row, 255.5 / 256, 0.0) == 256.0
    # the cross term is alpha * beta rounded to 1/256: 24/256 * 40/256 = 3.75/256 -> 4/256
    corner = np.array([[0.0, 0.0], [0.0, 256.0]])
    assert oracle_mod.bilinear_texture(corner, 24 / 256, 40 / 256) == 4.0
    assert _textbook(corner, 24 / 256, 40 / 256) == pytest.approx(3.75)
    # 8/256 * 48/256 = 1.5/256: a tie, rounded up
    assert oracle_mod.bilinear_texture(corner, 8 / 256, 48 / 256) == 2.0
    # affine images have no cross term: the value is exact at the rounded position
    yy, xx = np.mgrid[0:4, 0:5]
    ramp = 7.0 + 2.0 * xx + 5.0 * yy
    assert oracle_mod.bilinear_texture(ramp, 1 + 10.3 / 256, 2 + 99.7 / 256) == pytest.approx(
        7.0 + 2.0 * (1 + 10 / 256) + 5.0 * (2 + 100 / 256), abs=1e-12)


def test_texture_bilinear_error_bound_and_clamping(oracle_mod):
    rng = np.random.default_rng(4)
    img = rng.integers(0, 256, (8, 9)).astype(np.float64)
    worst = 0.0
    for _ in range(2000):
        x, y = rng.uniform(0, 8), rng.uniform(0, 7)
        x0, y0 = int(np.floor(x)), int(np.floor(y))
        if x0 >= 8 or y0 >= 7:
            continue
        a, b, c, d = img[y0, x0], img[y0, x0 + 1], img[y0 + 1, x0], img[y0 + 1, x0 + 1]
        bound = (abs(b - a) + abs(c - a) + 3 * abs(d - b - c + a)) / 512
        err = abs(oracle_mod.bilinear_texture(img, x, y) - _textbook(img, x, y))
        assert err <= bound + 1e-12
        worst = max(worst, err / max(bound, 1e-12))
    assert worst > 0.3          # the rounding is visible, not a no-op
    # outside the image the edge texels repeat (clamp-to-edge addressing)
    for x, y in ((1.5, 10.0), (-0.3, 2.75), (12.0, 3.25)):
        assert oracle_mod.bilinear_texture(img, x, y) == oracle_mod.bilinear_texture(
            img, min(max(x, 0.0), 8.0), min(max(y, 0.0), 7.0))
    assert oracle_mod.bilinear_texture(img, -3.0, -7.0) == img[0, 0]
    assert oracle_mod.bilinear_texture(img, 9.0, 1.0) == img[1, 8]


# --------------------------------------------------------------------------
# geometry: plane-induced homography
# --------------------------------------------------------------------------
def _random_rig(rng, n=3, W=64, H=48):
    from paper_1805_07920_gb300.synth import Camera, intrinsics, look_at
    cams = []
    for i in range(n):
        c = rng.uniform(-1, 1, 3) + np.array([0, 0, -5.0])
        R, t = look_at(c, rng.uniform(-0.3, 0.3, 3))
        K = intrinsics(W, H, rng.uniform(50, 90))
        K[0, 1] = rng.uniform(-0.5, 0.5)   # a little skew
        cams.append(Camera(K, R, t, W, H))
    return cams


def test_homography_transfers_points_on_the_plane(oracle_mod):
    rng = np.random.default_rng(1)
    cams = _random_rig(rng)
    imgs = [rng.uniform(0, 255, (c.height, c.width)) for c in cams]
    o = oracle_mod.Oracle(cams, imgs, 0, [1, 2])
    Kr, Rr, tr = cams[0].K, cams[0].R, cams[0].t
    for _ in range(50):
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        if n[2] > 0:
            n = -n
        d = rng.uniform(2, 8)
        for j, v in enumerate([1, 2]):
            H = o.homography(j, n, d)
            x = np.array([rng.uniform(0, 63), rng.uniform(0, 47), 1.0])
            ray = np.linalg.solve(Kr, x)
            X = ray * (-d / (n @ ray))                # on n.X + d = 0, camera frame
            Xw = Rr.T @ (X - tr)                      # world
            p = cams[v].K @ (cams[v].R @ Xw + cams[v].t)
            q = H @ x
            np.testing.assert_allclose(q[:2] / q[2], p[:2] / p[2], rtol=0, atol=1e-8)


# --------------------------------------------------------------------------
# matching cost, Eq. (8)
# --------------------------------------------------------------------------
def _plane_at(o, x, y, n, D):
    return np.array([n[0], n[1], n[2], D], np.float64)


def test_cost_zero_for_identical_patches(oracle_mod, tiny_scene):
    sc = tiny_scene
    cams = list(sc.cams) + [sc.cams[sc.ref]]
    imgs = list(sc.images) + [sc.images[sc.ref]]
    o = oracle_mod.Oracle(cams, imgs, sc.ref, [len(cams) - 1])
    rng = np.random.default_rng(2)
    Kinv = np.linalg.inv(sc.cams[sc.ref].K)
    for _ in range(100):
        x, y = int(rng.integers(6, sc.width - 6)), int(rng.integers(6, sc.height - 6))
        ray = Kinv @ [x, y, 1.0]
        n = -ray / np.linalg.norm(ray) + 0.4 * rng.normal(size=3)
        n /= np.linalg.norm(n)
        if n @ ray >= 0:
            n = -n
        assert o.cost(x, y, _plane_at(o, x, y, n, rng.uniform(2, 8)), 0) == pytest.approx(0.0, abs=1e-12)


def test_cost_affine_invariance(oracle_mod, tiny_scene):
    sc = tiny_scene
    j0 = sc.src[0]
    base = np.asarray(sc.images[j0], np.float64)
    rng = np.random.default_rng(3)
    pts = [(int(rng.integers(6, sc.width - 6)), int(rng.integers(6, sc.height - 6))) for _ in range(60)]
    gt = sc.gt_depth[sc.ref]
    gn = sc.gt_normal[sc.ref]
    planes = []
    for (x, y) in pts:
        D = gt[y, x] * rng.uniform(0.9, 1.1)
        planes.append(np.array([*gn[y, x], D]))

    def costs(img):
        imgs = list(map(np.asarray, sc.images))
        imgs[j0] = img
        o = oracle_mod.Oracle(sc.cams, imgs, sc.ref, [j0])
        return np.array([o.cost(x, y, pl, 0) for (x, y), pl in zip(pts, planes)])

    m0 = costs(base)
    assert np.all((m0 > 0) & (m0 < 2))
    np.testing.assert_allclose(costs(1.7 * base + 23.0), m0, atol=1e-9)
    np.testing.assert_allclose(costs(0.4 * base - 5.0), m0, atol=1e-9)
    # a negative gain flips the correlation: m -> 2 - m
    np.testing.assert_allclose(costs(-0.8 * base + 200.0), 2.0 - m0, atol=1e-9)


def _rectified_pair(rng, W=48, H=40, f=60.0, B=0.5):
    from paper_1805_07920_gb300.synth import Camera, intrinsics
    K = intrinsics(W, H, f)
    I = np.eye(3)
    ref = Camera(K, I, np.zeros(3), W, H)
    src = Camera(K, I, np.array([-B, 0.0, 0.0]), W, H)   # centre at (B, 0, 0)
    imgs = [rng.integers(0, 256, (H, W)).astype(np.float64), rng.integers(0, 256, (H, W)).astype(np.float64)]
    return [ref, src], imgs, f, B


def _bilateral_weights(r, Ic, offs, sI, sx):
    d = np.sqrt((offs ** 2).sum(1))
    return np.exp(-np.abs(r - Ic) / (2 * sI * sI) - d / (2 * sx * sx))


@pytest.mark.parametrize("shift,sI,sx", [(2, 3.0, 30.0), (5, 3.0, 30.0), (3, 10.0, 2.0), (4, 1e6, 1e6)])
def test_cost_rectified_pair_integer_shift(oracle_mod, shift, sI, sx):
    """Fronto-parallel plane z = D on a rectified pair warps by a pure shift of
    f B / D pixels; with an integer shift the cost is the weighted correlation
    of integer-indexed windows, computed here with numpy's weighted cov."""
    rng = np.random.default_rng(10 + shift)
    cams, imgs, f, B = _rectified_pair(rng)
    D = f * B / shift
    p = oracle_mod.default_params(sigma_I=sI, sigma_x=sx)
    o = oracle_mod.Oracle(cams, imgs, 0, [1], params=p)
    offs = np.array([(du, dv) for dv in range(-5, 6, 2) for du in range(-5, 6, 2)], np.float64)
    for (x, y) in [(20, 20), (30, 12), (25, 30), (14, 9)]:
        m = o.cost(x, y, np.array([0.0, 0.0, -1.0, D]), 0)
        r = np.array([imgs[0][y + int(dv), x + int(du)] for du, dv in offs])
        s = np.array([imgs[1][y + int(dv), x + int(du) - shift] for du, dv in offs])
        w = _bilateral_weights(r, imgs[0][y, x], offs, sI, sx)
        C = np.cov(np.stack([r, s]), aweights=w)
        expect = 1 - C[0, 1] / math.sqrt(C[0, 0] * C[1, 1])
        assert m == pytest.approx(expect, abs=1e-10)
        if sI > 1e5:   # uniform weights: the textbook Pearson correlation
            assert m == pytest.approx(1 - np.corrcoef(r, s)[0, 1], abs=1e-8)


def test_cost_worst_cases(oracle_mod):
    rng = np.random.default_rng(4)
    cams, imgs, f, B = _rectified_pair(rng)
    o = oracle_mod.Oracle(cams, imgs, 0, [1])
    # the plane does not face the pixel
    assert o.cost(20, 20, np.array([0.0, 0.0, 1.0, 3.0]), 0) == 2.0
    # non-positive depth
    assert o.cost(20, 20, np.array([0.0, 0.0, -1.0, -3.0]), 0) == 2.0
    # centre projects outside the source image: shift of 30 px at x = 10
    assert o.cost(10, 20, np.array([0.0, 0.0, -1.0, f * B / 30]), 0) == 2.0
    # textureless reference patch
    flat = [np.full_like(imgs[0], 77.0), imgs[1]]
    o2 = oracle_mod.Oracle(cams, flat, 0, [1])
    assert o2.cost(20, 20, np.array([0.0, 0.0, -1.0, f * B / 2]), 0) == 2.0
    # plane behind the source camera: view 1 sits 2 units ahead on the
    # optical axis, the plane is 1 unit in front of the reference
    from paper_1805_07920_gb300.synth import Camera
    ahead = Camera(cams[0].K, np.eye(3), np.array([0.0, 0.0, -2.0]), cams[0].width, cams[0].height)
    o3 = oracle_mod.Oracle([cams[0], ahead], imgs, 0, [1])
    assert o3.cost(24, 20, np.array([0.0, 0.0, -1.0, 1.0]), 0) == 2.0
    assert o3.cost(24, 20, np.array([0.0, 0.0, -1.0, 3.0]), 0) < 2.0
    # costs are always within [0, 2]
    for _ in range(200):
        nn = rng.normal(size=3)
        nn[2] = -abs(nn[2]) - 0.1
        nn /= np.linalg.norm(nn)
        c = o.cost(int(rng.integers(0, 48)), int(rng.integers(0, 40)), np.array([*nn, rng.uniform(1, 10)]), 0)
        assert 0.0 <= c <= 2.0


# --------------------------------------------------------------------------
# multi-hypothesis joint view selection, Eqs. (2)-(7)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("case", _golden("mhj_cases.json")["cases"], ids=lambda c: c["name"])
def test_mhj_hand_built_cases(oracle_mod, case):
    M = np.array(case["M_cols"], np.float64).T       # 8 x N
    w, S, v = oracle_mod.mhj(M, case.get("row_valid"), case["t"], case["S_prev"], case["v_prev"])
    assert S == case["S"]
    assert v == case["v"]
    if "weights" in case:
        np.testing.assert_allclose(w, case["weights"], rtol=0, atol=1e-15)
    if "nonzero" in case:
        assert sorted(np.nonzero(w > 0)[0].tolist()) == case["nonzero"]
    if "order" in case:
        nz = np.nonzero(w > 0)[0]
        assert nz[np.argsort(-w[nz], kind="stable")].tolist() == case["order"]


# --------------------------------------------------------------------------
# asymmetric checkerboard propagation (Sec. 3.1)
# --------------------------------------------------------------------------
def test_acp_region_geometry(oracle_mod):
    g = _golden("acp_regions.json")["regions"]
    allofs = set()
    for i, reg in enumerate(g):
        ofs = oracle_mod.acp_offsets(i)
        assert ofs == [tuple(o) for o in reg["offsets"]], reg["name"]
        assert len(ofs) == (7 if i < 4 else 11)         # Sec. 3.1: 7 near, 11 far
        for dx, dy in ofs:
            assert (abs(dx) + abs(dy)) % 2 == 1         # opposite checkerboard colour
            assert (dx, dy) not in allofs               # regions are disjoint
            allofs.add((dx, dy))
    # the four directions are rotations / mirrors of one another
    up = oracle_mod.acp_offsets(0)
    assert oracle_mod.acp_offsets(1) == [(dx, -dy) for dx, dy in up]
    assert oracle_mod.acp_offsets(2) == [(dy, dx) for dx, dy in up]
    assert oracle_mod.acp_offsets(3) == [(-dy, dx) for dx, dy in up]


def _flat_scene(oracle_mod, W=40, H=36):
    rng = np.random.default_rng(5)
    cams, imgs, f, B = _rectified_pair(rng, W=W, H=H)
    return oracle_mod.Oracle(cams, imgs, 0, [1])


def test_acp_pick_lowest_cost_and_bounds(oracle_mod):
    o = _flat_scene(oracle_mod, W=60, H=56)
    W, H = o.W, o.H
    cost = np.full((H, W), 1.5)
    x, y = 30, 28
    for gi in range(8):
        ofs = oracle_mod.acp_offsets(gi)
        k = (3 * gi + 2) % len(ofs)
        dx, dy = ofs[k]
        cost[y + dy, x + dx] = 0.1 * (gi + 1) / 10
    o.set_state(plane=np.tile([0, 0, -1.0, 5.0], (H, W, 1)), cost=cost)
    for gi in range(8):
        ofs = oracle_mod.acp_offsets(gi)
        dx, dy = ofs[(3 * gi + 2) % len(ofs)]
        assert o.acp_pick(x, y, gi) == (y + dy) * W + (x + dx)
    # equal costs: the nearest candidate wins
    o.set_state(cost=np.full((H, W), 0.5), plane=np.tile([0, 0, -1.0, 5.0], (H, W, 1)))
    for gi in range(8):
        dx, dy = oracle_mod.acp_offsets(gi)[0]
        assert o.acp_pick(x, y, gi) == (y + dy) * W + (x + dx)
    # near the border: far-up strip of row 2 has no candidate; far-left of x=3
    # has exactly one (distance 3)
    assert o.acp_pick(10, 2, 4) == -1
    assert o.acp_pick(3, 10, 6) == 10 * W + 0
    assert o.acp_row(10, 2, 4) is None


def test_acp_row_is_the_neighbours_plane(oracle_mod):
    """The propagated hypothesis at x is the neighbour's 3-D plane: the point
    at depth D_x on x's ray satisfies the neighbour's plane equation."""
    o = _flat_scene(oracle_mod)
    W, H = o.W, o.H
    rng = np.random.default_rng(6)
    plane = np.zeros((H, W, 4))
    n = rng.normal(size=(H, W, 3))
    n[..., 2] = -np.abs(n[..., 2]) - 1.0
    n /= np.linalg.norm(n, axis=2, keepdims=True)
    plane[..., :3] = n
    plane[..., 3] = rng.uniform(3, 6, (H, W))
    o.set_state(plane=plane, cost=rng.uniform(0, 2, (H, W)))
    Kinv = np.linalg.inv(np.array([[60.0, 0, 19.5], [0, 60.0, 17.5], [0, 0, 1]]))
    for (x, y) in [(20, 18), (10, 25), (30, 5)]:
        for gi in range(8):
            q = o.acp_pick(x, y, gi)
            row = o.acp_row(x, y, gi)
            if row is None:
                continue
            qx, qy = q % W, q // W
            nq, Dq = plane[qy, qx, :3], plane[qy, qx, 3]
            Xq = Dq * (Kinv @ [qx, qy, 1.0])
            Xx = row[3] * (Kinv @ [x, y, 1.0])
            np.testing.assert_allclose(row[:3], nq)
            assert nq @ (Xx - Xq) == pytest.approx(0.0, abs=1e-9)


# --------------------------------------------------------------------------
# random planes and refinement (Sec. 3.3)
# --------------------------------------------------------------------------
def test_random_planes(oracle_mod):
    o = _flat_scene(oracle_mod)
    Kinv = np.linalg.inv(np.array([[60.0, 0, 19.5], [0, 60.0, 17.5], [0, 0, 1]]))
    Ds, ns = [], []
    for y in range(o.H):
        for x in range(o.W):
            pl = o.random_plane(x, y)
            assert np.linalg.norm(pl[:3]) == pytest.approx(1.0, abs=1e-12)
            assert pl[:3] @ (Kinv @ [x, y, 1.0]) < 0
            Ds.append(pl[3])
            ns.append(pl[:3])
    Ds = np.array(Ds)
    p = oracle_mod.default_params()
    assert Ds.min() >= p.depth_min and Ds.max() < p.depth_max
    assert abs(Ds.mean() - 0.5 * (p.depth_min + p.depth_max)) < 0.2
    # the x component of a uniform unit vector is uniform in [-1, 1]
    nx = np.array(ns)[:, 0]
    assert abs(nx.mean()) < 0.06 and abs((nx ** 2).mean() - 1 / 3) < 0.03


def test_refinement_candidates(oracle_mod):
    o = _flat_scene(oracle_mod)
    Kinv = np.linalg.inv(np.array([[60.0, 0, 19.5], [0, 60.0, 17.5], [0, 0, 1]]))
    x, y = 11, 7
    ray = Kinv @ [x, y, 1.0]
    n0 = np.array([0.2, -0.1, -1.0])
    n0 /= np.linalg.norm(n0)
    pl = np.array([*n0, 4.0])
    for t in range(6):
        c = o.refine_candidates(x, y, pl, t)
        assert len(c) == (1 if t < 3 else 6)
        rho = 2.0 ** -(t + 1)
        for cand in c:
            assert np.linalg.norm(cand[:3]) == pytest.approx(1.0, abs=1e-12)
            assert cand[:3] @ ray < 0
        assert 4.0 * (1 - rho) <= c[0, 3] <= 4.0 * (1 + rho)
        # the perturbed normal stays within the angle a rho-box around n0 allows
        assert c[0, :3] @ n0 >= math.cos(math.asin(min(1.0, math.sqrt(3) * rho))) - 1e-12
        if t >= 3:
            np.testing.assert_array_equal(c[1, :3], n0)          # random depth, own normal
            assert c[2, 3] == 4.0                                # own depth, random normal
            np.testing.assert_array_equal(c[3, :3], c[2, :3])    # random depth and normal
            assert c[3, 3] == c[1, 3]
            np.testing.assert_array_equal(c[4, :3], n0)          # perturbed depth
            assert c[4, 3] == c[0, 3]
            np.testing.assert_array_equal(c[5, :3], c[0, :3])    # perturbed normal
            assert c[5, 3] == 4.0


def test_refinement_range_is_reached_on_both_sides(oracle_mod):
    """Two-sided pin of the bisection range rho_t = 2^-(t+1) of Sec. 3.3 (the
    range that halves every iteration, starting at one half): over every
    pixel of a 40 x 36 image (1440 independent draws per t) the perturbed
    depth D (1 + rho u), u uniform in (-1, 1), must fill the range on both
    sides -- its extremes beyond 0.9 rho above and below -- and never leave
    it; the perturbed normal n + rho delta (delta uniform in the unit cube)
    must turn further from n than any box of half-width rho / 2 allows
    (asin(sqrt(3) rho / 2): the ball around such a box), and never further
    than the rho box allows.  A range off by a factor of two either way
    fails one side."""
    o = _flat_scene(oracle_mod)
    n0 = np.array([0.2, -0.1, -1.0])
    n0 /= np.linalg.norm(n0)
    D0 = 4.0
    pl = np.array([*n0, D0])
    for t in range(6):
        rho = 2.0 ** -(t + 1)
        rel, ang = [], []
        for y in range(o.H):
            for x in range(o.W):
                c = o.refine_candidates(x, y, pl, t)[0]
                rel.append(c[3] / D0 - 1.0)
                ang.append(math.acos(min(1.0, abs(float(c[:3] @ n0)))))
        rel, ang = np.array(rel), np.array(ang)
        assert rel.max() > 0.9 * rho and rel.min() < -0.9 * rho, (t, rel.min(), rel.max())
        assert np.abs(rel).max() <= rho * (1 + 1e-12), t
        assert ang.max() > math.asin(min(1.0, math.sqrt(3) * rho / 2)), (t, ang.max())
        assert ang.max() <= math.asin(min(1.0, math.sqrt(3) * rho)) + 1e-12, (t, ang.max())


# --------------------------------------------------------------------------
# the checkerboard phase as a whole
# --------------------------------------------------------------------------
def test_phase_is_order_independent_and_colour_local(oracle_mod, tiny_scene):
    sc = tiny_scene
    a = oracle_mod.Oracle.from_scene(sc, seed=11)
    a.init_random()
    b = oracle_mod.Oracle.from_scene(sc, seed=11)
    b.init_random()
    before = a.get_state()
    a.step_phase(0)
    ys, xs = np.nonzero(((np.add.outer(np.arange(sc.height), np.arange(sc.width))) & 1) == 0)
    order = np.random.default_rng(7).permutation(len(xs))
    b.update_pixels(xs[order], ys[order])
    sa, sb = a.get_state(), b.get_state()
    for k in ("plane", "cost", "sel", "vprev", "choice"):
        np.testing.assert_array_equal(sa[k], sb[k], err_msg=k)
    red = ((np.add.outer(np.arange(sc.height), np.arange(sc.width))) & 1) == 1
    np.testing.assert_array_equal(sa["plane"][red], before["plane"][red])
    np.testing.assert_array_equal(sa["cost"][red], before["cost"][red])


def test_update_pixel_matches_phase(oracle_mod, tiny_scene):
    sc = tiny_scene
    o = oracle_mod.Oracle.from_scene(sc, seed=12)
    o.init_random()
    o.iterate(1)
    pre = [(x, y, o.update_pixel(x, y)) for (x, y) in [(5, 7), (80, 60), (159, 119), (0, 0), (33, 91)]
           if (x + y) % 2 == 0]
    o.step_phase(0)
    st = o.get_state()
    for x, y, u in pre:
        np.testing.assert_array_equal(st["plane"][y, x], u["plane"])
        assert st["cost"][y, x] == u["cost"]
        assert st["choice"][y, x] == u["choice"]


def test_initial_cost_is_mean_of_k_best_views(oracle_mod, medium_scene):
    sc = medium_scene
    o = oracle_mod.Oracle.from_scene(sc, seed=13)
    o.init_random()
    st = o.get_state()
    for (x, y) in [(100, 100), (320, 240), (600, 50)]:
        pl = st["plane"][y, x]
        m = sorted(o.cost(x, y, pl, j) for j in range(len(sc.src)))
        assert st["cost"][y, x] == pytest.approx(np.mean(m[:4]), abs=1e-15)
        assert st["sel"][y, x] == 0 and st["vprev"][y, x] == -1


def _textured_interior(sc, margin=6):
    img = sc.images[sc.ref].astype(np.float64)
    gy, gx = np.gradient(img)
    g = np.hypot(gx, gy)
    m = np.zeros(img.shape, bool)
    m[margin:-margin, margin:-margin] = True
    return m & (g > 2.0)


def test_brute_force_recovers_ground_truth(oracle_mod, tiny_scene):
    """Exhaustive search over depths around the truth with the true normal:
    the oracle's multi-view cost has its minimum at the ground truth."""
    sc = tiny_scene
    o = oracle_mod.Oracle.from_scene(sc)
    gt, gn = sc.gt_depth[sc.ref], sc.gt_normal[sc.ref]
    mask = _textured_interior(sc, margin=12)
    ys, xs = np.nonzero(mask)
    sel = np.random.default_rng(8).choice(len(xs), 150, replace=False)
    steps = np.linspace(-0.15, 0.15, 31)
    hits = 0
    for i in sel:
        x, y = int(xs[i]), int(ys[i])
        costs = [np.mean([o.cost(x, y, np.array([*gn[y, x], gt[y, x] * (1 + s)]), j) for j in range(2)])
                 for s in steps]
        hits += abs(steps[int(np.argmin(costs))]) <= 0.01 + 1e-12
    assert hits / len(sel) >= 0.9


def test_patchmatch_converges_on_tiny_scene(oracle_mod, tiny_scene):
    """Three iterations of the full update (ACP + MHJ + refinement) bring most
    textured pixels within 1 % of the ground-truth depth."""
    sc = tiny_scene
    o = oracle_mod.Oracle.from_scene(sc, seed=7)
    o.init_random()
    gt = sc.gt_depth[sc.ref]
    mask = _textured_interior(sc)
    fr = []
    for _ in range(3):
        o.iterate(1)
        D = o.depth_map()
        fr.append(np.mean(np.abs(D[mask] - gt[mask]) / gt[mask] < 0.01))
    assert fr[-1] >= 0.85
    assert fr[0] < fr[-1]


def test_own_plane_wins_exact_ties(oracle_mod, tiny_scene):
    """Eq. (7) keeps the minimal m_final; when a propagated hypothesis is the
    very same plane as the pixel's own, the own plane is kept."""
    sc = tiny_scene
    o = oracle_mod.Oracle.from_scene(sc, seed=14)
    H, W = sc.height, sc.width
    plane = np.tile([0.0, 0.0, -1.0, 5.0], (H, W, 1))   # one fronto-parallel plane
    o.set_state(plane=plane, cost=np.random.default_rng(9).uniform(0, 1, (H, W)), t=0)
    for (x, y) in [(20, 20), (50, 60), (101, 33), (140, 100)]:
        u = o.update_pixel(x, y)
        assert u["choice"] >= 8


def test_score_plane_is_eq7_from_pinned_parts(oracle_mod, tiny_scene):
    """score_plane (what classifies near-ties in the parity tests) is Eq. (7) for one plane:
    rebuilt here from the separately pinned parts -- the 8 ACP rows, the cost
    of Eq. (8) per view, the view weights of Eqs. (2)-(6) -- as
    sum_j w_j m(plane, j) / sum_j w_j; invalid rows count as cost 2 and stay
    out of the view selection."""
    sc = tiny_scene
    o = oracle_mod.Oracle.from_scene(sc, seed=15)
    o.init_random()
    o.iterate(1)
    st = o.get_state()
    N = len(sc.src)
    rng = np.random.default_rng(15)
    for _ in range(12):
        x, y = int(rng.integers(0, sc.width)), int(rng.integers(0, sc.height))
        M = np.full((8, N), 2.0)
        valid = np.zeros(8, np.int32)
        for g in range(8):
            row = o.acp_row(x, y, g)
            if row is None:
                continue
            valid[g] = 1
            M[g] = [o.cost(x, y, row, j) for j in range(N)]
        w, _, _ = oracle_mod.mhj(M, row_valid=valid, t=st["t"], S_prev=int(st["sel"][y, x]),
                                 v_prev=int(st["vprev"][y, x]), params=o.params)
        assert w.sum() > 0
        for plane in (st["plane"][y, x], o.random_plane(x, y)):
            expect = sum(w[j] * o.cost(x, y, plane, j) for j in range(N) if w[j] > 0) / w.sum()
            assert o.score_plane(x, y, plane) == pytest.approx(expect, rel=1e-12, abs=1e-15)


def test_symmetric_propagation_geometry(oracle_mod, tiny_scene):
    """The ablation without ACP: eight fixed candidates, the axis neighbours at
    distances 1 and 5 -- symmetric, opposite colour, no choice by cost."""
    offs = [oracle_mod.scp_offsets(g)[0] for g in range(8)]
    assert set(offs) == {(0, -1), (0, 1), (-1, 0), (1, 0), (0, -5), (0, 5), (-5, 0), (5, 0)}
    assert all((abs(dx) + abs(dy)) % 2 == 1 for dx, dy in offs)
    assert all((-dx, -dy) in offs for dx, dy in offs)
    sc = tiny_scene
    p = oracle_mod.default_params(depth_min=sc.depth_min, depth_max=sc.depth_max, seed=3,
                                  flags=oracle_mod.ORC_FLAG_SYMMETRIC)
    o = oracle_mod.Oracle.from_scene(sc, p)
    H, W = sc.height, sc.width
    o.set_state(plane=np.tile([0.0, 0.0, -1.0, 5.0], (H, W, 1)),
                cost=np.random.default_rng(4).uniform(0, 2, (H, W)), t=0)
    for (x, y) in [(10, 10), (2, 60), (157, 3), (80, 118)]:
        for g, (dx, dy) in enumerate(offs):
            qx, qy = x + dx, y + dy
            expect = qy * W + qx if 0 <= qx < W and 0 <= qy < H else -1
            assert o.acp_pick(x, y, g) == expect


@pytest.mark.parametrize("flags", ["heuristic", "both"])
def test_heuristic_view_selection(oracle_mod, tiny_scene, flags):
    """The ablation without MHJ: every hypothesis scored by the mean of its own
    k = 4 smallest per-view costs; the update keeps the smallest (own plane on
    ties), refinement included, and records no view selection."""
    sc = tiny_scene
    f = oracle_mod.ORC_FLAG_HEURISTIC | (oracle_mod.ORC_FLAG_SYMMETRIC if flags == "both" else 0)
    p = oracle_mod.default_params(depth_min=sc.depth_min, depth_max=sc.depth_max, seed=5, flags=f)
    o = oracle_mod.Oracle.from_scene(sc, p)
    o.init_random()
    o.iterate(1)
    st = o.get_state()
    N = len(sc.src)
    kb = lambda pl: float(np.mean(np.sort([o.cost(x, y, pl, j) for j in range(N)])[:min(4, N)]))
    rng = np.random.default_rng(6)
    for _ in range(10):
        x, y = int(rng.integers(0, sc.width)), int(rng.integers(0, sc.height))
        u = o.update_pixel(x, y)
        assert u["sel"] == 0 and u["v"] == -1
        assert u["cost"] == pytest.approx(kb(u["plane"]), rel=1e-12, abs=1e-15)
        own = kb(st["plane"][y, x])
        assert u["cost"] <= own + 1e-15
        for g in range(8):
            row = o.acp_row(x, y, g)
            if row is not None:
                assert u["cost"] <= kb(row) + 1e-15
        assert o.score_plane(x, y, u["plane"]) == pytest.approx(u["cost"], rel=1e-12, abs=1e-15)


def test_threaded_oracle_gives_identical_results(oracle_mod, tiny_scene):
    """The thread count of the oracle's pixel loops (used only to time it on
    all host cores) does not change any result: the pixels of one colour phase
    read only the other colour."""
    out = []
    try:
        for th in (1, 4):
            oracle_mod.set_threads(th)
            o = oracle_mod.Oracle.from_scene(tiny_scene, seed=12)
            o.init_random()
            o.iterate(1)
            out.append(o.get_state())
    finally:
        oracle_mod.set_threads(1)
    for k in ("plane", "cost", "sel", "vprev", "choice"):
        np.testing.assert_array_equal(out[0][k], out[1][k], err_msg=k)
