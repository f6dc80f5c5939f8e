"""Helpers shared by the GPU parity tests: identical-state set-up for the
oracle and the CUDA library, and the comparison rules.

Tolerances (floating point; the oracle is FP64, the kernels FP32):
  * cost: |m_gpu - m_oracle| <= 1e-4 per pixel;
  * same hypothesis: both sides keep the same plane -- depth within 1e-4
    relative and normals within 1e-6 of 1 - n.n' -- or the same winning row;
  * both on >= 99.9 % of the updated pixels that are not near-ties: a pixel
    where the two sides keep different planes whose unified costs, both
    scored by the oracle under that pixel's weights, differ by <= 2e-4 is a
    tie (several answers are correct there);
  * final depth after whole runs: within 1 % relative on >= 99 % of valid
    pixels (ground truth hit, >= 5 px from the border).
"""
import numpy as np

COST_TOL = 1e-4
TIE_TOL = 2e-4
FRACTION = 0.999
# The texture-filter form (AMH_FLAG_TEXTURE_BILINEAR) rounds the bilinear
# fractions to 1/256, so its cost is a step function of the sample positions
# (steps every 1/256 px).  The kernel's FP32 positions differ from the
# oracle's FP64 ones by about 1e-4 px (2-3 % of a step), so a sample near a
# step rounds the other way on the two sides and moves the cost of a few
# pairs past 1e-4 without any arithmetic error: that form is held to 99.8 %.
FRACTION_TEXTURE_FILTER = 0.998


def color_mask(H, W, color):
    return ((np.add.outer(np.arange(H), np.arange(W))) & 1) == color


def fp32_state(st):
    """Oracle state rounded to FP32 (the GPU's storage), back in FP64."""
    return dict(plane=st["plane"].astype(np.float32).astype(np.float64),
                cost=st["cost"].astype(np.float32).astype(np.float64),
                sel=st["sel"].astype(np.uint32), vprev=st["vprev"].astype(np.int32), t=st["t"])


def load_identical(orc, ctx, st):
    """Put the same (FP32-representable) state into the oracle and the GPU."""
    s = fp32_state(st)
    orc.set_state(plane=s["plane"], cost=s["cost"], sel=s["sel"], vprev=s["vprev"], t=s["t"])
    vb = np.where(s["vprev"] < 0, 255, s["vprev"]).astype(np.uint8)
    ctx.set_state(plane=s["plane"].astype(np.float32), cost=s["cost"].astype(np.float32),
                  sel=s["sel"], vbest=vb, t=s["t"])


def same_plane(pa, pb, rel_d=1e-4, ang=1e-6):
    da, db = pa[..., 3], pb[..., 3]
    dd = np.abs(da - db) / np.maximum(np.abs(da), 1e-12)
    na, nb = pa[..., :3], pb[..., :3]
    dot = (na * nb).sum(-1) / np.maximum(np.linalg.norm(na, axis=-1) * np.linalg.norm(nb, axis=-1), 1e-30)
    return (dd <= rel_d) & (1.0 - dot <= ang)


def compare_phase(o_st, g_st, mask):
    """Per-pixel agreement of one updated colour phase."""
    vg = g_st["vbest"].astype(np.int32)
    vg = np.where(vg == 255, -1, vg)
    same_h = same_plane(o_st["plane"], g_st["plane"].astype(np.float64)) | (o_st["choice"] == g_st["choice"])
    dcost = np.abs(o_st["cost"] - g_st["cost"].astype(np.float64))
    ok = same_h & (dcost <= COST_TOL)
    return dict(
        frac_ok=float(ok[mask].mean()),
        frac_same_hyp=float(same_h[mask].mean()),
        frac_cost=float((dcost[mask] <= COST_TOL).mean()),
        frac_sel=float((o_st["sel"] == g_st["sel"])[mask].mean()),
        frac_v=float((o_st["vprev"] == vg)[mask].mean()),
        max_dcost_same=float(dcost[mask & same_h].max()) if (mask & same_h).any() else 0.0,
        n=int(mask.sum()),
        bad=np.argwhere(mask & ~ok)[:10].tolist(),
    )


def valid_pixels(scene, margin=5):
    gt = scene.gt_depth[scene.ref]
    m = gt > 0
    m[:margin] = m[-margin:] = False
    m[:, :margin] = m[:, -margin:] = False
    return m


def phase_check(orc, ctx, st, color):
    """Identical state into both, one phase on each, per-pixel comparison with
    near-ties decided by the oracle.  Returns the report of compare_phase plus
    'ties' and 'frac_ok_nontie'."""
    load_identical(orc, ctx, st)
    orc.step_phase(color)
    ctx.step_phase(color)
    ctx.synchronize()
    o_st, g_st = orc.get_state(), ctx.get_state()
    mask = color_mask(ctx.H, ctx.W, color)
    r = compare_phase(o_st, g_st, mask)
    # classify the disagreements against the pre-phase state
    s = fp32_state(st)
    orc.set_state(plane=s["plane"], cost=s["cost"], sel=s["sel"], vprev=s["vprev"], t=s["t"])
    dcost = np.abs(o_st["cost"] - g_st["cost"].astype(np.float64))
    same_h = same_plane(o_st["plane"], g_st["plane"].astype(np.float64)) | (o_st["choice"] == g_st["choice"])
    bad = np.argwhere(mask & ~(same_h & (dcost <= COST_TOL)))
    ties = 0
    for (y, x) in bad:
        sg = orc.score_plane(int(x), int(y), g_st["plane"][y, x].astype(np.float64))
        if abs(sg - o_st["cost"][y, x]) <= TIE_TOL and dcost[y, x] <= TIE_TOL:
            ties += 1
    n = int(mask.sum())
    r["ties"] = ties
    r["n_bad"] = int(len(bad))
    r["frac_ok_nontie"] = 1.0 if n == ties else (n - len(bad)) / (n - ties)
    return r


def oracle_state_from_gpu(g_st):
    """A GPU state (FP32 planes and costs, vbest 255 = none) in the oracle's
    form (FP64, vprev -1 = none)."""
    vb = g_st["vbest"].astype(np.int32)
    return dict(plane=g_st["plane"].astype(np.float64), cost=g_st["cost"].astype(np.float64),
                sel=g_st["sel"].astype(np.uint32), vprev=np.where(vb == 255, -1, vb).astype(np.int32),
                t=g_st["t"])


def phase_check_states(orc, pre, post, color):
    """One phase the GPU has already run (its state before, `pre`, and after,
    `post`): the oracle runs the same phase from `pre` and the two are
    compared as in phase_check, near-ties decided by the oracle."""
    s = oracle_state_from_gpu(pre)
    orc.set_state(plane=s["plane"], cost=s["cost"], sel=s["sel"], vprev=s["vprev"], t=s["t"])
    orc.step_phase(color)
    o_st = orc.get_state()
    H, W = pre["cost"].shape
    mask = color_mask(H, W, color)
    r = compare_phase(o_st, post, mask)
    orc.set_state(plane=s["plane"], cost=s["cost"], sel=s["sel"], vprev=s["vprev"], t=s["t"])
    dcost = np.abs(o_st["cost"] - post["cost"].astype(np.float64))
    same_h = same_plane(o_st["plane"], post["plane"].astype(np.float64)) | (o_st["choice"] == post["choice"])
    bad = np.argwhere(mask & ~(same_h & (dcost <= COST_TOL)))
    ties = 0
    for (y, x) in bad:
        sg = orc.score_plane(int(x), int(y), post["plane"][y, x].astype(np.float64))
        if abs(sg - o_st["cost"][y, x]) <= TIE_TOL and dcost[y, x] <= TIE_TOL:
            ties += 1
    n = int(mask.sum())
    r["ties"] = ties
    r["n_bad"] = int(len(bad))
    r["frac_ok_nontie"] = 1.0 if n == ties else (n - len(bad)) / (n - ties)
    return r
