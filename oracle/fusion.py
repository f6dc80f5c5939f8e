"""FP64 CPU oracle of the depth-map post-processing (TEST INFRASTRUCTURE ONLY).

Sec. 3.3 ends the depth-map generation with a 4x4 median filter; Sec. 3.3's
last paragraph fuses the depth maps of all views with the consistency check
of Gipuma (its reference [9]) under the thresholds f_eps = 0.3 (disparity
difference), f_ang = 30 degrees (normal difference) and f_con = 2 (number of
consistent source images).  The paper leaves the details to [9]; the readings
written out here (and in the library) are:

* median4: the window is the 4 x 4 block of offsets -2..+1 in x and y around
  the pixel, clamped at the borders; the median of the 16 values is the mean
  of the 8th and 9th smallest.
* fuse: pixel p of view i with depth D > 0 back-projects to the world point X
  (normal n, in world coordinates).  Another view j is consistent when X lies
  in front of it, projects to a pixel q (nearest, ties rounded up) inside it
  with depth D_j(q) > 0, the disparity difference f_j * |C_i - C_j| *
  |1 / z_j(X) - 1 / D_j(q)| is at most f_eps (f_j the focal length of view j
  in pixels, C the camera centres, z_j(X) the depth of X in view j) and the
  angle between n and view j's normal at q is at most f_ang.  With at least
  f_con consistent views, the fused point is the mean of X and the consistent
  views' back-projected points X_j(q), its normal the normalised sum of the
  normals; otherwise p yields no point.
"""
from __future__ import annotations

import numpy as np


def median4(depth):
    """4 x 4 median of a depth map (offsets -2..+1, clamped borders)."""
    d = np.asarray(depth, np.float64)
    H, W = d.shape
    ys, xs = np.arange(H), np.arange(W)
    stack = []
    for dy in (-2, -1, 0, 1):
        for dx in (-2, -1, 0, 1):
            stack.append(d[np.clip(ys + dy, 0, H - 1)][:, np.clip(xs + dx, 0, W - 1)])
    s = np.sort(np.stack(stack), axis=0)
    return 0.5 * (s[7] + s[8])


def _cam(c):
    K = np.asarray(c.K, np.float64).reshape(3, 3)
    R = np.asarray(c.R, np.float64).reshape(3, 3)
    t = np.asarray(c.t, np.float64).reshape(3)
    return K, R, t, -R.T @ t


def fuse(cams, depths, normals, f_eps=0.3, f_ang_deg=30.0, f_con=2, near=1e-3):
    """Returns (points (V, H, W, 6) world x y z nx ny nz, valid (V, H, W),
    count (V, H, W) consistent views, ambiguous (V, H, W): some projection
    within `near` px of a rounding boundary or some test within `near`
    (relative) of its threshold -- where an FP32 implementation may decide
    otherwise)."""
    V = len(cams)
    P = [_cam(c) for c in cams]
    cos_ang = np.cos(np.deg2rad(f_ang_deg))
    out_pts, out_valid, out_cnt, out_amb = [], [], [], []
    for i in range(V):
        K, R, t, C = P[i]
        D = np.asarray(depths[i], np.float64)
        Nc = np.asarray(normals[i], np.float64)
        H, W = D.shape
        ys, xs = np.mgrid[0:H, 0:W].astype(np.float64)
        rays = np.stack([xs, ys, np.ones_like(xs)], -1) @ np.linalg.inv(K).T
        X = (D[..., None] * rays - t) @ R                        # R^T (X_cam - t)
        n = Nc @ R                                              # R^T n_cam
        has = D > 0
        sumX = X.copy()
        sumN = n.copy()
        cnt = np.zeros((H, W), np.int64)
        amb = np.zeros((H, W), bool)
        for j in range(V):
            if j == i:
                continue
            Kj, Rj, tj, Cj = P[j]
            Dj_map = np.asarray(depths[j], np.float64)
            Nj_map = np.asarray(normals[j], np.float64)
            Hj, Wj = Dj_map.shape
            Xc = X @ Rj.T + tj
            z = Xc[..., 2]
            front = has & (z > 0)
            with np.errstate(divide="ignore", invalid="ignore"):
                uv = (Xc @ Kj.T)[..., :2] / z[..., None]
            u, v = uv[..., 0], uv[..., 1]
            ui = np.floor(u + 0.5)
            vi = np.floor(v + 0.5)
            inside = front & (ui >= 0) & (ui < Wj) & (vi >= 0) & (vi < Hj)
            uic = np.where(inside, ui, 0).astype(np.int64)
            vic = np.where(inside, vi, 0).astype(np.int64)
            Dj = np.where(inside, Dj_map[vic, uic], 0.0)
            ok = inside & (Dj > 0)
            bij = np.linalg.norm(C - Cj)
            with np.errstate(divide="ignore", invalid="ignore"):
                disp = Kj[0, 0] * bij * np.abs(1.0 / z - 1.0 / np.where(ok, Dj, 1.0))
            nj = Nj_map[vic, uic] @ Rj
            dot = (n * nj).sum(-1) / np.maximum(np.linalg.norm(n, axis=-1) * np.linalg.norm(nj, axis=-1), 1e-300)
            cons = ok & (disp <= f_eps) & (dot >= cos_ang)
            # decisions an FP32 computation may take the other way
            fu, fv = u + 0.5 - ui, v + 0.5 - vi
            amb |= front & ((np.minimum(fu, 1 - fu) < near) | (np.minimum(fv, 1 - fv) < near))
            amb |= ok & ((np.abs(disp - f_eps) < near * f_eps) | (np.abs(dot - cos_ang) < near))
            rays_j = np.stack([uic, vic, np.ones_like(uic)], -1).astype(np.float64) @ np.linalg.inv(Kj).T
            Xj = (Dj[..., None] * rays_j - tj) @ Rj
            sumX += np.where(cons[..., None], Xj, 0.0)
            sumN += np.where(cons[..., None], nj, 0.0)
            cnt += cons
        valid = has & (cnt >= f_con)
        pts = np.zeros((H, W, 6))
        pts[..., :3] = sumX / (1 + cnt)[..., None]
        nn = np.linalg.norm(sumN, axis=-1, keepdims=True)
        pts[..., 3:] = sumN / np.maximum(nn, 1e-300)
        pts[~valid] = 0.0
        out_pts.append(pts)
        out_valid.append(valid)
        out_cnt.append(cnt)
        out_amb.append(amb)
    return out_pts, out_valid, out_cnt, out_amb
