"""FP64 CPU oracle of the source-view preselection (TEST INFRASTRUCTURE ONLY).

Sec. 2 and Sec. 4 take, for every reference image, N source images chosen by
viewing angle and baseline, leaving the rule open.  The reading written out
here (and in the library's ``amh_select_sources``): the point P at z-depth d
on the reference's optical axis stands for the scene; a view qualifies when P
lies in front of it and projects inside its image, and the triangulation
angle at P between the rays to the two camera centres lies in
[min_angle, max_angle] degrees -- a lower bound for baseline, an upper one
for similar appearance.  The qualifying views, ordered by increasing angle
(ties by index), are the sources; at most n_src of them are kept.
"""
from __future__ import annotations

import numpy as np


def _krt(c):
    K = np.asarray(c.K, np.float64).reshape(3, 3)
    R = np.asarray(c.R, np.float64).reshape(3, 3)
    t = np.asarray(c.t, np.float64).reshape(3)
    return K, R, t


def triangulation_angles(cams, ref, depth):
    """Per view: (angle in degrees or None when P is not seen, projection
    (u, v) or None).  The reference's own entry is None."""
    K, R, t = _krt(cams[ref])
    C = -R.T @ t
    P = R.T @ (np.array([0.0, 0.0, depth]) - t)          # camera point (0, 0, d) in the world
    out = []
    for v, c in enumerate(cams):
        if v == ref:
            out.append((None, None))
            continue
        Kv, Rv, tv = _krt(c)
        Xc = Rv @ P + tv
        if not Xc[2] > 0:
            out.append((None, None))
            continue
        u, w = (Kv @ Xc)[:2] / Xc[2]
        if not (0 <= u <= c.width - 1 and 0 <= w <= c.height - 1):
            out.append((None, (u, w)))
            continue
        a, b = C - P, -Rv.T @ tv - P
        cosang = np.clip(a @ b / (np.linalg.norm(a) * np.linalg.norm(b)), -1.0, 1.0)
        out.append((float(np.degrees(np.arccos(cosang))), (u, w)))
    return out


def select_sources(cams, ref, depth, n_src=10, min_angle_deg=1.0, max_angle_deg=60.0):
    angles = triangulation_angles(cams, ref, depth)
    cand = [(a, v) for v, (a, _) in enumerate(angles) if a is not None and min_angle_deg <= a <= max_angle_deg]
    cand.sort()
    return [v for _, v in cand[:n_src]]
