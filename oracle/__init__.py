"""Python access to the FP64 CPU oracle (``amh_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``.  The product library never imports,
links or calls it, and it shares no code with the CUDA path.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

ORACLE_DIR = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(ORACLE_DIR, "_lib", "liborc.so")
ORC_MAX_SRC = 32
NREGION = 8
ORC_FLAG_SQUARED = 1        # squared differences in the bilateral weight
ORC_FLAG_SYMMETRIC = 4      # ablation: symmetric checkerboard propagation
ORC_FLAG_HEURISTIC = 8      # ablation: heuristic (per-hypothesis k-best) view selection
ORC_FLAG_TEXTURE_BILINEAR = 16  # bilinear weights as a texture unit's linear filter forms them


def build_command() -> list[str]:
    return ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", LIB_PATH,
            os.path.join(ORACLE_DIR, "amh_oracle.c"), "-lm"]


def build() -> str:
    os.makedirs(os.path.dirname(LIB_PATH), exist_ok=True)
    r = subprocess.run(build_command(), capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("oracle build failed:\n" + r.stdout + r.stderr)
    return LIB_PATH


class OrcCamera(ctypes.Structure):
    _fields_ = [("K", ctypes.c_double * 9), ("R", ctypes.c_double * 9),
                ("t", ctypes.c_double * 3), ("width", ctypes.c_int), ("height", ctypes.c_int)]


class OrcParams(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("tau_mc_init", ctypes.c_double),
                ("alpha", ctypes.c_double), ("beta", ctypes.c_double), ("tau_up", ctypes.c_double),
                ("n1", ctypes.c_int), ("n2", ctypes.c_int), ("k", ctypes.c_int),
                ("sigma_I", ctypes.c_double), ("sigma_x", ctypes.c_double),
                ("win_radius", ctypes.c_int), ("win_stride", ctypes.c_int),
                ("depth_min", ctypes.c_double), ("depth_max", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("flags", ctypes.c_int)]


_LIB = None
_dp = ctypes.POINTER(ctypes.c_double)
_vp = ctypes.c_void_p


def lib():
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            build()
        L = ctypes.CDLL(LIB_PATH)
        L.orc_default_params.argtypes = [ctypes.POINTER(OrcParams)]
        L.orc_create.restype = _vp
        L.orc_create.argtypes = [ctypes.POINTER(OrcParams), ctypes.c_int, ctypes.POINTER(OrcCamera),
                                 ctypes.POINTER(_dp), ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                 ctypes.c_int]
        L.orc_destroy.argtypes = [_vp]
        L.orc_set_threads.argtypes = [ctypes.c_int]
        L.orc_width.argtypes = [_vp]
        L.orc_height.argtypes = [_vp]
        L.orc_set_state.argtypes = [_vp, _vp, _vp, _vp, _vp, ctypes.c_int]
        L.orc_get_state.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp, ctypes.POINTER(ctypes.c_int)]
        L.orc_init_random.argtypes = [_vp]
        L.orc_step_phase.argtypes = [_vp, ctypes.c_int]
        L.orc_iterate.argtypes = [_vp, ctypes.c_int]
        L.orc_update_pixel.argtypes = [_vp, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, _vp, _vp]
        L.orc_update_pixels.argtypes = [_vp, ctypes.c_int, _vp, _vp]
        L.orc_philox4x32_10.argtypes = [_vp, _vp, _vp]
        L.orc_u01.restype = ctypes.c_double
        L.orc_u01.argtypes = [ctypes.c_uint32]
        L.orc_tau_mc.restype = ctypes.c_double
        L.orc_tau_mc.argtypes = [ctypes.POINTER(OrcParams), ctypes.c_int]
        L.orc_confidence.restype = ctypes.c_double
        L.orc_confidence.argtypes = [ctypes.POINTER(OrcParams), ctypes.c_double]
        L.orc_homography.argtypes = [_vp, ctypes.c_int, _vp, ctypes.c_double, _vp]
        L.orc_bilinear.restype = ctypes.c_double
        L.orc_bilinear.argtypes = [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double]
        L.orc_bilinear_texture.restype = ctypes.c_double
        L.orc_bilinear_texture.argtypes = [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double]
        L.orc_cost.restype = ctypes.c_double
        L.orc_cost.argtypes = [_vp, ctypes.c_int, ctypes.c_int, _vp, ctypes.c_int]
        L.orc_mhj.argtypes = [ctypes.POINTER(OrcParams), ctypes.c_int, _vp, _vp, ctypes.c_int,
                              ctypes.c_uint32, ctypes.c_int, _vp, _vp, _vp]
        L.orc_acp_offsets.restype = ctypes.c_int
        L.orc_acp_offsets.argtypes = [ctypes.c_int, _vp, _vp]
        L.orc_scp_offsets.restype = ctypes.c_int
        L.orc_scp_offsets.argtypes = [ctypes.c_int, _vp, _vp]
        L.orc_acp_pick.restype = ctypes.c_int
        L.orc_acp_pick.argtypes = [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        L.orc_acp_row.restype = ctypes.c_int
        L.orc_acp_row.argtypes = [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp]
        L.orc_refine_candidates.restype = ctypes.c_int
        L.orc_refine_candidates.argtypes = [_vp, ctypes.c_int, ctypes.c_int, _vp, ctypes.c_int, _vp]
        L.orc_random_plane.argtypes = [_vp, ctypes.c_int, ctypes.c_int, _vp]
        L.orc_score_plane.restype = ctypes.c_double
        L.orc_score_plane.argtypes = [_vp, ctypes.c_int, ctypes.c_int, _vp]
        _LIB = L
    return _LIB


def default_params(**kw) -> OrcParams:
    p = OrcParams()
    lib().orc_default_params(ctypes.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def philox4x32_10(ctr, key):
    c = np.asarray(ctr, np.uint32).copy()
    k = np.asarray(key, np.uint32).copy()
    o = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(o))
    return o


def u01(x: int) -> float:
    return lib().orc_u01(ctypes.c_uint32(int(x)))


def tau_mc(t: int, params: OrcParams | None = None) -> float:
    p = params or default_params()
    return lib().orc_tau_mc(ctypes.byref(p), t)


def confidence(m: float, params: OrcParams | None = None) -> float:
    p = params or default_params()
    return lib().orc_confidence(ctypes.byref(p), m)


def set_threads(n: int) -> None:
    """Threads of the oracle's pixel loops (default 1; timing only -- the
    results do not depend on it)."""
    lib().orc_set_threads(int(n))


def bilinear(img: np.ndarray, x: float, y: float) -> float:
    a = np.ascontiguousarray(img, np.float64)
    return lib().orc_bilinear(_ptr(a), a.shape[1], a.shape[0], x, y)


def bilinear_texture(img: np.ndarray, x: float, y: float) -> float:
    a = np.ascontiguousarray(img, np.float64)
    return lib().orc_bilinear_texture(_ptr(a), a.shape[1], a.shape[0], x, y)


def acp_offsets(g: int):
    dx = np.zeros(16, np.int32)
    dy = np.zeros(16, np.int32)
    n = lib().orc_acp_offsets(g, _ptr(dx), _ptr(dy))
    return list(zip(dx[:n].tolist(), dy[:n].tolist()))


def scp_offsets(g: int):
    """The fixed candidate of region g under symmetric propagation."""
    dx = np.zeros(1, np.int32)
    dy = np.zeros(1, np.int32)
    lib().orc_scp_offsets(g, _ptr(dx), _ptr(dy))
    return [(int(dx[0]), int(dy[0]))]


def mhj(M, row_valid=None, t=0, S_prev=0, v_prev=-1, params: OrcParams | None = None):
    """Weights, S_t bitmask and v_t for an 8 x N cost matrix."""
    p = params or default_params()
    M = np.ascontiguousarray(M, np.float64)
    assert M.shape[0] == NREGION
    N = M.shape[1]
    rv = np.ones(NREGION, np.int32) if row_valid is None else np.asarray(row_valid, np.int32).copy()
    w = np.zeros(N, np.float64)
    S = np.zeros(1, np.uint32)
    v = np.zeros(1, np.int32)
    lib().orc_mhj(ctypes.byref(p), t, _ptr(M), _ptr(rv), N, ctypes.c_uint32(S_prev), v_prev,
                  _ptr(w), _ptr(S), _ptr(v))
    return w, int(S[0]), int(v[0])


class Oracle:
    """One reference view with its sources, as in the C-ABI library."""

    def __init__(self, cams, images, ref, src, params: OrcParams | None = None):
        L = lib()
        self.params = params or default_params()
        n = len(cams)
        carr = (OrcCamera * n)()
        for i, c in enumerate(cams):
            carr[i].K[:] = list(np.asarray(c.K, float).ravel())
            carr[i].R[:] = list(np.asarray(c.R, float).ravel())
            carr[i].t[:] = list(np.asarray(c.t, float).ravel())
            carr[i].width, carr[i].height = int(c.width), int(c.height)
        self._imgs = [np.ascontiguousarray(im, np.float64) for im in images]
        for c, im in zip(cams, self._imgs):
            assert im.shape == (c.height, c.width)
        iarr = (_dp * n)(*[im.ctypes.data_as(_dp) for im in self._imgs])
        sarr = (ctypes.c_int * len(src))(*src)
        self.ctx = L.orc_create(ctypes.byref(self.params), n, carr, iarr, ref, sarr, len(src))
        if not self.ctx:
            raise ValueError("oracle rejected the inputs")
        self.W, self.H = L.orc_width(self.ctx), L.orc_height(self.ctx)
        self.n_src = len(src)

    @classmethod
    def from_scene(cls, scene, params: OrcParams | None = None, **kw):
        p = params or default_params(depth_min=scene.depth_min, depth_max=scene.depth_max, **kw)
        return cls(scene.cams, scene.images, scene.ref, scene.src, p)

    def __del__(self):
        if getattr(self, "ctx", None):
            lib().orc_destroy(self.ctx)
            self.ctx = None

    # ---- state ----
    def get_state(self):
        n = self.W * self.H
        plane = np.zeros((self.H, self.W, 4), np.float64)
        cost = np.zeros((self.H, self.W), np.float64)
        sel = np.zeros((self.H, self.W), np.uint32)
        vprev = np.zeros((self.H, self.W), np.int32)
        choice = np.zeros((self.H, self.W), np.int32)
        t = ctypes.c_int(0)
        lib().orc_get_state(self.ctx, _ptr(plane), _ptr(cost), _ptr(sel), _ptr(vprev), _ptr(choice),
                            ctypes.byref(t))
        assert plane.size == 4 * n
        return dict(plane=plane, cost=cost, sel=sel, vprev=vprev, choice=choice, t=t.value)

    def set_state(self, plane=None, cost=None, sel=None, vprev=None, t=0):
        keep = []

        def arr(a, dt, shape):
            if a is None:
                return None
            a = np.ascontiguousarray(a, dt).reshape(shape)
            keep.append(a)
            return _ptr(a)
        lib().orc_set_state(self.ctx, arr(plane, np.float64, (self.H, self.W, 4)),
                            arr(cost, np.float64, (self.H, self.W)),
                            arr(sel, np.uint32, (self.H, self.W)),
                            arr(vprev, np.int32, (self.H, self.W)), int(t))

    # ---- method ----
    def init_random(self):
        lib().orc_init_random(self.ctx)

    def step_phase(self, color: int):
        lib().orc_step_phase(self.ctx, int(color))

    def iterate(self, k: int):
        lib().orc_iterate(self.ctx, int(k))

    def update_pixel(self, x: int, y: int):
        pl = np.zeros(4, np.float64)
        cost = np.zeros(1, np.float64)
        S = np.zeros(1, np.uint32)
        v = np.zeros(1, np.int32)
        ch = np.zeros(1, np.int32)
        lib().orc_update_pixel(self.ctx, x, y, _ptr(pl), _ptr(cost), _ptr(S), _ptr(v), _ptr(ch))
        return dict(plane=pl, cost=float(cost[0]), sel=int(S[0]), v=int(v[0]), choice=int(ch[0]))

    def update_pixels(self, xs, ys):
        xs = np.ascontiguousarray(xs, np.int32)
        ys = np.ascontiguousarray(ys, np.int32)
        lib().orc_update_pixels(self.ctx, len(xs), _ptr(xs), _ptr(ys))

    # ---- building blocks ----
    def homography(self, j: int, n, d: float):
        nn = np.ascontiguousarray(n, np.float64)
        H = np.zeros(9, np.float64)
        lib().orc_homography(self.ctx, j, _ptr(nn), d, _ptr(H))
        return H.reshape(3, 3)

    def cost(self, x: int, y: int, plane, j: int) -> float:
        pl = np.ascontiguousarray(plane, np.float64)
        return lib().orc_cost(self.ctx, x, y, _ptr(pl), j)

    def acp_pick(self, x, y, g):
        return lib().orc_acp_pick(self.ctx, x, y, g)

    def acp_row(self, x, y, g):
        out = np.zeros(4, np.float64)
        ok = lib().orc_acp_row(self.ctx, x, y, g, _ptr(out))
        return out if ok else None

    def refine_candidates(self, x, y, plane, t):
        pl = np.ascontiguousarray(plane, np.float64)
        out = np.zeros((6, 4), np.float64)
        n = lib().orc_refine_candidates(self.ctx, x, y, _ptr(pl), t, _ptr(out))
        return out[:n]

    def score_plane(self, x, y, plane) -> float:
        pl = np.ascontiguousarray(plane, np.float64)
        return lib().orc_score_plane(self.ctx, x, y, _ptr(pl))

    def random_plane(self, x, y):
        out = np.zeros(4, np.float64)
        lib().orc_random_plane(self.ctx, x, y, _ptr(out))
        return out

    def depth_map(self):
        return self.get_state()["plane"][..., 3]
