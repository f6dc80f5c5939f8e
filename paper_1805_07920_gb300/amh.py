"""Thin ctypes binding of the C-ABI in ``include/amh.h`` (``_lib/libamh.so``).

Argument marshalling only: every step of the update runs in the library's
CUDA kernels.  Host arrays are numpy arrays; device buffers are torch CUDA
tensors (their ``data_ptr()`` is passed, and by default the context runs on
torch's current stream).  There is no CPU fallback: if the library or a GPU is
missing, the calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "libamh.so")

AMH_OK, AMH_EINVAL, AMH_ECUDA, AMH_ENOMEM, AMH_EDEVICE, AMH_ESTATE = 0, -1, -2, -3, -4, -5
AMH_MEM_HOST, AMH_MEM_DEVICE = 0, 1
AMH_FLAG_BILATERAL_SQUARED = 1
AMH_FLAG_SYMMETRIC_PROPAGATION = 4   # ablation: symmetric checkerboard propagation
AMH_FLAG_HEURISTIC_VIEWS = 8         # ablation: per-hypothesis k-best view selection
AMH_FLAG_IMAGES_F16 = 2
AMH_FLAG_TEXTURE_BILINEAR = 16       # precision form: texture-unit bilinear interpolation
AMH_FLAG_STAGED_FETCH = 32           # fetch path: shared-memory staged matrix sweep (measured alternative)
MAX_SRC = 32
NOALLOC_MAX_PIXELS = 262144
BATCH_VARIANTS = 5                   # AMH_BATCH_VARIANTS: tile / warp-layout variants of the batched form

EXPORTS = ["amh_default_params", "amh_create", "amh_set_stream", "amh_init_random",
           "amh_step_phase", "amh_iterate", "amh_get_state", "amh_set_state", "amh_read_maps",
           "amh_get_info", "amh_pair_count", "amh_pair_counts", "amh_synchronize", "amh_last_error", "amh_destroy",
           "amh_read_maps_noalloc", "amh_batch_create", "amh_batch_init_random", "amh_batch_step_phase",
           "amh_batch_iterate", "amh_batch_run", "amh_batch_set_variant", "amh_batch_autotune",
           "amh_batch_info", "amh_batch_get_state", "amh_batch_pair_count", "amh_batch_synchronize",
           "amh_batch_last_error", "amh_batch_destroy", "amh_net_create", "amh_net_params", "amh_net_grads",
           "amh_net_set_input", "amh_net_set_example", "amh_net_features", "amh_net_targets", "amh_net_set_targets", "amh_net_forward",
           "amh_net_backward", "amh_net_adam", "amh_net_read", "amh_net_propose", "amh_clear_proposal", "amh_net_synchronize",
           "amh_net_last_error", "amh_net_destroy", "amh_gather_peak", "amh_median4", "amh_fuse", "amh_select_sources", "amh_set_proposal", "amh_bounds_checked"]


class AmhError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"amh error {code}: {msg}")
        self.code = code


class Camera(ctypes.Structure):
    _fields_ = [("K", ctypes.c_double * 9), ("R", ctypes.c_double * 9), ("t", ctypes.c_double * 3),
                ("width", ctypes.c_int32), ("height", ctypes.c_int32)]


class Params(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("tau_mc_init", ctypes.c_float), ("alpha", ctypes.c_float),
                ("beta", ctypes.c_float), ("tau_up", ctypes.c_float), ("n1", ctypes.c_int32),
                ("n2", ctypes.c_int32), ("k", ctypes.c_int32), ("sigma_I", ctypes.c_float),
                ("sigma_x", ctypes.c_float), ("win_radius", ctypes.c_int32), ("win_stride", ctypes.c_int32),
                ("depth_min", ctypes.c_float), ("depth_max", ctypes.c_float), ("seed", ctypes.c_uint64),
                ("flags", ctypes.c_int32)]


class State(ctypes.Structure):
    _fields_ = [("plane", ctypes.c_void_p), ("cost", ctypes.c_void_p), ("sel", ctypes.c_void_p),
                ("vbest", ctypes.c_void_p), ("wmask", ctypes.c_void_p), ("choice", ctypes.c_void_p),
                ("t", ctypes.c_int32)]


_LIB = None
_vp = ctypes.c_void_p
_i32 = ctypes.c_int32


def lib():
    """Load ``libamh.so``; raises if it has not been built."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run __graft_entry__.build() (no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        L.amh_default_params.argtypes = [ctypes.POINTER(Params)]
        L.amh_create.argtypes = [ctypes.POINTER(_vp), ctypes.POINTER(Params), _i32, ctypes.POINTER(Camera),
                                 ctypes.POINTER(_vp), _i32, _i32, ctypes.POINTER(_i32), _i32, _vp]
        L.amh_set_stream.argtypes = [_vp, _vp]
        L.amh_init_random.argtypes = [_vp]
        L.amh_step_phase.argtypes = [_vp, _i32]
        L.amh_iterate.argtypes = [_vp, _i32]
        L.amh_get_state.argtypes = [_vp, ctypes.POINTER(State), _i32]
        L.amh_set_state.argtypes = [_vp, ctypes.POINTER(State), _i32]
        L.amh_read_maps.argtypes = [_vp, _vp, _vp, _vp, _vp, _i32]
        L.amh_read_maps_noalloc.argtypes = [_vp, _vp, _vp, ctypes.c_int64, ctypes.c_int64]
        L.amh_get_info.argtypes = [_vp, ctypes.POINTER(_i32), ctypes.POINTER(_i32), ctypes.POINTER(_i32),
                                   ctypes.POINTER(_i32)]
        L.amh_pair_count.argtypes = [_vp, ctypes.POINTER(ctypes.c_uint64), _i32]
        L.amh_pair_counts.argtypes = [_vp, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64), _i32]
        L.amh_synchronize.argtypes = [_vp]
        L.amh_last_error.argtypes = [_vp]
        L.amh_last_error.restype = ctypes.c_char_p
        L.amh_destroy.argtypes = [_vp]
        L.amh_destroy.restype = None
        _LIB = L
    return _LIB


def select_sources(cams, ref, depth, n_src=10, min_angle_deg=1.0, max_angle_deg=60.0):
    """Source views for reference `ref` by triangulation angle at the point at
    z-depth `depth` on its optical axis (``amh_select_sources``)."""
    L = lib()
    L.amh_select_sources.argtypes = [_i32, ctypes.POINTER(Camera), _i32, ctypes.c_double, _i32, ctypes.c_double,
                                     ctypes.c_double, ctypes.POINTER(_i32), ctypes.POINTER(_i32)]
    out = (_i32 * int(n_src))()
    n = _i32()
    rc = L.amh_select_sources(len(cams), make_cameras(cams), int(ref), float(depth), int(n_src),
                              float(min_angle_deg), float(max_angle_deg), out, ctypes.byref(n))
    if rc != AMH_OK:
        raise AmhError(rc, L.amh_last_error(None).decode())
    return [int(out[i]) for i in range(n.value)]


def gather_peak() -> float:
    """Measured texture-gather rate of the GPU (gathers per second)."""
    L = lib()
    L.amh_gather_peak.argtypes = [ctypes.POINTER(ctypes.c_double)]
    v = ctypes.c_double()
    rc = L.amh_gather_peak(ctypes.byref(v))
    if rc != AMH_OK:
        raise AmhError(rc, "gather peak measurement failed")
    return v.value


def median4(depth):
    """4x4 median of a depth map (torch float32 CUDA tensor, H x W) into a new
    tensor, on the current stream (``amh_median4``)."""
    import torch
    d = depth.contiguous()
    out = torch.empty_like(d)
    L = lib()
    L.amh_median4.argtypes = [_vp, _vp, _i32, _i32, _vp]
    rc = L.amh_median4(_vp(d.data_ptr()), _vp(out.data_ptr()), d.shape[1], d.shape[0], _current_stream())
    if rc != AMH_OK:
        raise AmhError(rc, L.amh_last_error(None).decode())
    return out


def fuse(cams, depths, normals, f_eps=0.3, f_ang_deg=30.0, f_con=2):
    """Consistency fusion (``amh_fuse``) of per-view depth (H x W) and normal
    (H x W x 3, camera coordinates) torch float32 CUDA tensors; returns
    (points (H x W x 6 world coordinates and normal) and counts (H x W uint8))
    per view."""
    import torch
    V = len(cams)
    arr = make_cameras(cams)
    d = [x.contiguous() for x in depths]
    n = [x.contiguous() for x in normals]
    pts = [torch.zeros(x.shape[0], x.shape[1], 6, dtype=torch.float32, device=x.device) for x in d]
    cnt = [torch.zeros(x.shape[0], x.shape[1], dtype=torch.uint8, device=x.device) for x in d]
    keep = []

    def P(ts):
        a = (_vp * V)(*[_vp(t.data_ptr()) for t in ts])
        keep.append(a)
        return ctypes.cast(a, _vp)

    L = lib()
    L.amh_fuse.argtypes = [_i32, ctypes.POINTER(Camera), _vp, _vp, ctypes.c_float, ctypes.c_float, _i32, _vp, _vp, _vp]
    rc = L.amh_fuse(V, arr, P(d), P(n), float(f_eps), float(f_ang_deg), int(f_con), P(pts), P(cnt), _current_stream())
    if rc != AMH_OK:
        raise AmhError(rc, L.amh_last_error(None).decode())
    return pts, cnt


def default_params(**kw) -> Params:
    p = Params()
    lib().amh_default_params(ctypes.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def make_cameras(cams) -> ctypes.Array:
    arr = (Camera * len(cams))()
    for i, c in enumerate(cams):
        arr[i].K[:] = [float(v) for v in np.asarray(c.K, float).ravel()]
        arr[i].R[:] = [float(v) for v in np.asarray(c.R, float).ravel()]
        arr[i].t[:] = [float(v) for v in np.asarray(c.t, float).ravel()]
        arr[i].width, arr[i].height = int(c.width), int(c.height)
    return arr


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _ptr(x):
    if x is None:
        return None
    if _is_torch(x):
        assert x.is_cuda and x.is_contiguous()
        return ctypes.c_void_p(x.data_ptr())
    assert isinstance(x, np.ndarray) and x.flags["C_CONTIGUOUS"]
    return x.ctypes.data_as(ctypes.c_void_p)


def _current_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    except ImportError:
        pass
    return None


class Context:
    """One reference view and its sources on the GPU (``amh_create``).

    ``images`` are uint8 or float16 arrays (numpy on the host or torch on the
    GPU); float16 images select the FP16 texture storage."""

    def __init__(self, cams, images, ref: int, src, params: Params | None = None, stream=None):
        L = lib()
        self.params = params or default_params()
        self._cams = make_cameras(cams)
        n = len(cams)
        dev = _is_torch(images[0])
        half = str(images[0].dtype).endswith("float16")
        if half:
            self.params.flags |= AMH_FLAG_IMAGES_F16
        dt = np.float16 if half else np.uint8
        self._keep = [im if dev else np.ascontiguousarray(im, dt) for im in images]
        for c, im in zip(cams, self._keep):
            assert tuple(im.shape) == (c.height, c.width), "image shape must be (height, width)"
        ptrs = (_vp * n)(*[(_ptr(im).value if im is not None else None) for im in self._keep])
        srcs = (_i32 * len(src))(*[int(s) for s in src])
        self.ctx = _vp()
        if stream is None:
            stream = _current_stream()
        rc = L.amh_create(ctypes.byref(self.ctx), ctypes.byref(self.params), n, self._cams, ptrs,
                          AMH_MEM_DEVICE if dev else AMH_MEM_HOST, int(ref), srcs, len(src), stream)
        if rc != AMH_OK:
            raise AmhError(rc, L.amh_last_error(None).decode())
        self._keep = None
        w, h, ns, t = _i32(), _i32(), _i32(), _i32()
        L.amh_get_info(self.ctx, ctypes.byref(w), ctypes.byref(h), ctypes.byref(ns), ctypes.byref(t))
        self.W, self.H, self.n_src = w.value, h.value, ns.value

    @classmethod
    def from_scene(cls, scene, params: Params | None = None, images=None, **kw):
        p = params or default_params(depth_min=scene.depth_min, depth_max=scene.depth_max, **kw)
        return cls(scene.cams, images if images is not None else scene.images, scene.ref, scene.src, p)

    def _check(self, rc):
        if rc != AMH_OK:
            raise AmhError(rc, lib().amh_last_error(self.ctx).decode())

    def close(self):
        if getattr(self, "ctx", None) and self.ctx.value:
            lib().amh_destroy(self.ctx)
            self.ctx = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- method ----
    def set_stream(self, stream):
        self._check(lib().amh_set_stream(self.ctx, stream))

    def init_random(self):
        self._check(lib().amh_init_random(self.ctx))

    def step_phase(self, color: int):
        self._check(lib().amh_step_phase(self.ctx, int(color)))

    def iterate(self, k: int):
        self._check(lib().amh_iterate(self.ctx, int(k)))

    def synchronize(self):
        self._check(lib().amh_synchronize(self.ctx))

    @property
    def t(self) -> int:
        t = _i32()
        lib().amh_get_info(self.ctx, None, None, None, ctypes.byref(t))
        return t.value

    def pair_count(self, reset: bool = False) -> int:
        c = ctypes.c_uint64()
        self._check(lib().amh_pair_count(self.ctx, ctypes.byref(c), int(reset)))
        return c.value

    def pair_counts(self, reset: bool = False) -> tuple[int, int]:
        """(all evaluations, those sampled from shared-memory boxes) since the
        last reset."""
        c, st = ctypes.c_uint64(), ctypes.c_uint64()
        self._check(lib().amh_pair_counts(self.ctx, ctypes.byref(c), ctypes.byref(st), int(reset)))
        return c.value, st.value

    # ---- state ----
    def get_state(self):
        H, W = self.H, self.W
        st = dict(plane=np.zeros((H, W, 4), np.float32), cost=np.zeros((H, W), np.float32),
                  sel=np.zeros((H, W), np.uint32), vbest=np.zeros((H, W), np.uint8),
                  wmask=np.zeros((H, W), np.uint32), choice=np.zeros((H, W), np.uint8))
        s = State(*[_ptr(st[k]) for k in ("plane", "cost", "sel", "vbest", "wmask", "choice")], 0)
        self._check(lib().amh_get_state(self.ctx, ctypes.byref(s), AMH_MEM_HOST))
        st["t"] = s.t
        return st

    def get_state_device(self, out: dict):
        """Copy the state into torch CUDA tensors given in ``out`` (any subset)."""
        s = State(*[_ptr(out.get(k)) for k in ("plane", "cost", "sel", "vbest", "wmask", "choice")], 0)
        self._check(lib().amh_get_state(self.ctx, ctypes.byref(s), AMH_MEM_DEVICE))
        return s.t

    def set_state(self, plane, cost=None, sel=None, vbest=None, wmask=None, choice=None, t=0):
        dev = _is_torch(plane)
        H, W = self.H, self.W

        def conv(a, dt, shape):
            if a is None:
                return None
            if dev:
                return a.contiguous()
            return np.ascontiguousarray(np.asarray(a).reshape(shape), dt)
        arrs = [conv(plane, np.float32, (H, W, 4)), conv(cost, np.float32, (H, W)),
                conv(sel, np.uint32, (H, W)), conv(vbest, np.uint8, (H, W)),
                conv(wmask, np.uint32, (H, W)), conv(choice, np.uint8, (H, W))]
        s = State(*[_ptr(a) for a in arrs], int(t))
        self._check(lib().amh_set_state(self.ctx, ctypes.byref(s), AMH_MEM_DEVICE if dev else AMH_MEM_HOST))

    def read_maps(self):
        H, W = self.H, self.W
        depth = np.zeros((H, W), np.float32)
        normal = np.zeros((H, W, 3), np.float32)
        cost = np.zeros((H, W), np.float32)
        sel = np.zeros((H, W), np.uint32)
        self._check(lib().amh_read_maps(self.ctx, _ptr(depth), _ptr(normal), _ptr(cost), _ptr(sel),
                                        AMH_MEM_HOST))
        return dict(depth=depth, normal=normal, cost=cost, selected=sel)

    def read_maps_noalloc(self, depth=None, normal=None, first_pixel: int = 0, n_pixels: int | None = None):
        """Depth/normal of a pixel range into host arrays, without any device
        allocation (amh_read_maps_noalloc; at most NOALLOC_MAX_PIXELS per
        call).  depth / normal must be C-contiguous float32 numpy arrays of at
        least n_pixels / 3 * n_pixels elements.  Without n_pixels the call
        reads as many pixels from first_pixel on as remain in the image, fit
        the per-call maximum and fit the given arrays."""
        bufs = [(name, a, per) for name, a, per in (("depth", depth, 1), ("normal", normal, 3)) if a is not None]
        for name, a, _ in bufs:
            if not isinstance(a, np.ndarray) or a.dtype != np.float32 or not a.flags["C_CONTIGUOUS"]:
                raise ValueError(f"read_maps_noalloc: {name} must be a C-contiguous float32 numpy array")
        if n_pixels is None:
            n_pixels = min([self.W * self.H - int(first_pixel), NOALLOC_MAX_PIXELS] +
                           [a.size // per for _, a, per in bufs])
        n_pixels = int(n_pixels)
        for name, a, per in bufs:
            if a.size < per * max(n_pixels, 0):
                raise ValueError(f"read_maps_noalloc: {name} holds {a.size} floats, {per * n_pixels} needed")
        self._check(lib().amh_read_maps_noalloc(self.ctx, _ptr(depth), _ptr(normal), int(first_pixel),
                                                n_pixels))

    def read_maps_device(self, depth=None, normal=None, cost=None, selected=None):
        self._check(lib().amh_read_maps(self.ctx, _ptr(depth), _ptr(normal), _ptr(cost), _ptr(selected),
                                        AMH_MEM_DEVICE))


# ---------------------------------------------------------------------------
# batched form
# ---------------------------------------------------------------------------
_BATCH_READY = False


def _batch_lib():
    global _BATCH_READY
    L = lib()
    if not _BATCH_READY:
        L.amh_batch_create.argtypes = [ctypes.POINTER(_vp), ctypes.POINTER(Params), _i32, ctypes.POINTER(Camera),
                                       ctypes.POINTER(_vp), _i32, _i32, ctypes.POINTER(_i32),
                                       ctypes.POINTER(_i32), ctypes.POINTER(_i32), _vp]
        for name in ("amh_batch_init_random", "amh_batch_synchronize"):
            getattr(L, name).argtypes = [_vp]
        L.amh_batch_step_phase.argtypes = [_vp, _i32]
        L.amh_batch_iterate.argtypes = [_vp, _i32]
        L.amh_batch_run.argtypes = [_vp, _i32]
        L.amh_batch_set_variant.argtypes = [_vp, _i32]
        L.amh_batch_autotune.argtypes = [_vp, _i32, ctypes.POINTER(_i32), ctypes.POINTER(ctypes.c_float)]
        L.amh_batch_info.argtypes = [_vp, _i32, ctypes.POINTER(_i32), ctypes.POINTER(_i32), ctypes.POINTER(_i32),
                                     ctypes.POINTER(_i32)]
        L.amh_batch_get_state.argtypes = [_vp, _i32, ctypes.POINTER(State), _i32]
        L.amh_batch_pair_count.argtypes = [_vp, ctypes.POINTER(ctypes.c_uint64), _i32]
        L.amh_batch_last_error.argtypes = [_vp]
        L.amh_batch_last_error.restype = ctypes.c_char_p
        L.amh_batch_destroy.argtypes = [_vp]
        L.amh_batch_destroy.restype = None
        _BATCH_READY = True
    return L


class Batch:
    """Several references at once (``amh_batch_create``): refs[r] with the
    sources src_lists[r]."""

    def __init__(self, cams, images, refs, src_lists, params: Params | None = None, stream=None):
        L = _batch_lib()
        self.params = params or default_params()
        self._cams = make_cameras(cams)
        n = len(cams)
        half = str(images[0].dtype).endswith("float16")
        if half:
            self.params.flags |= AMH_FLAG_IMAGES_F16
        dt = np.float16 if half else np.uint8
        keep = [np.ascontiguousarray(im, dt) for im in images]
        ptrs = (_vp * n)(*[k.ctypes.data for k in keep])
        offs = [0]
        flat = []
        for s in src_lists:
            flat += [int(v) for v in s]
            offs.append(len(flat))
        self.ctx = _vp()
        rc = L.amh_batch_create(ctypes.byref(self.ctx), ctypes.byref(self.params), n, self._cams, ptrs,
                                AMH_MEM_HOST, len(refs), (_i32 * len(refs))(*refs), (_i32 * len(offs))(*offs),
                                (_i32 * len(flat))(*flat), stream)
        if rc != AMH_OK:
            raise AmhError(rc, L.amh_batch_last_error(None).decode())
        self.n_refs = len(refs)
        self.sizes = []
        for r in range(self.n_refs):
            w, h, ns = _i32(), _i32(), _i32()
            L.amh_batch_info(self.ctx, r, ctypes.byref(w), ctypes.byref(h), ctypes.byref(ns), None)
            self.sizes.append((w.value, h.value, ns.value))

    def _check(self, rc):
        if rc != AMH_OK:
            raise AmhError(rc, _batch_lib().amh_batch_last_error(self.ctx).decode())

    def close(self):
        if getattr(self, "ctx", None) and self.ctx.value:
            _batch_lib().amh_batch_destroy(self.ctx)
            self.ctx = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init_random(self):
        self._check(_batch_lib().amh_batch_init_random(self.ctx))

    def step_phase(self, color):
        self._check(_batch_lib().amh_batch_step_phase(self.ctx, int(color)))

    def iterate(self, k):
        self._check(_batch_lib().amh_batch_iterate(self.ctx, int(k)))

    def run(self, iters):
        self._check(_batch_lib().amh_batch_run(self.ctx, int(iters)))

    def set_variant(self, v):
        self._check(_batch_lib().amh_batch_set_variant(self.ctx, int(v)))

    def autotune(self, iters=1):
        ch = _i32()
        ms = (ctypes.c_float * BATCH_VARIANTS)()
        self._check(_batch_lib().amh_batch_autotune(self.ctx, int(iters), ctypes.byref(ch), ms))
        return ch.value, list(ms)

    def synchronize(self):
        self._check(_batch_lib().amh_batch_synchronize(self.ctx))

    def pair_count(self, reset=False):
        c = ctypes.c_uint64()
        self._check(_batch_lib().amh_batch_pair_count(self.ctx, ctypes.byref(c), int(reset)))
        return c.value

    def get_state(self, r):
        W, H, _ = self.sizes[r]
        st = dict(plane=np.zeros((H, W, 4), np.float32), cost=np.zeros((H, W), np.float32),
                  sel=np.zeros((H, W), np.uint32), vbest=np.zeros((H, W), np.uint8),
                  wmask=np.zeros((H, W), np.uint32), choice=np.zeros((H, W), np.uint8))
        s = State(*[_ptr(st[k]) for k in ("plane", "cost", "sel", "vbest", "wmask", "choice")], 0)
        self._check(_batch_lib().amh_batch_get_state(self.ctx, int(r), ctypes.byref(s), AMH_MEM_HOST))
        st["t"] = s.t
        return st


# ---------------------------------------------------------------------------
# learned proposal network
# ---------------------------------------------------------------------------
NET_LAYERS = [("e1", 16, 32), ("e2", 32, 64), ("e3", 64, 96), ("e4", 96, 128),
              ("d3", 128, 96), ("d2", 96, 64), ("d1", 64, 32), ("out", 32, 16)]
_NET_READY = False


def _net_lib():
    global _NET_READY
    L = lib()
    if not _NET_READY:
        _fp = ctypes.POINTER(ctypes.c_float)
        L.amh_net_create.argtypes = [ctypes.POINTER(_vp), _i32, _i32, ctypes.c_uint64, _vp]
        L.amh_net_params.argtypes = [_vp, _i32, _vp, _vp, _i32]
        L.amh_net_grads.argtypes = [_vp, _i32, _vp, _vp]
        L.amh_net_set_input.argtypes = [_vp, _vp]
        L.amh_net_set_example.argtypes = [_vp, _vp, _i32, _vp, _vp, _i32, _i32]
        L.amh_net_features.argtypes = [_vp, _vp]
        L.amh_net_targets.argtypes = [_vp, _vp, ctypes.c_float]
        L.amh_net_set_targets.argtypes = [_vp, _vp, _vp]
        L.amh_net_forward.argtypes = [_vp, _vp]
        L.amh_net_backward.argtypes = [_vp, _fp]
        L.amh_net_adam.argtypes = [_vp, ctypes.c_float]
        L.amh_net_read.argtypes = [_vp, _i32, _vp, ctypes.POINTER(ctypes.c_int64)]
        L.amh_net_propose.argtypes = [_vp, _vp]
        L.amh_clear_proposal.argtypes = [_vp]
        L.amh_net_synchronize.argtypes = [_vp]
        L.amh_net_last_error.argtypes = [_vp]
        L.amh_net_last_error.restype = ctypes.c_char_p
        L.amh_net_destroy.argtypes = [_vp]
        L.amh_net_destroy.restype = None
        _NET_READY = True
    return L


def net_size_for(width, height):
    """Network input size for a width x height reference: the (x/2, y/2) grid
    rounded up to multiples of 8."""
    r8 = lambda v: (v + 7) // 8 * 8
    return r8((width + 1) // 2), r8((height + 1) // 2)


class Net:
    """The learned proposal network (``amh_net_*``)."""

    def __init__(self, width2, height2, seed=0, stream=None):
        L = _net_lib()
        self.ctx = _vp()
        if stream is None:
            stream = _current_stream()
        rc = L.amh_net_create(ctypes.byref(self.ctx), int(width2), int(height2), ctypes.c_uint64(seed), stream)
        if rc != AMH_OK:
            raise AmhError(rc, L.amh_net_last_error(None).decode())
        self.w2, self.h2 = int(width2), int(height2)

    def _check(self, rc):
        if rc != AMH_OK:
            raise AmhError(rc, _net_lib().amh_net_last_error(self.ctx).decode())

    def close(self):
        if getattr(self, "ctx", None) and self.ctx.value:
            _net_lib().amh_net_destroy(self.ctx)
            self.ctx = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_params(self):
        out = {}
        for i, (name, cin, cout) in enumerate(NET_LAYERS):
            w = np.zeros((9, cout, cin), np.float32)
            b = np.zeros(cout, np.float32)
            self._check(_net_lib().amh_net_params(self.ctx, i, _ptr(w), _ptr(b), 0))
            out[name] = (w, b)
        return out

    def set_params(self, params):
        for i, (name, cin, cout) in enumerate(NET_LAYERS):
            w = np.ascontiguousarray(params[name][0], np.float32).reshape(9, cout, cin)
            b = np.ascontiguousarray(params[name][1], np.float32).reshape(cout)
            self._check(_net_lib().amh_net_params(self.ctx, i, _ptr(w), _ptr(b), 1))

    def get_grads(self):
        out = {}
        for i, (name, cin, cout) in enumerate(NET_LAYERS):
            w = np.zeros((9, cout, cin), np.float32)
            b = np.zeros(cout, np.float32)
            self._check(_net_lib().amh_net_grads(self.ctx, i, _ptr(w), _ptr(b)))
            out[name] = (w, b)
        return out

    def set_input(self, x0):
        x = np.ascontiguousarray(x0, np.float32).reshape(self.h2, self.w2, 16)
        self._check(_net_lib().amh_net_set_input(self.ctx, _ptr(x)))

    def set_example(self, x, target, mask, mirror_x=False, mirror_y=False):
        """One training example (amh_net_set_example): features x (h2, w2, C)
        float32 with C <= 16, targets (h2, w2, 4) float32, mask (h2, w2) uint8,
        all numpy arrays or all CUDA tensors (which then must stay alive until
        the network's stream has run the call); mirrored on the device."""
        dev = _is_torch(x)
        if dev:
            import torch
            ok = (x.dtype == torch.float32 and target.dtype == torch.float32 and mask.dtype == torch.uint8 and
                  all(a.is_cuda and a.is_contiguous() for a in (x, target, mask)))
            C = x.shape[-1]
        else:
            x = np.ascontiguousarray(x, np.float32)
            target = np.ascontiguousarray(target, np.float32)
            mask = np.ascontiguousarray(mask, np.uint8)
            ok = True
            C = x.shape[-1]
        if not ok:
            raise ValueError("set_example: float32 / float32 / uint8 contiguous CUDA tensors expected")
        n = self.h2 * self.w2
        if (x.numel() if dev else x.size) != n * C:
            raise ValueError(f"set_example: features must be ({self.h2}, {self.w2}, C)")
        if (target.numel() if dev else target.size) != n * 4 or (mask.numel() if dev else mask.size) != n:
            raise ValueError(f"set_example: targets ({self.h2}, {self.w2}, 4) and mask ({self.h2}, {self.w2}) expected")
        self._check(_net_lib().amh_net_set_example(self.ctx, _ptr(x), int(C), _ptr(target), _ptr(mask),
                                                   (1 if mirror_x else 0) | (2 if mirror_y else 0),
                                                   AMH_MEM_DEVICE if dev else AMH_MEM_HOST))
        if not dev:
            self.synchronize()

    def set_targets(self, target, mask):
        t = np.ascontiguousarray(target, np.float32).reshape(self.h2, self.w2, 4)
        m = np.ascontiguousarray(mask, np.uint8).reshape(self.h2, self.w2)
        self._check(_net_lib().amh_net_set_targets(self.ctx, _ptr(t), _ptr(m)))

    def features(self, ctx: Context):
        self._check(_net_lib().amh_net_features(self.ctx, ctx.ctx))

    def targets(self, ctx: Context, cost_max=0.5):
        self._check(_net_lib().amh_net_targets(self.ctx, ctx.ctx, float(cost_max)))

    def forward(self, want_output=False):
        out = np.zeros((self.h2, self.w2, 16), np.float32) if want_output else None
        self._check(_net_lib().amh_net_forward(self.ctx, _ptr(out) if want_output else None))
        return out

    def backward(self):
        loss = ctypes.c_float()
        self._check(_net_lib().amh_net_backward(self.ctx, ctypes.byref(loss)))
        return loss.value

    def adam(self, lr):
        self._check(_net_lib().amh_net_adam(self.ctx, float(lr)))

    def propose(self, ctx: Context):
        self._check(_net_lib().amh_net_propose(self.ctx, ctx.ctx))

    # name -> (level, channels); level k is (height2 >> k, width2 >> k)
    NET_TENSORS = {"x0": (0, 16), "e1": (0, 32), "in_e2": (1, 32), "e2": (1, 64), "in_e3": (2, 64), "e3": (2, 96),
                   "in_e4": (3, 96), "e4": (3, 128), "in_d3": (2, 128), "r3": (2, 96), "d3": (2, 96),
                   "in_d2": (1, 96), "r2": (1, 64), "d2": (1, 64), "in_d1": (0, 64), "r1": (0, 32), "d1": (0, 32),
                   "out": (0, 16)}
    LAYER_LEVEL = {"e1": 0, "e2": 1, "e3": 2, "e4": 3, "d3": 2, "d2": 1, "d1": 0, "out": 0}

    def read(self, name):
        """An internal tensor as float32 (H, W, C): a forward tensor of
        NET_TENSORS, "dy:<layer>" for the gradient at that layer's output
        after its ReLU mask (from the last backward), or "target" / "mask"."""
        names = [n for n, _, _ in NET_LAYERS]
        if name.startswith("dy:"):
            L = names.index(name[3:])
            which, level, ch = 32 + L, self.LAYER_LEVEL[name[3:]], NET_LAYERS[L][2]
        elif name in ("target", "mask"):
            which, level, ch = (64, 0, 4) if name == "target" else (65, 0, 1)
        else:
            which = list(self.NET_TENSORS).index(name)
            level, ch = self.NET_TENSORS[name]
        cnt = ctypes.c_int64((self.h2 >> level) * (self.w2 >> level) * ch)
        out = np.zeros(cnt.value, np.float32)
        self._check(_net_lib().amh_net_read(self.ctx, which, _ptr(out), ctypes.byref(cnt)))
        return out.reshape(self.h2 >> level, self.w2 >> level, ch)

    def synchronize(self):
        self._check(_net_lib().amh_net_synchronize(self.ctx))

    def save(self, path):
        p = self.get_params()
        np.savez_compressed(path, **{f"{k}_w": v[0] for k, v in p.items()}, **{f"{k}_b": v[1] for k, v in p.items()})

    def load(self, path):
        z = np.load(path)
        self.set_params({name: (z[f"{name}_w"], z[f"{name}_b"]) for name, _, _ in NET_LAYERS})


def set_proposal(ctx: Context, planes):
    """Caller-supplied proposals (``amh_set_proposal``): planes is a
    (ceil(H/2), ceil(W/2), 4) float32 array or CUDA tensor of (nx, ny, nz, d)
    with n . X + d = 0 in reference-camera coordinates."""
    L = lib()
    L.amh_set_proposal.argtypes = [_vp, _vp, _i32, _i32, _i32]
    if _is_torch(planes):
        buf = planes.contiguous().float()
        h2, w2 = int(buf.shape[0]), int(buf.shape[1])
        rc = L.amh_set_proposal(ctx.ctx, _vp(buf.data_ptr()), w2, h2, AMH_MEM_DEVICE)
    else:
        buf = np.ascontiguousarray(planes, np.float32)
        h2, w2 = buf.shape[0], buf.shape[1]
        rc = L.amh_set_proposal(ctx.ctx, buf.ctypes.data, w2, h2, AMH_MEM_HOST)
    ctx._check(rc)
    ctx.synchronize()      # the copy has read buf before it goes out of scope


def clear_proposal(ctx: Context):
    ctx._check(_net_lib().amh_clear_proposal(ctx.ctx))
