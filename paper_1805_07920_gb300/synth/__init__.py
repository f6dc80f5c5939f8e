"""Seeded synthetic multi-view scenes (input generator).

Holds none of the stereo method's arithmetic: it lays out planes, quads and
spheres from a seed, places pinhole cameras on an arc or a ring, and calls the
C ray caster (``scenegen.c``) for uint8 images and ground-truth depth/normal.
Every consumer -- the oracle tests, the CUDA parity tests and the benchmark --
draws its inputs from here.

Named workloads (sizes and structure of the paper's multi-view workloads):

``tiny``     160x120, 1 reference + 2 sources, two slanted planes with Perlin
             albedo, f = 150 px, cameras on a 15 degree arc.
``medium``   640x480, 1 + 5, three textured spheres over a slanted ground
             plane, depth 2..10, cameras on a 40 degree arc.
``large``    3200x2112, 1 + 10, multi-object scene with about 10 % textureless
             surface, per-view gain U(0.8, 1.2) and bias U(-0.2, 0.2) * 128.
``ring20``   20 cameras on a ring, every view a reference with its 10 nearest
             views as sources; 8 x 1920x1080, 6 x 2560x1440, 6 x 3200x2112.
``learned``  1600x1056, 1 + 10, multi-object scene whose layout depends on the
             seed (training and held-out scenes).
``fusion``   160x120, 5 cameras with ground truth in every view (fusion tests).
``many``     96x72, 1 + 32 cameras on a 60 degree arc (the largest source count).
"""
from __future__ import annotations

import ctypes
import math
import os
from dataclasses import dataclass, field

import numpy as np

_LIB = None
_LIB_PATH = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                         "_lib", "libscenegen.so")

SYN_PLANE, SYN_QUAD, SYN_SPHERE, SYN_SKY = 0, 1, 2, 3


class _Cam(ctypes.Structure):
    _fields_ = [("K", ctypes.c_double * 9), ("R", ctypes.c_double * 9),
                ("t", ctypes.c_double * 3), ("width", ctypes.c_int), ("height", ctypes.c_int)]


class _Prim(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("flat", ctypes.c_int),
                ("a", ctypes.c_double * 3), ("b", ctypes.c_double * 3), ("c", ctypes.c_double * 3),
                ("albedo", ctypes.c_double), ("tex_freq", ctypes.c_double),
                ("tex_amp", ctypes.c_double), ("tex_off", ctypes.c_double)]


def _lib():
    global _LIB
    if _LIB is None:
        if not os.path.exists(_LIB_PATH):
            from .. import _build
            _build.build()
        lib = ctypes.CDLL(_LIB_PATH)
        lib.syn_render_view.restype = ctypes.c_int
        lib.syn_render_view.argtypes = [
            ctypes.POINTER(_Cam), ctypes.POINTER(_Prim), ctypes.c_int, ctypes.POINTER(ctypes.c_int),
            ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
            ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        lib.syn_make_perm.argtypes = [ctypes.c_uint64, ctypes.POINTER(ctypes.c_int)]
        _LIB = lib
    return _LIB


@dataclass
class Camera:
    K: np.ndarray          # 3x3
    R: np.ndarray          # 3x3, x_cam = R X + t
    t: np.ndarray          # 3
    width: int
    height: int

    @property
    def centre(self) -> np.ndarray:
        return -self.R.T @ self.t


@dataclass
class Scene:
    name: str
    seed: int
    cams: list
    images: list                      # uint8 (H, W) per camera
    ref: int
    src: list
    depth_min: float
    depth_max: float
    gt_depth: dict = field(default_factory=dict)    # view -> float32 (H, W)
    gt_normal: dict = field(default_factory=dict)   # view -> float32 (H, W, 3)

    @property
    def width(self) -> int:
        return self.cams[self.ref].width

    @property
    def height(self) -> int:
        return self.cams[self.ref].height


def look_at(centre, target, up=(0.0, -1.0, 0.0)):
    """World-to-camera (R, t) of a camera at `centre` looking at `target`
    (camera x right, y down, z forward)."""
    c = np.asarray(centre, float)
    z = np.asarray(target, float) - c
    z /= np.linalg.norm(z)
    x = np.cross(np.asarray(up, float), z)
    x /= np.linalg.norm(x)
    y = np.cross(z, x)
    R = np.stack([x, y, z])
    return R, -R @ c


def intrinsics(width, height, f):
    return np.array([[f, 0.0, (width - 1) / 2.0], [0.0, f, (height - 1) / 2.0], [0.0, 0.0, 1.0]])


def _prim(kind, a, b=(0, 0, 0), c=(0, 0, 0), albedo=0.5, tex_freq=1.0, tex_amp=0.45,
          tex_off=0.0, flat=0):
    p = _Prim()
    p.kind, p.flat = kind, flat
    p.a[:], p.b[:], p.c[:] = list(map(float, a)), list(map(float, b)), list(map(float, c))
    p.albedo, p.tex_freq, p.tex_amp, p.tex_off = albedo, tex_freq, tex_amp, tex_off
    return p


def render(cams, prims, seed, *, gains=None, biases=None, ss=2, flat_freq=0.0,
           flat_thresh=1.0, flat_albedo=0.55, gt_views=()):
    """Ray-cast every camera; returns (images, gt_depth, gt_normal)."""
    lib = _lib()
    perm = (ctypes.c_int * 512)()
    lib.syn_make_perm(ctypes.c_uint64(seed), perm)
    parr = (_Prim * len(prims))(*prims)
    images, gd, gn = [], {}, {}
    for v, cam in enumerate(cams):
        cc = _Cam()
        cc.K[:] = list(cam.K.ravel())
        cc.R[:] = list(cam.R.ravel())
        cc.t[:] = list(cam.t.ravel())
        cc.width, cc.height = cam.width, cam.height
        img = np.empty((cam.height, cam.width), np.uint8)
        want = v in gt_views
        dep = np.empty((cam.height, cam.width), np.float32) if want else None
        nrm = np.empty((cam.height, cam.width, 3), np.float32) if want else None
        g = 1.0 if gains is None else float(gains[v])
        b = 0.0 if biases is None else float(biases[v])
        rc = lib.syn_render_view(ctypes.byref(cc), parr, len(prims), perm, flat_freq, flat_thresh,
                                 flat_albedo, g, b, ss, img.ctypes.data,
                                 dep.ctypes.data if want else None,
                                 nrm.ctypes.data if want else None)
        if rc != 0:
            raise RuntimeError("scene rendering failed (singular intrinsics)")
        images.append(img)
        if want:
            gd[v], gn[v] = dep, nrm
    return images, gd, gn


def _tex_freq(depth, f):
    # base noise period of about 24 px at this depth; the finest octave is ~3 px
    return 1.0 / (24.0 * depth / f)


def _arc_cams(n, width, height, f, radius, arc_deg, target=(0.0, 0.0, 0.0), height_off=0.0):
    cams = []
    for i in range(n):
        a = math.radians(-arc_deg / 2 + arc_deg * i / (n - 1)) if n > 1 else 0.0
        c = (target[0] + radius * math.sin(a), target[1] + height_off, target[2] - radius * math.cos(a))
        R, t = look_at(c, target)
        cams.append(Camera(intrinsics(width, height, f), R, t, width, height))
    return cams


def _centre_first(n):
    """Reference = middle camera, sources = the others sorted by distance."""
    ref = n // 2
    src = sorted([v for v in range(n) if v != ref], key=lambda v: (abs(v - ref), v))
    return ref, src


def scene_tiny(seed=1):
    W, H, f = 160, 120, 150.0
    cams = _arc_cams(3, W, H, f, radius=4.0, arc_deg=15.0)
    tf = _tex_freq(4.0, f)
    prims = [
        # left plane, turned 30 degrees about the vertical axis
        _prim(SYN_QUAD, a=(-0.9, 0, -0.3), b=(1.2 * math.cos(0.52), 0, 1.2 * math.sin(0.52)),
              c=(0, 2.5, 0), albedo=0.5, tex_freq=tf, tex_off=3.1),
        # back plane, tilted 25 degrees about the horizontal axis
        _prim(SYN_PLANE, a=(0, math.sin(0.44), -math.cos(0.44)), b=(1.2, 0, 0), albedo=0.5,
              tex_freq=tf, tex_off=11.7),
    ]
    ref, src = _centre_first(3)
    imgs, gd, gn = render(cams, prims, seed, gt_views=(ref,))
    return Scene("tiny", seed, cams, imgs, ref, src, 2.0, 8.0, gd, gn)


def scene_fusion(seed=6, n=5):
    """The tiny scene's two slanted planes seen by n cameras on a 20-degree
    arc, with ground-truth depth and normals for every view (depth-map fusion
    tests)."""
    W, H, f = 160, 120, 150.0
    cams = _arc_cams(n, W, H, f, radius=4.0, arc_deg=20.0)
    tf = _tex_freq(4.0, f)
    prims = [
        _prim(SYN_QUAD, a=(-0.9, 0, -0.3), b=(1.2 * math.cos(0.52), 0, 1.2 * math.sin(0.52)),
              c=(0, 2.5, 0), albedo=0.5, tex_freq=tf, tex_off=3.1),
        _prim(SYN_PLANE, a=(0, math.sin(0.44), -math.cos(0.44)), b=(1.2, 0, 0), albedo=0.5,
              tex_freq=tf, tex_off=11.7),
    ]
    ref, src = _centre_first(n)
    imgs, gd, gn = render(cams, prims, seed, gt_views=tuple(range(n)))
    return Scene("fusion", seed, cams, imgs, ref, src, 2.0, 8.0, gd, gn)


def scene_many(seed=7, n=33, width=96, height=72):
    """The tiny scene's two slanted planes seen by n cameras on a 60-degree
    arc at 96x72: the middle one is the reference, the other n - 1 its
    sources (n = 33 gives the largest source count, 32)."""
    f = 0.9 * width
    cams = _arc_cams(n, width, height, f, radius=4.0, arc_deg=60.0)
    tf = _tex_freq(4.0, f)
    prims = [
        _prim(SYN_QUAD, a=(-0.9, 0, -0.3), b=(1.2 * math.cos(0.52), 0, 1.2 * math.sin(0.52)),
              c=(0, 2.5, 0), albedo=0.5, tex_freq=tf, tex_off=3.1),
        _prim(SYN_PLANE, a=(0, math.sin(0.44), -math.cos(0.44)), b=(1.2, 0, 0), albedo=0.5,
              tex_freq=tf, tex_off=11.7),
    ]
    ref, src = _centre_first(n)
    imgs, gd, gn = render(cams, prims, seed, gt_views=(ref,))
    return Scene("many", seed, cams, imgs, ref, src, 2.0, 8.0, gd, gn)


def scene_medium(seed=2):
    W, H, f = 640, 480, 560.0
    cams = _arc_cams(6, W, H, f, radius=6.0, arc_deg=40.0, height_off=-0.8)
    rng = np.random.default_rng(seed)
    tf = _tex_freq(6.0, f)
    prims = [
        # slanted ground plane below the spheres
        _prim(SYN_PLANE, a=(0, -math.cos(0.2), math.sin(0.2)), b=(1.3, 0, 0), albedo=0.5,
              tex_freq=tf, tex_off=1.3),
        # back wall
        _prim(SYN_PLANE, a=(0, 0, -1), b=(3.0, 0, 0), albedo=0.45, tex_freq=tf * 0.8, tex_off=7.2),
    ]
    for i in range(3):
        r = rng.uniform(0.6, 1.0)
        c = (rng.uniform(-1.8, 1.8), 1.2 - r - rng.uniform(0, 0.3), rng.uniform(-1.5, 1.0))
        prims.append(_prim(SYN_SPHERE, a=c, b=(r, 0, 0), albedo=rng.uniform(0.4, 0.6),
                           tex_freq=tf * rng.uniform(0.9, 1.3), tex_off=rng.uniform(0, 50)))
    ref, src = _centre_first(6)
    imgs, gd, gn = render(cams, prims, seed, gt_views=(ref,))
    return Scene("medium", seed, cams, imgs, ref, src, 2.0, 10.0, gd, gn)


def _multi_object_prims(rng, tf, spread=2.5, n_spheres=4, n_boxes=4):
    prims = [
        _prim(SYN_PLANE, a=(0, -1, 0), b=(1.5, 0, 0), albedo=0.5, tex_freq=tf, tex_off=2.2),
        _prim(SYN_PLANE, a=(0, 0, -1), b=(4.0, 0, 0), albedo=0.5, tex_freq=tf * 0.8, tex_off=5.5),
    ]
    for _ in range(n_spheres):
        r = rng.uniform(0.35, 0.8)
        c = (rng.uniform(-spread, spread), 1.5 - r, rng.uniform(-1.5, 2.0))
        prims.append(_prim(SYN_SPHERE, a=c, b=(r, 0, 0), albedo=rng.uniform(0.35, 0.65),
                           tex_freq=tf * rng.uniform(0.8, 1.4), tex_off=rng.uniform(0, 50)))
    for _ in range(n_boxes):
        hw, hh, hd = rng.uniform(0.25, 0.6), rng.uniform(0.3, 0.9), rng.uniform(0.25, 0.6)
        cx, cz = rng.uniform(-spread, spread), rng.uniform(-1.5, 2.0)
        cy = 1.5 - hh
        yaw = rng.uniform(0, math.pi)
        ux = np.array([math.cos(yaw), 0, math.sin(yaw)])
        uz = np.array([-math.sin(yaw), 0, math.cos(yaw)])
        uy = np.array([0.0, 1.0, 0.0])
        ctr = np.array([cx, cy, cz])
        alb, off = rng.uniform(0.35, 0.65), rng.uniform(0, 50)
        for axis, h, (pa, ha), (pb, hb) in ((ux, hw, (uy, hh), (uz, hd)), (uz, hd, (ux, hw), (uy, hh)),
                                            (uy, hh, (ux, hw), (uz, hd))):
            for sgn in (-1, 1):
                prims.append(_prim(SYN_QUAD, a=ctr + sgn * h * axis, b=pa * ha, c=pb * hb, albedo=alb,
                                   tex_freq=tf * 1.1, tex_off=off))
    return prims


def scene_large(seed=3, width=3200, height=2112, n_src=10, name="large", arc_deg=30.0):
    f = 0.875 * width
    n = n_src + 1
    cams = _arc_cams(n, width, height, f, radius=7.0, arc_deg=arc_deg, height_off=-1.0)
    rng = np.random.default_rng(seed)
    tf = _tex_freq(7.0, f)
    prims = _multi_object_prims(rng, tf)
    gains = rng.uniform(0.8, 1.2, n)
    biases = rng.uniform(-0.2, 0.2, n) * 128.0
    ref, src = _centre_first(n)
    imgs, gd, gn = render(cams, prims, seed, gains=gains, biases=biases, flat_freq=0.9,
                          flat_thresh=0.28, flat_albedo=0.55, gt_views=(ref,))
    return Scene(name, seed, cams, imgs, ref, src, 2.0, 14.0, gd, gn)


def scene_learned(seed, width=1600, height=1056):
    return scene_large(seed=seed, width=width, height=height, name="learned")


RING20_SIZES = [(1920, 1080)] * 8 + [(2560, 1440)] * 6 + [(3200, 2112)] * 6


def ring20_layout(n=20):
    """Camera index -> size, interleaved around the ring so neighbours differ."""
    order = np.argsort((np.arange(n) * 7) % n, kind="stable")
    return [RING20_SIZES[int(i)] for i in order]


def scene_ring20(seed=4, n=20, n_src=10, sizes=None):
    rng = np.random.default_rng(seed)
    sizes = sizes or ring20_layout(n)
    cams = []
    radius = 7.0
    for i in range(n):
        a = 2 * math.pi * i / n
        c = (radius * math.sin(a), -1.2, -radius * math.cos(a))
        R, t = look_at(c, (0.0, 0.3, 0.0))
        w, h = sizes[i]
        cams.append(Camera(intrinsics(w, h, 0.875 * w), R, t, w, h))
    tf = _tex_freq(7.0, 0.875 * 1920)
    prims = _multi_object_prims(rng, tf, spread=1.5, n_spheres=3, n_boxes=3)
    del prims[1]   # no back wall inside a ring: a textured sky sphere instead
    prims.append(_prim(SYN_SKY, a=(0, 0, 0), b=(16.0, 0, 0), albedo=0.5, tex_freq=tf * 0.5, tex_off=9.0))
    imgs, gd, gn = render(cams, prims, seed)
    return Scene("ring20", seed, cams, imgs, 0, ring_sources(0, n, n_src), 1.0, 24.0, gd, gn)


def ring_sources(ref, n=20, n_src=10):
    """The n_src cameras nearest to `ref` along the ring (alternating sides)."""
    out = []
    for k in range(1, n):
        for s in (1, -1):
            v = (ref + s * k) % n
            if v != ref and v not in out:
                out.append(v)
    return out[:n_src]


SCENES = {"tiny": scene_tiny, "medium": scene_medium, "large": scene_large,
          "ring20": scene_ring20, "learned": scene_learned, "fusion": scene_fusion, "many": scene_many}


def make_scene(name: str, seed: int | None = None, cache_dir: str | None = None) -> Scene:
    """Build a named scene.  With ``cache_dir`` (or $AMH_SCENE_CACHE) the
    rendered scene is kept there as a pickle and reused."""
    cache_dir = cache_dir or os.environ.get("AMH_SCENE_CACHE")
    path = None
    if cache_dir:
        path = os.path.join(cache_dir, f"scene_{name}_{'default' if seed is None else seed}.pkl")
        if os.path.exists(path):
            import pickle
            with open(path, "rb") as f:
                return pickle.load(f)
    fn = SCENES[name]
    sc = fn() if seed is None else fn(seed)
    if path:
        import pickle
        os.makedirs(cache_dir, exist_ok=True)
        tmp = path + f".{os.getpid()}.tmp"
        with open(tmp, "wb") as f:
            pickle.dump(sc, f, protocol=pickle.HIGHEST_PROTOCOL)
        os.replace(tmp, path)
    return sc


def crop_scene(scene: Scene, x0: int, y0: int, w: int, h: int) -> Scene:
    """The same scene with the reference image cropped to (x0, y0, w, h): the
    reference intrinsics shift their principal point; sources stay whole."""
    cams = list(scene.cams)
    rc = scene.cams[scene.ref]
    K = rc.K.copy()
    K[0, 2] -= x0
    K[1, 2] -= y0
    cams[scene.ref] = Camera(K, rc.R, rc.t, w, h)
    imgs = list(scene.images)
    imgs[scene.ref] = np.ascontiguousarray(scene.images[scene.ref][y0:y0 + h, x0:x0 + w])
    gd = {k: (np.ascontiguousarray(v[y0:y0 + h, x0:x0 + w]) if k == scene.ref else v)
          for k, v in scene.gt_depth.items()}
    gn = {k: (np.ascontiguousarray(v[y0:y0 + h, x0:x0 + w]) if k == scene.ref else v)
          for k, v in scene.gt_normal.items()}
    return Scene(scene.name + "_crop", scene.seed, cams, imgs, scene.ref, list(scene.src),
                 scene.depth_min, scene.depth_max, gd, gn)
