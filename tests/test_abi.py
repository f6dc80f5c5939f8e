"""CPU checks of the C-ABI library: it builds for sm_103a, loads without a
GPU, exports every entry point include/*.h declares, and rejects invalid
arguments before touching the device."""
import ctypes
import glob
import os
import re
import subprocess

import numpy as np
import pytest

REPO = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def built():
    from paper_1805_07920_gb300 import _build
    outs = _build.build()
    assert all(os.path.exists(o) for o in outs)
    return outs


def _declared():
    names = []
    for h in glob.glob(os.path.join(REPO, "include", "*.h")):
        txt = open(h).read()
        names += re.findall(r"AMH_API\s+[\w\s\*]+?\b(amh\w+)\s*\(", txt)
    return sorted(set(names))


def _exported(path):
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    return {ln.split()[-1] for ln in out.splitlines() if ln.strip()}


def test_every_declared_symbol_is_exported(built):
    from paper_1805_07920_gb300 import amh
    decl = _declared()
    assert len(decl) >= 14
    exp = _exported(amh.LIB_PATH)
    missing = [d for d in decl if d not in exp]
    assert not missing, missing
    # and nothing but the declared C entry points is exported by the library
    ours = {e for e in exp if e.startswith("amh")}
    assert ours == set(decl), ours ^ set(decl)
    for name in amh.EXPORTS:
        assert name in decl


def test_library_loads_without_gpu(built):
    from paper_1805_07920_gb300 import amh
    L = amh.lib()
    for name in _declared():
        assert hasattr(L, name)


def test_default_params_are_the_papers(built):
    import json
    from paper_1805_07920_gb300 import amh
    g = json.load(open(os.path.join(REPO, "tests", "golden", "params_sec4.json")))
    p = amh.default_params()
    for k, v in g.items():
        if not k.startswith("_"):
            assert getattr(p, k) == pytest.approx(v, rel=1e-7), k


def _cams(n=3, W=16, H=12):
    from paper_1805_07920_gb300.synth import Camera, intrinsics
    return [Camera(intrinsics(W, H, 20.0), np.eye(3), np.array([0.1 * i, 0, 0]), W, H) for i in range(n)]


def _create(cams, images, ref, src, params=None, mem=0):
    from paper_1805_07920_gb300 import amh
    L = amh.lib()
    p = params or amh.default_params()
    carr = amh.make_cameras(cams)
    keep = [np.ascontiguousarray(i, np.uint8) if i is not None else None for i in images]
    ptrs = (ctypes.c_void_p * len(images))(*[(k.ctypes.data if k is not None else None) for k in keep])
    sarr = (ctypes.c_int32 * max(1, len(src)))(*src)
    ctx = ctypes.c_void_p()
    rc = L.amh_create(ctypes.byref(ctx), ctypes.byref(p), len(cams), carr, ptrs, mem, ref, sarr, len(src), None)
    return rc, L.amh_last_error(None).decode(), ctx


@pytest.mark.parametrize("case", ["n_src0", "n_src33", "src_is_ref", "src_repeat", "bad_ref", "bad_window",
                                  "bad_K", "null_image", "bad_mem", "bad_depth_range", "empty_image",
                                  "texture_f16", "texture_ablation"])
def test_invalid_arguments_rejected_on_host(built, case):
    from paper_1805_07920_gb300 import amh
    cams = _cams()
    imgs = [np.zeros((12, 16), np.uint8) for _ in cams]
    ref, src, p, mem = 0, [1, 2], amh.default_params(), 0
    if case == "n_src0":
        src = []
    elif case == "n_src33":
        cams, imgs = _cams(34), [np.zeros((12, 16), np.uint8)] * 34
        src = list(range(1, 34))
    elif case == "src_is_ref":
        src = [0, 1]
    elif case == "src_repeat":
        src = [1, 1]
    elif case == "bad_ref":
        ref = 5
    elif case == "bad_window":
        p.win_radius = 3
    elif case == "bad_K":
        cams[1].K = cams[1].K.copy()
        cams[1].K[2, 2] = 2.0
    elif case == "null_image":
        imgs[2] = None
    elif case == "bad_mem":
        mem = 7
    elif case == "bad_depth_range":
        p.depth_min, p.depth_max = 5.0, 1.0
    elif case == "empty_image":
        cams[2].width = 0
    elif case == "texture_f16":
        p.flags = amh.AMH_FLAG_TEXTURE_BILINEAR | amh.AMH_FLAG_IMAGES_F16
    elif case == "texture_ablation":
        p.flags = amh.AMH_FLAG_TEXTURE_BILINEAR | amh.AMH_FLAG_SYMMETRIC_PROPAGATION
    rc, msg, ctx = _create(cams, imgs, ref, src, p, mem)
    assert rc == amh.AMH_EINVAL, (rc, msg)
    assert msg and not ctx.value


def test_null_context_calls_fail_cleanly(built):
    from paper_1805_07920_gb300 import amh
    L = amh.lib()
    assert L.amh_init_random(None) == amh.AMH_EINVAL
    assert L.amh_step_phase(None, 0) == amh.AMH_EINVAL
    assert L.amh_iterate(None, 1) == amh.AMH_EINVAL
    assert L.amh_default_params(None) == amh.AMH_EINVAL
    assert L.amh_synchronize(None) == amh.AMH_EINVAL
    plane = (ctypes.c_float * 4)()
    assert L.amh_set_proposal(None, plane, 1, 1, 0) == amh.AMH_EINVAL
    L.amh_destroy(None)


def test_binding_has_no_cpu_fallback(tmp_path, monkeypatch):
    from paper_1805_07920_gb300 import amh
    monkeypatch.setattr(amh, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(amh, "_LIB", None)
    with pytest.raises(RuntimeError):
        amh.lib()


def test_create_without_a_device_fails_cleanly(built):
    """Valid arguments on a machine without a usable GPU: the first CUDA call
    of amh_create fails, the partial context is freed and the error comes
    back as a code and a message (no abort, no CPU path)."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1805_07920_gb300 import amh
    cams = _cams()
    imgs = [np.zeros((12, 16), np.uint8) for _ in cams]
    rc, msg, ctx = _create(cams, imgs, 0, [1, 2])
    assert rc in (amh.AMH_ECUDA, amh.AMH_ENOMEM), (rc, msg)
    assert "cuda" in msg.lower() and not ctx.value
    # and again: nothing left behind makes a second attempt behave differently
    rc2, msg2, ctx2 = _create(cams, imgs, 0, [1, 2])
    assert rc2 == rc and not ctx2.value


def test_post_processing_argument_errors_carry_a_message(built):
    from paper_1805_07920_gb300 import amh
    L = amh.lib()
    L.amh_last_error.restype = ctypes.c_char_p
    assert L.amh_median4(None, None, 4, 4, None) == amh.AMH_EINVAL
    assert b"amh_median4" in L.amh_last_error(None)
    assert L.amh_fuse(1, None, None, None, ctypes.c_float(0.3), ctypes.c_float(30.0), 2, None, None, None) == amh.AMH_EINVAL
    assert b"amh_fuse" in L.amh_last_error(None)

