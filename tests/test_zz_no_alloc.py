"""amh_read_maps_noalloc: the map read-back for callers that cannot allocate
device memory when they read results (a pooling allocator that owns the GPU,
loops that must not allocate after start-up).  It is a blocking read, made
outside stream capture.  It must return exactly what amh_read_maps returns,
call after call, through the C-ABI, and leave the device's free memory
where it was.

Kept in a file of its own, collected last."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def amh():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_07920_gb300 import amh as m
    m.lib()
    return m


def _read_sliced(ctx, amh, n_total):
    depth = np.full(n_total, np.nan, np.float32)
    normal = np.full((n_total, 3), np.nan, np.float32)
    step = amh.NOALLOC_MAX_PIXELS
    for first in range(0, n_total, step):
        n = min(step, n_total - first)
        d = np.empty(n, np.float32)
        nm = np.empty((n, 3), np.float32)
        ctx.read_maps_noalloc(d, nm, first, n)
        depth[first:first + n] = d
        normal[first:first + n] = nm
    return depth, normal


@pytest.mark.parametrize("scene", ["tiny", "medium"])
def test_noalloc_read_matches_read_maps_twice(amh, synth_mod, scene):
    sc = synth_mod.make_scene(scene)
    g = amh.Context.from_scene(sc, seed=17)
    g.init_random()
    for call in range(2):           # two calls in a row, the state moving between them
        g.iterate(1)
        ref = g.read_maps()
        n = sc.width * sc.height
        depth, normal = _read_sliced(g, amh, n)
        np.testing.assert_array_equal(depth, ref["depth"].ravel(), err_msg=f"call {call}")
        np.testing.assert_array_equal(normal, ref["normal"].reshape(-1, 3), err_msg=f"call {call}")


def test_noalloc_partial_and_single_buffer(amh, synth_mod):
    sc = synth_mod.make_scene("tiny")
    g = amh.Context.from_scene(sc, seed=18)
    g.init_random()
    g.iterate(1)
    ref = g.read_maps()
    d = np.empty(1000, np.float32)
    g.read_maps_noalloc(d, None, 5000, 1000)
    np.testing.assert_array_equal(d, ref["depth"].ravel()[5000:6000])
    nm = np.empty((7, 3), np.float32)
    g.read_maps_noalloc(None, nm, sc.width * sc.height - 7, 7)
    np.testing.assert_array_equal(nm, ref["normal"].reshape(-1, 3)[-7:])


def test_noalloc_rejects_oversize_and_bad_ranges(amh, synth_mod):
    sc = synth_mod.make_scene("medium")       # 307200 pixels > the per-call maximum
    g = amh.Context.from_scene(sc, seed=19)
    g.init_random()
    n = sc.width * sc.height
    big = np.empty(n, np.float32)
    with pytest.raises(amh.AmhError) as e:
        g.read_maps_noalloc(big, None, 0, n)
    assert e.value.code == amh.AMH_EINVAL and "AMH_NOALLOC_MAX_PIXELS" in str(e.value)
    with pytest.raises(amh.AmhError):
        g.read_maps_noalloc(big[:10], None, n - 5, 10)
    with pytest.raises(amh.AmhError):
        g.read_maps_noalloc(None, None, 0, 10)
    # the context is still usable afterwards
    d = np.empty(10, np.float32)
    g.read_maps_noalloc(d, None, 0, 10)
    np.testing.assert_array_equal(d, g.read_maps()["depth"].ravel()[:10])


def test_noalloc_leaves_device_memory_unchanged(amh, synth_mod):
    """After a first call (which looks up the scratch array and may load the
    library's kernels), further calls change the device's free memory by
    nothing: no staging buffer is allocated."""
    import torch
    sc = synth_mod.make_scene("tiny")
    g = amh.Context.from_scene(sc, seed=20)
    g.init_random()
    g.iterate(1)
    n = sc.width * sc.height
    d = np.empty(n, np.float32)
    nm = np.empty((n, 3), np.float32)
    g.read_maps_noalloc(d, nm, 0, n)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(5):
        g.read_maps_noalloc(d, nm, 0, n)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    np.testing.assert_array_equal(d, g.read_maps()["depth"].ravel())


def test_noalloc_binding_checks_buffers(amh, synth_mod):
    """The binding refuses buffers the C call would overrun or misread."""
    sc = synth_mod.make_scene("tiny")
    g = amh.Context.from_scene(sc, seed=21)
    g.init_random()
    with pytest.raises(ValueError):
        g.read_maps_noalloc(np.empty(10, np.float64), None, 0, 10)         # wrong dtype
    with pytest.raises(ValueError):
        g.read_maps_noalloc(np.empty(9, np.float32), None, 0, 10)          # too short
    with pytest.raises(ValueError):
        g.read_maps_noalloc(None, np.empty((9, 3), np.float32), 0, 10)     # normals too short
    with pytest.raises(ValueError):
        g.read_maps_noalloc(np.empty((20, 2), np.float32)[:, 0], None, 0, 10)   # not contiguous
    d = np.empty(37, np.float32)
    g.read_maps_noalloc(d, None, 100)           # the count follows the buffer
    np.testing.assert_array_equal(d, g.read_maps()["depth"].ravel()[100:137])
