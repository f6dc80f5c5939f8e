"""The per-pixel state is stored split by colour inside the library; every
call that takes or returns state uses row-major maps.  These tests check the
conversion both ways, from host and device memory, on odd and even widths
(where the two colours' runs of a row differ in length), and that a phase
leaves the other colour's entries untouched."""
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


def _random_state(rng, H, W):
    n = rng.normal(size=(H, W, 3))
    n /= np.linalg.norm(n, axis=-1, keepdims=True)
    plane = np.concatenate([n, rng.uniform(2.0, 8.0, (H, W, 1))], -1).astype(np.float32)
    return dict(plane=plane, cost=rng.uniform(0, 2, (H, W)).astype(np.float32),
                sel=rng.integers(0, 2**32, (H, W), dtype=np.uint64).astype(np.uint32),
                vbest=rng.integers(0, 256, (H, W)).astype(np.uint8),
                wmask=rng.integers(0, 2**32, (H, W), dtype=np.uint64).astype(np.uint32),
                choice=rng.integers(0, 16, (H, W)).astype(np.uint8))


@pytest.mark.parametrize("W,H", [(160, 120), (97, 61), (31, 17), (2, 3)])
def test_host_round_trip(amh, tiny_scene, synth_mod, W, H):
    sc = tiny_scene if (W, H) == (160, 120) else synth_mod.crop_scene(tiny_scene, 5, 7, W, H)
    g = amh.Context.from_scene(sc, seed=3)
    st = _random_state(np.random.default_rng(W * 1000 + H), H, W)
    g.set_state(st["plane"], st["cost"], st["sel"], st["vbest"], st["wmask"], st["choice"], t=4)
    back = g.get_state()
    assert back["t"] == 4
    for k in ("plane", "cost", "sel", "vbest", "wmask", "choice"):
        assert np.array_equal(back[k], st[k]), k
    maps = g.read_maps()
    assert np.array_equal(maps["depth"], st["plane"][..., 3])
    assert np.array_equal(maps["normal"], st["plane"][..., :3])
    assert np.array_equal(maps["cost"], st["cost"])
    assert np.array_equal(maps["selected"], st["wmask"])
    if H * W <= amh.NOALLOC_MAX_PIXELS:
        d = np.zeros(H * W, np.float32)
        nrm = np.zeros(3 * H * W, np.float32)
        g.read_maps_noalloc(d, nrm)
        assert np.array_equal(d, st["plane"][..., 3].ravel())
        assert np.array_equal(nrm, st["plane"][..., :3].ravel())
    g.close()


def test_device_round_trip(amh, tiny_scene, synth_mod):
    import torch
    sc = synth_mod.crop_scene(tiny_scene, 3, 2, 101, 77)
    g = amh.Context.from_scene(sc, seed=3)
    H, W = g.H, g.W
    st = _random_state(np.random.default_rng(7), H, W)
    dev = {k: torch.from_numpy(v.view(np.int32) if v.dtype == np.uint32 else v).cuda() for k, v in st.items()}
    g.set_state(dev["plane"], dev["cost"], dev["sel"], dev["vbest"], dev["wmask"], dev["choice"], t=2)
    out = {k: torch.empty_like(v) for k, v in dev.items()}
    assert g.get_state_device(out) == 2
    torch.cuda.synchronize()
    for k in st:
        got = out[k].cpu().numpy()
        if st[k].dtype == np.uint32:
            got = got.view(np.uint32)
        assert np.array_equal(got, st[k]), k
    g.close()


@pytest.mark.parametrize("W,H", [(97, 61), (160, 120)])
def test_phase_leaves_other_colour(amh, tiny_scene, synth_mod, W, H):
    """A phase of colour c rewrites exactly the pixels with (x + y) % 2 == c:
    the other colour's state comes back bit for bit (the split layout keeps
    the two colours' entries apart)."""
    sc = tiny_scene if (W, H) == (160, 120) else synth_mod.crop_scene(tiny_scene, 11, 13, W, H)
    g = amh.Context.from_scene(sc, seed=9)
    g.init_random()
    g.iterate(1)
    before = g.get_state()
    for colour in (0, 1):
        g.step_phase(colour)
        after = g.get_state()
        yy, xx = np.mgrid[0:H, 0:W]
        other = (xx + yy) % 2 != colour
        for k in ("plane", "cost", "sel", "vbest", "wmask", "choice"):
            assert np.array_equal(after[k][other], before[k][other]), (colour, k)
        # the updated colour was written (its winning-row codes are set again)
        assert (after["choice"][~other] <= 15).all()
        before = after
    g.close()
