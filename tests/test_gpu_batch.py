"""The batched form (several references, uneven sizes, one persistent launch
per colour phase, CUDA-graph replay, tile autotuning) through the C-ABI.

Every pixel's update depends only on its reference's state, so the batch must
reproduce single-reference contexts bit for bit (reference r draws with seed
+ r), whatever the tile variant and whether the launches are replayed from a
graph; and its phases are compared with the FP64 oracle directly
(test_batch_phases_match_oracle)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

KEYS = ("plane", "cost", "sel", "vbest", "wmask", "choice")


@pytest.fixture(scope="module")
def amh():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_07920_gb300 import amh as m
    m.lib()
    return m


@pytest.fixture(scope="module")
def ring(synth_mod):
    sizes = [(96, 64), (160, 120), (128, 96), (96, 64), (160, 120), (128, 96)]
    return synth_mod.scene_ring20(seed=9, n=6, n_src=3, sizes=sizes)


def _lists(ring, synth_mod, n=6, n_src=3):
    refs = list(range(n))
    return refs, [synth_mod.ring_sources(r, n, n_src) for r in refs]


def _single(amh, ring, r, src, seed, iters, flags=0):
    p = amh.default_params(depth_min=ring.depth_min, depth_max=ring.depth_max, seed=seed + r, flags=flags)
    g = amh.Context(ring.cams, ring.images, r, src, p)
    g.init_random()
    g.iterate(iters)
    return g.get_state()


def test_batch_equals_single_contexts(amh, ring, synth_mod):
    refs, srcs = _lists(ring, synth_mod)
    p = amh.default_params(depth_min=ring.depth_min, depth_max=ring.depth_max, seed=70)
    b = amh.Batch(ring.cams, ring.images, refs, srcs, p)
    b.init_random()
    b.iterate(2)
    for r in refs:
        s1 = _single(amh, ring, r, srcs[r], 70, 2)
        sb = b.get_state(r)
        assert sb["t"] == 2
        for k in KEYS:
            np.testing.assert_array_equal(sb[k], s1[k], err_msg=f"ref {r} {k}")


def test_batch_texture_form_equals_single_contexts(amh, ring, synth_mod):
    """The texture-filter precision form batched: bit for bit the single
    contexts of that form (those are parity-checked against the oracle's
    texture-unit sampling)."""
    refs, srcs = _lists(ring, synth_mod)
    f = amh.AMH_FLAG_TEXTURE_BILINEAR
    p = amh.default_params(depth_min=ring.depth_min, depth_max=ring.depth_max, seed=75, flags=f)
    b = amh.Batch(ring.cams, ring.images, refs, srcs, p)
    b.init_random()
    b.iterate(4)
    for r in refs:
        s1 = _single(amh, ring, r, srcs[r], 75, 4, flags=f)
        sb = b.get_state(r)
        for k in KEYS:
            np.testing.assert_array_equal(sb[k], s1[k], err_msg=f"ref {r} {k}")


def test_graph_replay_and_variants_agree(amh, ring, synth_mod):
    refs, srcs = _lists(ring, synth_mod)
    p = amh.default_params(depth_min=ring.depth_min, depth_max=ring.depth_max, seed=71)
    b = amh.Batch(ring.cams, ring.images, refs, srcs, p)
    b.init_random()
    b.iterate(3)
    ref_states = [b.get_state(r) for r in refs]
    for variant in range(amh.BATCH_VARIANTS):
        b.set_variant(variant)
        b.run(3)            # init + 3 iterations from a CUDA graph
        b.run(3)            # replayed
        b.synchronize()
        for r in refs:
            s = b.get_state(r)
            for k in KEYS:
                np.testing.assert_array_equal(s[k], ref_states[r][k], err_msg=f"variant {variant} ref {r} {k}")


def test_autotune_picks_a_variant(amh, ring, synth_mod):
    refs, srcs = _lists(ring, synth_mod)
    p = amh.default_params(depth_min=ring.depth_min, depth_max=ring.depth_max, seed=72)
    b = amh.Batch(ring.cams, ring.images, refs, srcs, p)
    chosen, ms = b.autotune(iters=1)
    assert chosen in range(amh.BATCH_VARIANTS) and len(ms) == amh.BATCH_VARIANTS
    assert all(m > 0 for m in ms) and ms[chosen] == min(ms)
    with pytest.raises(amh.AmhError):
        b.step_phase(0)     # the tuning run left no usable state
    b.init_random()
    b.iterate(1)
    s1 = _single(amh, ring, 0, srcs[0], 72, 1)
    np.testing.assert_array_equal(b.get_state(0)["plane"], s1["plane"])


def test_batch_rejects_bad_lists(amh, ring):
    with pytest.raises(amh.AmhError):
        amh.Batch(ring.cams, ring.images, [0, 1], [[1, 2], [1, 3]])   # ref 1 lists itself
    with pytest.raises(amh.AmhError):
        amh.Batch(ring.cams, ring.images, [0], [[]])                  # no source
    b = amh.Batch(ring.cams, ring.images, [0], [[1]])
    with pytest.raises(amh.AmhError):
        b.set_variant(amh.BATCH_VARIANTS)


@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4])
def test_batch_phases_match_oracle(amh, oracle_mod, synth_mod, variant):
    """The batched kernel against the FP64 oracle directly: three references
    of uneven, ragged sizes in one batch, each tile variant, the state first
    advanced by CUDA-graph replays (init + 1 iteration, built and replayed);
    then every colour phase at t = 1 and t = 4 is re-run by the oracle for
    each reference from the batch's own pre-phase state and compared pixel
    by pixel (same plane and |dcost| <= 1e-4 on >= 99.9 % of the non-tie
    pixels, view selection likewise)."""
    from parity_utils import FRACTION, phase_check_states
    sizes = [(97, 61), (160, 120), (130, 98), (97, 61), (160, 120), (130, 98)]
    ring = synth_mod.scene_ring20(seed=12, n=6, n_src=3, sizes=sizes)
    refs = [0, 1, 2]
    srcs = [synth_mod.ring_sources(r, 6, 3) for r in refs]
    seed = 90
    p = amh.default_params(depth_min=ring.depth_min, depth_max=ring.depth_max, seed=seed)
    b = amh.Batch(ring.cams, ring.images, refs, srcs, p)
    b.set_variant(variant)
    b.run(1)
    b.run(1)            # replayed: the same graph again from a fresh init
    b.synchronize()
    orcs = [oracle_mod.Oracle(ring.cams, ring.images, r, s,
                              oracle_mod.default_params(depth_min=ring.depth_min, depth_max=ring.depth_max,
                                                        seed=seed + r)) for r, s in zip(refs, srcs)]
    checked = 0
    for t in (1, 4):
        if t == 4:
            b.iterate(2)
        for color in (0, 1):
            pre = [b.get_state(i) for i in range(len(refs))]
            assert all(s["t"] == t for s in pre)
            b.step_phase(color)
            b.synchronize()
            for i in range(len(refs)):
                post = b.get_state(i)
                r = phase_check_states(orcs[i], pre[i], post, color)
                assert r["frac_ok_nontie"] >= FRACTION, (variant, t, color, refs[i], r)
                assert r["frac_sel"] >= FRACTION and r["frac_v"] >= FRACTION, (variant, t, color, refs[i], r)
                checked += r["n"]
    assert checked == 2 * sum(w * h for (w, h) in sizes[:3])
