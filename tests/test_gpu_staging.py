"""The staged matrix sweep (AMH_FLAG_STAGED_FETCH, a measured alternative to
the default texture-only fetch path): from t = 1 on, per block and source
view a shared-memory box of bilinear cells (built from the texture unit's
gathers) serves the window samples of every warp whose windows fit in it;
the other samples use the texture unit.  The staged path is held to the
per-phase parity bar against the FP64 oracle for every image form, ablation
and ragged size, at t where the boxes carry samples; once the planes have
settled most evaluations must actually come from the boxes; the default path
reports none."""
import dataclasses

import numpy as np
import pytest

from parity_utils import FRACTION, phase_check

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def amh():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_07920_gb300 import amh as m
    m.lib()
    return m


def _settled_state(oracle_mod, sc, seed, oflags):
    o = oracle_mod.Oracle.from_scene(sc, seed=seed, flags=oflags)
    o.init_random()
    o.iterate(2)
    return o, o.get_state()


@pytest.mark.parametrize("form", ["u8", "f16", "squared", "symmetric", "heuristic"])
def test_staged_phase_parity(oracle_mod, amh, synth_mod, form):
    sc = synth_mod.crop_scene(synth_mod.make_scene("medium"), 180, 140, 200, 150)
    gflags = {"u8": 0, "f16": 0, "squared": amh.AMH_FLAG_BILATERAL_SQUARED,
              "symmetric": amh.AMH_FLAG_SYMMETRIC_PROPAGATION, "heuristic": amh.AMH_FLAG_HEURISTIC_VIEWS}[form]
    oflags = {"u8": 0, "f16": 0, "squared": oracle_mod.ORC_FLAG_SQUARED, "symmetric": oracle_mod.ORC_FLAG_SYMMETRIC,
              "heuristic": oracle_mod.ORC_FLAG_HEURISTIC}[form]
    if form == "f16":
        sc = dataclasses.replace(sc, images=[im.astype(np.float16) for im in sc.images])
    o, st = _settled_state(oracle_mod, sc, 50, oflags)
    g = amh.Context.from_scene(sc, seed=50, flags=gflags | amh.AMH_FLAG_STAGED_FETCH)
    bar = 0.99 if form == "squared" else FRACTION
    for t in (2, 4):
        st["t"] = t
        for color in (0, 1):
            g.pair_counts(reset=True)
            r = phase_check(o, g, st, color)
            tot, staged = g.pair_counts(reset=True)
            assert r["frac_ok_nontie"] >= bar, (form, t, color, r)
            assert staged > 0.1 * tot, (form, t, color, staged, tot)


@pytest.mark.parametrize("size", [(37, 23), (7, 5), (1, 9), (33, 17)])
def test_staged_ragged_sizes(oracle_mod, amh, synth_mod, size):
    w, h = size
    sc = synth_mod.crop_scene(synth_mod.make_scene("tiny"), 60, 40, w, h)
    o, st = _settled_state(oracle_mod, sc, 51, 0)
    g = amh.Context.from_scene(sc, seed=51, flags=amh.AMH_FLAG_STAGED_FETCH)
    for color in (0, 1):
        r = phase_check(o, g, st, color)
        assert r["frac_ok_nontie"] >= FRACTION, (size, color, r)


def test_boxes_carry_settled_samples(amh, synth_mod):
    """After two iterations on the 640x480 scene the boxes serve a large part
    of the evaluations of the next iteration (matrix, own plane and
    refinement together); at t = 0 and on the default path none."""
    sc = synth_mod.make_scene("medium")
    g = amh.Context.from_scene(sc, seed=52, flags=amh.AMH_FLAG_STAGED_FETCH)
    g.init_random()
    g.pair_counts(reset=True)
    g.iterate(1)
    tot0, staged0 = g.pair_counts(reset=True)
    g.iterate(1)
    g.pair_counts(reset=True)
    g.iterate(1)
    tot, staged = g.pair_counts(reset=True)
    print(f"\nstaged evaluations at t = 2: {staged} of {tot} ({staged / tot:.3f})")
    assert tot0 > 0 and staged0 == 0
    assert tot > 0 and staged / tot > 0.3, (staged, tot)
    t = amh.Context.from_scene(sc, seed=52)
    t.init_random()
    t.iterate(3)
    tot2, staged2 = t.pair_counts()
    assert tot2 > 0 and staged2 == 0
