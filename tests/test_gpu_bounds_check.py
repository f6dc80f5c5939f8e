"""The bounds-checked build of the library (-DAMH_BOUNDS_CHECK): every index
the update computes into the state, the reference image or the proposals is
checked against its array and an out-of-range one is recorded in a status
word that amh_synchronize reports as AMH_EDEVICE.  Valid runs of every form
(uint8, FP16, texture filter, ablations, proposals, the batch) must report a
clean status and give bit for bit the normal build's states."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
REPO = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

RUN = r'''
import json, sys, numpy as np
sys.path.insert(0, {repo!r})
from paper_1805_07920_gb300 import amh, synth
amh.LIB_PATH = {lib!r}
L = amh.lib()
sc = synth.make_scene("tiny")
out = {{"checked": int(L.amh_bounds_checked())}}
cases = {{"u8": dict(flags=0), "texture": dict(flags=amh.AMH_FLAG_TEXTURE_BILINEAR),
         "symmetric": dict(flags=amh.AMH_FLAG_SYMMETRIC_PROPAGATION),
         "heuristic": dict(flags=amh.AMH_FLAG_HEURISTIC_VIEWS)}}
for name, kw in cases.items():
    c = amh.Context.from_scene(sc, seed=3, **kw)
    c.init_random()
    c.iterate(3)
    c.synchronize()
    st = c.get_state()
    out[name] = float(np.asarray(st["plane"], np.float64).sum()) + float(np.asarray(st["cost"], np.float64).sum())
    np.save({tmp!r} + "/" + name + ".npy", st["plane"])
c = amh.Context.from_scene(sc, seed=3, images=[im.astype(np.float16) for im in sc.images])
c.init_random(); c.iterate(2); c.synchronize()
np.save({tmp!r} + "/f16.npy", c.get_state()["plane"])
# a proposal on a grid smaller than the image (edge cells repeat)
c = amh.Context.from_scene(sc, seed=3)
c.init_random(); c.iterate(1)
prop = np.zeros((20, 30, 4), np.float32); prop[..., 2] = -1.0; prop[..., 3] = 4.0
amh.set_proposal(c, prop)
c.iterate(1); c.synchronize()
np.save({tmp!r} + "/prop.npy", c.get_state()["plane"])
ring = synth.scene_ring20(seed=9, n=4, n_src=2, sizes=[(96, 64), (64, 48), (96, 64), (64, 48)])
b = amh.Batch(ring.cams, ring.images, [0, 1, 2, 3], [synth.ring_sources(r, 4, 2) for r in range(4)],
              amh.default_params(depth_min=ring.depth_min, depth_max=ring.depth_max, seed=5))
b.init_random(); b.iterate(2); b.synchronize()
np.save({tmp!r} + "/batch.npy", np.concatenate([b.get_state(r)["plane"].ravel() for r in range(4)]))
print(json.dumps(out))
'''


def _run(lib, tmp):
    os.makedirs(tmp, exist_ok=True)
    r = subprocess.run([sys.executable, "-c", RUN.format(repo=REPO, lib=lib, tmp=str(tmp))],
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_bounds_checked_build_is_clean_and_identical(tmp_path):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sys.path.insert(0, REPO)
    from paper_1805_07920_gb300 import _build
    checked = _build.build(bounds_checked=True)[0]
    normal = os.path.join(os.path.dirname(checked), "libamh.so")
    a = _run(checked, tmp_path / "checked")      # every synchronize returned AMH_OK
    b = _run(normal, tmp_path / "normal")
    assert a["checked"] == 1 and b["checked"] == 0
    for name in ("u8", "texture", "symmetric", "heuristic", "f16", "prop", "batch"):
        np.testing.assert_array_equal(np.load(tmp_path / "checked" / f"{name}.npy"),
                                      np.load(tmp_path / "normal" / f"{name}.npy"), err_msg=name)
