"""Out-of-memory at context creation, injected on the host: with
AMH_FAIL_ALLOC_AT=k the k-th device allocation of amh_create reports an
out-of-memory error without allocating.  For every k the call must return
AMH_ENOMEM with a message, free what it had allocated (device memory back
where it was), and leave the library able to create a working context."""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
N_STATE_ALLOCS = 9       # reference, plane, cost, S, v, weight mask, choice, counters, status


@pytest.fixture(scope="module")
def amh():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_07920_gb300 import amh as m
    m.lib()
    return m


def test_injected_allocation_failures_clean_up(amh, synth_mod):
    import torch
    W, H, n = 2048, 2048, 3        # every allocation large enough that a leak shows
    rng = np.random.default_rng(0)
    cams = []
    for i in range(n):
        R, t = synth_mod.look_at((0.3 * i, 0.0, -5.0), (0.0, 0.0, 0.0))
        cams.append(synth_mod.Camera(synth_mod.intrinsics(W, H, 1800.0), R, t, W, H))
    imgs = [rng.integers(0, 256, (H, W), dtype=np.uint8) for _ in range(n)]
    p = amh.default_params(depth_min=2.0, depth_max=10.0)
    # a full run first: lazily loaded kernels and their local-memory
    # reservation claim device memory at the first launch, not at creation
    c = amh.Context(cams, imgs, 0, [1, 2], p)
    c.init_random()
    c.iterate(1)
    c.synchronize()
    c.close()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    n_allocs = N_STATE_ALLOCS + 2                           # + one texture array per source
    try:
        for k in range(1, n_allocs + 1):
            os.environ["AMH_FAIL_ALLOC_AT"] = str(k)
            with pytest.raises(amh.AmhError) as err:
                amh.Context(cams, imgs, 0, [1, 2], p)
            assert err.value.code == amh.AMH_ENOMEM, (k, str(err.value))
            assert "alloc" in str(err.value).lower() or "memory" in str(err.value).lower()
        os.environ["AMH_FAIL_ALLOC_AT"] = str(n_allocs + 1)   # past the last allocation: nothing fails
        c = amh.Context(cams, imgs, 0, [1, 2], p)
        c.init_random()
        c.iterate(1)
        c.synchronize()
        c.close()
    finally:
        del os.environ["AMH_FAIL_ALLOC_AT"]
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    # one leaked plane array alone would be 64 MB
    assert free0 - free1 < (8 << 20), (free0, free1)
