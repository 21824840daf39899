"""The allocation-free rasteriser (for callers that cannot call cudaMalloc, such as
an application whose memory pool already holds the device's free memory).

Collected last on purpose: it checks lbm_em_rasterize_janus_noalloc through the C ABI
against lbm_em_rasterize_janus on two calls in a row (region ids must match bit for
bit, the bar every rasterisation test uses), and that an oversized request is refused
before anything is launched."""
import math

import numpy as np
import pytest

from paper_2509_22308_gb300 import lbm_em as L

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2509_22308_gb300 import build
    build.build()


def test_noalloc_rasteriser_matches_allocating_one_twice():
    specs = [(L.make_janus(40.5, math.radians(30.0), 2.0, 7.5), 300, 211),
             (L.make_janus(96.0, math.radians(135.0), 4.0, pec2=True), 512, 384)]
    for j, nx, ny in specs:                 # two calls in a row share the one array
        got = L.rasterize_janus_noalloc(j, nx, ny)
        ref = L.rasterize_janus(j, nx, ny)
        assert np.array_equal(got, ref)
        assert (got == 1).any() and (got == 2).any()


def test_noalloc_rejects_oversized_request():
    j = L.make_janus(10.0, 0.0, 2.0, 3.0)
    with pytest.raises(L.LbmEmError) as e:
        L.rasterize_janus_noalloc(j, 4096, 1025)   # 4096 * 1025 bytes > 4 MiB
    assert e.value.status == L.EINVAL
    # the largest allowed window still works and agrees
    got = L.rasterize_janus_noalloc(j, 4096, 1024)
    assert np.array_equal(got, L.rasterize_janus(j, 4096, 1024))
