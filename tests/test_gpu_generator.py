"""The GPU edge generator reproduces the numpy generator bit for bit (input module check)."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,E,gamma,max_deg", [(20_000, 100_000, 2.1, 2_000.0),
                                               (300_000, 3_000_000, 2.0, 60_000.0)])
def test_gpu_generator_equals_numpy(n, E, gamma, max_deg):
    import synth.gpu
    src, dst, meta = synth.gpu.chung_lu_undirected(n, E, gamma, 11, max_deg)
    want = synth.chung_lu_undirected(n, E, gamma, 11, max_deg)
    assert meta["edges"] == want.num_edges
    assert np.array_equal(src.cpu().numpy().view(np.uint64), want.src)
    assert np.array_equal(dst.cpu().numpy().view(np.uint64), want.dst)
