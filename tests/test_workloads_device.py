"""The device-side source term used by the batch and serving benchmarks equals the
numpy source term it stands in for (both evaluate the same manufactured Laplacian)."""
import numpy as np
import pytest

import workloads as W


@pytest.mark.parametrize("which", ["batch2d", "serve3d"])
def test_source_term_device_matches_numpy(which):
    torch = pytest.importorskip("torch")
    if which == "batch2d":
        sp = W.batch_specs(1, seed=3, n_lo=64, n_hi=96)[0]
    else:
        sp = [s for _, s in W.serving_trace(40, seed=1, n3_lo=32, n3_hi=48, step=16) if s.dim == 3][0]
    n, d = sp.n, sp.dim
    ph = np.random.default_rng(0).random(n ** d) < 0.5
    ref = W.to_flat(W.source_term(sp, W.node_coords(n, d), W.from_flat(ph, n, d)))
    got = W.source_term_device(sp, torch.as_tensor(ph)).numpy()
    assert np.max(np.abs(ref - got)) <= 1e-13 * max(1.0, np.max(np.abs(ref)))
    assert np.all(got[~ph] == 0.0)
