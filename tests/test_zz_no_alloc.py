"""The allocation-free conservation sums (lbm_model_conserved_sums_noalloc) agree with
lbm_model_conserved_sums.

The entry point serves callers that cannot call cudaMalloc when they need the sums: hosts whose
device memory belongs to their own pool allocator or to a fixed budget, and diagnostics after an
out-of-memory error. Its reduction scratch is a static device array that
every call reuses, so the test calls it twice in a row, with a time step in between, and checks
that the second result is not contaminated by the first. This file is collected last and must
pass both alone in a fresh process and after the other GPU tests.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _model(lbm_lib):
    import torch  # noqa: F401
    from paper_2512_16230_gb300 import inputs as I
    from paper_2512_16230_gb300 import lbm
    from paper_2512_16230_gb300 import workloads as W
    spec = W.LATTICES["rD3Q53"]
    lat = lbm.Lattice(spec.kind, spec.c, spec.cs2, spec.free_w)
    n = (23, 17, 11)
    m = lbm.Model(lat, "nse", n, store="f64")
    m.set_relaxation(np.linspace(0.8, 1.7, spec.R), 1.1)
    m.set_force(0, 2, 1e-3, 0, 1.0)      # uniform force: the momentum sum changes every step
    m.set_populations(I.random_populations(n, lat.Q, seed=31))
    return lat, m


def test_noalloc_sums_match_the_allocating_entry_point(lbm_lib):
    import torch
    lat, m = _model(lbm_lib)
    out = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
    for _ in range(2):
        want = m.conserved_sums()
        m.conserved_sums_noalloc(out)
        m.synchronize()
        got = out.cpu().numpy()
        assert np.allclose(got[:4], want, rtol=1e-12, atol=1e-12), (got, want)
        m.step(1)
    # after the two calls the sums must have moved (the force changes the momentum)
    assert not np.allclose(m.conserved_sums()[1], want[1], rtol=1e-12, atol=1e-12)


def test_noalloc_rejects_bad_output(lbm_lib):
    from paper_2512_16230_gb300 import lbm
    lat, m = _model(lbm_lib)
    assert lbm.load().lbm_model_conserved_sums_noalloc(m.handle, None) == 1    # LBM_ERR_ARG
    assert lbm.load().lbm_model_conserved_sums_noalloc(None, None) == 1
    host = np.zeros(4)                                                          # host memory: rejected
    assert lbm.load().lbm_model_conserved_sums_noalloc(m.handle, host.ctypes.data) == 1
    assert np.all(host == 0.0)
