"""Tensor-core (tcgen05) collide-stream kernel for 16-bit deviation storage.

The contractions with the integer monomial table run as matrix products with exact 16-bit
operands (the stored deviations and mono_k(e_i)) and FP32 accumulation; the back projection
splits the per-cell coefficients into a high and a low 16-bit part. Against the FP64 oracle fed
the stored deviations, one step must stay within the rounding of input and output, like the
CUDA-core kernel; over a flow the error must match the CUDA-core kernel's per-dtype bounds.
"""
import numpy as np
import pytest

from paper_2512_16230_gb300 import inputs as I
from paper_2512_16230_gb300 import workloads as W

from _harness import ALL_SPECS, RAGGED, gpu_model, oracle_model, rel_l2, workload_pair
from test_gpu_reduced_precision import _stored_deviation

pytestmark = pytest.mark.gpu

UNIT = {"bf16_dev": 2.0 ** -8, "f16_dev": 2.0 ** -11}


@pytest.fixture(autouse=True)
def _lib(lbm_lib):
    return lbm_lib


def _pair(name, eq, store, seed):
    spec = ALL_SPECS[name]
    d = spec.d
    n = RAGGED[d]
    s = np.random.default_rng(seed).uniform(0.6, 1.9, spec.R)
    kw = dict(s_high=1.3)
    if eq == "nse":
        kw["force"] = (0, d - 1, 1e-3, 1, 0.2)
    else:
        kw["u_const"] = tuple(np.linspace(0.03, 0.06, d))
        kw["nonlin"] = 1.0
    gm = gpu_model(spec, eq, n, s, store=store, **kw)
    om = oracle_model(spec, eq, n, s, **kw)
    return spec, n, gm, om


@pytest.mark.parametrize("store", ["f16_dev", "bf16_dev"])
@pytest.mark.parametrize("eq", ["nse", "ncde"])
@pytest.mark.parametrize("name", ["rD2Q13", "rD2Q17", "rD2Q25", "rD3Q33", "rD3Q45", "rD3Q53", "rD2Q9", "rD3Q27"])
def test_tensor_core_step_against_oracle(name, eq, store):
    """One step on tcgen05 from stored deviations: the new deviations f - w agree with the FP64
    oracle (fed the same stored values) within the rounding of input and output."""
    spec, n, gm, om = _pair(name, eq, store, 21)
    gm.set_tensor_cores(1)
    w = om.lat.w.reshape((-1,) + (1,) * spec.d)
    r = np.random.default_rng(5).uniform(-0.1, 0.1, size=(gm.Q,) + n[::-1])
    f_in = w * (1.0 + r)
    gm.set_populations(f_in)
    om.set_populations(w + _stored_deviation(f_in, w, store))
    gm.step(1)
    om.step(1)
    err = rel_l2(gm.get_populations() - w, om.f - w)
    print(f"{name} {eq} {store}: deviation rel L2 after one tensor-core step {err:.2e}")
    assert err <= 4 * UNIT[store]


@pytest.mark.parametrize("store", ["f16_dev", "bf16_dev"])
@pytest.mark.parametrize("name", ["rD2Q25", "rD3Q53"])
def test_tensor_core_matches_cuda_core_kernel(name, store):
    """The tensor-core and CUDA-core kernels compute the same FP32 collision up to summation
    order: after 5 steps from the same state the stored deviations differ by at most a few units
    in the last place of the 16-bit format."""
    spec, n, gm, _ = _pair(name, "nse", store, 3)
    spec, n, gc, _ = _pair(name, "nse", store, 3)
    gm.set_tensor_cores(1)
    w = gm.lattice.tables["w"].reshape((-1,) + (1,) * spec.d)
    f_in = w * (1.0 + np.random.default_rng(9).uniform(-0.05, 0.05, size=(gm.Q,) + n[::-1]))
    gm.set_populations(f_in)
    gc.set_populations(f_in)
    gm.step(5)
    gc.step(5)
    a, b = gm.get_populations() - w, gc.get_populations() - w
    scale = np.abs(b).max()
    assert np.abs(a - b).max() <= 8 * UNIT[store] * scale


@pytest.mark.parametrize("store,bound,rho_bound", [("f16_dev", 1e-3, 5e-5), ("bf16_dev", 6e-3, 3e-4)])
def test_tensor_core_taylor_green_copy(store, bound, rho_bound):
    """Config 4 with the contractions on tensor cores: the rD3Q53 Taylor-Green copy (48 x 48 x 36,
    188 steps) against the FP64 oracle, within the same per-dtype bounds as the CUDA-core kernel."""
    wl = W.taylor_green_3d(n=(48, 48, 36), steps=188)
    om, gm = workload_pair(wl, store=store)
    gm.set_tensor_cores(1)
    om.step(wl.steps)
    gm.step(wl.steps)
    r_g, u_g = gm.read_fields()
    r_o, u_o = om.fields()
    eu, er = rel_l2(u_g, u_o), rel_l2(r_g, r_o)
    print(f"{store} tensor cores: u rel L2 {eu:.3e}, rho rel L2 {er:.3e}")
    assert eu <= bound
    assert er <= rho_bound


HIGH_RATES = {4: 0.8, 5: 1.35, 6: 1.6, 7: 0.9, 8: 1.25}


def test_tensor_core_timeout_is_reported():
    """The bounded waits: with the test hook no matrix product is issued, every CTA's wait runs
    out, the status word reports LBM_ERR_TIMEOUT at the next synchronisation, and the model (and
    the context) keep working afterwards."""
    from paper_2512_16230_gb300 import lbm
    spec = W.LATTICES["rD2Q25"]
    n = (64, 48)
    gm = gpu_model(spec, "nse", n, np.ones(spec.R), store="f16_dev")
    gm.init_fields(*I.rest_state(n, 2))
    gm.set_tensor_cores(2)
    gm.step(1)
    with pytest.raises(lbm.LBMError, match="LBM_ERR_TIMEOUT"):
        gm.synchronize()
    gm.synchronize()                      # the status word was cleared
    gm.set_tensor_cores(1)
    gm.init_fields(*I.rest_state(n, 2))
    gm.step(3)
    rho, u = gm.read_fields()
    assert np.allclose(rho, 1.0, atol=1e-3) and np.abs(u).max() < 1e-3


def test_tensor_core_timeout_is_reported_fp32_high_rates():
    """The same hook on the FP32 kernel with per-order rates (the higher rows' operator on
    tcgen05): every wait runs out, LBM_ERR_TIMEOUT is reported, and the model steps correctly
    afterwards (rest state, per-order rates: a fixed point)."""
    from paper_2512_16230_gb300 import lbm
    spec = W.LATTICES["rD3Q33"]
    n = (16, 12, 10)
    gm = gpu_model(spec, "nse", n, np.ones(spec.R), s_high=1.2, store="f32", s_orders=HIGH_RATES)
    gm.init_fields(*I.rest_state(n, 3))
    gm.set_tensor_cores(2)
    gm.step(1)
    with pytest.raises(lbm.LBMError, match="LBM_ERR_TIMEOUT"):
        gm.synchronize()
    gm.synchronize()
    gm.set_tensor_cores(1)
    gm.init_fields(*I.rest_state(n, 3))
    gm.step(3)
    rho, u = gm.read_fields()
    assert np.allclose(rho, 1.0, atol=1e-6) and np.abs(u).max() < 1e-6


def test_tensor_cores_not_for_fp64():
    from paper_2512_16230_gb300 import lbm
    spec = W.LATTICES["rD2Q13"]
    gm = gpu_model(spec, "nse", (8, 8), np.ones(spec.R), store="f64")
    with pytest.raises(lbm.LBMError, match="LBM_ERR_ARG"):
        gm.set_tensor_cores(1)


@pytest.mark.parametrize("store", ["f16_dev", "bf16_dev"])
@pytest.mark.parametrize("name", ["rD2Q13", "rD2Q25", "rD3Q33", "rD3Q45", "rD3Q53", "rD2Q9", "rD3Q27"])
def test_tensor_core_high_order_rates_step(name, store):
    """The full Q x Q collision with one rate per order >= 4 on tcgen05 (the higher rows join both
    products): one step against the FP64 oracle with the same per-order rates, within the
    rounding of input and output."""
    spec = ALL_SPECS[name]
    d = spec.d
    n = RAGGED[d]
    s = np.random.default_rng(31).uniform(0.6, 1.9, spec.R)
    kw = dict(s_high=1.2, force=(0, d - 1, 1e-3, 1, 0.2), s_orders=HIGH_RATES)
    gm = gpu_model(spec, "nse", n, s, store=store, **kw)
    om = oracle_model(spec, "nse", n, s, **kw)
    gm.set_tensor_cores(1)
    w = om.lat.w.reshape((-1,) + (1,) * d)
    r = np.random.default_rng(6).uniform(-0.1, 0.1, size=(gm.Q,) + n[::-1])
    f_in = w * (1.0 + r)
    gm.set_populations(f_in)
    om.set_populations(w + _stored_deviation(f_in, w, store))
    gm.step(1)
    om.step(1)
    err = rel_l2(gm.get_populations() - w, om.f - w)
    print(f"{name} {store}: deviation rel L2 after one tensor-core step with per-order rates {err:.2e}")
    assert err <= 4 * UNIT[store]


def test_tensor_core_high_order_rates_flow():
    """A Taylor-Green flow (24 x 24 x 18 rD3Q53, Re 100) with per-order rates over 40 steps with
    FP16 deviations, where tcgen05 is the default kernel: velocity against the FP64 oracle within
    the FP16 bound."""
    wl = W.taylor_green_3d(n=(24, 24, 18), steps=40, re=100.0)
    spec = wl.lattice
    om = oracle_model(spec, wl.eq, wl.n, wl.s, wl.s_high, s_orders=HIGH_RATES)
    gm = gpu_model(spec, wl.eq, wl.n, wl.s, wl.s_high, store="f16_dev", s_orders=HIGH_RATES)
    rho, u = wl.fields()
    om.init_fields(rho, u)
    gm.init_fields(rho, u)
    om.step(wl.steps)
    gm.step(wl.steps)
    assert rel_l2(gm.read_fields()[1], om.fields()[1]) <= 1e-3


@pytest.mark.parametrize("store", ["f16_dev", "bf16_dev"])
@pytest.mark.parametrize("name", ["rD2Q9", "rD3Q27"])
def test_tensor_core_m2g_anisotropy_step(name, store):
    """The density-gradient term of Eq. (M2Ga) in the 16-bit tensor-core kernel: one step against
    the FP64 oracle fed the stored deviations (the previous-step density is the density of that
    state on both sides), within the rounding of input and output."""
    spec = ALL_SPECS[name]
    d = spec.d
    n = RAGGED[d]
    s = np.random.default_rng(41).uniform(0.6, 1.9, spec.R)
    kw = dict(s_high=1.3, force=(0, d - 1, 1e-3, 1, 0.2), m2g_aniso=True)
    gm = gpu_model(spec, "nse", n, s, store=store, **kw)
    om = oracle_model(spec, "nse", n, s, **kw)
    gm.set_tensor_cores(1)
    w = om.lat.w.reshape((-1,) + (1,) * d)
    r = np.random.default_rng(7).uniform(-0.1, 0.1, size=(gm.Q,) + n[::-1])
    f_in = w * (1.0 + r)
    gm.set_populations(f_in)
    om.set_populations(w + _stored_deviation(f_in, w, store))
    gm.step(1)
    om.step(1)
    err = rel_l2(gm.get_populations() - w, om.f - w)
    assert err <= 4 * UNIT[store]


@pytest.mark.parametrize("store", ["f16_dev", "bf16_dev"])
@pytest.mark.parametrize("name", ["rD2Q13", "rD2Q25", "rD3Q53"])
def test_tensor_core_ncde_cross_diffusion_step(name, store):
    """The cross-diffusion term of Eq. (GNCDE) in the 16-bit tensor-core kernel (psi rounded to
    FP32 on both sides): one step against the FP64 oracle fed the stored deviations."""
    from _harness import round_to_store
    spec = ALL_SPECS[name]
    d = spec.d
    n = RAGGED[d]
    s = np.random.default_rng(43).uniform(0.6, 1.9, spec.R)
    psi = round_to_store(I.random_scalar(n, seed=3), "f32")
    kw = dict(s_high=1.3, u_const=tuple(np.linspace(0.03, 0.06, d)), nonlin=1.0, a2=0.05, psi=psi)
    gm = gpu_model(spec, "ncde", n, s, store=store, **kw)
    om = oracle_model(spec, "ncde", n, s, **kw)
    gm.set_tensor_cores(1)
    w = om.lat.w.reshape((-1,) + (1,) * d)
    r = np.random.default_rng(8).uniform(-0.1, 0.1, size=(gm.Q,) + n[::-1])
    f_in = w * (1.0 + r)
    gm.set_populations(f_in)
    om.set_populations(w + _stored_deviation(f_in, w, store))
    gm.step(1)
    om.step(1)
    err = rel_l2(gm.get_populations() - w, om.f - w)
    assert err <= 4 * UNIT[store]
