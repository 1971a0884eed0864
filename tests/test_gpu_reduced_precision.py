"""Reduced-precision storage: populations stored as BF16 / FP16 deviations f_i - w_i rho_ref,
collision in FP32 (the same kernels). Errors against the FP64 oracle, per dtype.

Bounds: storage rounds each deviation to 2^-9 (BF16) or 2^-12 (FP16) relative; the deviations of
a near-equilibrium flow are O(|u|/c_s) w_i, so one step perturbs u by a few 1e-4 (BF16) or a few
1e-5 (FP16) relative, and the bounds below allow the accumulation over the run.
"""
import json
import os

import numpy as np
import pytest

from paper_2512_16230_gb300 import inputs as I
from paper_2512_16230_gb300 import workloads as W

from _harness import gpu_model, oracle_model, rel_l2, workload_pair

pytestmark = pytest.mark.gpu

OUT = os.environ.get("LBM_PRECISION_REPORT")


@pytest.fixture(autouse=True)
def _lib(lbm_lib):
    return lbm_lib


def _report(key, value):
    if OUT:
        data = json.load(open(OUT)) if os.path.exists(OUT) else {}
        data[key] = value
        json.dump(data, open(OUT, "w"), indent=1)


@pytest.mark.parametrize("store,bound,rho_bound", [("bf16_dev", 6e-3, 3e-4), ("f16_dev", 1e-3, 5e-5),
                                                   ("f32", 1e-5, 1e-5)])
def test_taylor_green_3d_copy_per_dtype(store, bound, rho_bound):
    """Config 4 error study: the rD3Q53 Taylor-Green copy (48 x 48 x 36, Ma 0.3, Re 1600, 188 steps)
    with each storage dtype against the FP64 oracle: relative L2 of u and rho."""
    wl = W.taylor_green_3d(n=(48, 48, 36), steps=188)
    om, gm = workload_pair(wl, store=store)
    om.step(wl.steps)
    gm.step(wl.steps)
    r_g, u_g = gm.read_fields()
    r_o, u_o = om.fields()
    eu, er = rel_l2(u_g, u_o), rel_l2(r_g, r_o)
    _report(f"tgv3d_48x48x36_188steps_{store}", {"u_rel_l2": eu, "rho_rel_l2": er})
    print(f"{store}: u rel L2 {eu:.3e}, rho rel L2 {er:.3e}")
    assert eu <= bound
    assert er <= rho_bound


@pytest.mark.parametrize("store,bound", [("bf16_dev", 5e-3), ("f16_dev", 7e-4)])
def test_kolmogorov_serving_flow_per_dtype(store, bound):
    """A serving-mix flow (3D Kolmogorov on cubic rD3Q45 cells, forced through M2G) after 300
    steps: velocity error of reduced storage against the FP64 oracle."""
    wl = W.kolmogorov_3d(lattice="rD3Q45", n=(16, 24, 16), steps=300)
    om, gm = workload_pair(wl, store=store)
    om.step(wl.steps)
    gm.step(wl.steps)
    eu = rel_l2(gm.read_fields()[1], om.fields()[1])
    _report(f"kolmogorov3d_rD3Q45_16x24x16_300steps_{store}", {"u_rel_l2": eu})
    print(f"{store}: u rel L2 {eu:.3e}")
    assert eu <= bound


@pytest.mark.parametrize("store", ["bf16_dev", "f16_dev"])
def test_deviation_roundtrip(store):
    """set/get of populations through deviation storage: the deviation f - w rho_ref is rounded
    once to the storage format (relative 2^-8 for BF16, 2^-11 for FP16, FP16 subnormals below
    2^-14 absolute 2^-25), the rest is FP32 arithmetic."""
    spec = W.LATTICES["rD2Q25"]
    n = (37, 29)
    gm = gpu_model(spec, "nse", n, np.ones(spec.R), store=store)
    w = gm.lattice.tables["w"].reshape(-1, 1, 1)
    r = np.random.default_rng(3).uniform(-0.2, 0.2, size=(gm.Q,) + n[::-1])
    f0 = w * (1.0 + r)
    gm.set_populations(f0)
    got = gm.get_populations()
    dev = np.abs(f0 - w)
    rel, absl = (2.0 ** -8, 0.0) if store == "bf16_dev" else (2.0 ** -11, 2.0 ** -25)
    bound = rel * dev + absl + 2.0 ** -22 * np.abs(f0)
    assert np.all(np.abs(got - f0) <= bound)


def _round_bf16(x32):
    """float32 -> bfloat16 (round to nearest even) -> float64, on the host."""
    b = np.ascontiguousarray(x32, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = ((b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return b.view(np.float32).astype(np.float64)


def _stored_deviation(f, w, store):
    """The deviation the library stores for f: FP32 difference f - w rounded to the format."""
    dev32 = np.float32(f).astype(np.float32) - np.float32(w).astype(np.float32)
    if store == "f16_dev":
        return dev32.astype(np.float16).astype(np.float64)
    return _round_bf16(dev32)


@pytest.mark.parametrize("store,unit", [("bf16_dev", 2.0 ** -8), ("f16_dev", 2.0 ** -11)])
@pytest.mark.parametrize("name", ["rD2Q25", "rD3Q53"])
def test_deviation_storage_one_step(name, store, unit):
    """One collide-stream step in deviation storage: the kernel collides the deviations directly
    (reference moments added back, s_h rho_ref folded into h_0). Against the FP64 oracle from the
    same stored input, the error of the new deviations f - w is bounded by the rounding of the
    input and of the output (each <= unit relative), times the O(1) gain of the collision."""
    spec = W.LATTICES[name]
    d = spec.d
    n = (37, 29) if d == 2 else (13, 11, 9)
    s = np.random.default_rng(1).uniform(0.6, 1.9, spec.R)
    gm = gpu_model(spec, "nse", n, s, 1.3, store=store, force=(0, d - 1, 1e-3, 1, 0.2))
    om = oracle_model(spec, "nse", n, s, 1.3, force=(0, d - 1, 1e-3, 1, 0.2))
    w = om.lat.w.reshape((-1,) + (1,) * d)
    r = np.random.default_rng(5).uniform(-0.1, 0.1, size=(gm.Q,) + n[::-1])
    f_in = w * (1.0 + r)
    gm.set_populations(f_in)
    om.set_populations(w + _stored_deviation(f_in, w, store))   # the value the GPU holds
    gm.step(1)
    om.step(1)
    err = rel_l2(gm.get_populations() - w, om.f - w)
    print(f"{name} {store}: deviation rel L2 after one step {err:.2e}")
    assert err <= 4 * unit
