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


@pytest.mark.parametrize("store,bound", [("bf16_dev", 5e-2), ("f16_dev", 5e-3), ("f32", 1e-5)])
def test_taylor_green_3d_copy_per_dtype(store, bound):
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
    assert er <= bound


@pytest.mark.parametrize("store,bound", [("bf16_dev", 1e-2), ("f16_dev", 2e-3)])
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
