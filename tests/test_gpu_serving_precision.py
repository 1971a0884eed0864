"""Per-class error of the served reduced-precision flows against the FP64 oracle.

The serving mix (config 5) has nine flow classes: the 2D Taylor-Green vortex and the 2D nonlinear
convection-diffusion hill (App. A, Eq. (M-NCDE-6)) on rD2Q17 / rD2Q21 / rD2Q25 (Sec. 5), and the 3D
Kolmogorov flow forced through M2G on cubic rD3Q33 / rD3Q45 / rD3Q53 (App. D). Each class is run
with the served parameters (``workloads.serving_workload``) in FP32, FP16 and BF16 storage and
compared with the oracle at 200, 500 and 1000 steps: relative L2 of u (NSE) or phi (NCDE), and of
rho. The 16-bit rounding error grows with the run, so the serving policy stores a request as FP16
deviations only up to its class's threshold (``serve.F16_MAX_STEPS``); these tests check that the
FP16 error stays within the 1e-3 bound up to that threshold, on the oracle's grid and, against the
library's FP64 path (itself pinned to the oracle at 1e-12), on the largest served grids.
"""
import json
import os

import numpy as np
import pytest

from paper_2512_16230_gb300 import serve as S
from paper_2512_16230_gb300 import workloads as W

from _harness import gpu_model, rel_l2, workload_pair

pytestmark = pytest.mark.gpu

OUT = os.environ.get("LBM_PRECISION_REPORT")
GRID = {"tgv2d": (64, 48), "ncde": (64, 48), "kolmogorov": (16, 24, 16)}
LARGEST = {"tgv2d": (1024, 768), "ncde": (1024, 768), "kolmogorov": (160, 160, 160)}
CHECKPOINTS = (200, 500, 1000)
BOUND = 1e-3


@pytest.fixture(autouse=True)
def _lib(lbm_lib):
    return lbm_lib


def _report(key, value):
    if OUT:
        data = json.load(open(OUT)) if os.path.exists(OUT) else {}
        data[key] = value
        json.dump(data, open(OUT, "w"), indent=1)


def _gpu(wl, store):
    """The library model of a workload alone (no oracle: the grid is too large for it)."""
    gm = gpu_model(wl.lattice, wl.eq, wl.n, wl.s, wl.s_high, force=wl.force, u_const=wl.u_const,
                   nonlin=wl.nonlin, store=store)
    rho, u = wl.fields()
    gm.init_fields(rho, None if u is None else np.ascontiguousarray(u))
    return gm


def _errors(wl, om, gm):
    if wl.eq == "nse":
        r_g, u_g = gm.read_fields()
        r_o, u_o = om.fields() if hasattr(om, "fields") else om.read_fields()
        return {"u": rel_l2(u_g, u_o), "rho": rel_l2(r_g, r_o)}
    p_g, _ = gm.read_fields()
    p_o, _ = om.fields() if hasattr(om, "fields") else om.read_fields()
    return {"phi": rel_l2(p_g, p_o)}


@pytest.mark.parametrize("flow,lattice", S.SERVING_CLASSES)
def test_served_class_error_per_dtype(flow, lattice):
    """FP32, FP16 and BF16 storage of one served class against the FP64 oracle at 200, 500 and 1000
    steps. FP32 stays within 1e-4 on u (phi); FP16 within the 1e-3 bound at every checkpoint up to
    the class's FP16 threshold."""
    req = dict(rid=0, flow=flow, lattice=lattice, grid=GRID[flow], steps=CHECKPOINTS[-1], seed=7, store="16bit")
    wl = W.serving_workload(req, "f32")
    om, _ = workload_pair(wl, store="f32")
    models = {}
    for store in ("f32", "f16_dev", "bf16_dev"):
        _, models[store] = workload_pair(W.serving_workload(req, store), store=store)
    res, done = {}, 0
    for c in CHECKPOINTS:
        om.step(c - done)
        for gm in models.values():
            gm.step(c - done)
        done = c
        res[c] = {store: _errors(wl, om, gm) for store, gm in models.items()}
    for gm in models.values():
        gm.close()
    key = f"{flow}|{lattice}|{'x'.join(map(str, GRID[flow]))}"
    _report(key, res)
    print(key, json.dumps(res))
    main = "u" if wl.eq == "nse" else "phi"
    top = S.F16_MAX_STEPS[flow, lattice]
    for c in CHECKPOINTS:
        assert res[c]["f32"][main] <= 1e-4, (key, c, res[c])
        if c <= top:
            assert res[c]["f16_dev"][main] <= BOUND, (key, c, res[c])


@pytest.mark.parametrize("flow,lattice", S.SERVING_CLASSES)
def test_served_threshold_at_largest_grid(flow, lattice):
    """The FP16 threshold of each class on its largest served grid (1024 x 768 in 2D, 160^3 in 3D):
    FP16 storage against the library's FP64 path after F16_MAX_STEPS steps, within the bound."""
    steps = S.F16_MAX_STEPS[flow, lattice]
    if steps == 0:
        pytest.skip("the class is always served in FP32")
    req = dict(rid=0, flow=flow, lattice=lattice, grid=LARGEST[flow], steps=steps, seed=7, store="16bit")
    wl = W.serving_workload(req, "f64")
    ref, g16 = _gpu(wl, "f64"), _gpu(W.serving_workload(req, "f16_dev"), "f16_dev")
    ref.step(steps)
    g16.step(steps)
    err = _errors(wl, ref, g16)
    ref.close()
    g16.close()
    key = f"{flow}|{lattice}|{'x'.join(map(str, LARGEST[flow]))}|{steps}steps|f16_vs_gpu_f64"
    _report(key, err)
    print(key, json.dumps(err))
    assert err["u" if wl.eq == "nse" else "phi"] <= BOUND, (key, err)
