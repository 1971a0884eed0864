"""The row-staged gather of 16-bit deviation storage (lbm_model_set_gather "rows"): each CTA
moves the source x-rows of its row's populations into shared memory with bulk copies, reads the
pull sources (Eq. (2-2b)) there, and sends the collided row back with bulk copies.

Checks: propagation alone is bit-exact against the oracle's periodic shift (pure data movement,
every wrap in x, y and z, row lengths from 8 cells to the 256-cell pitch); a collide-stream
step gives bitwise the populations of the per-thread gather (same collision code, same inputs),
and one step stays within the 16-bit bounds of the FP64 oracle; the model extensions that read
neighbour fields (the M2G density gradient, the NCDE cross diffusion) agree bitwise too.
"""
import numpy as np
import pytest

from paper_2512_16230_gb300 import inputs as I
from paper_2512_16230_gb300 import workloads as W

from _harness import gpu_model, oracle_lattice, oracle_model, rel_l2

pytestmark = pytest.mark.gpu

# n_x a multiple of 8 (16-byte rows); the smallest extents make every pull wrap, n_x = 256 fills
# the row buffers
ROW_GRIDS = {2: [(8, 3), (48, 13), (256, 5)], 3: [(8, 2, 2), (24, 7, 5), (256, 3, 2)]}
LATTICES = ["rD2Q13", "rD2Q17", "rD2Q21", "rD2Q25", "rD2Q9", "rD3Q27", "rD3Q33", "rD3Q45", "rD3Q53"]
UNIT = {"bf16_dev": 2.0 ** -8, "f16_dev": 2.0 ** -11}


@pytest.fixture(autouse=True)
def _lib(lbm_lib):
    return lbm_lib


@pytest.mark.parametrize("store", ["f16_dev", "bf16_dev"])
@pytest.mark.parametrize("name", LATTICES)
def test_row_gather_stream_only_is_bit_exact(name, store):
    """Eq. (2-2b) alone through the row buffers: the same bits as the oracle's periodic shift of the
    stored state, on every grid of ROW_GRIDS."""
    spec = W.LATTICES[name]
    for n in ROW_GRIDS[spec.d]:
        gm = gpu_model(spec, "nse", n, np.ones(spec.R), store=store)
        gm.set_gather("rows")
        gm.set_populations(I.random_populations(n, gm.Q, seed=7))
        g0 = gm.get_populations()          # the stored (16-bit) state, decoded
        om = oracle_model(spec, "nse", n, np.ones(spec.R))
        om.set_populations(g0)
        gm.stream_only(3)
        om.stream_only(3)
        assert np.array_equal(gm.get_populations(), om.f), n
        gm.close()


def _step_kwargs(eq, d):
    if eq == "nse":
        return dict(s_high=1.3, cs2_eq=0.55, force=(0, d - 1, 3e-3, 1, 0.4))
    return dict(s_high=1.3, cs2_eq=0.55, u_const=tuple(np.linspace(0.03, 0.06, d)), nonlin=1.0)


def _near_equilibrium(w, n, Q, seed, eq):
    r = np.random.default_rng(seed).uniform(-0.1, 0.1, size=(Q,) + tuple(reversed(n)))
    base = 1.0 if eq == "nse" else 0.7
    return w.reshape((-1,) + (1,) * len(n)) * base * (1.0 + r)


@pytest.mark.parametrize("store", ["f16_dev", "bf16_dev"])
@pytest.mark.parametrize("eq", ["nse", "ncde"])
@pytest.mark.parametrize("name", LATTICES)
def test_row_gather_step_matches_thread_gather(name, eq, store):
    """Three collide-stream steps (NSE with a body force through M1F and M2G; NCDE with M1G and the
    nonlinear D(phi)) with random rates: the row-staged and the per-thread gather give bitwise the
    same populations; after the first step both are within the 16-bit bound of the FP64 oracle
    started from the same stored state (the input and output roundings, each <= one unit of the
    format relative to the deviation, times the O(1) gain of the collision)."""
    spec = W.LATTICES[name]
    d = spec.d
    n = ROW_GRIDS[d][1]
    s = np.random.default_rng(3).uniform(0.6, 1.9, spec.R)
    kw = _step_kwargs(eq, d)
    om = oracle_model(spec, eq, n, s, **kw)
    w = om.lat.w
    f0 = _near_equilibrium(w, n, om.lat.Q, 5, eq)
    out = {}
    for mode in ("rows", "threads"):
        gm = gpu_model(spec, eq, n, s, store=store, **kw)
        gm.set_gather(mode)
        gm.set_populations(f0)
        if mode == "rows":
            om.set_populations(gm.get_populations())     # the value the GPU holds
            om.step(1)
        gm.step(1)
        out[mode, 1] = gm.get_populations()
        gm.step(2)
        out[mode, 3] = gm.get_populations()
        gm.close()
    assert np.array_equal(out["rows", 1], out["threads", 1])
    assert np.array_equal(out["rows", 3], out["threads", 3])
    ref = w.reshape((-1,) + (1,) * d) * (1.0 if eq == "nse" else 0.0)
    err = rel_l2(out["rows", 1] - ref, om.f - ref)
    assert err <= 4 * UNIT[store], err


@pytest.mark.parametrize("store", ["f16_dev", "bf16_dev"])
def test_row_gather_with_gradient_terms(store):
    """The extensions that read neighbour cells besides the populations: the delta4 term of M2G on
    rD3Q27 (previous-step density at the 2d neighbours) and, on rD2Q13, the per-cell-rate NCDE with
    the mixed-derivative and cross-diffusion terms (psi at the neighbours): bitwise the same with
    both gathers over four steps."""
    cases = []
    spec = W.LATTICES["rD3Q27"]
    n = (24, 7, 5)
    cases.append((spec, "nse", n, dict(force=(0, 2, 2e-3, 1, 0.1)), lambda m: m.set_m2g_anisotropy(1)))
    spec2 = W.LATTICES["rD2Q13"]
    n2 = (48, 13)
    psi = I.random_scalar(n2, seed=2)

    def rate_cross(m):
        m.set_ncde_variant("rate", -0.2)
        m.set_ncde_cross_diffusion(0.02, psi)
    cases.append((spec2, "ncde", n2, dict(u_const=(0.03, 0.02), nonlin=1.0), rate_cross))
    for spec, eq, n, kw, extra in cases:
        s = np.random.default_rng(4).uniform(0.7, 1.8, spec.R)
        w = oracle_lattice(spec).w
        f0 = _near_equilibrium(w, n, len(w), 9, eq)
        res = {}
        for mode in ("rows", "threads"):
            gm = gpu_model(spec, eq, n, s, store=store, **kw)
            extra(gm)
            gm.set_gather(mode)
            gm.set_populations(f0)
            gm.step(4)
            res[mode] = gm.get_populations()
            gm.close()
        assert np.array_equal(res["rows"], res["threads"]), spec.kind


def test_row_gather_errors():
    """ROWS is refused where it does not apply (n_x not a multiple of 8, above the pitch, FP32
    storage) and a forced ROWS step with a kernel that has no row-staged form (per-order rates on
    the CUDA cores) reports LBM_ERR_NOT_IMPLEMENTED; nothing runs in either case."""
    from paper_2512_16230_gb300 import lbm
    spec = W.LATTICES["rD3Q53"]
    for n, store in (((37, 8, 8), "f16_dev"), ((264, 4, 4), "f16_dev"), ((16, 8, 8), "f32")):
        gm = gpu_model(spec, "nse", n, np.ones(spec.R), store=store)
        with pytest.raises(lbm.LBMError, match="LBM_ERR_ARG"):
            gm.set_gather("rows")
        gm.close()
    gm = gpu_model(spec, "nse", (16, 8, 8), np.ones(spec.R), store="f16_dev")
    gm.set_gather("rows")
    gm.set_tensor_cores(0)
    gm.set_high_rates([0.9, 1.2])       # per-order rates on the CUDA cores have no row-staged kernel
    with pytest.raises(lbm.LBMError, match="LBM_ERR_NOT_IMPLEMENTED"):
        gm.step(1)
    assert gm.counters() == (0, 0)
    assert lbm.load().lbm_model_set_gather(gm.handle, 7) == 1    # unknown mode: LBM_ERR_ARG


@pytest.mark.parametrize("store", ["f16_dev", "bf16_dev"])
@pytest.mark.parametrize("eq", ["nse", "ncde"])
@pytest.mark.parametrize("name", LATTICES)
def test_row_gather_tensor_cores_step(name, eq, store):
    """The row-staged kernel with the contractions on tcgen05 (A operands written into tensor memory
    by the threads): one step within the 16-bit bound of the FP64 oracle from the same stored state;
    after three steps bitwise the per-thread tcgen05 kernel (the same products on the same operands,
    A from shared memory there) and within the 16-bit bound of the CUDA-core row kernel."""
    spec = W.LATTICES[name]
    d = spec.d
    n = ROW_GRIDS[d][1]
    s = np.random.default_rng(3).uniform(0.6, 1.9, spec.R)
    kw = _step_kwargs(eq, d)
    om = oracle_model(spec, eq, n, s, **kw)
    w = om.lat.w
    f0 = _near_equilibrium(w, n, om.lat.Q, 5, eq)
    out = {}
    for mode, tensor in (("rows", 1), ("rows", 0), ("threads", 1)):
        gm = gpu_model(spec, eq, n, s, store=store, **kw)
        gm.set_gather(mode)
        gm.set_tensor_cores(tensor)
        gm.set_populations(f0)
        if mode == "rows" and tensor:
            om.set_populations(gm.get_populations())
            om.step(1)
        gm.step(1)
        out[mode, tensor, 1] = gm.get_populations()
        gm.step(2)
        out[mode, tensor, 3] = gm.get_populations()
        gm.synchronize()
        gm.close()
    ref = w.reshape((-1,) + (1,) * d) * (1.0 if eq == "nse" else 0.0)
    assert rel_l2(out["rows", 1, 1] - ref, om.f - ref) <= 4 * UNIT[store]
    assert np.array_equal(out["rows", 1, 3], out["threads", 1, 3])
    assert rel_l2(out["rows", 1, 3] - ref, out["rows", 0, 3] - ref) <= 4 * UNIT[store]


HIGH_RATES = {4: 0.8, 5: 1.35, 6: 1.6, 7: 0.9, 8: 1.25}


@pytest.mark.parametrize("store", ["f16_dev", "bf16_dev"])
@pytest.mark.parametrize("name", ["rD2Q13", "rD2Q25", "rD3Q33", "rD3Q45", "rD3Q53", "rD2Q9", "rD3Q27"])
def test_row_gather_tensor_cores_high_order_rates(name, store):
    """The full Q x Q collision with one rate per order >= 4 in the row-staged tensor-core kernel
    (the higher rows join both products): one step within the 16-bit bound of the FP64 oracle with
    the same per-order rates, and three steps bitwise the per-thread tcgen05 kernel."""
    spec = W.LATTICES[name]
    d = spec.d
    n = ROW_GRIDS[d][1]
    s = np.random.default_rng(31).uniform(0.6, 1.9, spec.R)
    kw = dict(s_high=1.2, force=(0, d - 1, 1e-3, 1, 0.2), s_orders=HIGH_RATES)
    om = oracle_model(spec, "nse", n, s, **kw)
    w = om.lat.w
    f0 = _near_equilibrium(w, n, om.lat.Q, 6, "nse")
    out = {}
    for mode in ("rows", "threads"):
        gm = gpu_model(spec, "nse", n, s, store=store, **kw)
        gm.set_gather(mode)
        gm.set_tensor_cores(1)
        gm.set_populations(f0)
        if mode == "rows":
            om.set_populations(gm.get_populations())
            om.step(1)
        gm.step(1)
        out[mode, 1] = gm.get_populations()
        gm.step(2)
        out[mode, 3] = gm.get_populations()
        gm.close()
    wr = w.reshape((-1,) + (1,) * d)
    assert rel_l2(out["rows", 1] - wr, om.f - wr) <= 4 * UNIT[store]
    assert np.array_equal(out["rows", 3], out["threads", 3])


@pytest.mark.parametrize("tensor", [0, 1])
def test_row_gather_timeout_is_reported(tensor):
    """The bounded waits of the row-staged kernels: with the test hook no row copy is issued, every
    CTA's wait on its first row buffer runs out, the status word reports LBM_ERR_TIMEOUT at the next
    synchronisation, and the model (and the context) keep working afterwards."""
    from paper_2512_16230_gb300 import lbm
    spec = W.LATTICES["rD3Q53"]
    n = (32, 12, 10)
    gm = gpu_model(spec, "nse", n, np.ones(spec.R), store="f16_dev")
    gm.init_fields(*I.rest_state(n, 3))
    gm.set_tensor_cores(tensor)
    assert lbm.load().lbm_model_set_gather(gm.handle, 3) == 0
    gm.step(1)
    with pytest.raises(lbm.LBMError, match="LBM_ERR_TIMEOUT"):
        gm.synchronize()
    gm.synchronize()                      # the status word was cleared
    gm.set_gather("rows")
    gm.init_fields(*I.rest_state(n, 3))
    gm.step(3)
    rho, u = gm.read_fields()
    assert np.allclose(rho, 1.0, atol=1e-3) and np.abs(u).max() < 1e-3
