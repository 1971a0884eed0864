"""GPU parity of the CUDA library (through its C ABI) against the FP64 oracle.

Tolerances: streaming and population I/O are data movement and must be bit-exact. The FP64 path
must agree with the oracle to <= 1e-12 relative (the oracle applies the full Q x Q matrix
Lambda = H^{-1} S H while the kernel uses the reduced Hermite form, so agreement is up to rounding
order; one collision differs by O(1e-15) and 200 steps stay well below 1e-12). The FP32 path must
agree to <= 1e-5 relative L2 (FP32 unit round-off 6e-8 times the O(10) condition of the moment
transforms, accumulated over the run).
"""
import math

import numpy as np
import pytest

from paper_2512_16230_gb300 import inputs as I
from paper_2512_16230_gb300 import workloads as W

from _harness import (ALL_SPECS, RAGGED, gpu_lattice, gpu_model, oracle_lattice, oracle_model, rel_l2, rel_max,
                      round_to_store, workload_pair)

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5}


@pytest.fixture(autouse=True)
def _lib(lbm_lib):
    return lbm_lib


def _monomials(d):
    return W.row_orders(d)


@pytest.mark.parametrize("name", sorted(ALL_SPECS))
def test_setup_tables_match_oracle(name):
    """The FP64 GPU set-up (weights by solving the moment equations, Hermite rows by weighted
    Gram-Schmidt) equals the oracle's closed-form weights and projected Hermite rows."""
    spec = ALL_SPECS[name]
    g = gpu_lattice(spec).tables
    o = oracle_lattice(spec)
    assert np.array_equal(g["e"], o.e)
    assert np.abs(g["w"] - o.w).max() <= 1e-14 * np.abs(o.w).max()
    assert np.abs(g["H"] - o.H).max() <= 1e-13 * np.abs(o.H).max()
    N_o = np.sum(o.w * o.H ** 2, axis=1)
    assert np.abs(g["N"] / N_o - 1).max() <= 1e-13
    assert np.array_equal(np.diag(g["T"]), np.ones(o.R))
    assert np.all(np.triu(g["T"], 1) == 0.0)


@pytest.mark.parametrize("store", ["f64", "f32"])
@pytest.mark.parametrize("name", ["rD2Q13", "rD2Q17", "rD2Q21", "rD2Q25", "rD3Q33", "rD3Q45", "rD3Q53"])
def test_stream_only_is_bit_exact(name, store):
    """Eq. (2-2b) alone: pure data movement, identical bits to the oracle's periodic shift."""
    spec = W.LATTICES[name]
    n = RAGGED[spec.d]
    om = oracle_model(spec, "nse", n, np.ones(spec.R))
    gm = gpu_model(spec, "nse", n, np.ones(spec.R), store=store)
    f0 = round_to_store(I.random_populations(n, om.lat.Q, seed=7), store)
    gm.set_populations(f0)
    assert np.array_equal(gm.get_populations(), f0)
    om.set_populations(f0)
    gm.stream_only(3)
    om.stream_only(3)
    assert np.array_equal(gm.get_populations(), om.f)


def _random_rates(R, seed):
    return np.random.default_rng(seed).uniform(0.6, 1.9, R)


@pytest.mark.parametrize("store", ["f64", "f32"])
@pytest.mark.parametrize("eq", ["nse", "ncde"])
@pytest.mark.parametrize("name", sorted(ALL_SPECS))
def test_one_collision_stream_step(name, eq, store):
    """One full step from far-from-equilibrium populations with random rates (NSE with a body
    force through M1F/M2G, NCDE with its M1G and nonlinear D(phi)), element by element."""
    spec = ALL_SPECS[name]
    d = spec.d
    n = RAGGED[d]
    s = _random_rates(spec.R, 3)
    kw = dict(s_high=1.3, cs2_eq=0.55)
    if eq == "nse":
        kw["force"] = (0, d - 1, 3e-3, 1, 0.4)
    else:
        kw["u_const"] = tuple(np.linspace(0.03, 0.06, d))
        kw["nonlin"] = 1.0
    om = oracle_model(spec, eq, n, s, **kw)
    gm = gpu_model(spec, eq, n, s, store=store, **kw)
    f0 = round_to_store(I.random_populations(n, om.lat.Q, seed=11), store)
    om.set_populations(f0)
    gm.set_populations(f0)
    om.step(1)
    gm.step(1)
    g = gm.get_populations()
    tol = TOL[store]
    assert rel_l2(g, om.f) <= tol
    assert rel_max(g, om.f) <= 10 * tol
    # a second step exercises phi^{n-1} (NCDE) and the post-collision state
    om.step(1)
    gm.step(1)
    assert rel_l2(gm.get_populations(), om.f) <= tol


@pytest.mark.parametrize("store", ["f64", "f32"])
@pytest.mark.parametrize("name", ["rD2Q25", "rD2Q13", "rD3Q53", "rD3Q33"])
def test_init_fields_and_readout(name, store):
    """Initialisation f-bar = f^eq (Eq. (feq-1)) and the field readout (Eq. (2-4-2))."""
    spec = W.LATTICES[name]
    d = spec.d
    n = RAGGED[d]
    rho, u = I.random_fields(n, d, seed=5)
    om = oracle_model(spec, "nse", n, np.ones(spec.R), force=(d - 1, 0, 1e-3, 2, 0.0))
    gm = gpu_model(spec, "nse", n, np.ones(spec.R), store=store, force=(d - 1, 0, 1e-3, 2, 0.0))
    om.init_fields(rho, u)
    gm.init_fields(rho, u)
    assert rel_max(gm.get_populations(), om.f) <= TOL[store]
    r_g, u_g = gm.read_fields()
    r_o, u_o = om.fields()
    assert rel_max(r_g, r_o) <= TOL[store]
    assert rel_max(u_g, u_o) <= 10 * TOL[store]


@pytest.mark.parametrize("name", ["rD2Q25", "rD2Q13", "rD3Q53", "rD3Q45"])
def test_conservation_sums(name):
    """FP64 global sums equal the oracle's; mass is conserved and momentum changes by sum F."""
    spec = W.LATTICES[name]
    d = spec.d
    n = RAGGED[d]
    force = (0, d - 1, 2e-3, 0, 1.0)    # uniform-in-x profile with non-zero mean
    om = oracle_model(spec, "nse", n, _random_rates(spec.R, 1), 1.2, force=force)
    gm = gpu_model(spec, "nse", n, _random_rates(spec.R, 1), 1.2, force=force, store="f64")
    f0 = I.random_populations(n, om.lat.Q, seed=2)
    om.set_populations(f0)
    gm.set_populations(f0)
    s0 = gm.conserved_sums()
    assert np.allclose(s0, om.conserved_sums(), rtol=1e-13, atol=1e-13)
    gm.step(4)
    om.step(4)
    s4 = gm.conserved_sums()
    assert np.allclose(s4, om.conserved_sums(), rtol=1e-12, atol=1e-12)
    assert abs(s4[0] / s0[0] - 1) < 1e-13
    F = om.force_field()
    for a in range(d):
        assert abs(s4[1 + a] - s0[1 + a] - 4 * F[a].sum()) < 1e-11
    assert np.array_equal(gm.conserved_sums(), s4)   # deterministic reduction order


def test_taylor_green_2d_config_fp64():
    """Config: rD2Q25 Taylor-Green, 64 x 48 (dy/dx = 4/3), Re = 100, FP64, 200 steps."""
    wl = W.taylor_green_2d()
    om, gm = workload_pair(wl, store="f64")
    om.step(wl.steps)
    gm.step(wl.steps)
    r_g, u_g = gm.read_fields()
    r_o, u_o = om.fields()
    assert rel_l2(r_g, r_o) <= 1e-12
    assert rel_l2(u_g, u_o) <= 1e-12
    assert rel_l2(gm.get_populations(), om.f) <= 1e-12


@pytest.mark.parametrize("store", ["f64", "f32"])
def test_ncde_config_reduced_size(store):
    """Config 2 at reduced size: rD2Q13 nonlinear CDE (dy/dx = 1.25), sigma = 20, noise 1e-3."""
    wl = W.ncde_hill(n=(96, 80), steps=150, store=store)
    om, gm = workload_pair(wl)
    om.step(wl.steps)
    gm.step(wl.steps)
    assert rel_l2(gm.read_fields()[0], om.fields()[0]) <= TOL[store]


def test_taylor_green_3d_copy_fp32():
    """Config 3 on its 48 x 48 x 36 copy (same Ma = 0.3 and Re = 1600, 188 steps = the same
    convective time as 1000 steps at 256 x 256 x 192): FP32 kernel against the FP64 oracle."""
    wl = W.taylor_green_3d(n=(48, 48, 36), steps=188)
    om, gm = workload_pair(wl, store="f32")
    om.step(wl.steps)
    gm.step(wl.steps)
    r_g, u_g = gm.read_fields()
    r_o, u_o = om.fields()
    assert rel_l2(u_g, u_o) <= 1e-5
    assert rel_l2(r_g, r_o) <= 1e-5


@pytest.mark.parametrize("name", ["rD2Q13", "rD2Q25", "rD3Q33", "rD3Q53"])
def test_minimal_grid_wraps(name):
    """Smallest allowed grid (every extent equal to the largest velocity component): every pull
    wraps around the periodic box."""
    spec = W.LATTICES[name]
    rm = 3 if spec.kind in ("rD2Q17", "rD2Q21", "rD2Q25") else 2
    n = (rm,) * spec.d
    s = _random_rates(spec.R, 9)
    om = oracle_model(spec, "nse", n, s, 1.1)
    gm = gpu_model(spec, "nse", n, s, 1.1, store="f64")
    f0 = I.random_populations(n, om.lat.Q, seed=4)
    om.set_populations(f0)
    gm.set_populations(f0)
    om.step(3)
    gm.step(3)
    assert rel_l2(gm.get_populations(), om.f) <= 1e-12


def test_invalid_arguments_are_rejected():
    """Bad arguments return an error status on the host; no kernel runs."""
    from paper_2512_16230_gb300 import lbm
    spec = W.LATTICES["rD3Q53"]
    lat = gpu_lattice(spec)
    with pytest.raises(lbm.LBMError, match="LBM_ERR_ARG"):
        lbm.Model(lat, "nse", (1, 8, 8))
    with pytest.raises(lbm.LBMError, match="LBM_ERR_ARG"):        # 2^31 cells: rejected before any allocation
        lbm.Model(lat, "nse", (2048, 2048, 512))
    # the largest accepted cell count is 2^31 - 2^21 (checked without allocating: workspace_bytes)
    assert 1024 * 1024 * 2046 == 2 ** 31 - 2 ** 21
    assert lbm.workspace_bytes(lat, "nse", (1024, 1024, 2046), "f16_dev") > 0
    with pytest.raises(lbm.LBMError, match="LBM_ERR_ARG"):
        lbm.workspace_bytes(lat, "nse", (1024, 1024, 2047), "f16_dev")
    with pytest.raises(lbm.LBMError, match="LBM_ERR_ARG"):
        lbm.Lattice("rD3Q53", spec.c, spec.cs2, ())
    with pytest.raises(lbm.LBMError, match="LBM_ERR_ARG"):
        lbm.Lattice("rD2Q13", (1.0, -1.0), (0.8, 0.8))
    m = lbm.Model(lat, "nse", (8, 8, 8))
    with pytest.raises(lbm.LBMError, match="LBM_ERR_ARG"):
        m.set_relaxation(np.full(20, 2.5))
    with pytest.raises(lbm.LBMError, match="LBM_ERR_ARG"):
        m.set_force(0, 5, 1.0, 1)
    m.step(0)
    assert m.counters() == (0, 0)


def test_infeasible_lattice_is_reported():
    """rD2Q13 outside 1/3 < d0 < 1 (Eq. (Q13lattice)): a Hermite norm is not positive."""
    from paper_2512_16230_gb300 import lbm
    with pytest.raises(lbm.LBMError, match="LATTICE_INFEASIBLE"):
        lbm.Lattice("rD2Q13", (1.0, 1.0), (0.2, 0.2))
    # rD3Q53 on dz/dx = 4/3 with one shared sound speed: the corrected H_zzz has N < 0
    spec = W.RD3Q53_SHARED_CS
    with pytest.raises(lbm.LBMError, match="LATTICE_INFEASIBLE"):
        lbm.Lattice(spec.kind, spec.c, spec.cs2, spec.free_w)


def test_steps_are_deterministic():
    spec = W.LATTICES["rD3Q53"]
    n = RAGGED[3]
    runs = []
    for _ in range(2):
        gm = gpu_model(spec, "nse", n, _random_rates(spec.R, 5), store="f32")
        gm.set_populations(round_to_store(I.random_populations(n, 53, seed=1), "f32"))
        gm.step(5)
        runs.append((gm.get_populations(), gm.conserved_sums()))
    assert np.array_equal(runs[0][0], runs[1][0])
    assert np.array_equal(runs[0][1], runs[1][1])


@pytest.mark.parametrize("store", ["f64", "f32"])
@pytest.mark.parametrize("name", ["rD2Q25", "rD2Q13", "rD3Q53", "rD3Q45", "rD3Q53-aniso", "rD2Q9", "rD3Q27"])
def test_bulk_viscosity_step(name, store):
    """Independent bulk viscosity (Eq. (4-27), k = 0): the normal second-order block of S couples
    the rows through s_b, also inside (I - S2/2) M2G (body force on)."""
    spec = ALL_SPECS[name]
    d = spec.d
    n = RAGGED[d]
    s = _random_rates(spec.R, 8)
    kw = dict(s_high=1.2, force=(d - 1, 0, 2e-3, 1, 0.1), s_bulk=0.9)
    om = oracle_model(spec, "nse", n, s, **kw)
    gm = gpu_model(spec, "nse", n, s, store=store, **kw)
    f0 = round_to_store(I.random_populations(n, om.lat.Q, seed=21), store)
    om.set_populations(f0)
    gm.set_populations(f0)
    om.step(2)
    gm.step(2)
    assert rel_l2(gm.get_populations(), om.f) <= TOL[store]


def _order_projectors(H, orders, w):
    """W H_k^T (H_k W H_k^T)^-1 H_k for every order k of the given rows (any basis of a block)."""
    out = {}
    for k in sorted(set(orders)):
        Hk = H[[r for r, o in enumerate(orders) if o == k]]
        out[k] = (w[:, None] * Hk.T) @ np.linalg.solve((Hk * w) @ Hk.T, Hk)
    return out


@pytest.mark.parametrize("name", sorted(ALL_SPECS))
def test_high_rows_match_oracle_blocks(name):
    """The GPU set-up completes the Hermite matrix with graded rows of order >= 4. Any basis of an
    order block gives the same collision, so the comparison is of the W-projector of each order,
    against the oracle's full matrix (built by its own selection and orthogonalisation)."""
    spec = ALL_SPECS[name]
    glat = gpu_lattice(spec)
    hi = glat.query_high()
    olat = oracle_lattice(spec)
    R = olat.R
    assert len(hi["orders"]) == olat.Q - R
    assert sorted(hi["orders"]) == sorted(olat.full_orders[R:])
    assert np.allclose(hi["N"], np.einsum("ri,i,ri->r", hi["H"], glat.tables["w"], hi["H"]), rtol=1e-12, atol=0)
    Pg = _order_projectors(hi["H"], list(hi["orders"]), glat.tables["w"])
    Po = _order_projectors(olat.Hfull[R:], olat.full_orders[R:], olat.w)
    for k in Po:
        assert np.abs(Pg[k] - Po[k]).max() < 1e-10, k
    # W-orthogonal to the rows of order <= 3 and to each other (the kernel divides by N_r row by row)
    w = glat.tables["w"]
    G = (hi["H"] * w) @ glat.tables["H"].T
    assert np.abs(G).max() < 1e-12 * np.sqrt(np.abs(hi["N"])).max() * np.sqrt(glat.tables["N"]).max()
    Gh = (hi["H"] * w) @ hi["H"].T
    sc = np.sqrt(np.abs(np.diag(Gh)))
    assert np.abs(Gh / np.outer(sc, sc) - np.eye(len(sc))).max() < 1e-12


def test_high_rows_need_nonzero_weights():
    """With w45 = 0 the eight (+-2)^3 velocities of rD3Q53 carry no weight, so a higher row living on
    them has zero W-norm: the lattice builds, but distinct higher-order rates are refused."""
    from paper_2512_16230_gb300 import lbm
    lat = lbm.Lattice("rD3Q53", (1.0, 1.0, 1.0), (0.6, 0.6, 0.6), (0.0,))
    with pytest.raises(lbm.LBMError, match="LATTICE_INFEASIBLE"):
        lat.query_high()
    m = lbm.Model(lat, "nse", (4, 4, 4), store="f64")
    m.set_high_rates([])                 # shared rate: nothing to refuse
    with pytest.raises(lbm.LBMError, match="LATTICE_INFEASIBLE"):
        m.set_high_rates([1.3])


HIGH_RATES = {4: 0.8, 5: 1.35, 6: 1.6, 7: 0.9, 8: 1.25}


@pytest.mark.parametrize("store,tensor", [("f64", 0), ("f32", 0), ("f32", 1)])
@pytest.mark.parametrize("name", ["rD2Q25", "rD2Q17", "rD2Q13", "rD3Q53", "rD3Q45", "rD3Q33", "rD3Q53-aniso",
                                  "rD2Q9", "rD3Q27"])
def test_high_order_rates_step(name, store, tensor):
    """The full Q x Q collision with one rate per order >= 4 against the oracle's
    Lambda = H^{-1} S H with the same per-order rates, body force on: the CUDA-core kernel with
    explicit higher rows (tensor = 0) and, on FP32, the higher rows on tcgen05 as FP16 high/low
    splits next to the CUDA-core reduced form (tensor = 1, the default with per-order rates)."""
    spec = ALL_SPECS[name]
    d = spec.d
    n = RAGGED[d]
    s = _random_rates(spec.R, 9)
    kw = dict(s_high=1.15, force=(d - 1, 0, 2e-3, 1, 0.1), s_orders=HIGH_RATES)
    om = oracle_model(spec, "nse", n, s, **kw)
    gm = gpu_model(spec, "nse", n, s, store=store, **kw)
    if store != "f64":
        gm.set_tensor_cores(tensor)
    f0 = round_to_store(I.random_populations(n, om.lat.Q, seed=23), store)
    om.set_populations(f0)
    gm.set_populations(f0)
    om.step(2)
    gm.step(2)
    assert rel_l2(gm.get_populations(), om.f) <= TOL[store]


@pytest.mark.parametrize("store", ["f32", "f16_dev"])
def test_high_order_rates_flow(store):
    """A Taylor-Green flow on rD3Q53 with distinct higher-order rates over 40 steps: the explicit
    rows also work on deviation storage (the reference state has no moment of order >= 4)."""
    wl = W.taylor_green_3d(n=(24, 24, 18), steps=40, re=100.0)
    spec = wl.lattice
    kw = dict(force=wl.force, u_const=wl.u_const, nonlin=wl.nonlin, s_orders=HIGH_RATES)
    om = oracle_model(spec, wl.eq, wl.n, wl.s, wl.s_high, **kw)
    gm = gpu_model(spec, wl.eq, wl.n, wl.s, wl.s_high, store=store, **kw)
    rho, u = wl.fields()
    om.init_fields(rho, u)
    gm.init_fields(rho, u)
    om.step(wl.steps)
    gm.step(wl.steps)
    eu = rel_l2(gm.read_fields()[1], om.fields()[1])
    assert eu <= (1e-5 if store == "f32" else 1e-3)


NCDE_VARIANTS = [("moment", 0.7), ("rate", 0.0), ("rate", -0.5), ("cde", 0.0)]


@pytest.mark.parametrize("store", ["f64", "f32"])
@pytest.mark.parametrize("variant,a1", NCDE_VARIANTS)
@pytest.mark.parametrize("name", ["rD2Q13", "rD2Q25", "rD3Q33", "rD3Q53"])
def test_ncde_variant_steps(name, variant, a1, store):
    """App. A variants against the oracle from far-from-equilibrium populations over three steps
    (so that phi^{n-1} enters): the mixed-derivative term a1 of Eq. (GNCDE), the per-cell rates
    s1(phi) and the diffusion-based CDE with its local-gradient source S_G."""
    spec = ALL_SPECS[name]
    d = spec.d
    n = RAGGED[d]
    s = _random_rates(spec.R, 13)
    kw = dict(s_high=1.2, u_const=tuple(np.linspace(0.04, 0.08, d)), nonlin=0.0 if variant == "cde" else 1.0,
              ncde_mode=variant, a1=a1)
    om = oracle_model(spec, "ncde", n, s, **kw)
    gm = gpu_model(spec, "ncde", n, s, store=store, **kw)
    f0 = round_to_store(I.random_populations(n, om.lat.Q, seed=17), store)
    om.set_populations(f0)
    gm.set_populations(f0)
    for _ in range(3):
        om.step(1)
        gm.step(1)
        assert rel_l2(gm.get_populations(), om.f) <= TOL[store]
    phi_g, _ = gm.read_fields()
    phi_o, _ = om.fields()
    assert rel_l2(phi_g, phi_o) <= TOL[store]


@pytest.mark.parametrize("variant", ["rate", "cde"])
def test_ncde_variant_hill_flow(variant):
    """A Gaussian hill (config 2 in miniature, 96 x 80 rD2Q13, FP32) over 300 steps in the rate and
    CDE variants: phi against the FP64 oracle."""
    spec = W.LATTICES["rD2Q13"]
    n = (96, 80)
    s = np.ones(spec.R)
    s[1:3] = 1.6
    kw = dict(u_const=(0.02, 0.01), nonlin=0.0 if variant == "cde" else 1.0, ncde_mode=variant)
    om = oracle_model(spec, "ncde", n, s, **kw)
    gm = gpu_model(spec, "ncde", n, s, store="f32", **kw)
    phi0 = I.gaussian_hill(n, spec.c, 20.0, 1.0, noise=1e-3, seed=0)
    om.init_fields(phi0)
    gm.init_fields(phi0)
    om.step(300)
    gm.step(300)
    assert rel_l2(gm.read_fields()[0], om.fields()[0]) <= 1e-5


def test_ncde_variant_errors():
    from paper_2512_16230_gb300 import lbm
    spec = W.LATTICES["rD2Q13"]
    nse = gpu_model(spec, "nse", (8, 8), np.ones(spec.R), store="f32")
    with pytest.raises(lbm.LBMError, match="LBM_ERR_ARG"):
        nse.set_ncde_variant("rate")
    m = gpu_model(spec, "ncde", (8, 8), np.ones(spec.R), store="f32", u_const=(0.01, 0.0))
    with pytest.raises(lbm.LBMError, match="LBM_ERR_ARG"):
        m.set_ncde_variant("cde", 0.5)
    b = lbm.Batch(4)
    b.add(m)
    m.set_ncde_variant("rate")             # every variant runs inside a batch
    m.set_ncde_variant("moment", 0.3)
    b.remove(m)
    b.close()


@pytest.mark.parametrize("store", ["f64", "f32"])
@pytest.mark.parametrize("lattice,n", [("rD2Q9", (64, 48)), ("rD3Q27", (24, 24, 18))])
def test_single_speed_taylor_green(lattice, n, store):
    """Single-speed rectangular lattices (k = 1) with the per-axis normal rates of Eq. (4-29):
    a Taylor-Green vortex over 100 steps against the FP64 oracle."""
    if len(n) == 2:
        wl = W.taylor_green_2d(n=n, steps=100, store=store, lattice=lattice)
    else:
        wl = W.taylor_green_3d(n=n, steps=100, store=store, re=100.0, ma=0.1, lattice=lattice)
    om, gm = workload_pair(wl)
    om.step(wl.steps)
    gm.step(wl.steps)
    r_g, u_g = gm.read_fields()
    r_o, u_o = om.fields()
    assert rel_l2(u_g, u_o) <= TOL[store]
    assert rel_l2(r_g, r_o) <= TOL[store]




M2G_VARIANTS = [  # (store, per-order rates, tensor cores): k_step FP64 / FP32, k_step_high, k_step_tc32_high
    ("f64", False, 0), ("f32", False, 0), ("f64", True, 0), ("f32", True, 0), ("f32", True, 1)]


@pytest.mark.parametrize("store,high,tensor", M2G_VARIANTS)
@pytest.mark.parametrize("s_bulk", [None, 0.9])
@pytest.mark.parametrize("name", ["rD2Q9", "rD3Q27"])
def test_m2g_anisotropy_steps(name, s_bulk, store, high, tensor):
    """The (delta4 . u) . grad rho term of Eq. (M2Ga) on the single-speed lattices, from
    far-from-equilibrium populations (O(1) density gradients, every wrap of the central
    difference on a ragged grid): three steps against the FP64 oracle. The first takes the density
    of the initial state as the previous one; the next two read the density the kernel stored (the
    two-field history). Covers the bulk block of Eq. (4-27) inside (I - S2/2), the per-order-rate
    kernels and the FP32 tensor-core kernel. The term moves the oracle's populations by more than
    20 times the GPU-oracle difference (about 2e-4 relative after three steps)."""
    spec = ALL_SPECS[name]
    d = spec.d
    n = RAGGED[d]
    s = _random_rates(spec.R, 12)
    kw = dict(s_high=1.2, force=(d - 1, 0, 2e-3, 1, 0.1), s_bulk=s_bulk, s_orders=HIGH_RATES if high else None)
    om = oracle_model(spec, "nse", n, s, m2g_aniso=True, **kw)
    ref = oracle_model(spec, "nse", n, s, **kw)
    gm = gpu_model(spec, "nse", n, s, store=store, m2g_aniso=True, **kw)
    if store != "f64":
        gm.set_tensor_cores(tensor)
    f0 = round_to_store(I.random_populations(n, om.lat.Q, seed=23), store)
    for m in (om, ref, gm):
        m.set_populations(f0)
    for _ in range(3):
        om.step(1)
        ref.step(1)
        gm.step(1)
        err = rel_l2(gm.get_populations(), om.f)
        assert err <= TOL[store]
    assert rel_l2(ref.f, om.f) > max(20 * err, 1e-5)


@pytest.mark.parametrize("store", ["f64", "f32"])
@pytest.mark.parametrize("name,n", [("rD2Q9", (4, 32)), ("rD3Q27", (4, 4, 32))])
def test_m2g_anisotropy_sound_wave(name, n, store):
    """A sound wave along the long axis (c = 4/3) on a background flow of 0.1 along it, the flow
    whose downstream / upstream damping split the term removes: 300 steps with the term on against
    the FP64 oracle (density and velocity)."""
    spec = ALL_SPECS[name]
    d = spec.d
    s = np.ones(spec.R)
    olat = oracle_lattice(spec)
    for r, p in enumerate(olat.polys):
        if olat.orders[r] == 2 and max(max(p, key=sum)) == 2:
            s[r] = 1.2
    om = oracle_model(spec, "nse", n, s, m2g_aniso=True)
    gm = gpu_model(spec, "nse", n, s, store=store, m2g_aniso=True)
    c = spec.c[d - 1]
    z = np.arange(n[d - 1]) * c
    shape = tuple(reversed(n))
    prof = np.cos(2 * math.pi * z / (n[d - 1] * c)).reshape((n[d - 1],) + (1,) * (d - 1))
    rho = 1.0 + 1e-3 * np.broadcast_to(prof, shape)
    u = np.zeros((d,) + shape)
    u[d - 1] = 0.1
    om.init_fields(rho, u)
    gm.init_fields(rho, u)
    om.step(300)
    gm.step(300)
    r_g, u_g = gm.read_fields()
    r_o, u_o = om.fields()
    # FP32: on this nearly uniform state every cell rounds alike, so the rounding of a step does not
    # average out over the grid; the mean density drifts by ~3e-8 per step (and u = j / rho with it)
    tol = TOL[store] if store == "f64" else 5e-5
    assert rel_l2(u_g, u_o) <= tol
    assert rel_l2(r_g, r_o) <= tol
    if store == "f64":
        # the wave itself: the perturbations (~4e-5 against rho = 1 and the 0.1 background) carry
        # the FP64 rounding of the full values, ~1e-13 absolute, while the term changes them by
        # ~1e-2 relative over the run
        assert rel_l2(r_g - 1.0, r_o - 1.0) <= 1e-8
        bg = 0.1 * (np.arange(d) == d - 1).reshape((-1,) + (1,) * d)
        assert rel_l2(u_g - bg, u_o - bg) <= 1e-8


def test_m2g_anisotropy_errors():
    from paper_2512_16230_gb300 import lbm
    spec = ALL_SPECS["rD2Q25"]
    gm = gpu_model(spec, "nse", (8, 8), np.ones(spec.R))
    with pytest.raises(lbm.LBMError, match="LBM_ERR_ARG"):
        gm.set_m2g_anisotropy(1)
    spec = ALL_SPECS["rD2Q9"]
    gm = gpu_model(spec, "ncde", (8, 8), np.ones(spec.R), u_const=(0.01, 0.0))
    with pytest.raises(lbm.LBMError, match="LBM_ERR_ARG"):
        gm.set_m2g_anisotropy(1)
    gm = gpu_model(spec, "nse", (8, 8), np.ones(spec.R))
    with pytest.raises(lbm.LBMError, match="LBM_ERR_ARG"):
        gm.set_m2g_anisotropy(2)
    gm.set_m2g_anisotropy(1)
    gm.set_m2g_anisotropy(0)


CROSS_VARIANTS = [  # (store, NCDE variant, a1, per-order rates, tensor cores)
    ("f64", "moment", 0.0, False, 0), ("f32", "moment", 0.4, False, 0), ("f64", "rate", 0.0, False, 0),
    ("f32", "rate", -0.3, False, 0), ("f32", "moment", 0.0, True, 0), ("f32", "moment", 0.0, True, 1)]


@pytest.mark.parametrize("store,variant,a1,high,tensor", CROSS_VARIANTS)
@pytest.mark.parametrize("name", ["rD2Q13", "rD2Q25", "rD3Q33", "rD3Q53", "rD2Q9"])
def test_ncde_cross_diffusion_steps(name, store, variant, a1, high, tensor):
    """The cross-diffusion term of Eq. (GNCDE) (A2 = a2 I, D-bar = psi I, grad psi by central
    differences) with a random psi on a ragged grid: three steps from far-from-equilibrium
    populations against the oracle, with the moment and per-cell-rate variants, the mixed
    derivative, the per-order-rate kernels and the FP32 tensor-core kernel. The term moves the
    oracle's populations by more than 20 times the GPU-oracle difference."""
    spec = ALL_SPECS[name]
    d = spec.d
    n = RAGGED[d]
    s = _random_rates(spec.R, 19)
    psi = round_to_store(I.random_scalar(n, seed=29), store)
    kw = dict(s_high=1.2, u_const=tuple(np.linspace(0.04, 0.08, d)), nonlin=1.0, ncde_mode=variant, a1=a1,
              s_orders=HIGH_RATES if high else None)
    om = oracle_model(spec, "ncde", n, s, a2=0.05, psi=psi, **kw)
    ref = oracle_model(spec, "ncde", n, s, **kw)
    gm = gpu_model(spec, "ncde", n, s, store=store, a2=0.05, psi=psi, **kw)
    if store != "f64":
        gm.set_tensor_cores(tensor)
    f0 = round_to_store(I.random_populations(n, om.lat.Q, seed=31), store)
    for m in (om, ref, gm):
        m.set_populations(f0)
    for _ in range(3):
        om.step(1)
        ref.step(1)
        gm.step(1)
        err = rel_l2(gm.get_populations(), om.f)
        assert err <= TOL[store]
    assert rel_l2(ref.f, om.f) > max(20 * err, 1e-5)


@pytest.mark.parametrize("store", ["f64", "f32"])
def test_ncde_cross_diffusion_driven_mode(store):
    """rD2Q13 at rest driven by psi = cos(k y) (the mode of the oracle pin, along the c = 1.25
    axis): 300 steps against the oracle, phi within the per-dtype tolerance of its driven part."""
    spec = ALL_SPECS["rD2Q13"]
    n = (4, 64)
    s = np.ones(spec.R)
    s[1] = s[2] = 1.5
    c = spec.c[1]
    y = np.arange(n[1]) * c
    psi = np.broadcast_to(np.cos(2 * math.pi * y / (n[1] * c)).reshape(n[1], 1), (n[1], n[0])).copy()
    kw = dict(u_const=(0.0, 0.0), a2=0.02, psi=round_to_store(psi, store))
    om = oracle_model(spec, "ncde", n, s, **kw)
    gm = gpu_model(spec, "ncde", n, s, store=store, **kw)
    phi0 = np.ones((n[1], n[0]))
    om.init_fields(phi0)
    gm.init_fields(phi0)
    om.step(300)
    gm.step(300)
    phi_g, _ = gm.read_fields()
    phi_o, _ = om.fields()
    assert rel_l2(phi_g - 1.0, phi_o - 1.0) <= (1e-10 if store == "f64" else 1e-3)


def test_ncde_cross_diffusion_errors():
    from paper_2512_16230_gb300 import lbm
    spec = ALL_SPECS["rD2Q13"]
    gm = gpu_model(spec, "nse", (8, 8), np.ones(spec.R))
    with pytest.raises(lbm.LBMError, match="LBM_ERR_ARG"):
        gm.set_ncde_cross_diffusion(0.1, np.zeros((8, 8)))
    gm = gpu_model(spec, "ncde", (8, 8), np.ones(spec.R), u_const=(0.01, 0.0))
    with pytest.raises(lbm.LBMError, match="LBM_ERR_ARG"):
        gm.set_ncde_cross_diffusion(0.1, None)
    gm.set_ncde_cross_diffusion(0.1, np.zeros((8, 8)))
    with pytest.raises(lbm.LBMError, match="LBM_ERR_ARG"):
        gm.set_ncde_variant("cde")
    gm.set_ncde_cross_diffusion(0.0)
    gm.set_ncde_variant("cde")
    with pytest.raises(lbm.LBMError, match="LBM_ERR_ARG"):
        gm.set_ncde_cross_diffusion(0.1, np.zeros((8, 8)))
    with pytest.raises(ValueError):
        gm.set_ncde_cross_diffusion(0.1, np.zeros((4, 8)))


COMBINED = [  # (lattice, eq, settings): several extensions on one solve
    ("rD2Q25", "nse", dict(s_bulk=0.9, s_orders={4: 0.8, 5: 1.35, 6: 1.6}, cs2_eq=0.7, force=(1, 0, 2e-3, 1, 0.1))),
    ("rD3Q53", "nse", dict(s_bulk=1.1, s_orders={4: 0.9, 5: 1.2, 6: 1.5, 7: 1.0, 8: 1.3}, force=(2, 0, 2e-3, 1, 0.1))),
    ("rD3Q27", "nse", dict(s_bulk=0.95, s_orders={4: 0.85, 5: 1.25, 6: 1.4}, m2g_aniso=True, force=(0, 2, 2e-3, 1, 0.1))),
    ("rD2Q13", "ncde", dict(ncde_mode="rate", a1=-0.2, a2=0.03, s_orders={4: 1.3, 5: 0.8},
                            u_const=(0.04, 0.02), nonlin=1.0)),
]


@pytest.mark.parametrize("store,tensor", [("f64", 0), ("f32", 0), ("f32", 1)])
@pytest.mark.parametrize("name,eq,settings", COMBINED)
def test_combined_extensions_step(name, eq, settings, store, tensor):
    """The extensions together on one solve (bulk block, per-order rates, p = rho RT, body force,
    the M2G density-gradient term; NCDE per-cell rates with the mixed-derivative and
    cross-diffusion terms and per-order rates): three steps from far-from-equilibrium populations
    against the oracle, on the CUDA cores and (FP32) with the higher rows on tcgen05."""
    spec = ALL_SPECS[name]
    n = RAGGED[spec.d]
    s = _random_rates(spec.R, 51)
    kw = dict(settings)
    if "a2" in kw:
        kw["psi"] = round_to_store(I.random_scalar(n, seed=9), store)
    om = oracle_model(spec, eq, n, s, 1.15, **kw)
    gm = gpu_model(spec, eq, n, s, 1.15, store=store, **kw)
    if store != "f64":
        gm.set_tensor_cores(tensor)
    f0 = round_to_store(I.random_populations(n, om.lat.Q, seed=27), store)
    om.set_populations(f0)
    gm.set_populations(f0)
    for _ in range(3):
        om.step(1)
        gm.step(1)
        assert rel_l2(gm.get_populations(), om.f) <= TOL[store]
