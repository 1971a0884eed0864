"""Parity at the full sizes of the benchmark configurations, in the launch configuration the
benchmark times (one lbm.Model, default kernel choice, the workload's own storage).

The oracle cannot run these grids, so the checks are (1) sampled outputs the oracle computes one
by one: after the first step from the analytic initial fields, f_i(x) = f~_i(x - e_i), so the
oracle collides just the source cells x - e_i of each sampled cell x (the equilibrium of the
initial fields there), including cells on every face and corner of the periodic box; and (2)
properties that hold at any size (conservation of mass and momentum, energy decay).
"""
import numpy as np
import pytest

from paper_2512_16230_gb300 import workloads as W

from _harness import gpu_model, oracle_lattice, oracle_model, rel_l2

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5}


@pytest.fixture(autouse=True)
def _lib(lbm_lib):
    return lbm_lib


def _sample_cells(n, count, seed):
    """Cell coordinates (x, y[, z]): every corner of the box plus seeded interior and face cells."""
    rng = np.random.default_rng(seed)
    d = len(n)
    corners = [tuple((n[a] - 1) * ((k >> a) & 1) for a in range(d)) for k in range(2 ** d)]
    rest = [tuple(int(rng.integers(0, n[a])) if a != (k % d) else int((n[a] - 1) * (k % 2))
                  for a in range(d)) for k in range(count // 2)]
    inner = [tuple(int(rng.integers(0, n[a])) for a in range(d)) for _ in range(count - count // 2)]
    return corners + rest + inner


def _oracle_first_step(wl, cells, rho, u):
    """f_i(x) after one step for each sampled cell x: the oracle collides, on a one-dimensional
    list of cells, the equilibrium of the initial fields at every source cell x - e_i."""
    spec = wl.lattice
    lat = oracle_lattice(spec)
    d, Q = lat.d, lat.Q
    n = wl.n
    src = []
    for x in cells:
        for i in range(Q):
            src.append(tuple((x[a] - int(lat.e[i, a])) % n[a] for a in range(d)))
    idx = tuple(np.array([y[a] for y in src]) for a in reversed(range(d)))   # numpy order (z, y, x)
    M = len(src)
    grid = (M,) + (1,) * (d - 1)
    shape = tuple(reversed(grid))
    om = oracle_model(spec, wl.eq, grid, wl.s, wl.s_high, force=wl.force, u_const=wl.u_const,
                      nonlin=wl.nonlin)
    if wl.eq == "nse":
        om.init_fields(rho[idx].reshape(shape), np.stack([u[a][idx] for a in range(d)]).reshape((d,) + shape))
    else:
        om.init_fields(rho[idx].reshape(shape))
    ft = om.collide().reshape(Q, M)
    return np.array([[ft[i, s * Q + i] for s in range(len(cells))] for i in range(Q)])


def _gpu_first_step(wl, cells, rho, u, tensor=0):
    import torch
    spec = wl.lattice
    gm = gpu_model(spec, wl.eq, wl.n, wl.s, wl.s_high, force=wl.force, u_const=wl.u_const, nonlin=wl.nonlin,
                   store=wl.store)
    if tensor:
        gm.set_tensor_cores(1)
    gm.init_fields(rho, None if u is None else np.ascontiguousarray(u))
    gm.step(1)
    out = torch.empty((gm.Q,) + tuple(reversed(wl.n)), dtype=torch.float64, device="cuda")
    gm.get_populations(out)
    gm.synchronize()
    idx = tuple(torch.tensor([x[a] for x in cells], device="cuda") for a in reversed(range(len(wl.n))))
    got = out[(slice(None),) + idx].cpu().numpy()
    del out
    gm.close()
    torch.cuda.empty_cache()
    return got


def test_config3_full_size_first_step_sampled():
    """rD3Q53 Taylor-Green, 256 x 256 x 192, FP32 (the benchmark workload): one step from the
    analytic fields, all 53 populations at 72 sampled cells (the 8 corners, cells on the faces and
    inside) against the oracle's per-cell collisions, within the FP32 parity bound."""
    wl = W.taylor_green_3d()
    rho, u = wl.fields()
    cells = _sample_cells(wl.n, 64, seed=5)
    got = _gpu_first_step(wl, cells, rho, u)
    want = _oracle_first_step(wl, cells, rho, u)
    assert rel_l2(got, want) <= TOL["f32"]
    assert np.abs(got - want).max() <= 10 * TOL["f32"] * np.abs(want).max()


@pytest.mark.parametrize("tensor", [0, 1])
@pytest.mark.parametrize("store,unit", [("f16_dev", 2.0 ** -11), ("bf16_dev", 2.0 ** -8)])
def test_config4_full_size_first_step_sampled(store, unit, tensor):
    """The reduced-precision configuration: the benchmark workload with 16-bit deviation storage
    (f - w rho_ref stored, collision in FP32), in the launch the benchmark times (the row-staged
    kernel, with the contractions on the CUDA cores or on tcgen05). One step at 72 sampled cells
    against the oracle's per-cell collisions of the FP64 equilibrium: the deviations agree within
    the rounding of the stored input and output (4 units of the 16-bit format)."""
    wl = W.taylor_green_3d(store=store)
    rho, u = wl.fields()
    cells = _sample_cells(wl.n, 64, seed=7)
    got = _gpu_first_step(wl, cells, rho, u, tensor)
    want = _oracle_first_step(wl, cells, rho, u)
    w = oracle_lattice(wl.lattice).w[:, None]
    assert rel_l2(got - w, want - w) <= 4 * unit


@pytest.mark.parametrize("store", ["f16_dev", "bf16_dev"])
def test_config4_full_size_row_gather_is_bitwise_thread_gather(store):
    """The benchmark workload in 16-bit storage, two steps, with the launch the benchmark times (the
    row-staged gather, chosen automatically for n_x = 256) and with the per-thread gather: the
    whole population arrays are bitwise equal (compared on the device)."""
    import torch
    wl = W.taylor_green_3d(store=store)
    rho, u = wl.fields()
    out = {}
    for mode in ("auto", "threads"):
        gm = gpu_model(wl.lattice, wl.eq, wl.n, wl.s, wl.s_high, store=store)
        gm.set_gather(mode)
        gm.init_fields(rho, np.ascontiguousarray(u))
        gm.step(2)
        out[mode] = torch.empty((gm.Q,) + tuple(reversed(wl.n)), dtype=torch.float64, device="cuda")
        gm.get_populations(out[mode])
        gm.synchronize()
        gm.close()
    assert torch.equal(out["auto"], out["threads"])
    del out
    torch.cuda.empty_cache()


HIGH_RATES = {4: 0.8, 5: 1.35, 6: 1.6, 7: 0.9, 8: 1.25}


def _wave_populations(n, w, seed, amp=0.05):
    """Non-equilibrium populations on the whole grid, (Q, nz, ny, nx) float64:
    f_i(x) = w_i (1 + amp sin(2 pi sum_a k_ia x_a / n_a + phase_i)) with seeded integer wave vectors
    and phases per population, so that every moment order, the rows of order >= 4 included, is
    excited and varies from cell to cell."""
    rng = np.random.default_rng(seed)
    Q = len(w)
    k = rng.integers(-3, 4, size=(Q, 3))
    ph = rng.uniform(0.0, 2.0 * np.pi, Q)
    x = [2.0 * np.pi * np.arange(n[a]) / n[a] for a in range(3)]
    f = np.empty((Q, n[2], n[1], n[0]))
    for i in range(Q):
        arg = (k[i, 0] * x[0][None, None, :] + k[i, 1] * x[1][None, :, None] + k[i, 2] * x[2][:, None, None]
               + ph[i])
        f[i] = w[i] * (1.0 + amp * np.sin(arg))
    return f


@pytest.mark.parametrize("store,tol", [("f32", 1e-5), ("f16_dev", 4 * 2.0 ** -11)])
def test_config3_high_order_rates_full_size_sampled(store, tol):
    """The per-order-rate variant of the benchmark solve at its full size (rD3Q53, 256 x 256 x 192),
    in the launch the benchmark times (FP32: the CUDA-core reduced form with the higher rows'
    operator on tcgen05; FP16 deviations: the row-staged tcgen05 kernel with the higher rows): one
    step from seeded non-equilibrium populations (every order excited), all 53 populations at 72
    sampled cells against the oracle's full Q x Q collision Lambda = H^-1 S H of the source cells
    x - e_i, within the FP32 bound (FP32) or 4 units of FP16 on the deviations (FP16)."""
    import torch
    wl = W.taylor_green_3d(store=store)
    spec = wl.lattice
    lat = oracle_lattice(spec)
    f0 = _wave_populations(wl.n, lat.w, seed=31)
    w4 = lat.w[:, None, None, None]
    if store == "f32":
        f0 = f0.astype(np.float32).astype(np.float64)
    else:
        f0 = w4 + (f0 - w4).astype(np.float16).astype(np.float64)
    cells = _sample_cells(wl.n, 64, seed=9)
    gm = gpu_model(spec, wl.eq, wl.n, wl.s, wl.s_high, store=store, s_orders=HIGH_RATES)
    gm.set_populations(f0)
    gm.step(1)
    out = torch.empty((gm.Q,) + tuple(reversed(wl.n)), dtype=torch.float64, device="cuda")
    gm.get_populations(out)
    gm.synchronize()
    idx = tuple(torch.tensor([x[a] for x in cells], device="cuda") for a in (2, 1, 0))
    got = out[(slice(None),) + idx].cpu().numpy()
    del out
    gm.close()
    torch.cuda.empty_cache()
    # the oracle: the full collision of every source cell x - e_i, on a one-dimensional list of cells
    Q, n = lat.Q, wl.n
    src = [tuple((x[a] - int(lat.e[i, a])) % n[a] for a in range(3)) for x in cells for i in range(Q)]
    fs = f0[:, [c[2] for c in src], [c[1] for c in src], [c[0] for c in src]]
    del f0
    M = len(src)
    om = oracle_model(spec, wl.eq, (M, 1, 1), wl.s, wl.s_high, s_orders=HIGH_RATES)
    om.set_populations(fs.reshape(Q, 1, 1, M))
    ft = om.collide().reshape(Q, M)
    want = np.array([[ft[i, s * Q + i] for s in range(len(cells))] for i in range(Q)])
    if store == "f32":
        assert rel_l2(got, want) <= tol
    else:
        w = lat.w[:, None]
        assert rel_l2(got - w, want - w) <= tol


@pytest.mark.parametrize("store", ["f32", "f64"])
def test_config2_full_size_first_step_sampled(store):
    """rD2Q13 nonlinear CDE hill, 1024 x 768, FP32 and FP64: one step from the seeded fields at
    68 sampled cells against the oracle's per-cell collisions (phi^{-1} = phi^0 on both sides)."""
    wl = W.ncde_hill(store=store)
    phi, _ = wl.fields()
    cells = _sample_cells(wl.n, 64, seed=6)
    got = _gpu_first_step(wl, cells, phi, None)
    want = _oracle_first_step(wl, cells, phi, None)
    assert rel_l2(got, want) <= TOL[store]


def _mirror(a, axis):
    """a(-x) along numpy axis `axis` of a periodic grid (cell i -> (n - i) mod n)."""
    return np.roll(np.flip(a, axis=axis), 1, axis=axis)


def test_config3_full_size_invariants():
    """The benchmark workload over 100 steps: mass and momentum are conserved (no force, no net
    momentum), and the mirror symmetries of the Taylor-Green field (x -> -x, y -> -y, z -> -z about
    the origin of the periodic box, under which u_a is odd along axis a and even along the others,
    and rho is even) survive on the symmetric lattice to FP32 rounding, through every wrap."""
    wl = W.taylor_green_3d()
    spec = wl.lattice
    gm = gpu_model(spec, wl.eq, wl.n, wl.s, wl.s_high, store=wl.store)
    rho, u = wl.fields()
    gm.init_fields(rho, np.ascontiguousarray(u))
    s0 = gm.conserved_sums()
    gm.step(100)
    s1 = gm.conserved_sums()
    r, v = gm.read_fields()
    gm.close()
    u0 = wl.init["u0"]
    assert abs(s1[0] - s0[0]) <= 1e-5 * s0[0]
    assert np.abs(s1[1:]).max() <= 1e-5 * wl.ncells * u0
    for a in range(3):
        ax = 2 - a                                   # numpy axis of spatial axis a
        assert np.abs(_mirror(r, ax) - r).max() <= 1e-5
        for b in range(3):
            sign = -1.0 if b == a else 1.0
            assert np.abs(_mirror(v[b], ax) - sign * v[b]).max() <= 1e-5 * u0
