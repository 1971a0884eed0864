"""Test helpers: build the oracle and the CUDA model of the same workload side by side.

Only tests import this module. The oracle and the library receive the same plain inputs
(lattice settings, rates, seeded fields or populations); nothing computed by one side is fed
to the other.
"""
import numpy as np

from oracle import lattice as OL
from oracle import mrt as OM
from paper_2512_16230_gb300 import workloads as W

ANISO = {
    "rD2Q25-aniso": W.LatticeSpec("rD2Q25", (1.0, 1.2), (0.7, 0.9), (2e-4, 1e-4, 3e-4, 5e-5)),
    "rD3Q53-aniso": W.LatticeSpec("rD3Q53", (1.0, 1.2, 4.0 / 3.0), (0.85, 1.152, 0.7 * 16.0 / 9.0), (5e-4,)),
}
ALL_SPECS = dict(W.LATTICES, **ANISO)

# Ragged grids spanning several 128-cell blocks with a partial last block.
RAGGED = {2: (37, 29), 3: (13, 11, 9)}


def oracle_lattice(spec):
    return OL.build(spec.kind, spec.c, spec.cs2, spec.free_w)


def gpu_lattice(spec):
    from paper_2512_16230_gb300 import lbm
    return lbm.Lattice(spec.kind, spec.c, spec.cs2, spec.free_w)


def oracle_model(spec, eq, n, s, s_high=1.0, force=None, u_const=None, nonlin=0.0, cs2_eq=None, lat=None,
                 s_bulk=None, s_orders=None, ncde_mode="moment", a1=0.0, m2g_aniso=False, a2=0.0, psi=None):
    lat = lat or oracle_lattice(spec)
    return OM.Model(lat, eq, n, np.asarray(s, dtype=float), s_high, cs2_eq=cs2_eq, force=force,
                    u_const=None if u_const is None else np.asarray(u_const, dtype=float), nonlin=nonlin,
                    s_bulk=s_bulk, s_orders=s_orders, ncde_mode=ncde_mode, a1=a1, m2g_aniso=m2g_aniso,
                    a2=a2, psi=psi)


def gpu_model(spec, eq, n, s, s_high=1.0, force=None, u_const=None, nonlin=0.0, cs2_eq=None, store="f32",
              lat=None, s_bulk=None, s_orders=None, ncde_mode="moment", a1=0.0, m2g_aniso=False, a2=0.0,
              psi=None):
    from paper_2512_16230_gb300 import lbm
    lat = lat or gpu_lattice(spec)
    m = lbm.Model(lat, eq, n, store=store)
    m.set_relaxation(s, s_high)
    if cs2_eq is not None:
        m.set_eos(cs2_eq)
    if force is not None:
        m.set_force(*force)
    if u_const is not None:
        m.set_ncde(u_const, nonlin)
    if s_bulk is not None:
        m.set_bulk(s_bulk)
    if s_orders:
        m.set_high_rates([s_orders.get(k, s_high) for k in range(4, max(s_orders) + 1)])
    if ncde_mode != "moment" or a1:
        m.set_ncde_variant(ncde_mode, a1)
    if m2g_aniso:
        m.set_m2g_anisotropy(1)
    if a2:
        m.set_ncde_cross_diffusion(a2, psi)
    return m


def workload_pair(wl, store=None):
    """(oracle model, GPU model) of a Workload, both initialised from the same fields."""
    rho, u = wl.fields()
    om = oracle_model(wl.lattice, wl.eq, wl.n, wl.s, wl.s_high, force=wl.force, u_const=wl.u_const,
                      nonlin=wl.nonlin)
    gm = gpu_model(wl.lattice, wl.eq, wl.n, wl.s, wl.s_high, force=wl.force, u_const=wl.u_const,
                   nonlin=wl.nonlin, store=store or wl.store)
    om.init_fields(rho, u)
    gm.init_fields(rho, u)
    return om, gm


def rel_l2(a, b):
    a = np.asarray(a, dtype=float)
    b = np.asarray(b, dtype=float)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def rel_max(a, b):
    a = np.asarray(a, dtype=float)
    b = np.asarray(b, dtype=float)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def round_to_store(x, store):
    """Values exactly representable in the storage dtype (for bit-exact data movement checks)."""
    if store == "f32":
        return np.asarray(x, dtype=np.float32).astype(np.float64)
    return np.asarray(x, dtype=np.float64)
