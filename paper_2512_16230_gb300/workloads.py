"""Workload parameters: lattice settings, relaxation rates and grids of the benchmark configs.

These are inputs to the method (plain numbers), shared by the tests, the benchmark and the
oracle harness so that every side solves the same problem. The only formulas here invert the
viscosity law nu = cs2 (1/s - 1/2) (Eq. (4-29), compressible, k = 0) and the diffusivity law
K = cs2 (1/s1 - 1/2) (Eq. (ME-NCDE-3)) to choose rates; lattice arithmetic lives in the library
and, independently, in the oracle.

Free weights and sound speeds were chosen to maximise the smallest weight (all positive on the
2D lattices and on cubic 3D cells). On rD3Q53 with dz/dx = 4/3 and one shared sound speed no
all-positive setting exists: the max-min choice c_s^2 = 0.624, w45 = 2.9625e-4 leaves a minimum
weight of -2.0e-3 and a negative norm of the corrected H_zzz row, and the FP64 oracle diverges on
the 48 x 48 x 36 Taylor-Green copy. The rD3Q53 workload therefore uses per-axis sound speeds
(Remark 2): d_0z / d_0x = 0.75 with c_sx^2 = c_sy^2 = 0.96, c_sz^2 = 1.28, w45 = 8e-4 (minimum
weight 8e-4, near the max-min optimum at that ratio) and the isothermal pressure p = 0.96 rho.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import inputs as I


@dataclass(frozen=True)
class LatticeSpec:
    kind: str
    c: tuple
    cs2: tuple
    free_w: tuple = ()

    @property
    def d(self):
        return len(self.c)

    @property
    def single(self):
        """Single-speed lattice (components in {0, +-1}; k = 1 of Sec. 3.4)."""
        return self.kind in SINGLE_SPEED

    @property
    def R(self):
        return len(row_orders(self.d, self.single))


SINGLE_SPEED = ("rD2Q9", "rD3Q27")

# Shared-c_s setting of rD3Q53 on dz/dx = 4/3 (negative weights and a negative H_zzz norm).
RD3Q53_SHARED_CS = LatticeSpec("rD3Q53", (1.0, 1.0, 4.0 / 3.0), (0.624,) * 3, (2.9625e-4,))

LATTICES = {
    "rD2Q25": LatticeSpec("rD2Q25", (1.0, 4.0 / 3.0), (0.8, 0.8), (3.125e-4,) * 4),
    "rD2Q21": LatticeSpec("rD2Q21", (1.0, 4.0 / 3.0), (0.8, 0.8), (7.29e-4,) * 3),
    "rD2Q17": LatticeSpec("rD2Q17", (1.0, 4.0 / 3.0), (0.8, 0.8), (2.1875e-3,)),
    "rD2Q13": LatticeSpec("rD2Q13", (1.0, 1.25), (0.8, 0.8), ()),
    "rD3Q53": LatticeSpec("rD3Q53", (1.0, 1.0, 4.0 / 3.0), (0.96, 0.96, 1.28), (8e-4,)),
    "rD3Q53-cubic": LatticeSpec("rD3Q53", (1.0, 1.0, 1.0), (0.6,) * 3, (2.4e-4,)),
    "rD3Q45": LatticeSpec("rD3Q45", (1.0, 1.0, 1.0), (0.6,) * 3, ()),
    "rD3Q33": LatticeSpec("rD3Q33", (1.0, 1.0, 1.0), (0.5,) * 3, ()),
    # single-speed lattices on rectangular cells (d_0 = c_s^2 / c_a^2 < 1 keeps every weight positive)
    "rD2Q9": LatticeSpec("rD2Q9", (1.0, 4.0 / 3.0), (1.0 / 3.0, 1.0 / 3.0), ()),
    "rD3Q27": LatticeSpec("rD3Q27", (1.0, 1.0, 4.0 / 3.0), (1.0 / 3.0,) * 3, ()),
}


def row_orders(d, single=False):
    """Order (0..3) of each Hermite row in the paper's order (2D: App. C, 3D: App. D); the
    single-speed lattices have no pure-cube rows (the last d)."""
    o = [0, 1, 1, 2, 2, 2, 3, 3, 3, 3] if d == 2 else [0, 1, 1, 1] + [2] * 6 + [3] * 10
    return o[:len(o) - d] if single else o


def rates_nse(d, nu, cs2, s3=1.0, spec=None):
    """s_nu = 1 / (nu / cs2 + 1/2) on every second-order row, s3 on the third-order rows. On a
    single-speed lattice (k = 1) the normal rows c_a^2 - c_sa^2 take s_a = 1 / (2 nu / (c_a^2 - cs2)
    + 1/2) per axis, which makes the normal viscosity of Eq. (4-29) equal to the shear one."""
    single = spec is not None and spec.single
    o = np.array(row_orders(d, single))
    s = np.ones(len(o))
    s[o == 2] = 1.0 / (nu / cs2 + 0.5)
    s[o == 3] = s3
    if single:
        normal = (3, 5) if d == 2 else (4, 5, 6)
        for a, r in enumerate(normal):
            s[r] = 1.0 / (2.0 * nu / (spec.c[a] ** 2 - cs2) + 0.5)
    return s


def rates_ncde(d, K, cs2, spec=None):
    """s_1 = 1 / (K / cs2 + 1/2) on the first-order rows."""
    o = np.array(row_orders(d, spec is not None and spec.single))
    s = np.ones(len(o))
    s[o == 1] = 1.0 / (K / cs2 + 0.5)
    return s


@dataclass
class Workload:
    name: str
    lattice: LatticeSpec
    eq: str
    n: tuple
    steps: int
    s: np.ndarray
    s_high: float = 1.0
    store: str = "f32"
    force: tuple | None = None
    u_const: tuple | None = None
    nonlin: float = 0.0
    init: dict = field(default_factory=dict)

    @property
    def ncells(self):
        return int(np.prod(self.n))

    def fields(self):
        """Seeded initial fields (rho, u) or (phi, None)."""
        kind = self.init["kind"]
        lat = self.lattice
        if kind == "tgv2d":
            return I.taylor_green_2d(self.n, lat.c, self.init["u0"], 1.0, lat.cs2[0])
        if kind == "tgv3d":
            return I.taylor_green_3d(self.n, lat.c, self.init["u0"], 1.0, lat.cs2[0])
        if kind == "hill":
            return I.gaussian_hill(self.n, lat.c, self.init["sigma"], self.init.get("amplitude", 1.0),
                                   self.init.get("noise", 0.0), self.init.get("seed", 0)), None
        if kind == "rest":
            return I.rest_state(self.n, lat.d)
        raise ValueError(kind)


def taylor_green_2d(n=(64, 48), steps=200, store="f64", re=100.0, ma=0.05, lattice="rD2Q25"):
    """Config: rD2Q25 Taylor-Green vortex, L = 2 pi on rectangular cells (dy/dx = 4/3),
    u0 = 0.05 c_s, Re = u0 L / nu with L = L_x / (2 pi)."""
    lat = LATTICES[lattice]
    u0 = ma * math.sqrt(lat.cs2[0])
    nu = u0 * (n[0] * lat.c[0] / (2 * math.pi)) / re
    return Workload(f"{lat.kind} Taylor-Green 2D", lat, "nse", tuple(n), steps, rates_nse(2, nu, lat.cs2[0], spec=lat),
                    store=store, init=dict(kind="tgv2d", u0=u0, nu=nu))


def ncde_hill(n=(1024, 768), steps=5000, store="f32", D0=0.1, nonlin=1.0, sigma=20.0, noise=1e-3, seed=0,
              u=(0.02, 0.01)):
    """Config: rD2Q13 nonlinear convection-diffusion d_t phi + div(u phi) = div(D0 (1 + phi^2) grad phi),
    u = (0.02, 0.01), dy/dx = 1.25, Gaussian hill A = 1, sigma = 20 dx plus U[-1e-3, 1e-3] noise."""
    lat = LATTICES["rD2Q13"]
    return Workload("rD2Q13 nonlinear CDE", lat, "ncde", tuple(n), steps, rates_ncde(2, D0, lat.cs2[0], spec=lat),
                    store=store, u_const=tuple(u), nonlin=nonlin,
                    init=dict(kind="hill", sigma=sigma, noise=noise, seed=seed, D0=D0))


def taylor_green_3d(n=(256, 256, 192), steps=1000, store="f32", re=1600.0, ma=0.3, lattice="rD3Q53"):
    """Config: rD3Q53 compressible isothermal Taylor-Green vortex on dz/dx = 4/3 cells,
    Ma = U0 / c_s = 0.3, Re = U0 L / nu with L = L_x / (2 pi)."""
    lat = LATTICES[lattice]
    u0 = ma * math.sqrt(lat.cs2[0])
    nu = u0 * (n[0] * lat.c[0] / (2 * math.pi)) / re
    return Workload(f"{lat.kind} Taylor-Green 3D", lat, "nse", tuple(n), steps, rates_nse(3, nu, lat.cs2[0], spec=lat),
                    store=store, init=dict(kind="tgv3d", u0=u0, nu=nu))


def kolmogorov_3d(lattice="rD3Q53-cubic", n=(32, 32, 32), steps=200, store="f32", nu=0.05, umax_ma=0.05):
    """Serving-mix flow: F = (A sin(2 pi y / L_y), 0, 0) with A set so the steady u_max = 0.05 c_s."""
    lat = LATTICES[lattice]
    ly = n[1] * lat.c[1]
    umax = umax_ma * math.sqrt(lat.cs2[0])
    A = umax * nu * (2 * math.pi / ly) ** 2
    return Workload(f"{lat.kind} Kolmogorov 3D", lat, "nse", tuple(n), steps, rates_nse(3, nu, lat.cs2[0], spec=lat),
                    store=store, force=(0, 1, A, 1, 0.0), init=dict(kind="rest"))


def serving_workload(req, store):
    """The Workload of one serving request (see inputs.serving_requests): 2D Taylor-Green at
    Re = 100 and u0 = 0.05 c_s, 2D nonlinear CDE hill (D0 = 0.1, sigma = n_x / 8, u = (0.02, 0.01)),
    or 3D Kolmogorov flow with nu = 0.05 and steady u_max = 0.05 c_s."""
    n = tuple(req["grid"])
    if req["flow"] == "kolmogorov":
        wl = kolmogorov_3d(lattice=req["lattice"], n=n, steps=req["steps"], store=store)
    elif req["flow"] == "tgv2d":
        lat = LATTICES[req["lattice"]]
        u0 = 0.05 * math.sqrt(lat.cs2[0])
        nu = u0 * (n[0] * lat.c[0] / (2 * math.pi)) / 100.0
        wl = Workload(f"{lat.kind} Taylor-Green 2D", lat, "nse", n, req["steps"], rates_nse(2, nu, lat.cs2[0], spec=lat),
                      store=store, init=dict(kind="tgv2d", u0=u0, nu=nu))
    else:
        lat = LATTICES[req["lattice"]]
        wl = Workload(f"{lat.kind} nonlinear CDE", lat, "ncde", n, req["steps"], rates_ncde(2, 0.1, lat.cs2[0], spec=lat),
                      store=store, u_const=(0.02, 0.01), nonlin=1.0,
                      init=dict(kind="hill", sigma=max(2.0, n[0] / 8.0), noise=1e-3, seed=req["seed"]))
    return wl
