"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle harness.

This module produces initial fields and raw population arrays only; it holds none of the
lattice-Boltzmann arithmetic (no weights, moments, equilibria or collision). Random numbers
come from numpy's counter-based Philox generator keyed by an explicit seed, so every caller
gets the same arrays on any machine.

Layout conventions (shared by the C ABI and the oracle): a field on a grid of
n = (n_x, n_y[, n_z]) cells is a C-order array of shape (n_z, n_y, n_x) (x fastest);
a velocity field has a leading axis of length d (u[0] = u_x); populations have a leading
axis of length Q. Physical coordinates are in units of the first grid spacing: the cell with
index i_a sits at x_a = i_a * c_a where c_a = dx_a / dx_1.
"""
from __future__ import annotations

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=int(seed)))


def coords(n, c):
    """Physical cell coordinates x_a = i_a * c_a as a list of broadcastable arrays (x first)."""
    d = len(n)
    shape = tuple(reversed(n))
    out = []
    for a in range(d):
        s = [1] * d
        s[d - 1 - a] = n[a]
        out.append((np.arange(n[a], dtype=np.float64) * c[a]).reshape(s) * np.ones(shape))
    return out


def taylor_green_2d(n, c, u0, rho0=1.0, cs2=1.0 / 3.0):
    """2D Taylor-Green vortex on the periodic box L_a = n_a c_a:
    u_x = -u0 (k_y/k) cos(k_x x) sin(k_y y), u_y = u0 (k_x/k) sin(k_x x) cos(k_y y),
    p = p0 - rho0 u0^2 / 4 [(k_y/k)^2 cos(2 k_x x) + (k_x/k)^2 cos(2 k_y y)], rho = p / cs2."""
    x, y = coords(n, c)
    kx = 2.0 * np.pi / (n[0] * c[0])
    ky = 2.0 * np.pi / (n[1] * c[1])
    k = np.hypot(kx, ky) / np.sqrt(2.0)
    ux = -u0 * (ky / k) * np.cos(kx * x) * np.sin(ky * y)
    uy = u0 * (kx / k) * np.sin(kx * x) * np.cos(ky * y)
    dp = -0.25 * rho0 * u0 ** 2 * ((ky / k) ** 2 * np.cos(2 * kx * x) + (kx / k) ** 2 * np.cos(2 * ky * y))
    rho = rho0 + dp / cs2
    return rho, np.stack([ux, uy])


def taylor_green_3d(n, c, u0, rho0=1.0, cs2=1.0 / 3.0):
    """3D Taylor-Green vortex on the periodic box L_a = n_a c_a (phases k_a x_a):
    u = u0 (sin X cos Y cos Z, -cos X sin Y cos Z, 0),
    p = p0 + rho0 u0^2 / 16 (cos 2X + cos 2Y)(cos 2Z + 2), rho = p / cs2 with p0 = rho0 cs2."""
    x, y, z = coords(n, c)
    X = 2.0 * np.pi * x / (n[0] * c[0])
    Y = 2.0 * np.pi * y / (n[1] * c[1])
    Z = 2.0 * np.pi * z / (n[2] * c[2])
    ux = u0 * np.sin(X) * np.cos(Y) * np.cos(Z)
    uy = -u0 * np.cos(X) * np.sin(Y) * np.cos(Z)
    uz = np.zeros_like(ux)
    dp = rho0 * u0 ** 2 / 16.0 * (np.cos(2 * X) + np.cos(2 * Y)) * (np.cos(2 * Z) + 2.0)
    rho = rho0 + dp / cs2
    return rho, np.stack([ux, uy, uz])


def gaussian_hill(n, c, sigma, amplitude=1.0, noise=0.0, seed=0, center=None):
    """phi = A exp(-|x - x0|^2 / (2 sigma^2)) + U[-noise, noise] (sigma in units of dx_1)."""
    xs = coords(n, c)
    if center is None:
        center = [0.5 * n[a] * c[a] for a in range(len(n))]
    r2 = sum((xs[a] - center[a]) ** 2 for a in range(len(n)))
    phi = amplitude * np.exp(-r2 / (2.0 * sigma ** 2))
    if noise:
        phi = phi + _rng(seed).uniform(-noise, noise, size=phi.shape)
    return phi


def rest_state(n, d, rho0=1.0):
    shape = tuple(reversed(n))
    return np.full(shape, rho0), np.zeros((d,) + shape)


def random_fields(n, d, seed, rho_amp=0.02, u_amp=0.05):
    """rho = 1 + U[-rho_amp, rho_amp], u_a = U[-u_amp, u_amp] per cell."""
    g = _rng(seed)
    shape = tuple(reversed(n))
    rho = 1.0 + g.uniform(-rho_amp, rho_amp, size=shape)
    u = g.uniform(-u_amp, u_amp, size=(d,) + shape)
    return rho, u


def random_populations(n, Q, seed, lo=0.5, hi=1.5):
    """f_i(x) = U[lo, hi] / Q: a positive, far-from-equilibrium population array (Q, *grid)."""
    shape = (Q,) + tuple(reversed(n))
    return _rng(seed).uniform(lo, hi, size=shape) / Q


def random_scalar(n, seed, lo=-1.0, hi=1.0):
    return _rng(seed).uniform(lo, hi, size=tuple(reversed(n)))


SERVING_2D = ("rD2Q17", "rD2Q21", "rD2Q25")
SERVING_3D = ("rD3Q33", "rD3Q45", "rD3Q53-cubic")


def serving_requests(n, seed=0, rate_per_s=50.0, steps=(200, 5000), side2d=(32, 1024), ny2d=(32, 768),
                     side3d=(32, 160), frac_3d=0.5, frac_16bit=0.5):
    """A seeded stream of LB solve requests: Poisson arrivals at ``rate_per_s``; half 2D
    (rD2Q17/21/25, Taylor-Green or NCDE hill, n_x log-uniform in [32, 1024], n_y in [32, 768]),
    half 3D Kolmogorov on cubic cells (rD3Q33/45/53, side log-uniform in [32, 160]); steps
    uniform in [200, 5000]; storage FP32 or 16-bit. Each request is a dict."""
    g = _rng(seed)
    t = 0.0
    out = []
    for rid in range(int(n)):
        t += g.exponential(1.0 / rate_per_s)
        three_d = g.random() < frac_3d
        if three_d:
            lat = SERVING_3D[int(g.integers(0, 3))]
            side = int(round(np.exp(g.uniform(np.log(side3d[0]), np.log(side3d[1])))))
            grid = (side, side, side)
            flow = "kolmogorov"
        else:
            lat = SERVING_2D[int(g.integers(0, 3))]
            grid = (int(round(np.exp(g.uniform(np.log(side2d[0]), np.log(side2d[1]))))),
                    int(round(np.exp(g.uniform(np.log(ny2d[0]), np.log(ny2d[1]))))))
            flow = "tgv2d" if g.random() < 0.5 else "ncde"
        out.append(dict(rid=rid, arrival=t, lattice=lat, flow=flow, grid=grid,
                        steps=int(g.integers(steps[0], steps[1] + 1)),
                        store="16bit" if g.random() < frac_16bit else "f32", seed=int(seed * 100003 + rid)))
    return out
