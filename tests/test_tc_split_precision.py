"""Precision of the FP16 high/low split products used by the tensor-core kernels, emulated in numpy
against FP64 (no GPU).

On FP32 storage with one rate per order >= 4 the correction of the higher rows,
Delta_i = w_i sum_r a_r H_r(c_i) sum_j H_r(c_j) f_j (the rows of order >= 4 of Eq. (H-MRT-LB), with
a_r = -(s_r - s_high) / N_r), is applied as one dense Q x Q operator G_ij = sum_r a_r H_r(c_i)
H_r(c_j) whose rows are scaled to unit max by powers of two, times the populations scaled per cell
by a power of two; both are split into FP16 high and low parts and three products are summed
(hi.hi + hi.lo + lo.hi). These tests emulate exactly that arithmetic with the oracle's higher rows
and check it against the FP64 correction, and against the two-contraction form (y = H f, z = a y,
Delta = W H^T z, each operand split the same way) that it replaces.
"""
import numpy as np
import pytest

from oracle import lattice as OL
from paper_2512_16230_gb300 import workloads as W

RATES = {4: 0.8, 5: 1.35, 6: 1.6, 7: 0.9, 8: 1.25}
S_HIGH = 1.15
LATTICES = ["rD2Q9", "rD2Q13", "rD2Q17", "rD2Q21", "rD2Q25", "rD3Q27", "rD3Q33", "rD3Q45", "rD3Q53"]


def _f16(x):
    return np.asarray(x, dtype=np.float64).astype(np.float16).astype(np.float64)


def _split(x):
    hi = _f16(x)
    return hi, _f16(x - hi)


def _pow2(v):
    """The power of two that brings v > 0 into [1, 2) when multiplied by it."""
    return 2.0 ** -(np.frexp(v)[1] - 1)


def _higher(name):
    spec = W.LATTICES[name]
    lat = OL.build(spec.kind, spec.c, spec.cs2, spec.free_w)
    Hh = lat.Hfull[lat.R:]
    N = (Hh ** 2 * lat.w).sum(axis=1)
    a = -np.array([RATES.get(o, S_HIGH) - S_HIGH for o in lat.full_orders[lat.R:]]) / N
    return lat, Hh, a


def _dense(lat, Hh, a, f):
    G = (Hh.T * a) @ Hh
    rs = np.array([_pow2(np.abs(row).max()) if np.abs(row).max() > 0 else 1.0 for row in G])
    gh, gl = _split(G * rs[:, None])
    sa = _pow2(np.abs(f).max())
    fh, fl = _split(f * sa)
    D = gh @ fh + gl @ fh + gh @ fl
    return lat.w * D / rs / sa


def _two_contractions(lat, Hh, a, f):
    hs = np.array([_pow2(np.abs(row).max()) for row in Hh])
    Hhi, Hlo = _split(Hh * hs[:, None])
    sa = _pow2(np.abs(f).max())
    fh, fl = _split(f * sa)
    y = (Hhi @ fh + Hlo @ fh + Hhi @ fl) / hs / sa
    z = a * y
    sz = _pow2(np.abs(z).max())
    zh, zl = _split(z * sz)
    return lat.w * ((Hhi.T @ (zh / hs) + Hlo.T @ (zh / hs) + Hhi.T @ (zl / hs)) / sz)


@pytest.mark.parametrize("name", LATTICES)
def test_dense_operator_split_keeps_fp32_level_precision(name):
    lat, Hh, a = _higher(name)
    rng = np.random.default_rng(11)
    worst_dense = worst_two = 0.0
    for _ in range(40):
        f = lat.w * (1.0 + rng.uniform(-0.1, 0.1, lat.Q))
        exact = lat.w * (((Hh.T * a) @ Hh) @ f)
        # the dense operator is the two contractions associated the other way
        assert np.allclose(exact, lat.w * (Hh.T @ (a * (Hh @ f))), rtol=0, atol=1e-14 * np.abs(f).max())
        worst_dense = max(worst_dense, np.linalg.norm(_dense(lat, Hh, a, f) - exact) / np.linalg.norm(f))
        worst_two = max(worst_two, np.linalg.norm(_two_contractions(lat, Hh, a, f) - exact) / np.linalg.norm(f))
    assert worst_dense <= 1e-6
    assert worst_dense <= 2.0 * worst_two + 1e-8


def test_unscaled_operator_would_lose_bits():
    """Without the row scaling (one power of two for the whole operator) the large-weight rows of G,
    which are small next to the rows of the small weights, keep fewer bits: the row scaling is what
    holds the split at FP32 level on rD2Q25 (weights from 3e-4 to 0.27)."""
    lat, Hh, a = _higher("rD2Q25")
    G = (Hh.T * a) @ Hh
    s = _pow2(np.abs(G).max())
    gh, gl = _split(G * s)
    rng = np.random.default_rng(3)
    f = lat.w * (1.0 + rng.uniform(-0.1, 0.1, lat.Q))
    sa = _pow2(np.abs(f).max())
    fh, fl = _split(f * sa)
    unscaled = lat.w * (gh @ fh + gl @ fh + gh @ fl) / s / sa
    exact = lat.w * (G @ f)
    row_scaled = _dense(lat, Hh, a, f)
    e_unscaled = np.abs(unscaled - exact).max() / np.abs(exact).max()
    e_rows = np.abs(row_scaled - exact).max() / np.abs(exact).max()
    assert e_rows < e_unscaled
