"""Oracle, part 1: multispeed rectangular lattices and their Hermite matrices (FP64, numpy).

TEST INFRASTRUCTURE ONLY. Nothing in the product path may import this module; only
``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` use it.
It shares no code, tables or constants with the CUDA library.

Everything here follows Sec. 5 and Appendices C/D of Shi, Yuan & Chai (arXiv 2512.16230):

* velocity sets in the paper's column order: Eq. (3-1) (rD2Q25), Eq. (Q13lattice) (rD2Q13),
  App. D (rD3Q53, rD3Q33); rD2Q21/rD2Q17 are the sub-lattices of Sec. 5 (i)-(ii) obtained by
  zeroing weights of rD2Q25, rD3Q45 is rD3Q53 with omega_45 = 0;
* weights from the printed closed forms: Eq. (WeightQ25) / (WeightQ25-1), Eq. (Q13lattice),
  the rD3Q53 / rD3Q33 weight lists of App. D, with d_0a = c_sa^2 / c_a^2 (the definition given
  with Eq. (new11); App. D prints the inverse ratio, which contradicts its own range and every
  identity of Eq. (Cont1-5));
* Hermite rows H0..H3 as defined in Sec. 5 (H2 = <EE> - Delta2, H3 = ccc - <c Delta2>), with the
  third-order rows corrected for rectangular cells by the W-projections of Eq. (CorrectQ25)
  (2D) and App. D (3D);
* rows of order >= 4 (left to the modeller by App. C/D) taken from the paper's own lists where it
  prints one (rD2Q13: Eq. (TransM); rD3Q33: the symbolic rows M21..M33 of App. D), otherwise
  graded monomials kept greedily when they raise the rank; the rows of degree k are
  W-orthogonalised against every row of lower degree, so that HWH^T is block diagonal as Sec. 4
  requires and each order k >= 4 is a block that can carry its own rate.

Polynomials are dicts {exponent tuple: coefficient} in the physical velocity c = diag(c_a) e.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass, field

import numpy as np

KINDS = ("rD2Q13", "rD2Q17", "rD2Q21", "rD2Q25", "rD3Q33", "rD3Q45", "rD3Q53", "rD2Q9", "rD3Q27")

# Single-speed (standard) lattices on rectangular cells: the special case of Sec. 3.4 with k = 1,
# whose velocity components are 0 and +-1 only.
SINGLE_SPEED = ("rD2Q9", "rD3Q27")

# ---------------------------------------------------------------------------------------------
# Velocity sets (integer multiples e_j of the axis speeds c_a), columns in the paper's order.
# ---------------------------------------------------------------------------------------------

# Eq. (3-1): rD2Q25.
E_RD2Q25 = np.array([
    [0, 1, 0, -1, 0, 1, -1, -1, 1, 2, 0, -2, 0, 2, -2, -2, 2, 3, 0, -3, 0, 3, -3, -3, 3],
    [0, 0, 1, 0, -1, 1, 1, -1, -1, 0, 2, 0, -2, 2, 2, -2, -2, 0, 3, 0, -3, 3, 3, -3, -3],
], dtype=np.int64).T

# App. D, rD3Q53: the 27 single-speed vectors followed by the 26 doubled non-zero ones.
_E27 = np.array([
    [0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, -1, 1],
    [0, 0, 0, 1, -1, 0, 0, 1, -1, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, 1, -1, -1, 1, 1, -1],
    [0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 1, -1, -1, 1, 1, -1, 1, -1],
], dtype=np.int64).T
E_RD3Q53 = np.concatenate([_E27, 2 * _E27[1:]], axis=0)

# Sub-lattices keep the parent's column order (Sec. 5 (i)-(iii); App. D rD3Q33 lists the first
# 33 columns of rD3Q53; rD3Q45 drops the eight (+-2,+-2,+-2) vectors, i.e. omega_45 = 0).
VELOCITIES = {
    "rD2Q25": E_RD2Q25,
    "rD2Q21": E_RD2Q25[:21],
    "rD2Q17": E_RD2Q25[:17],
    "rD2Q13": E_RD2Q25[:13],
    "rD3Q53": E_RD3Q53,
    "rD3Q45": E_RD3Q53[:45],
    "rD3Q33": E_RD3Q53[:33],
    "rD2Q9": E_RD2Q25[:9],       # rest, the four axis and the four diagonal vectors
    "rD3Q27": E_RD3Q53[:27],     # every vector with components in {-1, 0, 1}
}

# App. C: the special D2Q21 lattice with knight-move velocities (a CHECK case, not a runtime lattice).
E_SPECIAL_D2Q21 = np.array([
    [0, 1, 0, -1, 0, 1, -1, -1, 1, 2, 1, -1, -2, -2, -1, 1, 2, 3, 0, -3, 0],
    [0, 0, 1, 0, -1, 1, 1, -1, -1, 1, 2, 2, 1, -1, -2, -2, -1, 0, 3, 0, -3],
], dtype=np.int64).T

# Number of free weights each kind takes, in this order:
#   rD2Q25: (w13, w17, w18, w21)   Eq. (WeightQ25)
#   rD2Q21: (w13, w17, w18)        rD2Q25 with w21 = 0
#   rD2Q17: (w13,)                 rD2Q25 with w21 = w17 = w18 = 0
#   rD2Q13: ()                     Eq. (Q13lattice)
#   rD3Q53: (w45,)                 App. D
#   rD3Q45: ()                     rD3Q53 with w45 = 0
#   rD3Q33: ()                     App. D (w33 = w37 = w41 = w45 = 0)
N_FREE = {"rD2Q25": 4, "rD2Q21": 3, "rD2Q17": 1, "rD2Q13": 0,
          "rD3Q53": 1, "rD3Q45": 0, "rD3Q33": 0, "rD2Q9": 0, "rD3Q27": 0}


def dim_of(kind: str) -> int:
    return 2 if kind.startswith("rD2") else 3


# ---------------------------------------------------------------------------------------------
# Weights
# ---------------------------------------------------------------------------------------------

def d0(c, cs2):
    """d_0a = c_sa^2 / c_a^2, the definition stated with Eq. (new11)."""
    return np.asarray(cs2, dtype=np.float64) / np.asarray(c, dtype=np.float64) ** 2


def weights_rd2q25_classes(d01, d02, w13, w17, w18, w21):
    """Eq. (WeightQ25): free w13, w17, w18, w21; returns the ten weight classes of Eq. (3-1-2)."""
    w5 = 0.25 * (d01 * d02 - 64.0 * w13 - 324.0 * w21)
    w9 = (d01 * (3.0 * d01 - 1.0) - 48.0 * w13 - 144.0 * w17 - 288.0 * w21) / 24.0
    w10 = (d02 * (3.0 * d02 - 1.0) - 48.0 * w13 - 144.0 * w18 - 288.0 * w21) / 24.0
    w1 = 0.5 * d01 - (2.0 * w5 + 4.0 * w9 + 8.0 * w13 + 9.0 * w17 + 18.0 * w21)
    w2 = 0.5 * d02 - (2.0 * w5 + 4.0 * w10 + 8.0 * w13 + 9.0 * w18 + 18.0 * w21)
    return dict(w1=w1, w2=w2, w5=w5, w9=w9, w10=w10, w13=w13, w17=w17, w18=w18, w21=w21)


def weights_rd2q25_classes_alt(d01, d02, w9, w10, w13, w21):
    """Eq. (WeightQ25-1): the same system solved with w9, w10, w13, w21 free."""
    w5 = 0.25 * (d01 * d02 - 64.0 * w13 - 324.0 * w21)
    w17 = (d01 * (3.0 * d01 - 1.0) - 24.0 * w9 - 48.0 * w13 - 288.0 * w21) / 144.0
    w18 = (d02 * (3.0 * d02 - 1.0) - 24.0 * w10 - 48.0 * w13 - 288.0 * w21) / 144.0
    w1 = 0.5 * d01 - (2.0 * w5 + 4.0 * w9 + 8.0 * w13 + 9.0 * w17 + 18.0 * w21)
    w2 = 0.5 * d02 - (2.0 * w5 + 4.0 * w10 + 8.0 * w13 + 9.0 * w18 + 18.0 * w21)
    return dict(w1=w1, w2=w2, w5=w5, w9=w9, w10=w10, w13=w13, w17=w17, w18=w18, w21=w21)


def expand_rd2q25(cls) -> np.ndarray:
    """Eq. (3-1-2): per-velocity weights of rD2Q25 from its classes; w0 = 1 - sum_{j>0} w_j."""
    w = np.empty(25)
    for j, name in enumerate(["w1", "w2", "w1", "w2"], start=1):
        w[j] = cls[name]
    w[5:9] = cls["w5"]
    w[9], w[10], w[11], w[12] = cls["w9"], cls["w10"], cls["w9"], cls["w10"]
    w[13:17] = cls["w13"]
    w[17], w[18], w[19], w[20] = cls["w17"], cls["w18"], cls["w17"], cls["w18"]
    w[21:25] = cls["w21"]
    w[0] = 1.0 - w[1:].sum()
    return w


def weights_rd2q13(d01, d02) -> np.ndarray:
    """Eq. (Q13lattice): closed-form rD2Q13 weights, W = diag{w0,w1,w2,w1,w2,w5 x4,w9,w10,w9,w10}."""
    w9 = d01 * (3.0 * d01 - 1.0) / 24.0
    w10 = d02 * (3.0 * d02 - 1.0) / 24.0
    w0 = (1.0 - d01) * (1.0 - d02) + 6.0 * (w9 + w10)
    w1 = 0.5 * d01 * (1.0 - d02) - 4.0 * w9
    w2 = 0.5 * d02 * (1.0 - d01) - 4.0 * w10
    w5 = 0.25 * d01 * d02
    return np.array([w0, w1, w2, w1, w2, w5, w5, w5, w5, w9, w10, w9, w10])


def weights_rd3q53_classes(d01, d02, d03, w45):
    """App. D, rD3Q53 weight list (free w45); returns the 15 weight classes."""
    w19 = d01 * d02 * d03 / 8.0 - 64.0 * w45
    w33 = d01 * d02 * (3.0 * d01 - 1.0) / 192.0 - 2.0 * w45
    w37 = d01 * d03 * (3.0 * d01 - 1.0) / 192.0 - 2.0 * w45
    w41 = d02 * d03 * (3.0 * d02 - 1.0) / 192.0 - 2.0 * w45
    w7 = d01 * d02 / 4.0 - 2.0 * w19 - 16.0 * w33 - 32.0 * w45
    w11 = d01 * d03 / 4.0 - 2.0 * w19 - 16.0 * w37 - 32.0 * w45
    w15 = d02 * d03 / 4.0 - 2.0 * w19 - 16.0 * w41 - 32.0 * w45
    w27 = d01 * (3.0 * d01 - 1.0) / 24.0 - 2.0 * (w33 + w37) - 4.0 * w45
    w28 = d02 * (3.0 * d02 - 1.0) / 24.0 - 2.0 * (w33 + w41) - 4.0 * w45
    w29 = d03 * (3.0 * d03 - 1.0) / 24.0 - 2.0 * (w41 + w37) - 4.0 * w45
    w1 = d01 / 2.0 - 2.0 * (w7 + w11) - 4.0 * w19 - 4.0 * w27 - 8.0 * (w33 + w37) - 16.0 * w45
    w2 = d02 / 2.0 - 2.0 * (w7 + w15) - 4.0 * w19 - 4.0 * w28 - 8.0 * (w33 + w41) - 16.0 * w45
    w3 = d03 / 2.0 - 2.0 * (w11 + w15) - 4.0 * w19 - 4.0 * w29 - 8.0 * (w41 + w37) - 16.0 * w45
    w0 = (1.0 - 2.0 * (w1 + w2 + w3 + w27 + w28 + w29)
          - 4.0 * (w7 + w11 + w15 + w33 + w37 + w41) - 8.0 * (w19 + w45))
    return dict(w0=w0, w1=w1, w2=w2, w3=w3, w7=w7, w11=w11, w15=w15, w19=w19, w27=w27,
                w28=w28, w29=w29, w33=w33, w37=w37, w41=w41, w45=w45)


def weights_rd3q33_classes(d01, d02, d03):
    """App. D, rD3Q33 weight list (w33 = w37 = w41 = w45 = 0)."""
    w19 = d01 * d02 * d03 / 8.0
    w7 = d01 * d02 / 4.0 - 2.0 * w19
    w11 = d01 * d03 / 4.0 - 2.0 * w19
    w15 = d02 * d03 / 4.0 - 2.0 * w19
    w27 = d01 * (3.0 * d01 - 1.0) / 24.0
    w28 = d02 * (3.0 * d02 - 1.0) / 24.0
    w29 = d03 * (3.0 * d03 - 1.0) / 24.0
    w1 = d01 / 2.0 - 2.0 * (w7 + w11) - 4.0 * w19 - 4.0 * w27
    w2 = d02 / 2.0 - 2.0 * (w7 + w15) - 4.0 * w19 - 4.0 * w28
    w3 = d03 / 2.0 - 2.0 * (w11 + w15) - 4.0 * w19 - 4.0 * w29
    w0 = 1.0 - 2.0 * (w1 + w2 + w3 + w27 + w28 + w29) - 4.0 * (w7 + w11 + w15) - 8.0 * w19
    return dict(w0=w0, w1=w1, w2=w2, w3=w3, w7=w7, w11=w11, w15=w15, w19=w19,
                w27=w27, w28=w28, w29=w29)


def expand_rd3(cls, q: int) -> np.ndarray:
    """App. D weight matrices W: per-velocity weights for the first q columns of rD3Q53."""
    order = (["w0"] + ["w1"] * 2 + ["w2"] * 2 + ["w3"] * 2 + ["w7"] * 4 + ["w11"] * 4
             + ["w15"] * 4 + ["w19"] * 8 + ["w27"] * 2 + ["w28"] * 2 + ["w29"] * 2
             + ["w33"] * 4 + ["w37"] * 4 + ["w41"] * 4 + ["w45"] * 8)
    return np.array([cls.get(name, 0.0) for name in order[:q]])


def weights(kind: str, c, cs2, free_w=()) -> np.ndarray:
    """Per-velocity weights of ``kind`` for axis speeds ``c`` and squared sound speeds ``cs2``."""
    dd = d0(c, cs2)
    free_w = tuple(float(v) for v in free_w)
    if len(free_w) != N_FREE[kind]:
        raise ValueError(f"{kind} takes {N_FREE[kind]} free weights, got {len(free_w)}")
    if kind == "rD2Q13":
        return weights_rd2q13(dd[0], dd[1])
    if kind in ("rD2Q25", "rD2Q21", "rD2Q17"):
        w13, w17, w18, w21 = {"rD2Q25": lambda f: f,
                              "rD2Q21": lambda f: (f[0], f[1], f[2], 0.0),
                              "rD2Q17": lambda f: (f[0], 0.0, 0.0, 0.0)}[kind](free_w)
        w = expand_rd2q25(weights_rd2q25_classes(dd[0], dd[1], w13, w17, w18, w21))
        q = int(kind[4:])
        assert np.all(w[q:] == 0.0)
        return w[:q]
    if kind in ("rD3Q53", "rD3Q45"):
        w45 = free_w[0] if kind == "rD3Q53" else 0.0
        cls = weights_rd3q53_classes(dd[0], dd[1], dd[2], w45)
        return expand_rd3(cls, int(kind[4:]))
    if kind == "rD3Q33":
        return expand_rd3(weights_rd3q33_classes(dd[0], dd[1], dd[2]), 33)
    if kind in SINGLE_SPEED:
        return weights_single_speed(VELOCITIES[kind], dd)
    raise ValueError(kind)


def weights_single_speed(e, dd) -> np.ndarray:
    """Single-speed lattices: the weight conditions of Eq. (new11) that a velocity set with
    components in {0, +-1} can meet are sum w = 1, Delta2_aa = c_sa^2 and the mixed fourth (and,
    in 3D, sixth) moments Delta4_aabb = Delta2_aa Delta2_bb, Delta6_xxyyzz = Delta2_xx Delta2_yy
    Delta2_zz (the axis condition Delta4_aaaa = 3 Delta2_aa^2 fails unless d_0a = 1/3: that defect
    is the delta^(4) of k = 1). With one weight per reflection class these conditions are solved
    by the product of the one-dimensional weights w(0) = 1 - d_0a, w(+-1) = d_0a / 2."""
    w = np.ones(e.shape[0])
    for a in range(e.shape[1]):
        w = w * np.where(e[:, a] == 0, 1.0 - dd[a], 0.5 * dd[a])
    return w


def lattice_moment(w, cvel, idx) -> float:
    """Eq. (new0): Delta^(k)_{i1..ik} = sum_j w_j c_{j,i1} ... c_{j,ik} (brute force)."""
    prod = np.ones(len(w))
    for a in idx:
        prod = prod * cvel[:, a]
    return float(np.sum(w * prod))


# ---------------------------------------------------------------------------------------------
# Polynomials in the velocity components
# ---------------------------------------------------------------------------------------------

def _unit(d, axes):
    ex = [0] * d
    for a in axes:
        ex[a] += 1
    return tuple(ex)


def poly_add(p, q, scale=1.0):
    out = dict(p)
    for k, v in q.items():
        out[k] = out.get(k, 0.0) + scale * v
    return {k: v for k, v in out.items() if v != 0.0}


def poly_eval(p, cvel) -> np.ndarray:
    """Evaluate a polynomial at every lattice velocity c_j (rows of ``cvel``)."""
    out = np.zeros(cvel.shape[0])
    for ex, coef in p.items():
        term = np.full(cvel.shape[0], coef)
        for a, k in enumerate(ex):
            term = term * cvel[:, a] ** k
        out += term
    return out


def poly_degree(p) -> int:
    return max(sum(ex) for ex in p) if p else 0


# Row labels in the paper's order: 2D rows as in App. C (H_1..H_10), 3D rows as in App. D (H_1..H_20).
ROWS_2D = [(), (0,), (1,), (0, 0), (0, 1), (1, 1), (0, 1, 1), (0, 0, 1), (0, 0, 0), (1, 1, 1)]
ROWS_3D = [(), (0,), (1,), (2,), (0, 0), (1, 1), (2, 2), (0, 1), (2, 0), (1, 2),
           (0, 1, 1), (2, 2, 0), (0, 0, 1), (1, 2, 2), (2, 0, 0), (1, 1, 2), (0, 1, 2),
           (0, 0, 0), (1, 1, 1), (2, 2, 2)]

# Third-order rows corrected for rectangular cells and the rows they are projected against:
# Eq. (CorrectQ25) in 2D (H_xxx against H_xyy, H_yyy against H_xxy) and App. D in 3D
# (H18 against H11, H12; H19 against H13, H14; H20 against H15, H16; 1-based row numbers).
CORRECTIONS_2D = {8: (6,), 9: (7,)}
CORRECTIONS_3D = {17: (10, 11), 18: (12, 13), 19: (14, 15)}


def hermite_polys(d, w, cvel, correct=True, single=False):
    """Sec. 5: H0 = e, H1 = E, H2 = <EE> - Delta2, H3 = ccc - <c Delta2>, then the
    rectangular-cell correction of the third-order rows by W-projection (Eq. (CorrectQ25), App. D).

    Delta2 is the lattice tensor of Eq. (new0) computed from the weights. Returns the list of
    polynomials and the projection coefficients used by the correction. ``single``: a
    single-speed lattice, where c_a^3 is c_a^2 times c_a, so the pure cubes (the last d rows, the
    only corrected ones) are dependent on the first-order rows and are left out."""
    rows = row_list(d, single)
    delta2 = np.array([[lattice_moment(w, cvel, (a, b)) for b in range(d)] for a in range(d)])
    polys = []
    for axes in rows:
        p = {_unit(d, axes): 1.0}
        if len(axes) == 2:
            a, b = axes
            p = poly_add(p, {_unit(d, ()): -delta2[a, b]})
        elif len(axes) == 3:
            a, b, g = axes
            p = poly_add(p, {_unit(d, (a,)): -delta2[b, g]})
            p = poly_add(p, {_unit(d, (b,)): -delta2[a, g]})
            p = poly_add(p, {_unit(d, (g,)): -delta2[a, b]})
        polys.append(p)
    coefs = {}
    if correct and not single:
        corr = CORRECTIONS_2D if d == 2 else CORRECTIONS_3D
        for r, against in corr.items():
            hbar = poly_eval(polys[r], cvel)
            p = polys[r]
            for s in against:
                hs = poly_eval(polys[s], cvel)
                a = float(np.sum(w * hbar * hs) / np.sum(w * hs * hs))
                coefs[(r, s)] = a
                p = poly_add(p, polys[s], -a)
            polys[r] = p
    return polys, coefs


def row_list(d, single=False):
    """Rows of order <= 3 in the paper's order; single-speed lattices drop the pure cubes."""
    rows = ROWS_2D if d == 2 else ROWS_3D
    return rows[:len(rows) - d] if single else rows


# Orders of the rows above (0..3), used for the blocks H_k of Eq. (feq-1).
def row_orders(d, single=False):
    return [len(a) for a in row_list(d, single)]


# Higher rows printed by the paper: rD2Q13 rows 11-13 of Eq. (TransM) and rD3Q33 rows M21..M33 (App. D).
HIGH_ROWS_PRINTED = {
    "rD2Q13": [(4, 0), (2, 2), (0, 4)],
    "rD3Q33": [(2, 2, 0), (2, 0, 2), (0, 2, 2), (2, 1, 1), (1, 2, 1), (1, 1, 2), (4, 0, 0),
               (0, 4, 0), (0, 0, 4), (2, 2, 1), (2, 1, 2), (1, 2, 2), (2, 2, 2)],
}


def graded_monomials(d, start_degree, max_degree=12):
    for deg in range(start_degree, max_degree + 1):
        for ex in sorted((e for e in itertools.product(range(deg + 1), repeat=d) if sum(e) == deg),
                         reverse=True):
            yield ex


@dataclass
class Lattice:
    kind: str
    d: int
    c: np.ndarray          # axis speeds c_a = dx_a / dt (lattice units, c_1 = 1)
    cs2: np.ndarray        # per-axis squared sound speeds c_sa^2 (Remark 2)
    e: np.ndarray          # (Q, d) integer velocities
    cvel: np.ndarray       # (Q, d) physical velocities c_j = diag(c) e_j
    w: np.ndarray          # (Q,) weights
    polys: list            # R Hermite polynomials (orders 0..3), paper's order
    H: np.ndarray          # (R, Q) Hermite rows evaluated on the lattice
    orders: list           # order of each of the R rows
    corr: dict             # rectangular-correction projection coefficients
    Hfull: np.ndarray      # (Q, Q) full Hermite matrix: H0..H3 then W-orthogonalised higher rows
    high_monomials: list = field(default_factory=list)
    full_orders: list = field(default_factory=list)   # order (degree) of every row of Hfull

    @property
    def Q(self):
        return self.e.shape[0]

    @property
    def R(self):
        return self.H.shape[0]

    def block(self, k):
        """Row indices of the order-k block H_k."""
        return [r for r, o in enumerate(self.orders) if o == k]


def build(kind: str, c, cs2, free_w=(), correct=True, high_rows=None) -> Lattice:
    """Construct a lattice: velocities, weights, Hermite rows H0..H3 and the full Q x Q matrix."""
    if kind not in VELOCITIES:
        raise ValueError(kind)
    d = dim_of(kind)
    c = np.asarray(c, dtype=np.float64)
    cs2 = np.asarray(cs2, dtype=np.float64)
    e = VELOCITIES[kind]
    cvel = e * c[None, :]
    w = weights(kind, c, cs2, free_w)
    return build_from(kind, d, c, cs2, e, w, correct=correct, high_rows=high_rows)


def build_from(kind, d, c, cs2, e, w, correct=True, high_rows=None) -> Lattice:
    cvel = e * np.asarray(c)[None, :]
    single = kind in SINGLE_SPEED
    polys, coefs = hermite_polys(d, w, cvel, correct=correct, single=single)
    H = np.stack([poly_eval(p, cvel) for p in polys])
    orders = row_orders(d, single)
    Q = e.shape[0]
    # Higher rows, graded by degree: the order-k block is the W-orthogonal complement of all rows of
    # lower degree inside the span of the monomials of degree <= k on the lattice (a subspace fixed
    # by the lattice alone, so a rate per order is well defined whichever monomials are listed).
    # Candidates come from the paper's lists where printed, otherwise graded monomials; a
    # candidate is kept when it raises the rank.
    cands = high_rows if high_rows is not None else HIGH_ROWS_PRINTED.get(kind)
    cands = list(cands) if cands is not None else list(graded_monomials(d, 4))
    cands = sorted(cands, key=sum)
    rows = [H[r] for r in range(H.shape[0])]
    degs = list(orders)
    chosen = []
    for deg in sorted({sum(ex) for ex in cands}):
        block = []
        for ex in [c for c in cands if sum(c) == deg]:
            v = poly_eval({tuple(ex): 1.0}, cvel)
            v = v / np.abs(v).max()
            trial = np.vstack(rows + block + [v[None, :]])
            if np.linalg.matrix_rank(trial, tol=1e-9 * np.abs(trial).max()) == trial.shape[0]:
                block.append(v)
                chosen.append(tuple(ex))
            if len(rows) + len(block) == Q:
                break
        if not block:
            continue
        # W-orthogonalise the block against every lower-degree row (block-diagonal H W H^T, Sec. 4),
        # then take an orthonormal basis of its span (any basis of the block gives the same
        # collision when the block shares one rate)
        prev = np.vstack(rows)
        G = (prev * w) @ prev.T
        B = np.vstack(block)
        # (pseudo-inverse: G is singular when a weight class is zero and the rows outnumber the
        # velocities of non-zero weight; the projection is then still W-orthogonal)
        # (applied twice: one projection in floating point leaves O(eps cond) overlap)
        Gi = np.linalg.pinv(G, rcond=1e-13)
        for _ in range(2):
            B = B - ((B * w) @ prev.T) @ Gi @ prev
        qmat, _ = np.linalg.qr(B.T)
        for q in qmat.T:
            rows.append(q)
            degs.append(deg)
        if len(rows) == Q:
            break
    if len(rows) != Q:
        raise ValueError(f"{kind}: could not complete the Hermite matrix ({len(rows)} of {Q})")
    Hfull = np.vstack(rows)
    high_orders = degs
    return Lattice(kind=kind, d=d, c=np.asarray(c), cs2=np.asarray(cs2), e=e, cvel=cvel, w=w,
                   polys=polys, H=H, orders=orders, corr=coefs, Hfull=Hfull, high_monomials=chosen,
                   full_orders=high_orders)


def hermite_inverse(lat: Lattice) -> np.ndarray:
    """H^{-1} of the full Q x Q Hermite matrix (plain LU inverse)."""
    return np.linalg.inv(lat.Hfull)


def hermite_inverse_weighted(lat: Lattice) -> np.ndarray:
    """Sec. 4: H^{-1} = W H^T (H W H^T)^{-1}, valid when HWH^T is block diagonal."""
    W = np.diag(lat.w)
    return W @ lat.Hfull.T @ np.linalg.inv(lat.Hfull @ W @ lat.Hfull.T)
