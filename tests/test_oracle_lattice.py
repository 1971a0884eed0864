"""Pins of the oracle's lattice construction against what the paper fixes (CPU only).

Each test compares the oracle with something other than itself: printed worked examples
(App. C D2Q17 cases, Eq. (TransM), Eq. (TransM33)), printed closed forms (Eq. (Q13lattice),
the App. C/D correction coefficients), brute-force lattice moments (Eq. (new0)) against the
identities Eq. (Cont1-5), and the invariant HWH^T = diag (Sec. 4).
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

from oracle import lattice as L

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _ev(expr, env=None):
    scope = {"sqrt": math.sqrt, "__builtins__": {}}
    scope.update(env or {})
    return float(eval(expr, scope))


# Parameter points: the workload settings plus anisotropic ones (per-axis c_sa, Remark 2).
POINTS = [
    ("rD2Q25", (1.0, 4.0 / 3.0), (0.8, 0.8), (3.13e-4,) * 4),
    ("rD2Q25", (1.0, 1.2), (0.7, 0.9), (2e-4, 1e-4, 3e-4, 5e-5)),
    ("rD2Q21", (1.0, 4.0 / 3.0), (0.8, 0.8), (7.29e-4,) * 3),
    ("rD2Q17", (1.0, 4.0 / 3.0), (0.8, 0.8), (2.19e-3,)),
    ("rD2Q13", (1.0, 1.25), (0.8, 0.8), ()),
    ("rD2Q13", (1.0, 1.1), (0.6, 0.7), ()),
    ("rD3Q53", (1.0, 1.0, 4.0 / 3.0), (0.624,) * 3, (2.96e-4,)),
    ("rD3Q53", (1.0, 1.2, 4.0 / 3.0), (0.6, 0.62, 0.64), (1e-4,)),
    ("rD3Q53", (1.0, 1.0, 1.0), (0.6,) * 3, (2e-4,)),
    ("rD3Q45", (1.0, 1.0, 1.0), (0.6,) * 3, ()),
    ("rD3Q45", (1.0, 1.1, 1.25), (0.6, 0.62, 0.58), ()),
    ("rD3Q33", (1.0, 1.0, 1.0), (0.5,) * 3, ()),
    ("rD3Q33", (1.0, 1.1, 1.3), (0.5, 0.55, 0.6), ()),
]


def _id(p):
    return f"{p[0]}-c{'x'.join(f'{v:.3g}' for v in p[1])}-cs{'x'.join(f'{v:.3g}' for v in p[2])}"


@pytest.mark.parametrize("point", POINTS, ids=_id)
def test_weight_identities(point):
    """Eq. (Cont1-5), Eq. (new11): brute-force lattice moments of the closed-form weights."""
    kind, c, cs2, fw = point
    lat = L.build(kind, c, cs2, fw)
    w, cv, d = lat.w, lat.cvel, lat.d
    cs2 = np.asarray(cs2)
    assert abs(w.sum() - 1.0) < 1e-14                                   # Eq. (new11a)
    for a, b in itertools.product(range(d), repeat=2):
        want = cs2[a] if a == b else 0.0                                # Eq. (Cont1-5a), (new5)
        assert abs(L.lattice_moment(w, cv, (a, b)) - want) < 1e-14
    for a in range(d):
        assert abs(L.lattice_moment(w, cv, (a,) * 4) - 3 * cs2[a] ** 2) < 1e-13   # (Cont1-5c)
        for b in range(d):
            if a != b:                                                  # (Cont1-5b)
                assert abs(L.lattice_moment(w, cv, (a, a, b, b)) - cs2[a] * cs2[b]) < 1e-13
    if d == 3:                                                          # (Cont1-5e), (new11f)
        assert abs(L.lattice_moment(w, cv, (0, 0, 1, 1, 2, 2)) - np.prod(cs2)) < 1e-13
        if kind in ("rD3Q53", "rD3Q45"):
            # App. D imposes Eq. (new11e) in one direction only (alpha < beta)
            for a, b in [(0, 1), (0, 2), (1, 2)]:
                got = L.lattice_moment(w, cv, (a, a, a, a, b, b))
                assert abs(got - 3 * cs2[a] ** 2 * cs2[b]) < 1e-13
    # odd moments vanish by symmetry (Sec. 5)
    for order in (1, 3, 5):
        for idx in itertools.combinations_with_replacement(range(d), order):
            assert abs(L.lattice_moment(w, cv, idx)) < 1e-13


def test_rd2q13_closed_form_equals_rd2q25_subset():
    """Eq. (Q13lattice) equals Eq. (WeightQ25) with w13 = w17 = w18 = w21 = 0 (Sec. 5 (iii))."""
    for d01, d02 in [(0.8, 0.45), (0.6, 0.5), (0.9, 0.4)]:
        q13 = L.weights_rd2q13(d01, d02)
        q25 = L.expand_rd2q25(L.weights_rd2q25_classes(d01, d02, 0.0, 0.0, 0.0, 0.0))
        assert np.allclose(q13, q25[:13], rtol=0, atol=1e-15)
        assert np.all(q25[13:] == 0.0)


def test_weightq25_forms_agree():
    """Eq. (WeightQ25) and Eq. (WeightQ25-1) solve the same system with different free weights."""
    d01, d02 = 0.8, 0.45
    a = L.weights_rd2q25_classes(d01, d02, 3e-4, 2e-4, 1e-4, 5e-5)
    b = L.weights_rd2q25_classes_alt(d01, d02, a["w9"], a["w10"], a["w13"], a["w21"])
    for k in a:
        assert abs(a[k] - b[k]) < 1e-16


def _case_lattice(case):
    e = np.array([case["ex"], case["ey"]]).T
    W = {k: _ev(v) for k, v in case["w"].items()}
    w = np.array([W["w0"]] + [W["w1"]] * 4 + [W["w5"]] * 4 + [W["w9"]] * 4 + [W["w13"]] * 4)
    return e, w, W, _ev(case["cs2"])


@pytest.mark.parametrize("name", ["case1", "case2", "case3", "case4", "case5"])
def test_d2q17_worked_examples(name):
    """App. C: the printed D2Q17 weights satisfy Eq. (Cont1-5) on the printed velocity sets,
    and the oracle's rD2Q25 closed forms reproduce them from the sub-lattice's free weights."""
    case = json.load(open(os.path.join(GOLDEN, "d2q17_cases.json")))[name]
    e, w, W, cs2 = _case_lattice(case)
    tol = 2e-6 if name == "case5" else 1e-14      # case 5 is printed to 7 digits
    cv = e.astype(np.float64)
    assert abs(w.sum() - 1.0) < tol
    assert abs(L.lattice_moment(w, cv, (0, 0)) - cs2) < tol
    assert abs(L.lattice_moment(w, cv, (1, 1)) - cs2) < tol
    assert abs(L.lattice_moment(w, cv, (0, 0, 1, 1)) - cs2 ** 2) < 5 * tol
    assert abs(L.lattice_moment(w, cv, (0, 0, 0, 0)) - 3 * cs2 ** 2) < 5 * tol
    assert abs(L.lattice_moment(w, cv, (0, 0, 0, 0, 1, 1)) - 3 * cs2 ** 3) < 5 * tol
    if name != "case5":
        # cases 1-4 are also sixth-order isotropic
        assert abs(L.lattice_moment(w, cv, (0,) * 6) - 15 * cs2 ** 3) < 1e-13
    # the case as a sub-lattice of rD2Q25 (square, c = 1): the oracle's closed forms with the
    # case's own free weights give back every printed weight, and zero for removed velocities
    want = {k: _ev(v, W) for k, v in case["rd2q25"].items()}
    if want["w17"] == 0.0 and want["w18"] == 0.0:
        got = L.weights_rd2q25_classes(cs2, cs2, want["w13"], 0.0, 0.0, want["w21"])
    else:
        got = L.weights_rd2q25_classes_alt(cs2, cs2, want["w9"], want["w10"], want["w13"], want["w21"])
    for k in want:
        assert abs(got[k] - want[k]) < 5 * tol, (k, got[k], want[k])
    w25 = L.expand_rd2q25(got)
    assert abs(w25[0] - W["w0"]) < 5 * tol


def test_d2q17_case2_misprint():
    """App. C case 2 prints w9 and w13 ten times too small: the printed values violate
    sum w = 1 and Eq. (Cont1-5a) by many orders of round-off, the tenfold ones satisfy Eq. (Cont1-5) exactly (the reading used)."""
    case = json.load(open(os.path.join(GOLDEN, "d2q17_cases.json")))["case2"]
    e, w, W, cs2 = _case_lattice(case)
    wp = w.copy()
    wp[9:13] = _ev(case["printed_w9"])
    wp[13:17] = _ev(case["printed_w13"])
    assert abs(wp.sum() - 1.0) > 1e-4
    assert abs(L.lattice_moment(wp, e.astype(float), (0, 0)) - cs2) > 1e-3
    assert abs(w.sum() - 1.0) < 1e-14


def _mono_on(e, ex):
    return np.prod(e.astype(np.float64) ** np.asarray(ex)[None, :], axis=1)


def test_printed_transformation_matrix_rd2q13():
    """Eq. (TransM)/(TransM-D): the printed rD2Q13 M equals the monomials on the velocity set,
    and the oracle's Hermite rows H0..H3 are the stated polynomials of those monomials."""
    g = json.load(open(os.path.join(GOLDEN, "transm_rd2q13.json")))
    mono = {"1": (0, 0), "x": (1, 0), "y": (0, 1), "xx": (2, 0), "xy": (1, 1), "yy": (0, 2),
            "xyy": (1, 2), "xxy": (2, 1), "xxx": (3, 0), "yyy": (0, 3), "xxxx": (4, 0),
            "xxyy": (2, 2), "yyyy": (0, 4)}
    e = L.VELOCITIES["rD2Q13"]
    for name, row in zip(g["rows"], g["M"]):
        assert np.array_equal(_mono_on(e, mono[name]), np.array(row, dtype=float)), name
    M = np.array(g["M"], dtype=float)
    assert np.linalg.matrix_rank(M) == 13


def test_printed_transformation_matrix_rd3q33_misprints():
    """Eq. (TransM33): all printed rows but rows 12 and 17 (1-based) equal the symbolic
    monomials of App. D; row 12 is shifted and row 17 repeats row 16, so the printed matrix has
    rank 32 while the symbolic one has full rank 33 (the symbolic rows are used)."""
    g = json.load(open(os.path.join(GOLDEN, "transm_rd3q33.json")))
    e = L.VELOCITIES["rD3Q33"]
    M = np.array(g["M"], dtype=float)
    sym = np.stack([_mono_on(e, ex) for ex in g["monomials"]])
    bad = [r - 1 for r in g["misprinted_rows_1based"]]
    for r in range(33):
        if r in bad:
            assert not np.array_equal(M[r], sym[r])
        else:
            assert np.array_equal(M[r], sym[r]), r
    assert np.array_equal(M[16], M[15])
    assert np.linalg.matrix_rank(M) == 32
    assert np.linalg.matrix_rank(sym) == 33


@pytest.mark.parametrize("point", POINTS, ids=_id)
def test_hermite_orthogonality(point):
    """Sec. 4: HWH^T is block diagonal; after the rectangular correction H0..H3 are mutually
    W-orthogonal row by row, and the higher rows are W-orthogonal to H0..H3."""
    kind, c, cs2, fw = point
    lat = L.build(kind, c, cs2, fw)
    G = (lat.Hfull * lat.w) @ lat.Hfull.T
    R = lat.R
    scale = np.sqrt(np.abs(np.diag(G)))
    rel = np.abs(G) / np.outer(scale, scale)
    low = rel[:R, :R] - np.eye(R)
    assert np.abs(low).max() < 1e-13
    assert np.abs(rel[:R, R:]).max() < 1e-12   # high rows carry W-norms down to ~1e-5
    # H^{-1} = W H^T (H W H^T)^{-1} (Sec. 4) agrees with the LU inverse
    Hi = L.hermite_inverse(lat)
    Hw = L.hermite_inverse_weighted(lat)
    assert np.abs(Hi - Hw).max() < 1e-11 * np.abs(Hi).max()


def test_correction_is_needed_on_rectangular_cells():
    """Remark 3: without the correction, H_xxx and H_xyy are not W-orthogonal on a rectangular
    rD2Q25 lattice; with it they are."""
    lat = L.build("rD2Q25", (1.0, 4.0 / 3.0), (0.8, 0.8), (3.13e-4,) * 4)
    polys, _ = L.hermite_polys(2, lat.w, lat.cvel, correct=False)
    hxxx = L.poly_eval(polys[8], lat.cvel)
    hxyy = L.poly_eval(polys[6], lat.cvel)
    raw = np.sum(lat.w * hxxx * hxyy) / np.sqrt(np.sum(lat.w * hxxx ** 2) * np.sum(lat.w * hxyy ** 2))
    assert abs(raw) > 1e-2
    assert abs(np.sum(lat.w * lat.H[8] * lat.H[6])) < 1e-15


def test_explicit_rows_app_d():
    """App. D: H5 = E1^2 - cs1^2, H11 = E1 (E2^2 - cs2^2), H17 = E1 E2 E3 and the uncorrected
    H18 = E1^3 - 3 cs1^2 E1 (explicit rows) equal the oracle's generic Sec. 5 construction."""
    c, cs2 = (1.0, 1.2, 4.0 / 3.0), (0.6, 0.62, 0.64)
    lat = L.build("rD3Q53", c, cs2, (1e-4,))
    E = lat.cvel.T
    polys, _ = L.hermite_polys(3, lat.w, lat.cvel, correct=False)
    H = np.stack([L.poly_eval(p, lat.cvel) for p in polys])
    assert np.allclose(H[4], E[0] ** 2 - cs2[0], atol=1e-14)
    assert np.allclose(H[9], E[1] * E[2], atol=1e-14)
    assert np.allclose(H[10], E[0] * (E[1] ** 2 - cs2[1]), atol=1e-14)
    assert np.allclose(H[11], (E[2] ** 2 - cs2[2]) * E[0], atol=1e-14)
    assert np.allclose(H[16], E[0] * E[1] * E[2], atol=1e-14)
    assert np.allclose(H[17], E[0] ** 3 - 3 * cs2[0] * E[0], atol=1e-13)


@pytest.mark.parametrize("c,cs2,w45", [((1.0, 1.2, 4.0 / 3.0), (0.6, 0.62, 0.64), 1e-4),
                                       ((1.0, 1.2, 4.0 / 3.0), (0.624,) * 3, 2.96e-4),
                                       ((1.0, 1.1, 1.25), (0.58, 0.6, 0.61), 0.0)])
def test_rd3q53_correction_closed_form(c, cs2, w45):
    """App. D: the printed a_i, b_i of the rD3Q53 third-order correction equal the W-projections."""
    lat = L.build("rD3Q53", c, cs2, (w45,))
    d1, d2, d3 = np.asarray(cs2) / np.asarray(c) ** 2
    cls = L.weights_rd3q53_classes(d1, d2, d3, w45)
    a0 = 192 * cls["w33"] + 384 * w45
    b0 = 192 * cls["w37"] + 384 * w45
    c0 = 192 * cls["w41"] + 384 * w45
    c1, c2, c3 = c
    a1 = c1 ** 2 / c2 ** 2 * (d1 * d2 * (1 - 3 * d1) + a0) / (d2 * d1 * (1 - d2) + a0)
    a2 = c2 ** 2 / c1 ** 2 * (d2 * d1 * (1 - 3 * d2) + a0) / (d1 * d2 * (1 - d1) + a0)
    a3 = c3 ** 2 / c1 ** 2 * (d3 * d1 * (1 - 3 * d3) + b0) / (d1 * d3 * (1 - d1) + b0)
    b1 = c1 ** 2 / c3 ** 2 * (d1 * d3 * (1 - 3 * d1) + b0) / (d3 * d1 * (1 - d3) + b0)
    b2 = c2 ** 2 / c3 ** 2 * (d2 * d3 * (1 - 3 * d2) + c0) / (d3 * d2 * (1 - d3) + c0)
    b3 = c3 ** 2 / c2 ** 2 * (d3 * d2 * (1 - 3 * d3) + c0) / (d2 * d3 * (1 - d2) + c0)
    got = lat.corr
    for key, want in [((17, 10), a1), ((17, 11), b1), ((18, 12), a2), ((18, 13), b2),
                      ((19, 14), a3), ((19, 15), b3)]:
        assert abs(got[key] - want) < 1e-12 * max(1.0, abs(want)), (key, got[key], want)


@pytest.mark.parametrize("c,cs2", [((1.0, 1.0, 1.0), (0.5,) * 3),
                                   ((1.0, 1.1, 1.3), (0.5, 0.55, 0.6))])
def test_rd3q33_correction_closed_form(c, cs2):
    """App. D, rD3Q33: H18 = H18bar - a1 (H11/b2 + H12/b3) etc. with a_a = 3 cs_a^2 - c_a^2 and
    b_a = cs_a^2 - c_a^2: the printed coefficients equal the W-projections."""
    lat = L.build("rD3Q33", c, cs2)
    a = [3 * cs2[k] - c[k] ** 2 for k in range(3)]
    b = [cs2[k] - c[k] ** 2 for k in range(3)]
    want = {(17, 10): a[0] / b[1], (17, 11): a[0] / b[2], (18, 12): a[1] / b[0],
            (18, 13): a[1] / b[2], (19, 14): a[2] / b[0], (19, 15): a[2] / b[1]}
    for key, v in want.items():
        assert abs(lat.corr[key] - v) < 1e-12 * max(1.0, abs(v)), (key, lat.corr[key], v)


@pytest.mark.parametrize("c,cs2,w9", [((1.0, 4.0 / 3.0), (0.8, 0.8), 1e-3),
                                      ((1.0, 1.25), (0.7, 0.75), 5e-4)])
def test_special_d2q21_correction_closed_form(c, cs2, w9):
    """App. C special D2Q21 (knight moves): its printed weights satisfy Eq. (Cont1-5a-d) and the
    printed a1/b1, a2/b2 equal the W-projections of H9 on H7 and H10 on H8."""
    d1, d2 = np.asarray(cs2) / np.asarray(c) ** 2
    w5 = d1 * d2 / 4 - 8 * w9
    w17 = (d1 * (3 * d1 - 1) - 48 * w9) / 144
    w18 = (d2 * (3 * d2 - 1) - 48 * w9) / 144
    w1 = d1 / 2 - 2 * w5 - 10 * w9 - 9 * w17
    w2 = d2 / 2 - 2 * w5 - 10 * w9 - 9 * w18
    w0 = 1 - 2 * (w1 + w2 + 2 * w5 + 4 * w9 + w17 + w18)
    w = np.array([w0, w1, w2, w1, w2] + [w5] * 4 + [w9] * 8 + [w17, w18, w17, w18])
    e = L.E_SPECIAL_D2Q21
    lat = L.build_from("special-D2Q21", 2, np.asarray(c), np.asarray(cs2), e, w)
    cv = lat.cvel
    assert abs(w.sum() - 1) < 1e-15
    for a in range(2):
        assert abs(L.lattice_moment(w, cv, (a, a)) - cs2[a]) < 1e-14
        assert abs(L.lattice_moment(w, cv, (a,) * 4) - 3 * cs2[a] ** 2) < 1e-14
    assert abs(L.lattice_moment(w, cv, (0, 0, 1, 1)) - cs2[0] * cs2[1]) < 1e-14
    c1, c2 = c
    a1 = c1 ** 4 * c2 ** 2 * (-3 * d2 * d1 ** 2 + d2 * d1 + 48 * w9)
    b1 = c1 ** 2 * c2 ** 4 * (-d1 * d2 ** 2 + d1 * d2 + 48 * w9)
    a2 = c1 ** 2 * c2 ** 4 * (-3 * d1 * d2 ** 2 + d1 * d2 + 48 * w9)
    b2 = c1 ** 4 * c2 ** 2 * (-d2 * d1 ** 2 + d2 * d1 + 48 * w9)
    assert abs(lat.corr[(8, 6)] - a1 / b1) < 1e-12 * max(1, abs(a1 / b1))
    assert abs(lat.corr[(9, 7)] - a2 / b2) < 1e-12 * max(1, abs(a2 / b2))


def test_workload_weights_sign():
    """The workload parameter choices: all weights positive on the 2D lattices, on the cubic 3D
    serving lattices and on rD3Q53 with dz/dx = 4/3 and per-axis sound speeds (Remark 2)."""
    for kind, c, cs2, fw in POINTS[:1] + POINTS[2:5]:
        assert L.build(kind, c, cs2, fw).w.min() > 0
    assert L.build("rD3Q53", (1, 1, 1), (0.6,) * 3, (2.4e-4,)).w.min() > 0
    assert L.build("rD3Q45", (1, 1, 1), (0.6,) * 3).w.min() > 0
    assert L.build("rD3Q33", (1, 1, 1), (0.5,) * 3).w.min() > 0
    lat = L.build("rD3Q53", (1, 1, 4.0 / 3.0), (0.96, 0.96, 1.28), (8e-4,))
    assert lat.w.min() > 7.9e-4
    assert np.sum(lat.w * lat.H ** 2, axis=1).min() > 0


def test_shared_sound_speed_rd3q53_is_indefinite():
    """With dz/dx = 4/3 and one shared c_s the App. D weights cannot all be positive: the max-min
    choice (c_s^2 = 0.624, w45 = 2.96e-4) leaves a minimum weight of about -2.0e-3 and the
    corrected H_zzz row gets a negative W-norm, so H W H^T is diagonal but indefinite."""
    lat = L.build("rD3Q53", (1, 1, 4.0 / 3.0), (0.624,) * 3, (2.9625e-4,))
    assert -2.1e-3 < lat.w.min() < -1.9e-3
    N = np.sum(lat.w * lat.H ** 2, axis=1)
    assert N[19] < 0 and np.all(N[:19] > 0)


@pytest.mark.parametrize("kind,c,cs2", [("rD2Q9", (1.0, 1.0), (1 / 3, 1 / 3)), ("rD2Q9", (1.0, 4 / 3), (0.3, 0.3)),
                                        ("rD3Q27", (1.0, 1.0, 1.0), (1 / 3,) * 3),
                                        ("rD3Q27", (1.0, 1.2, 4 / 3), (0.3, 0.32, 0.34))])
def test_single_speed_weights(kind, c, cs2):
    """Single-speed lattices: sum w = 1, Delta2_aa = c_sa^2 and the mixed fourth/sixth moments are
    products (Eq. (new11a), (Cont1-5a), (Cont1-5b), (Cont1-5e)), while the axis fourth moment is
    c_a^2 c_sa^2 instead of 3 c_sa^4 (the anisotropy delta^(4) of k = 1); odd moments vanish; on
    the square D2Q9 / D3Q27 at c_s^2 = 1/3 the weights are the textbook 4/9, 1/9, 1/36 and
    8/27, 2/27, 1/54, 1/216."""
    lat = L.build(kind, c, cs2)
    d = lat.d
    m = lambda *idx: L.lattice_moment(lat.w, lat.cvel, idx)
    assert abs(lat.w.sum() - 1) < 1e-15
    for a in range(d):
        assert abs(m(a, a) - cs2[a]) < 1e-15
        assert abs(m(a) ) < 1e-15 and abs(m(a, a, a)) < 1e-15
        assert abs(m(a, a, a, a) - c[a] ** 2 * cs2[a]) < 1e-14
        for b in range(a + 1, d):
            assert abs(m(a, a, b, b) - cs2[a] * cs2[b]) < 1e-15
            assert abs(m(a, b)) < 1e-15
    if d == 3:
        assert abs(m(0, 0, 1, 1, 2, 2) - cs2[0] * cs2[1] * cs2[2]) < 1e-15
    if c == (1.0,) * d:
        want = [4 / 9, 1 / 9, 1 / 36] if d == 2 else [8 / 27, 2 / 27, 1 / 54, 1 / 216]
        near = np.abs(lat.w[:, None] - np.array(want)[None, :])
        assert near.min(axis=1).max() < 1e-15
        assert set(near.argmin(axis=1)) == set(range(len(want)))
    # the rows of order <= 3 are the paper's list without the pure cubes, mutually W-orthogonal
    # and W-orthogonal to the higher rows
    R = lat.R
    assert R == (8 if d == 2 else 17)
    G = (lat.Hfull * lat.w) @ lat.Hfull.T
    sc = np.sqrt(np.diag(G))
    rel = G / np.outer(sc, sc)
    assert np.abs(rel[:R, :R] - np.eye(R)).max() < 1e-13
    assert np.abs(rel[:R, R:]).max() < 1e-12
