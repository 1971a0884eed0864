"""Oracle, part 2: the MRT-LB time step (FP64, numpy).

TEST INFRASTRUCTURE ONLY. Nothing in the product path may import this module; only
``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` use it.

The step follows Shi, Yuan & Chai (arXiv 2512.16230) in the paper's order:

* state: the transformed distribution f-bar of the full-correction scheme, Eq. (2-3);
* macroscopic fields with the half-source correction: Eq. (2-4-2) (NSE) and Eq. (2-4-1) (NCDE);
* equilibrium moments in the Hermite basis from the continuous moments M0..M3 of
  Eq. (M-NSEs-6a) / (M-NSEs-6-1) with k = 0 and M30 = rho u u u (Sec. 3.4: multispeed lattices),
  p = rho * cs2_eq (isothermal); for the NCDE from Eq. (M-NCDE-6): M0 = phi, M1 = u phi,
  M2 = cs2_eq D(phi) I with M20 = 0;
* the EDF and the source distributions from their Hermite moments by Eq. (feq-1) / Eq. (geq);
* the collision f~ = f - Lambda f^ne + dt [G + (I - Lambda/2) F] of Eq. (2-3) with
  Lambda = H^{-1} S H built from the full Q x Q Hermite matrix (Sec. 4, Eq. (H-MRT-LB));
* propagation f(x + c_j dt, t + dt) = f~(x, t), Eq. (2-2b), periodic.

Readings of points the paper leaves open (each is listed in the design notes):
* NSE source split (Eq. (M-NSEs-2), (M-NSEs-5)): S = 0, F_F = F, F_G = 0, so the SDF F has
  M0F = 0, M1F = F, M2F = 0 and G carries only M2G = (I - S2/2)(uF + Fu) (Eq. (M2Ga-1) with
  S = 0); third-order Hermite moments of F and G are zero.
* NCDE (App. A): S = 0, M1F = 0, G carries only M1G = (I - S1/2) d_t(u phi) with constant u
  and d_t phi by the backward difference (phi^n - phi^{n-1}) / dt, phi^{-1} = phi^0;
  the third-order Hermite moments of the NCDE equilibrium are zero.
* NCDE variants of App. A: ``ncde_mode="rate"`` puts the nonlinearity into per-cell first-order
  rates, K(phi) = K0 (1 + nonlin phi^2) = cs2_eq (1/s1(phi) - 1/2), with D(phi) = phi in M2;
  ``ncde_mode="cde"`` is special case (3), the diffusion-based CDE (M1 = 0, M2 = cs2_eq phi I,
  lambda = 1, S_G = -u . grad phi from the local gradient of Eq. (M-NCDE-3-00), M0G =
  (1 - s0/2) S_G); ``a1`` adds the mixed-derivative term of Eq. (GNCDE) with A1 = a1 I and
  B-bar = u phi, whose coefficient is dt A1 by the derivation (the printed K1 = dt S1 A1 carries
  the same slip as the printed K). ``a2`` with ``psi`` adds the cross-diffusion term of
  Eq. (GNCDE): A2 = a2 I and D-bar = psi I for a prescribed cell field psi, so M1G gains
  -S1 A2 grad psi (grad psi by central differences over the cell spacing c_a dt) and the
  equation gains div(dt A2 grad psi) (K2 = dt A2 by the derivation, as for K1).
* rows of order >= 4 (left to the designer by the paper) relax with one shared rate s_high, or
  with ``s_orders`` one rate per order k on the graded block: the W-orthogonal complement of the
  lower orders inside the lattice functions spanned by the monomials of degree <= k.
* the anisotropy term of Eq. (M2Ga) on the single-speed lattices (``m2g_aniso``): the bracket
  of M2G gains (delta4 . u) . grad rho, which is diagonal, (c_a^2 - 3 cs2_eq) u_a d_a rho on the
  normal row of axis a (delta4_aaaa = c_a^2 - 3 c_s^2, zero elsewhere, Sec. 3.4). grad rho is
  the second-order central difference, over the cell spacing c_a dt, of the density of the
  previous step; the first step after init_fields / set_populations takes the density of that
  state (rho^{-1} = rho^0, as for phi).
* bulk viscosity (Eq. (4-27)): with ``s_bulk`` the normal second-order rows relax through
  the inverse of S2^(1) = diag(1/s_s) + a b^T / d, with a = 1/s_b - 1/s_s, b = 1 on the
  multispeed lattices (k = 0) and the printed (c_a^2 - c_s^2) factors on the single-speed ones.

Arrays use the grid in C order with x fastest: a field has shape (n_z, n_y, n_x) in 3D and
(n_y, n_x) in 2D; populations have a leading Q axis; velocity fields a leading d axis (u[0]=u_x).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import lattice as L


def grid_shape(n):
    """numpy shape of a field on a grid with n = (n_x, n_y[, n_z]) cells."""
    return tuple(int(v) for v in reversed(n))


def axis_of(alpha: int, d: int, lead: int = 1) -> int:
    """numpy axis index of spatial axis alpha (0 = x) in an array with ``lead`` leading axes."""
    return lead + (d - 1 - alpha)


# ---------------------------------------------------------------------------------------------
# Continuous moments and Hermite moments of the equilibrium
# ---------------------------------------------------------------------------------------------

def continuous_moment_nse(ex, rho, j, p, m30=True):
    """Raw continuous moment of the monomial with exponents ``ex`` for the NSE equilibrium:
    M0 = rho, M1 = rho u, M2 = rho u u + p I, M3 = p (u_a d_bg + u_b d_ag + u_g d_ab) + M30
    (Eq. (M-NSEs-6a), Eq. (M-NSEs-6-1)): multispeed lattices take k = 0 and M30 = rho u u u;
    single-speed lattices (k = 1) take M30 = 0 as the standard-lattice case of Sec. 3.4 does, and
    have no pure-cube rows, so the k delta^(4) part of M3 never enters a row."""
    axes = [a for a, k in enumerate(ex) for _ in range(k)]
    u = [j[a] / rho for a in range(len(j))]
    if len(axes) == 0:
        return rho
    if len(axes) == 1:
        return j[axes[0]]
    if len(axes) == 2:
        a, b = axes
        return rho * u[a] * u[b] + (p if a == b else 0.0)
    if len(axes) == 3:
        a, b, g = axes
        out = rho * u[a] * u[b] * u[g] if m30 else 0.0 * rho
        if b == g:
            out = out + p * u[a]
        if a == g:
            out = out + p * u[b]
        if a == b:
            out = out + p * u[g]
        return out
    raise ValueError("NSE equilibrium moments are specified up to third order")


def hermite_moments_eq_nse(lat: L.Lattice, rho, j, cs2_eq):
    """m^eq_r = P_r(M): each Hermite polynomial with its monomials replaced by the moments."""
    p = rho * cs2_eq
    m30 = lat.kind not in L.SINGLE_SPEED
    out = []
    for poly in lat.polys:
        m = np.zeros_like(rho)
        for ex, coef in poly.items():
            m = m + coef * continuous_moment_nse(ex, rho, j, p, m30)
        out.append(m)
    return np.stack(out)


def hermite_moments_eq_ncde(lat: L.Lattice, phi, u_const, cs2_eq, nonlin, mode="moment"):
    """App. A, Eq. (M-NCDE-6): M0 = phi, M1 = B = u phi, M2 = cs2_eq D(phi) I (+ M20 = 0) with
    D(phi) = phi + nonlin * phi^3 / 3 ("moment"), D(phi) = phi ("rate": the nonlinearity sits in
    the relaxation rate instead); the diffusion-based CDE of App. A special case (3) ("cde") has
    M1 = 0 and M2 = cs2_eq phi I. Third-order Hermite moments zero."""
    Dphi = phi + nonlin * phi ** 3 / 3.0 if mode == "moment" else phi
    flux = 0.0 if mode == "cde" else 1.0
    out = []
    for poly, order in zip(lat.polys, lat.orders):
        if order == 3:
            out.append(np.zeros_like(phi))
            continue
        m = np.zeros_like(phi)
        for ex, coef in poly.items():
            axes = [a for a, k in enumerate(ex) for _ in range(k)]
            if len(axes) == 0:
                term = phi
            elif len(axes) == 1:
                term = flux * u_const[axes[0]] * phi
            else:
                term = cs2_eq * Dphi if axes[0] == axes[1] else np.zeros_like(phi)
            m = m + coef * term
        out.append(m)
    return np.stack(out)


def from_hermite_moments(lat: L.Lattice, m):
    """Eq. (feq-1) / Eq. (geq): g_i = w_i sum_k (H_k^T)_i (H_k W H_k^T)^{-1} m_{H,k}, k = 0..3.

    ``m`` has shape (R, ncells); returns (Q, ncells)."""
    out = np.zeros((lat.Q,) + m.shape[1:])
    for k in range(4):
        rows = lat.block(k)
        Hk = lat.H[rows]                                  # (n_k, Q)
        Gk = Hk @ np.diag(lat.w) @ Hk.T                   # H_k W H_k^T
        coef = np.linalg.inv(Gk) @ m[rows].reshape(len(rows), -1)
        out += (lat.w[:, None] * (Hk.T @ coef)).reshape(out.shape)
    return out


# ---------------------------------------------------------------------------------------------
# Model
# ---------------------------------------------------------------------------------------------

@dataclass
class Model:
    """One MRT-LB solve on a periodic grid of n = (n_x, n_y[, n_z]) cells."""
    lat: L.Lattice
    eq: str                                  # "nse" or "ncde"
    n: tuple
    s: np.ndarray                            # relaxation rate of each Hermite row (R values)
    s_high: float = 1.0                      # shared rate of all rows of order >= 4
    cs2_eq: float | None = None              # p / rho (NSE); prefactor of D(phi) (NCDE)
    force: tuple | None = None               # (a, b, A, k[, phase]): F = A sin(2 pi k x_b / L_b + phase) e_a
    u_const: np.ndarray | None = None        # NCDE convection velocity
    nonlin: float = 0.0                      # NCDE: D(phi) = phi + nonlin phi^3 / 3
    s_bulk: float | None = None              # NSE: bulk rate s_b of Eq. (4-27) (None: diagonal S)
    s_orders: dict | None = None             # rate of each order >= 4 ({4: s4, 5: s5, ...}; else s_high)
    ncde_mode: str = "moment"                # NCDE: "moment", "rate" (per-cell s1(phi)) or "cde"
    a1: float = 0.0                          # NCDE: A1 = a1 I of Eq. (GNCDE) with B-bar = u phi
    m2g_aniso: bool = False                  # NSE, single speed: (delta4 . u) . grad rho in M2G
    a2: float = 0.0                          # NCDE: A2 = a2 I of Eq. (GNCDE) with D-bar = psi I
    psi: np.ndarray | None = None            # NCDE: the prescribed field of D-bar (grid shape)
    f: np.ndarray = field(default=None, repr=False)          # f-bar, shape (Q, *grid)
    phi_prev: np.ndarray = field(default=None, repr=False)   # NCDE: phi at the previous step
    rho_prev: np.ndarray = field(default=None, repr=False)   # NSE: rho at the previous step
    step_count: int = 0

    def __post_init__(self):
        self.n = tuple(int(v) for v in self.n)
        self.s = np.asarray(self.s, dtype=np.float64)
        if self.cs2_eq is None:
            self.cs2_eq = float(self.lat.cs2[0])
        Q = self.lat.Q
        high = [(self.s_orders or {}).get(o, self.s_high) for o in self.lat.full_orders[self.lat.R:]]
        S = np.diag(np.concatenate([self.s, np.array(high, dtype=np.float64)]))
        self.normal = [r for r, p in enumerate(self.lat.polys)
                       if self.lat.orders[r] == 2 and max(max(p, key=sum)) == 2]
        if self.s_bulk is not None:
            S[np.ix_(self.normal, self.normal)] = self.normal_block()
        self.S = S
        self.Hinv = L.hermite_inverse(self.lat)
        self.Lam = self.Hinv @ S @ self.lat.Hfull       # Lambda = H^{-1} S H
        self.shape = grid_shape(self.n)
        if self.u_const is not None:
            self.u_const = np.asarray(self.u_const, dtype=np.float64)
        if self.m2g_aniso and (self.eq != "nse" or self.lat.kind not in L.SINGLE_SPEED):
            raise ValueError("the delta4 term of M2G is the single-speed (k = 1) NSE case")
        if self.a2 != 0.0 and (self.eq != "ncde" or self.ncde_mode == "cde" or self.psi is None):
            raise ValueError("the cross-diffusion term needs the NCDE (not the CDE variant) and psi")

    def normal_block(self):
        """Eq. (4-27): the relaxation of the normal second moments is the inverse of
        S2^(1) = diag(1/s_sa) + a b^T / d. Multispeed lattices (k = 0): a_a = 1/s_b - 1/s_sa and
        b = 1, so that the trace relaxes with s_b and the deviatoric part with s_s (Eq. (4-29):
        mu = (1/s_s - 1/2) p dt, mu_b = (2/d)(1/s_b - 1/2) p dt). Single-speed lattices (k = 1):
        a_a = (1/s_b - 1/s_sa)(c_a^2 - c_s^2) and b_b = 1/(c_b^2 - c_s^2) as printed, c_s^2 = cs2_eq,
        because there the normal moments are driven by (c_a^2 - c_s^2) rho d_a u_a."""
        d = self.lat.d
        ss = self.s[self.normal]
        if self.lat.kind in L.SINGLE_SPEED:
            D = self.lat.c ** 2 - self.cs2_eq
        else:
            D = np.ones(d)
        a = (1.0 / self.s_bulk - 1.0 / ss) * D
        return np.linalg.inv(np.diag(1.0 / ss) + np.outer(a, 1.0 / D) / d)

    # -- body force ---------------------------------------------------------------------------
    def force_field(self):
        """F(x) = A sin(2 pi k x_b / L_b + phase) e_a, x_b = i_b c_b the cell coordinate, L_b = n_b c_b."""
        d = self.lat.d
        F = np.zeros((d,) + self.shape)
        if self.force is None:
            return F
        a, b, A, k = self.force[:4]
        phase = self.force[4] if len(self.force) > 4 else 0.0
        idx = np.arange(self.n[b])
        prof = A * np.sin(2.0 * np.pi * k * idx / self.n[b] + phase)
        bshape = [1] * d
        bshape[axis_of(b, d, lead=0)] = self.n[b]
        F[a] = np.broadcast_to(prof.reshape(bshape), self.shape)
        return F

    # -- fields ----------------------------------------------------------------------------------
    def fields(self, f=None):
        """Eq. (2-4-2) (NSE, S = 0, F_F = F): rho = sum f, u = (sum c f + dt F / 2) / rho;
        Eq. (2-4-1) (NCDE, S = 0): phi = sum f."""
        f = self.f if f is None else f
        if self.eq == "ncde":
            if self.ncde_mode == "cde":
                # Eq. (2-4-1) with lambda = 1, S_F = 0: phi = sum f + S_G / 2
                return np.sum(f, axis=0) + 0.5 * self.cde_source(f), None
            return np.sum(f, axis=0), None
        rho = np.sum(f, axis=0)
        F = self.force_field()
        j = np.stack([np.tensordot(self.lat.cvel[:, a], f, axes=(0, 0)) for a in range(self.lat.d)])
        u = (j + 0.5 * F) / rho
        return rho, u

    def cde_source(self, f):
        """App. A special case (3): S_G = -u . grad phi with the local gradient of
        Eq. (M-NCDE-3-00a), grad_a phi = -s_a M1_a^ne / (dt cs2_eq), where M1^ne = sum_j c_j f_j
        (M1 = 0; the printed sum of f_j is read as the first moment)."""
        lat = self.lat
        out = np.zeros(f.shape[1:])
        for r, poly in enumerate(lat.polys):
            if lat.orders[r] == 1:
                (ex,) = poly.keys()
                a = ex.index(1)
                m1 = np.tensordot(lat.cvel[:, a], f, axes=(0, 0))
                out = out + self.u_const[a] * self.s[r] * m1 / self.cs2_eq
        return out

    def rate_of(self, r, phi):
        """Order-1 rate of row r in the "rate" reading: K(phi) = K0 (1 + nonlin phi^2) with
        K0 = cs2_eq (1/s_r - 1/2), and s_r(phi) = 1 / (K(phi) / cs2_eq + 1/2) (Eq. (GNCDE-0)
        read with S1^-1)."""
        K0 = self.cs2_eq * (1.0 / self.s[r] - 0.5)
        return 1.0 / (K0 * (1.0 + self.nonlin * phi ** 2) / self.cs2_eq + 0.5)

    def equilibrium(self, rho_or_phi, u=None):
        """Eq. (feq-1) for the fields given."""
        flat = rho_or_phi.reshape(-1)
        if self.eq == "nse":
            j = (u * rho_or_phi[None]).reshape(self.lat.d, -1)
            m = hermite_moments_eq_nse(self.lat, flat, j, self.cs2_eq)
        else:
            m = hermite_moments_eq_ncde(self.lat, flat, self.u_const, self.cs2_eq, self.nonlin, self.ncde_mode)
        return from_hermite_moments(self.lat, m).reshape((self.lat.Q,) + self.shape)

    def init_fields(self, rho_or_phi, u=None):
        """f-bar(t=0) = f^eq(rho, u) (or f^eq(phi)); for the NCDE phi^{-1} = phi^0."""
        rho_or_phi = np.asarray(rho_or_phi, dtype=np.float64)
        self.f = self.equilibrium(rho_or_phi, None if u is None else np.asarray(u, dtype=np.float64))
        self.phi_prev = rho_or_phi.copy() if self.eq == "ncde" else None
        self.rho_prev = rho_or_phi.copy() if self.eq == "nse" else None
        self.step_count = 0

    def set_populations(self, f):
        self.f = np.array(f, dtype=np.float64, copy=True)
        if self.eq == "ncde" and self.phi_prev is None:
            self.phi_prev = np.sum(self.f, axis=0)
        if self.eq == "nse":
            self.rho_prev = np.sum(self.f, axis=0)

    def central_gradient(self, g):
        """Second-order central differences on the periodic grid,
        d_a g = (g(x + e_a) - g(x - e_a)) / (2 c_a dt), c_a dt being the cell spacing along axis a
        (dt = 1)."""
        d = self.lat.d
        out = np.zeros((d,) + self.shape)
        for a in range(d):
            ax = axis_of(a, d, lead=0)
            out[a] = (np.roll(g, -1, axis=ax) - np.roll(g, 1, axis=ax)) / (2.0 * self.lat.c[a])
        return out

    def density_gradient(self):
        """grad rho from the density of the previous step (central differences)."""
        return self.central_gradient(self.rho_prev)

    # -- sources --------------------------------------------------------------------------------
    def source_moments(self, fields):
        """Hermite moments of the SDF F and of the auxiliary G (shape (R, ncells) each)."""
        lat = self.lat
        R = lat.R
        ncell = int(np.prod(self.shape))
        mF = np.zeros((R, ncell))
        mG = np.zeros((R, ncell))
        if self.eq == "nse":
            if self.force is None and not self.m2g_aniso:
                return mF, mG
            F = self.force_field().reshape(lat.d, -1)
            u = fields[1].reshape(lat.d, -1)
            S2 = self.S[:R, :R]
            raw = np.zeros((R, ncell))          # uF + Fu on the second-order rows
            if self.m2g_aniso:
                grad = self.density_gradient().reshape(lat.d, -1)
            for r, poly in enumerate(lat.polys):
                if lat.orders[r] == 2:
                    axes = [a for a, k in enumerate(max(poly, key=sum)) for _ in range(k)]
                    a, b = axes
                    raw[r] = u[a] * F[b] + F[a] * u[b]
                    if self.m2g_aniso and a == b:
                        # Eq. (M2Ga): [(delta4 . u) . grad rho]_aa = (c_a^2 - 3 c_s^2) u_a d_a rho
                        raw[r] = raw[r] + (lat.c[a] ** 2 - 3.0 * self.cs2_eq) * u[a] * grad[a]
            for r, poly in enumerate(lat.polys):
                o = lat.orders[r]
                if o == 1:
                    # M1F = F_F = F (Eq. (M-NSEs-2)); the row H_a = c_a carries F_a
                    (ex,) = poly.keys()
                    mF[r] = F[ex.index(1)]
                elif o == 2:
                    # M2G = (I - S2/2)(uF + Fu) (Eq. (M2Ga-1), S = 0; with m2g_aniso the
                    # bracket of Eq. (M2Ga) carries the delta4 term too), M0G = 0 so the H2
                    # Hermite moment equals the raw second moment; S2 is the second-order block
                    # of S (diagonal, or with the bulk coupling of Eq. (4-27))
                    rows2 = [q for q in range(R) if lat.orders[q] == 2]
                    mG[r] = raw[r] - 0.5 * (S2[r, rows2] @ raw[rows2])
            return mF, mG
        if self.ncde_mode == "cde":
            # App. A special case (3): M0G = (1 - s0/2) S_G (Eq. (M-NCDE-4), lambda = 1), M1G = 0
            mG[0] = (1.0 - 0.5 * self.s[0]) * self.cde_source(self.f).reshape(-1)
            return mF, mG
        # NCDE: M1G = (I - S1/2) u d_t phi - S1 (A1 d_t(u phi) + A2 div(psi I)) (Eq. (M-NCDE-6)
        # with M20 = 0, B-bar = u phi, D-bar = psi I); S1 per cell in the "rate" reading
        phi = fields[0].reshape(-1)
        dphi = phi - self.phi_prev.reshape(-1)
        gpsi = self.central_gradient(self.psi).reshape(lat.d, -1) if self.a2 != 0.0 else None
        for r, poly in enumerate(lat.polys):
            if lat.orders[r] == 1:
                (ex,) = poly.keys()
                a = ex.index(1)
                s1 = self.rate_of(r, phi) if self.ncde_mode == "rate" else self.s[r]
                mG[r] = (1.0 - 0.5 * s1 - s1 * self.a1) * self.u_const[a] * dphi
                if gpsi is not None:
                    mG[r] = mG[r] - s1 * self.a2 * gpsi[a]
        return mF, mG

    # -- one step --------------------------------------------------------------------------------
    def collide(self):
        """Eq. (2-3) collision: f~ = f - Lambda (f - f^eq) + dt [G + (I - Lambda/2) F]."""
        lat = self.lat
        rho_or_phi, u = self.fields()
        feq = self.equilibrium(rho_or_phi, u)
        mF, mG = self.source_moments((rho_or_phi, u))
        Fd = from_hermite_moments(lat, mF).reshape(lat.Q, -1)
        Gd = from_hermite_moments(lat, mG).reshape(lat.Q, -1)
        f = self.f.reshape(lat.Q, -1)
        fne = f - feq.reshape(lat.Q, -1)
        ft = f - self.Lam @ fne + Gd + Fd - 0.5 * (self.Lam @ Fd)
        if self.eq == "ncde" and self.ncde_mode == "rate":
            # per-cell S: Lambda(x) = Lambda + sum_r (s_r(phi(x)) - s_r) H^-1[:, r] H[r, :] over the
            # first-order rows (a change of S on those rows only)
            phi = rho_or_phi.reshape(-1)
            for r in lat.block(1):
                ds = self.rate_of(r, phi) - self.s[r]
                ft = ft - np.outer(self.Hinv[:, r], lat.Hfull[r] @ fne) * ds[None, :]
        if self.eq == "ncde":
            self.phi_prev = rho_or_phi.copy()
        elif self.m2g_aniso:
            self.rho_prev = rho_or_phi.copy()
        return ft.reshape(self.f.shape)

    def stream(self, ft):
        """Eq. (2-2b): f_j(x + c_j dt, t + dt) = f~_j(x, t) on the periodic grid."""
        out = np.empty_like(ft)
        d = self.lat.d
        for i in range(self.lat.Q):
            shifts = tuple(int(self.lat.e[i, a]) for a in range(d))
            axes = tuple(axis_of(a, d, lead=0) for a in range(d))
            out[i] = np.roll(ft[i], shifts, axis=axes)
        return out

    def step(self, nsteps=1):
        for _ in range(int(nsteps)):
            self.f = self.stream(self.collide())
            self.step_count += 1

    def stream_only(self, nsteps=1):
        for _ in range(int(nsteps)):
            self.f = self.stream(self.f)

    # -- diagnostics -----------------------------------------------------------------------------
    def conserved_sums(self):
        """Global sum_x sum_j f_j and sum_x sum_j c_j f_j (FP64)."""
        tot = np.sum(self.f, axis=tuple(range(1, self.f.ndim)))
        return np.concatenate([[tot.sum()], self.lat.cvel.T @ tot])
