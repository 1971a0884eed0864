// The per-cell MRT collision in the Hermite basis and the fused pull collide-stream kernel.
//
// One thread owns one cell. It gathers the Q populations of its cell from the neighbours
// x - e_i of the previous step (pull form of the propagation, Eq. (2-2b)), collides them
// (Eq. (2-3) with the Hermite-moment collision Eq. (H-MRT-LB-1)) and writes the post-collision
// populations back at its own cell (aligned, coalesced stores). The stored array is therefore
// the post-collision state of the last step; the pre-collision f-bar(x, t_n) of the paper is
// its pull-gather.
//
// The collision is evaluated in the reduced form that Eq. (H-MRT-LB-1) gives when every row
// of order >= 4 relaxes with one rate s_h:
//   f*_i = (1 - s_h) f_i + w_i sum_{r<R} H_ri / N_r [ s_h m^eq_r - (s_r - s_h)(m_r - m^eq_r)
//                                                     + sigma_r ],
// because the W-orthogonal complement of span(H0..H3) carries the same rate in every row.
// The two contractions with the Hermite matrix are factored through the monomials:
// H_r(c_i) = sum_k T_rk D_k mono_k(e_i), where mono_k(e_i) are small integers known at
// compile time (so zero products vanish and the +-e pairs share one pass), T is the
// lower-triangular, parity-block-diagonal Gram-Schmidt factor and D_k the axis-speed scale.
#pragma once

#include "lbm_internal.cuh"

// Tuning knobs of the collide-stream kernel (defaults measured best on GB300 for rD3Q53 on
// 256x256x192: 4 blocks of 128 threads per SM leave the kernel 128 registers without spills,
// 0.833 ms per FP32 step and 0.686 ms per FP16-deviation step, against 0.883 / 0.732 ms with
// 5 blocks (96 registers) and 0.989 / 0.756 ms with 6; evict-first loads or stores were slower):
//   LBM_K1_MIN_BLOCKS  minimum resident blocks per SM requested through __launch_bounds__
//   LBM_K1_LOAD        0: ld.global.nc (__ldg), 1: evict-first (__ldcs), 2: plain load
//   LBM_K1_STORE       0: plain store, 1: evict-first streaming store (__stcs)
#ifndef LBM_K1_MIN_BLOCKS
#define LBM_K1_MIN_BLOCKS 4
#endif
#ifndef LBM_K1_LOAD
#define LBM_K1_LOAD 0
#endif
#ifndef LBM_K1_STORE
#define LBM_K1_STORE 0
#endif

namespace lbm {

template <class T>
__device__ __forceinline__ T k1_load(const T* p) {
#if LBM_K1_LOAD == 0
  return __ldg(p);
#elif LBM_K1_LOAD == 1
  return __ldcs(p);
#else
  return *p;
#endif
}

template <class T>
__device__ __forceinline__ void k1_store(T* p, T v) {
#if LBM_K1_STORE == 1
  __stcs(p, v);
#else
  *p = v;
#endif
}

template <class CT>
__device__ __forceinline__ CT fmaf_t(CT a, CT b, CT c) {
  return fma(a, b, c);
}

// acc + c * x for a compile-time integer c
template <int C, class CT>
__device__ __forceinline__ CT axpy_c(CT x, CT acc) {
  if constexpr (C == 1) return acc + x;
  else if constexpr (C == -1) return acc - x;
  else return fma(CT(C), x, acc);
}

__host__ __device__ constexpr int axis_n(Mono m, int n) {
  // n-th axis (0-based) in the sorted list of axes of monomial m, e.g. xyy -> x, y, y
  return n < m.a ? 0 : (n < m.a + m.b ? 1 : 2);
}

// Raw moments mu_k = sum_i mono_k(e_i) f_i, k < R. Per primitive direction d the populations of
// +-m d are first combined per degree (s_deg = sum_m m^deg (f_md +- f_-md), + for even degree,
// - for odd), then mu_k += mono_k(d) s_deg(k): zero products vanish at compile time and each
// monomial product is shared by every speed of the direction.
template <int DEG, class CT>
__device__ __forceinline__ CT pick_degree(CT s0, CT s1, CT s2, CT s3) {
  if constexpr (DEG == 0) return s0;
  else if constexpr (DEG == 1) return s1;
  else if constexpr (DEG == 2) return s2;
  else return s3;
}

template <class L, class CT>
__device__ __forceinline__ void raw_moments(const CT (&f)[L::Q], CT (&mu)[L::R]) {
  static_for<L::R>([&](auto k) { mu[decltype(k)::value] = CT(0); });
  mu[0] = f[0];
  static_for<num_directions<L>()>([&](auto dk) {
    CT s0 = CT(0), s1 = CT(0), s2 = CT(0), s3 = CT(0);
    static_for<3>([&](auto mm) {
      constexpr int M = decltype(mm)::value + 1;
      constexpr int ip = velocity_index<L>(direction<L>(decltype(dk)::value), M);
      constexpr int im = velocity_index<L>(direction<L>(decltype(dk)::value), -M);
      if constexpr (ip >= 0) {
        const CT sp = f[ip] + f[im];
        const CT sm = f[ip] - f[im];
        s0 += sp;
        s1 = axpy_c<M>(sm, s1);
        s2 = axpy_c<M * M>(sp, s2);
        s3 = axpy_c<M * M * M>(sm, s3);
      }
    });
    static_for<L::R>([&](auto k) {
      constexpr int K = decltype(k)::value;
      constexpr int cv = mono_value(direction<L>(decltype(dk)::value), mono<L::D>(K));
      if constexpr (cv != 0) mu[K] = axpy_c<cv>(pick_degree<degree(mono<L::D>(K))>(s0, s1, s2, s3), mu[K]);
    });
  });
}

// Continuous raw moments of the NSE equilibrium (Eq. (M-NSEs-6a), Eq. (M-NSEs-6-1) with k = 0,
// M30 = rho u u u, p = rho cs2_eq): M0 = rho, M1 = j, M2 = j u + p I,
// M3 = j u u + p (u delta)_sym, for every monomial of the paper's row order. Single-speed
// lattices (k = 1) take M30 = 0 and have no pure-cube rows.
template <class L, class CT>
__device__ __forceinline__ void eq_raw_nse(CT rho, const CT (&j)[3], const CT (&u)[3], CT P,
                                           CT (&me)[L::R]) {
  static_for<L::R>([&](auto k) {
    constexpr int K = decltype(k)::value;
    constexpr int deg = degree(mono<L::D>(K));
    constexpr int a0 = axis_n(mono<L::D>(K), 0), a1 = axis_n(mono<L::D>(K), 1),
                  a2 = axis_n(mono<L::D>(K), 2);
    if constexpr (deg == 0) {
      me[K] = rho;
    } else if constexpr (deg == 1) {
      me[K] = j[a0];
    } else if constexpr (deg == 2) {
      if constexpr (a0 == a1) me[K] = fma(j[a0], u[a1], P);
      else me[K] = j[a0] * u[a1];
    } else {
      CT v = L::SINGLE ? CT(0) : j[a0] * u[a1] * u[a2];  // M30 = rho u u u (multispeed) or 0 (single speed)
      if constexpr (a1 == a2) v = fma(P, u[a0], v);
      if constexpr (a0 == a2) v = fma(P, u[a1], v);
      if constexpr (a0 == a1) v = fma(P, u[a2], v);
      me[K] = v;
    }
  });
}

// Continuous raw moments of the NCDE equilibrium up to second order (Eq. (M-NCDE-6), M20 = 0):
// M0 = phi, M1 = u phi, M2 = cs2_eq D(phi) I. Third-order entries are unused.
template <class L, class CT, class P>
__device__ __forceinline__ void eq_raw_ncde(CT phi, CT Dphi, const P& p,
                                            CT (&me)[L::R]) {
  static_for<L::R>([&](auto k) {
    constexpr int K = decltype(k)::value;
    constexpr int deg = degree(mono<L::D>(K));
    constexpr int a0 = axis_n(mono<L::D>(K), 0), a1 = axis_n(mono<L::D>(K), 1);
    if constexpr (deg == 0) me[K] = phi;
    else if constexpr (deg == 1) me[K] = p.u_const[a0] * phi;
    else if constexpr (deg == 2) me[K] = (a0 == a1) ? p.cs2_eq * Dphi : CT(0);
    else me[K] = CT(0);
  });
}

// sum_{k < r, same parity class as r} T_rk v_k + v_r   (T is monic: T_rr = 1)
template <class L, class CT, int r, class P>
__device__ __forceinline__ CT row_dot(const P& p, const CT (&v)[L::R]) {
  CT acc = v[r];
  static_for<r>([&](auto k) {
    constexpr int K = decltype(k)::value;
    if constexpr (parity_class(mono<L::D>(K)) == parity_class(mono<L::D>(r)))
      acc = fma(p.T[r][K], v[K], acc);
  });
  return acc;
}

// Hermite moments of the equilibrium, m^eq_r = sum_k T_rk me_k.
// For the NCDE the third-order Hermite moments of the equilibrium are zero.
template <class L, class CT, int EQ, int r, class P>
__device__ __forceinline__ CT hermite_eq(const P& p, const CT (&me)[L::R]) {
  if constexpr (EQ == LBM_NCDE && degree(mono<L::D>(r)) == 3) return CT(0);
  else return row_dot<L, CT, r>(p, me);
}

// f_i = (1 - s_h) f_i + w_i sum_k mono_k(e_i) h_k  (h already scaled by D_k). Per primitive
// direction d: E_deg = sum_{deg(k) = deg} mono_k(d) h_k, then for every speed m present
// f_{+-md} = (1 - s_h) f + w (E_0 + m^2 E_2 +- (m E_1 + m^3 E_3)).
template <class L, class CT, class P>
__device__ __forceinline__ void back_project(CT (&f)[L::Q], const P& p,
                                             const CT (&h)[L::R], CT oms) {
  f[0] = fma(oms, f[0], p.w[0] * h[0]);
  static_for<num_directions<L>()>([&](auto dk) {
    CT E1 = CT(0), E2 = CT(0), E3 = CT(0);
    static_for<L::R>([&](auto k) {
      constexpr int K = decltype(k)::value;
      constexpr int cv = mono_value(direction<L>(decltype(dk)::value), mono<L::D>(K));
      constexpr int deg = degree(mono<L::D>(K));
      if constexpr (cv != 0 && deg == 1) E1 = axpy_c<cv>(h[K], E1);
      if constexpr (cv != 0 && deg == 2) E2 = axpy_c<cv>(h[K], E2);
      if constexpr (cv != 0 && deg == 3) E3 = axpy_c<cv>(h[K], E3);
    });
    static_for<3>([&](auto mm) {
      constexpr int M = decltype(mm)::value + 1;
      constexpr int ip = velocity_index<L>(direction<L>(decltype(dk)::value), M);
      constexpr int im = velocity_index<L>(direction<L>(decltype(dk)::value), -M);
      if constexpr (ip >= 0) {
        const CT even = axpy_c<M * M>(E2, h[0]);
        const CT odd = (M == 1) ? E1 + E3 : fma(CT(M * M * M), E3, CT(M) * E1);
        f[ip] = fma(oms, f[ip], p.w[ip] * (even + odd));
        f[im] = fma(oms, f[im], p.w[im] * (even - odd));
      }
    });
  });
}

// h_k = D_k sum_{r >= k, same parity class} T_rk gN_r   (the transpose contraction)
template <class L, class CT, class P>
__device__ __forceinline__ void hermite_to_monomial(const P& p, const CT (&gN)[L::R],
                                                    CT (&h)[L::R]) {
  static_for<L::R>([&](auto k) {
    constexpr int K = decltype(k)::value;
    CT acc = gN[K];
    static_for<L::R>([&](auto r) {
      constexpr int Rr = decltype(r)::value;
      constexpr int Kk = decltype(k)::value;
      if constexpr (Rr > Kk && parity_class(mono<L::D>(Rr)) == parity_class(mono<L::D>(Kk)))
        acc = fma(p.T[Rr][Kk], gN[Rr], acc);
    });
    if constexpr (K == 0) h[K] = acc;
    else h[K] = acc * p.D[K];
  });
}

// Hermite moments of row r: the equilibrium m^eq_r and the non-equilibrium m_r - m^eq_r.
template <class L, class CT, int EQ, int r, class P>
__device__ __forceinline__ void row_moments(const P& p, const CT (&mu)[L::R], const CT (&me)[L::R], CT& meq,
                                            CT& neq) {
  meq = hermite_eq<L, CT, EQ, r>(p, me);
  if constexpr (EQ == LBM_NCDE && degree(mono<L::D>(r)) == 3) {
    neq = row_dot<L, CT, r>(p, mu);
  } else {
    CT dm[L::R];
    static_for<r + 1>([&](auto k) {
      constexpr int K = decltype(k)::value;
      if constexpr (parity_class(mono<L::D>(K)) == parity_class(mono<L::D>(r))) dm[K] = mu[K] - me[K];
      else dm[K] = CT(0);
    });
    neq = row_dot<L, CT, r>(p, dm);
  }
}

// Per-cell first-order factors of the NCDE (from the parameters, or per cell for the rate
// variant) and the CDE source S_G (zero otherwise).
template <class CT>
struct NcdeCell {
  CT sd1[3];    // s_a - s_high on the first-order rows
  CT half1[3];  // factor of u d_t phi in M1G
  CT sg;        // S_G of the CDE variant
};

// g_r / N_r with g = s_h m^eq - (S - s_h I)(m - m^eq) + sigma. S is diagonal except on the normal
// second-order rows, where the d x d block S_n carries the bulk coupling of Eq. (4-27).
// sigma: NSE (I - S/2) M1F = (1 - s/2) F on order 1 and M2G = (I - S2/2)(uF + Fu) on order 2,
// plus, given gr (single-speed lattices), the diagonal (delta4 . u) . grad rho of Eq. (M2Ga) with
// gr_a = (c_a^2 - 3 c_s^2) d_a rho; NCDE M1G = (I - S1/2) u d_t phi - S1 A1 d_t(u phi) on order 1
// (factor half1), minus S1 A2 grad psi given gr_a = a2 d_a psi (Eq. (M-NCDE-6), D-bar = psi I),
// and, for the CDE variant, M0G = (1 - s0/2) S_G on order 0.
template <class L, class CT, int EQ, int r, class P>
__device__ __forceinline__ CT row_update(const P& p, const CT (&meq)[L::R], const CT (&neq)[L::R],
                                         const CT (&u)[3], const CT (&F)[3], CT dphi, const NcdeCell<CT>& nc,
                                         const CT* gr) {
  constexpr int deg = degree(mono<L::D>(r));
  constexpr int na = normal_index<L::D>(r);
  CT relax, sig = CT(0);
  if constexpr (na >= 0) {
    relax = CT(0);
    static_for<L::D>([&](auto b) {
      constexpr int B = decltype(b)::value;
      relax = fma(p.sdn[na][B], neq[normal_row<L::D>(B)], relax);
      if constexpr (EQ == LBM_NSE) {
        CT t = CT(2) * u[B] * F[B];
        if (gr != nullptr) t = fma(u[B], gr[B], t);
        sig = fma(p.halfn[na][B], t, sig);
      }
    });
  } else {
    relax = p.sd[r] * neq[r];
    if constexpr (deg == 1) {
      constexpr int a = axis_n(mono<L::D>(r), 0);
      if constexpr (EQ == LBM_NSE) {
        sig = p.half[r] * F[a];
      } else {
        relax = nc.sd1[a] * neq[r];
        sig = nc.half1[a] * p.u_const[a] * dphi;
        if (gr != nullptr) sig = fma(-(nc.sd1[a] + p.s_high), gr[a], sig);
      }
    } else if constexpr (deg == 0 && EQ == LBM_NCDE && P::kNcdeVariants) {
      sig = p.half0 * nc.sg;
    } else if constexpr (deg == 2 && EQ == LBM_NSE) {
      constexpr int a = axis_n(mono<L::D>(r), 0), b = axis_n(mono<L::D>(r), 1);
      sig = p.half[r] * fma(u[a], F[b], u[b] * F[a]);
    }
  }
  const CT g = fma(p.s_high, meq[r], sig - relax);
  return g * p.invN[r];
}

// Coefficients of the rows of order >= 4 staged in shared memory, row-major (the values of one
// row at the rest velocity, c = 0, and at the + member of each +-e pair, c = P + 1, adjacent, so
// that one vector load serves four pairs), with a per-thread slot for each row's z_r. The row
// loops run at run time (rows outermost, pairs unrolled), which keeps the register footprint at
// the populations plus one accumulator per pair.
template <class L, class CT>
struct HighTable {
  static constexpr int HE = high_even<L>(), HO = high_odd<L>();
  static constexpr int NP = num_pairs<L>();
  static constexpr int CE = (NP + 1 + 3) / 4 * 4, CO = (NP + 3) / 4 * 4;  // padded row lengths
  alignas(16) CT he[HE * CE];
  alignas(16) CT ho[(HO > 0 ? HO : 1) * CO];
  CT ae[HE];
  CT ao[HO > 0 ? HO : 1];
  CT z[(HE + HO) * kBlock];  // z_r of thread t at z[r * kBlock + t]
  // block-wide copy from the kernel parameters (call before any thread returns)
  __device__ __forceinline__ void fill(const HighParams<CT>& hp) {
    for (int idx = threadIdx.x; idx < HE * (NP + 1); idx += blockDim.x)
      he[(idx / (NP + 1)) * CE + idx % (NP + 1)] = hp.he[idx / (NP + 1)][idx % (NP + 1)];
    for (int idx = threadIdx.x; idx < HO * NP; idx += blockDim.x) ho[(idx / NP) * CO + idx % NP] = hp.ho[idx / NP][idx % NP];
    for (int idx = threadIdx.x; idx < HE; idx += blockDim.x) ae[idx] = hp.ae[idx];
    for (int idx = threadIdx.x; idx < HO; idx += blockDim.x) ao[idx] = hp.ao[idx];
  }
};

// Four consecutive coefficients of a 16-byte-aligned shared-memory row.
template <class CT>
__device__ __forceinline__ void load4(const CT* p, CT (&v)[4]) {
  if constexpr (std::is_same<CT, float>::value) {
    const float4 q = *reinterpret_cast<const float4*>(p);
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
  } else {
    const double2 a = *reinterpret_cast<const double2*>(p);
    const double2 b = *reinterpret_cast<const double2*>(p + 2);
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
  }
}

// Rows of order >= 4 with their own rates: z_r = a_r sum_j h_r(c_j) f_j, a_r = -(s_r - s_h) / N_r,
// kept in the table's per-thread slots. Even rows take f_+ + f_- of each +-e pair, odd rows
// f_+ - f_- (h_r(-c) = +-h_r(c)). For deviation storage the reference state drops out (every
// such row is W-orthogonal to H_0).
template <class L, class CT>
__device__ __forceinline__ void high_moments(const CT (&f)[L::Q], HighTable<L, CT>& tb) {
  using T = HighTable<L, CT>;
  constexpr int NP = T::NP;
  CT sp[NP], sm[NP];
  static_for<NP>([&](auto q) {
    constexpr int P = decltype(q)::value;
    constexpr int ip = pair_plus<L>(P);
    constexpr int im = opposite<L>(ip);
    sp[P] = f[ip] + f[im];
    sm[P] = f[ip] - f[im];
  });
#pragma unroll 1
  for (int r = 0; r < T::HE; ++r) {
    const CT* h = tb.he + r * T::CE;
    CT acc = CT(0);
    static_for<T::CE / 4>([&](auto g) {
      CT v[4];
      load4(h + 4 * decltype(g)::value, v);
      static_for<4>([&](auto j) {
        constexpr int C = 4 * decltype(g)::value + decltype(j)::value;  // c = 0: rest, c = P + 1: pair P
        if constexpr (C == 0) acc = fma(v[decltype(j)::value], f[0], acc);
        else if constexpr (C <= NP) acc = fma(v[decltype(j)::value], sp[C - 1], acc);
      });
    });
    tb.z[r * kBlock + threadIdx.x] = acc * tb.ae[r];
  }
#pragma unroll 1
  for (int r = 0; r < T::HO; ++r) {
    const CT* h = tb.ho + r * T::CO;
    CT acc = CT(0);
    static_for<T::CO / 4>([&](auto g) {
      CT v[4];
      load4(h + 4 * decltype(g)::value, v);
      static_for<4>([&](auto j) {
        constexpr int C = 4 * decltype(g)::value + decltype(j)::value;
        if constexpr (C < NP) acc = fma(v[decltype(j)::value], sm[C], acc);
      });
    });
    tb.z[(T::HE + r) * kBlock + threadIdx.x] = acc * tb.ao[r];
  }
}

// f_i += w_i sum_r h_r(c_i) z_r over the rows of order >= 4 (the weights of a +-e pair are equal).
template <class L, class CT, class P>
__device__ __forceinline__ void high_back(CT (&f)[L::Q], const P& p, const HighTable<L, CT>& tb) {
  using T = HighTable<L, CT>;
  constexpr int NP = T::NP;
  CT ev[NP + 1], od[NP];
  static_for<NP + 1>([&](auto q) { ev[decltype(q)::value] = CT(0); });
  static_for<NP>([&](auto q) { od[decltype(q)::value] = CT(0); });
#pragma unroll 1
  for (int r = 0; r < T::HE; ++r) {
    const CT* h = tb.he + r * T::CE;
    const CT zr = tb.z[r * kBlock + threadIdx.x];
    static_for<T::CE / 4>([&](auto g) {
      CT v[4];
      load4(h + 4 * decltype(g)::value, v);
      static_for<4>([&](auto j) {
        constexpr int C = 4 * decltype(g)::value + decltype(j)::value;
        if constexpr (C <= NP) ev[C] = fma(v[decltype(j)::value], zr, ev[C]);
      });
    });
  }
#pragma unroll 1
  for (int r = 0; r < T::HO; ++r) {
    const CT* h = tb.ho + r * T::CO;
    const CT zr = tb.z[(T::HE + r) * kBlock + threadIdx.x];
    static_for<T::CO / 4>([&](auto g) {
      CT v[4];
      load4(h + 4 * decltype(g)::value, v);
      static_for<4>([&](auto j) {
        constexpr int C = 4 * decltype(g)::value + decltype(j)::value;
        if constexpr (C < NP) od[C] = fma(v[decltype(j)::value], zr, od[C]);
      });
    });
  }
  f[0] = fma(p.w[0], ev[0], f[0]);
  static_for<NP>([&](auto q) {
    constexpr int Pq = decltype(q)::value;
    constexpr int ip = pair_plus<L>(Pq);
    constexpr int im = opposite<L>(ip);
    f[ip] = fma(p.w[ip], ev[Pq + 1] + od[Pq], f[ip]);
    f[im] = fma(p.w[im], ev[Pq + 1] - od[Pq], f[im]);
  });
}

// One collision (Eq. (2-3)) of the populations f of one cell, in place.
// F: body force at the cell (NSE); phi_prev / phi_now: the NCDE field at t_{n-1} and t_n.
// DEV: f holds deviations f - w rho_ref (16-bit storage). The moments of the reference state are
// added back (only 1 and the squares c_a^2 have non-zero lattice moments), and the update
// f* - w rho_ref = (1 - s_h)(f - w rho_ref) + w H(h) - s_h w rho_ref folds the last term into h_0.
// HP = HighTable<L, CT>: the rows of order >= 4 relax with the rates in hp (the full Q x Q
// collision); HP = NoHigh: they share s_high (the reduced form alone).
struct NoHigh {};

// The collision in moment space: from the raw moments mu_k = sum_i mono_k(e_i) f_i (k < R) to
// the monomial-basis coefficients h of the update f*_i = (1 - s_h) f_i + w_i sum_k mono_k(e_i) h_k.
// phi_now receives phi (NCDE) or rho (NSE); gr, if given, the M2G density-gradient term.
template <class L, class CT, int EQ, bool DEV, class P>
__device__ __forceinline__ void collide_moments(CT (&mu)[L::R], const P& p, const CT (&F)[3], CT phi_prev,
                                                CT& phi_now, CT (&h)[L::R], const CT* gr = nullptr) {
  constexpr int R = L::R, D = L::D;
  if constexpr (DEV) {
    static_for<R>([&](auto k) {
      constexpr Mono mk = mono<L::D>(decltype(k)::value);
      if constexpr ((mk.a & 1) == 0 && (mk.b & 1) == 0 && (mk.c & 1) == 0 && degree(mk) <= 2 &&
                    (degree(mk) == 0 || mk.a == 2 || mk.b == 2 || mk.c == 2))
        mu[decltype(k)::value] += p.wmom_ref[decltype(k)::value];
    });
  }
  static_for<R>([&](auto k) {
    constexpr int K = decltype(k)::value;
    if constexpr (K > 0) mu[K] *= p.D[K];
  });
  CT me[R];
  CT u[3] = {CT(0), CT(0), CT(0)};
  CT dphi = CT(0);
  NcdeCell<CT> nc;
  if constexpr (EQ == LBM_NSE) {
    // Eq. (2-4-2) with S = 0, F_F = F: rho = sum f, rho u = sum c f + F / 2
    const CT rho = mu[0];
    const CT inv = CT(1) / rho;
    CT j[3] = {CT(0), CT(0), CT(0)};
    static_for<D>([&](auto a) {
      constexpr int A = decltype(a)::value;
      j[A] = fma(CT(0.5), F[A], mu[1 + A]);
      u[A] = j[A] * inv;
    });
    eq_raw_nse<L>(rho, j, u, rho * p.cs2_eq, me);
    phi_now = rho;
  } else {
    // Eq. (2-4-1) with S = 0: phi = sum f (+ S_G / 2, lambda = 1, for the CDE variant)
    CT phi = mu[0];
    static_for<3>([&](auto a) {
      nc.sd1[decltype(a)::value] = p.sd[decltype(a)::value + 1];
      nc.half1[decltype(a)::value] = p.half[decltype(a)::value + 1];
    });
    nc.sg = CT(0);
    if constexpr (P::kNcdeVariants) {
      if (p.ncde_variant == LBM_NCDE_CDE) {
        // S_G = -u . grad phi with grad_a phi = -s_a M1_a^ne / cs2 (M1 = 0)
        CT sg = CT(0);
        static_for<D>([&](auto a) { sg = fma(p.cde_coef[decltype(a)::value], mu[1 + decltype(a)::value], sg); });
        nc.sg = sg;
        phi = fma(CT(0.5), sg, phi);
      } else if (p.ncde_variant == LBM_NCDE_RATE) {
        // s_a(phi) = 1 / ((1/s_a - 1/2)(1 + nonlin phi^2) + 1/2)
        const CT g = fma(p.nonlin_rate, phi * phi, CT(1));
        static_for<D>([&](auto a) {
          constexpr int A = decltype(a)::value;
          const CT s1 = CT(1) / fma(p.kfac[A], g, CT(0.5));
          nc.sd1[A] = s1 - p.s_high;
          nc.half1[A] = fma(-s1, CT(0.5) + p.a1, CT(1));
        });
      }
    }
    phi_now = phi;
    dphi = phi - phi_prev;
    eq_raw_ncde<L>(phi, fma(p.nonlin_third, phi * phi * phi, phi), p, me);
  }
  CT meq[R], neq[R];
  static_for<R>([&](auto r) {
    constexpr int Rr = decltype(r)::value;
    row_moments<L, CT, EQ, Rr>(p, mu, me, meq[Rr], neq[Rr]);
  });
  CT gN[R];
  static_for<R>([&](auto r) {
    constexpr int Rr = decltype(r)::value;
    gN[Rr] = row_update<L, CT, EQ, Rr>(p, meq, neq, u, F, dphi, nc, gr);
  });
  hermite_to_monomial<L>(p, gN, h);
  if constexpr (DEV) h[0] -= p.sh_rho_ref;
}

template <class L, class CT, int EQ, bool DEV = false, class P, class HP = NoHigh>
__device__ __forceinline__ void collide(CT (&f)[L::Q], const P& p, const CT (&F)[3],
                                        CT phi_prev, CT& phi_now, HP* hp = nullptr, const CT* gr = nullptr) {
  constexpr bool HI = !std::is_same<HP, NoHigh>::value;
  if constexpr (HI) high_moments<L>(f, *hp);
  CT mu[L::R];
  raw_moments<L>(f, mu);
  CT h[L::R];
  collide_moments<L, CT, EQ, DEV>(mu, p, F, phi_prev, phi_now, h, gr);
  back_project<L>(f, p, h, p.one_minus_sh);
  if constexpr (HI) high_back<L>(f, p, *hp);
}

// Equilibrium populations of given fields, Eq. (feq-1): f^eq_i = w_i sum_r H_ri m^eq_r / N_r.
template <class L, class CT, int EQ, class P>
__device__ __forceinline__ void equilibrium(CT (&f)[L::Q], const P& p, CT rho_or_phi,
                                            const CT (&uin)[3]) {
  constexpr int R = L::R;
  CT me[R];
  if constexpr (EQ == LBM_NSE) {
    CT j[3], u[3];
    for (int a = 0; a < 3; ++a) {
      u[a] = uin[a];
      j[a] = rho_or_phi * uin[a];
    }
    eq_raw_nse<L>(rho_or_phi, j, u, rho_or_phi * p.cs2_eq, me);
  } else {
    const CT phi = rho_or_phi;
    eq_raw_ncde<L>(phi, fma(p.nonlin_third, phi * phi * phi, phi), p, me);
  }
  CT gN[R];
  static_for<R>([&](auto r) {
    constexpr int Rr = decltype(r)::value;
    gN[Rr] = hermite_eq<L, CT, EQ, Rr>(p, me) * p.invN[Rr];
  });
  CT h[R];
  hermite_to_monomial<L>(p, gN, h);
  static_for<L::Q>([&](auto i) { f[decltype(i)::value] = CT(0); });
  back_project<L>(f, p, h, CT(0));
}

// Cell coordinates and periodic neighbour offsets.
template <class L>
struct Neigh {
  static constexpr int RM = L::RMAX;
  int xo[2 * RM + 1], yo[2 * RM + 1], zo[2 * RM + 1];
  int x, y, z;
  template <class CT>
  __device__ __forceinline__ Neigh(int cell, const StepParams<CT>& p) : Neigh(cell, p.n, p.div_m, p.div_s) {}
  __device__ __forceinline__ Neigh(int cell, const int (&n)[3], const unsigned (&div_m)[2], const int (&div_s)[2]) {
    const int nx = n[0], ny = n[1];
    // the velocity components are at most RM <= every extent, so one wrap suffices and only on
    // the side a displacement can cross
    const int t = int(__umulhi(unsigned(cell), div_m[0]) >> div_s[0]);
    x = cell - t * nx;
    if constexpr (L::D == 2) {
      y = t;
      z = 0;
    } else {
      z = int(__umulhi(unsigned(t), div_m[1]) >> div_s[1]);
      y = t - z * ny;
    }
#pragma unroll
    for (int s = -RM; s <= RM; ++s) {
      xo[s + RM] = wrap1(x - s, s, nx);
      yo[s + RM] = wrap1(y - s, s, ny) * nx;
      if constexpr (L::D == 3) zo[s + RM] = wrap1(z - s, s, n[2]) * nx * ny;
      else zo[s + RM] = 0;
    }
  }
  __device__ __forceinline__ static int wrap1(int v, int s, int n) {
    if (s > 0) return v < 0 ? v + n : v;
    if (s < 0) return v >= n ? v - n : v;
    return v;
  }
  // cell index of x - e (pull source) for a compile-time velocity
  template <int I>
  __device__ __forceinline__ int src() const {
    constexpr Vel v = L::e(I);
    return xo[RM + v.x] + yo[RM + v.y] + (L::D == 3 ? zo[RM + v.z] : 0);
  }
  // cell index of x + e
  template <int I>
  __device__ __forceinline__ int dst() const {
    constexpr Vel v = L::e(I);
    return xo[RM - v.x] + yo[RM - v.y] + (L::D == 3 ? zo[RM - v.z] : 0);
  }
};

template <class CT>
__device__ __forceinline__ void body_force(int force_a, int force_b, const CT* force_tab, int x, int y,
                                           int z, CT (&F)[3]) {
  F[0] = F[1] = F[2] = CT(0);
  if (force_b >= 0) {
    const int ib = force_b == 0 ? x : (force_b == 1 ? y : z);
    const CT v = force_tab[ib];
    F[0] = force_a == 0 ? v : CT(0);
    F[1] = force_a == 1 ? v : CT(0);
    F[2] = force_a == 2 ? v : CT(0);
  }
}

// Gradient terms of the source moments: the delta4 term of M2G (Eq. (M2Ga)) on the single-speed
// lattices needs grad rho, the cross-diffusion term of M1G (Eq. (M-NCDE-6)) grad psi. Both take
// gr_a = gscale_a (g(x + e_a) - g(x - e_a)), the central difference of the cell field p.grad_in at
// the periodic neighbours of cell (x, y, z); zero when the term is off.
template <class L, int EQ>
struct GradTerm {
  static constexpr bool kOn = (L::SINGLE && EQ == LBM_NSE) || EQ == LBM_NCDE;
};
template <class L, class CT, class P>
__device__ __forceinline__ void cell_field_gradient(const P& p, int cell, int x, int y, int z, CT (&gr)[3]) {
  gr[0] = gr[1] = gr[2] = CT(0);
  if (!p.grad_on) return;
  const int nx = p.n[0], ny = p.n[1];
  const CT* g = p.grad_in;
  const int xp = x + 1 == nx ? -x : 1, xm = x == 0 ? nx - 1 : -1;
  gr[0] = p.gscale[0] * (g[cell + xp] - g[cell + xm]);
  const int yp = (y + 1 == ny ? -y : 1) * nx, ym = (y == 0 ? ny - 1 : -1) * nx;
  gr[1] = p.gscale[1] * (g[cell + yp] - g[cell + ym]);
  if constexpr (L::D == 3) {
    const int nz = p.n[2], nxy = nx * ny;
    const int zp = (z + 1 == nz ? -z : 1) * nxy, zm = (z == 0 ? nz - 1 : -1) * nxy;
    gr[2] = p.gscale[2] * (g[cell + zp] - g[cell + zm]);
  }
}

// K1 (COLLIDE) / K2 (stream only): pull gather, collide, aligned store.
template <class L, class CT, class ST, int EQ, bool COLLIDE>
__global__ void __launch_bounds__(kBlock, LBM_K1_MIN_BLOCKS) k_step(const StepParams<CT> p,
                                                 const ST* __restrict__ fin,
                                                 ST* __restrict__ fout, CT* __restrict__ phi) {
  const int cell = blockIdx.x * kBlock + threadIdx.x;
  if (cell >= p.ncells) return;
  const Neigh<L> nb(cell, p);
  const size_t N = size_t(p.ncells);
  CT f[L::Q];
  constexpr bool DEV = is_deviation_storage<ST>();
  static_for<L::Q>([&](auto i) {
    constexpr int I = decltype(i)::value;
    if constexpr (DEV) f[I] = RawCodec<ST>::dec(k1_load(fin + size_t(I) * N + nb.template src<I>()));
    else f[I] = Codec<ST>::dec(k1_load(fin + size_t(I) * N + nb.template src<I>()), p.wref[I]);
  });
  if constexpr (COLLIDE) {
    CT F[3];
    body_force(p.force_a, p.force_b, p.force_tab, nb.x, nb.y, nb.z, F);
    CT phi_prev = CT(0), phi_now = CT(0);
    if constexpr (EQ == LBM_NCDE) phi_prev = phi[cell];
    constexpr bool AG = GradTerm<L, EQ>::kOn;
    CT gr[3];
    if constexpr (AG) cell_field_gradient<L>(p, cell, nb.x, nb.y, nb.z, gr);
    collide<L, CT, EQ, DEV>(f, p, F, phi_prev, phi_now, static_cast<NoHigh*>(nullptr), AG ? gr : nullptr);
    if constexpr (EQ == LBM_NCDE) phi[cell] = phi_now;
    if constexpr (AG && EQ == LBM_NSE) {
      if (p.grad_on) p.rho_out[cell] = phi_now;
    }
  }
  static_for<L::Q>([&](auto i) {
    constexpr int I = decltype(i)::value;
    if constexpr (DEV) k1_store(fout + size_t(I) * N + cell, RawCodec<ST>::enc(f[I]));
    else k1_store(fout + size_t(I) * N + cell, Codec<ST>::enc(f[I], p.wref[I]));
  });
}

// K1 with distinct rates for the orders >= 4: the same gather / collide / store plus the two
// contractions with the higher rows (about 2 (Q - 1) (Q - R) / 2 more FMAs per cell, so the
// kernel is bound by instruction issue rather than HBM; 3 resident blocks leave it 168 registers).
template <class L, class CT, class ST, int EQ>
__global__ void __launch_bounds__(kBlock, 3) k_step_high(const StepParams<CT> p,
                                                          const HighParams<CT> hp,
                                                          const ST* __restrict__ fin,
                                                          ST* __restrict__ fout, CT* __restrict__ phi) {
  __shared__ HighTable<L, CT> tab;
  tab.fill(hp);
  __syncthreads();
  const int cell = blockIdx.x * kBlock + threadIdx.x;
  if (cell >= p.ncells) return;
  const Neigh<L> nb(cell, p);
  const size_t N = size_t(p.ncells);
  CT f[L::Q];
  constexpr bool DEV = is_deviation_storage<ST>();
  static_for<L::Q>([&](auto i) {
    constexpr int I = decltype(i)::value;
    if constexpr (DEV) f[I] = RawCodec<ST>::dec(k1_load(fin + size_t(I) * N + nb.template src<I>()));
    else f[I] = Codec<ST>::dec(k1_load(fin + size_t(I) * N + nb.template src<I>()), p.wref[I]);
  });
  CT F[3];
  body_force(p.force_a, p.force_b, p.force_tab, nb.x, nb.y, nb.z, F);
  CT phi_prev = CT(0), phi_now = CT(0);
  if constexpr (EQ == LBM_NCDE) phi_prev = phi[cell];
  constexpr bool AG = GradTerm<L, EQ>::kOn;
  CT gr[3];
  if constexpr (AG) cell_field_gradient<L>(p, cell, nb.x, nb.y, nb.z, gr);
  collide<L, CT, EQ, DEV>(f, p, F, phi_prev, phi_now, &tab, AG ? gr : nullptr);
  if constexpr (EQ == LBM_NCDE) phi[cell] = phi_now;
  if constexpr (AG && EQ == LBM_NSE) {
    if (p.grad_on) p.rho_out[cell] = phi_now;
  }
  static_for<L::Q>([&](auto i) {
    constexpr int I = decltype(i)::value;
    if constexpr (DEV) k1_store(fout + size_t(I) * N + cell, RawCodec<ST>::enc(f[I]));
    else k1_store(fout + size_t(I) * N + cell, Codec<ST>::enc(f[I], p.wref[I]));
  });
}

// Initialisation: f-bar(t=0) = f^eq(fields), written to the stored array at x - e_i so that the
// next pull gather yields it; the NCDE previous-step field starts at phi^0, the previous-step
// density of the single-speed NSE (phi non-null) at rho^0.
template <class L, class CT, class ST, int EQ>
__global__ void __launch_bounds__(kBlock) k_init(const StepParams<CT> p, const double* rho_or_phi,
                                                 const double* u, ST* __restrict__ fout,
                                                 CT* __restrict__ phi) {
  const int cell = blockIdx.x * kBlock + threadIdx.x;
  if (cell >= p.ncells) return;
  const Neigh<L> nb(cell, p);
  const size_t N = size_t(p.ncells);
  const CT r = CT(rho_or_phi[cell]);
  CT uu[3] = {CT(0), CT(0), CT(0)};
  if constexpr (EQ == LBM_NSE) {
    for (int a = 0; a < L::D; ++a) uu[a] = CT(u[size_t(a) * N + cell]);
    if (phi != nullptr) phi[cell] = r;
  } else {
    phi[cell] = r;
  }
  CT f[L::Q];
  equilibrium<L, CT, EQ>(f, p, r, uu);
  static_for<L::Q>([&](auto i) {
    constexpr int I = decltype(i)::value;
    fout[size_t(I) * N + nb.template src<I>()] = Codec<ST>::enc(f[I], p.wref[I]);
  });
}

// Parameter view of a batched step: lattice tables from the kernel parameter, per-solve values
// from the shared-memory copy of the solve's descriptor (same member names as StepParams).
template <class CT>
struct BatchView {
  const CT (&T)[kMaxR][kMaxR];
  const CT (&D)[kMaxR];
  const CT (&invN)[kMaxR];
  const CT (&w)[kMaxQ];
  const CT (&wref)[kMaxQ];
  const CT (&wmom_ref)[kMaxR];
  const CT (&sd)[kMaxR];
  const CT (&half)[kMaxR];
  const CT (&sdn)[3][3];
  const CT (&halfn)[3][3];
  const CT (&u_const)[3];
  CT s_high, one_minus_sh, sh_rho_ref, cs2_eq, nonlin_third;
  int ncde_variant;
  const CT (&kfac)[3];
  CT nonlin_rate, a1;
  const CT (&cde_coef)[3];
  CT half0;
  const int (&n)[3];
  int grad_on;
  const CT (&gscale)[3];
  const CT* grad_in;
  CT* rho_out;
  static constexpr bool kNcdeVariants = true;
  __device__ __forceinline__ BatchView(const BatchTables<CT>& t, const SolveDesc<CT>& d, int parity)
      : T(t.T), D(t.D), invN(t.invN), w(t.w), wref(t.wref), wmom_ref(t.wmom_ref), sd(d.sd), half(d.half),
        sdn(d.sdn), halfn(d.halfn), u_const(d.u_const), s_high(d.s_high), one_minus_sh(d.one_minus_sh), sh_rho_ref(d.sh_rho_ref),
        cs2_eq(d.cs2_eq), nonlin_third(d.nonlin_third), ncde_variant(d.ncde_variant), kfac(d.kfac),
        nonlin_rate(d.nonlin_rate), a1(d.a1), cde_coef(d.cde_coef), half0(d.half0), n(d.n), grad_on(d.grad_on),
        gscale(d.gscale), grad_in(d.grad_in[parity]), rho_out(d.rho_out[parity]) {}
};

// K6: persistent batched collide-stream. The grid is the resident capacity of the GPU; each
// block walks the tile work-list of the group (tiles of BLOCK cells from every solve), stages
// the descriptor of the tile's solve in shared memory when it changes, and runs the same per-cell
// gather / collide / store as k_step.
template <int BLOCK>
constexpr int batch_min_blocks() {
  return BLOCK >= 256 ? 2 : (BLOCK >= 128 ? LBM_K1_MIN_BLOCKS : 10);
}

// One cell of a batched step: the same gather / collide / store as k_step, with the solve's
// parameters from its staged descriptor (HP: the higher-row table of a per-order-rate group).
template <class L, class CT, class ST, int EQ, class HP>
__device__ __forceinline__ void batch_cell(const BatchTables<CT>& t, const SolveDesc<CT>& sd, int cell, int parity,
                                           HP* hp) {
  const Neigh<L> nb(cell, sd.n, sd.div_m, sd.div_s);
  const size_t N = size_t(sd.ncells);
  const ST* __restrict__ fin = static_cast<const ST*>(sd.f[parity]);
  ST* __restrict__ fout = static_cast<ST*>(sd.f[parity ^ 1]);
  const BatchView<CT> p(t, sd, parity);
  constexpr bool DEV = is_deviation_storage<ST>();
  CT f[L::Q];
  static_for<L::Q>([&](auto i) {
    constexpr int I = decltype(i)::value;
    if constexpr (DEV) f[I] = RawCodec<ST>::dec(k1_load(fin + size_t(I) * N + nb.template src<I>()));
    else f[I] = Codec<ST>::dec(k1_load(fin + size_t(I) * N + nb.template src<I>()), p.wref[I]);
  });
  CT F[3];
  body_force(sd.force_a, sd.force_b, sd.force_tab, nb.x, nb.y, nb.z, F);
  CT phi_prev = CT(0), phi_now = CT(0);
  if constexpr (EQ == LBM_NCDE) phi_prev = sd.phi[cell];
  constexpr bool AG = GradTerm<L, EQ>::kOn;
  CT gr[3];
  if constexpr (AG) cell_field_gradient<L>(p, cell, nb.x, nb.y, nb.z, gr);
  collide<L, CT, EQ, DEV>(f, p, F, phi_prev, phi_now, hp, AG ? gr : nullptr);
  if constexpr (EQ == LBM_NCDE) sd.phi[cell] = phi_now;
  if constexpr (AG && EQ == LBM_NSE) {
    if (p.grad_on) p.rho_out[cell] = phi_now;
  }
  static_for<L::Q>([&](auto i) {
    constexpr int I = decltype(i)::value;
    if constexpr (DEV) k1_store(fout + size_t(I) * N + cell, RawCodec<ST>::enc(f[I]));
    else k1_store(fout + size_t(I) * N + cell, Codec<ST>::enc(f[I], p.wref[I]));
  });
}

// Stage the descriptor of solve `solve` in shared memory (block-wide; call with the whole block).
template <class CT, int BLOCK>
__device__ __forceinline__ void stage_desc(SolveDesc<CT>& sd, const SolveDesc<CT>* __restrict__ descs, int solve) {
  constexpr int kWords = int(sizeof(SolveDesc<CT>) / sizeof(int4));
  static_assert(sizeof(SolveDesc<CT>) % sizeof(int4) == 0, "descriptor must be a whole number of int4");
  const int4* src = reinterpret_cast<const int4*>(descs + solve);
  int4* dst = reinterpret_cast<int4*>(&sd);
  for (int w = threadIdx.x; w < kWords; w += BLOCK) dst[w] = src[w];
}

template <class L, class CT, class ST, int EQ, int BLOCK>
__global__ void __launch_bounds__(BLOCK, batch_min_blocks<BLOCK>())
    k_step_batch(const BatchTables<CT> t, const SolveDesc<CT>* __restrict__ descs,
                 const Tile* __restrict__ tiles, int ntiles, int parity) {
  __shared__ SolveDesc<CT> sd;
  int staged = -1;
  for (int ti = blockIdx.x; ti < ntiles; ti += gridDim.x) {
    const Tile tile = tiles[ti];
    if (tile.solve != staged) {
      __syncthreads();
      stage_desc<CT, BLOCK>(sd, descs, tile.solve);
      __syncthreads();
      staged = tile.solve;
    }
    const int cell = tile.cell0 + int(threadIdx.x);
    if (cell >= sd.ncells) continue;
    batch_cell<L, CT, ST, EQ>(t, sd, cell, parity, static_cast<NoHigh*>(nullptr));
  }
}

// The batched step of a group whose solves have one rate per order >= 4: tiles of kBlock cells,
// and the solve's higher-row table (rows of the lattice, rates of the solve) staged in shared
// memory with its descriptor, as k_step_high does for one solve.
template <class L, class CT, class ST, int EQ>
__global__ void __launch_bounds__(kBlock, 3)
    k_step_batch_high(const BatchTables<CT> t, const SolveDesc<CT>* __restrict__ descs,
                      const HighParams<CT>* __restrict__ highs, const Tile* __restrict__ tiles, int ntiles,
                      int parity) {
  __shared__ SolveDesc<CT> sd;
  __shared__ HighTable<L, CT> tab;
  int staged = -1;
  for (int ti = blockIdx.x; ti < ntiles; ti += gridDim.x) {
    const Tile tile = tiles[ti];
    if (tile.solve != staged) {
      __syncthreads();
      stage_desc<CT, kBlock>(sd, descs, tile.solve);
      tab.fill(highs[tile.solve]);
      __syncthreads();
      staged = tile.solve;
    }
    const int cell = tile.cell0 + int(threadIdx.x);
    if (cell >= sd.ncells) continue;
    batch_cell<L, CT, ST, EQ>(t, sd, cell, parity, &tab);
  }
}

}  // namespace lbm

#include "tc_kernels.cuh"

namespace lbm {

template <class L, class CT, class ST, int EQ, class F>
lbm_status batch_by_block(int block, F&& fn) {
  switch (block) {
    case 64: return fn(k_step_batch<L, CT, ST, EQ, 64>);
    case 128: return fn(k_step_batch<L, CT, ST, EQ, 128>);
    case 256: return fn(k_step_batch<L, CT, ST, EQ, 256>);
  }
  return set_error(LBM_ERR_ARG, "batched tile size must be 64, 128 or 256 cells");
}

template <class L, class F>
lbm_status batch_kernel_high(int store, int eq, F&& fn) {
  if (store == LBM_F32) {
    if (eq == LBM_NSE) return fn(k_step_batch_high<L, float, float, LBM_NSE>);
    return fn(k_step_batch_high<L, float, float, LBM_NCDE>);
  }
  if (store == LBM_F16_DEV) {
    if (eq == LBM_NSE) return fn(k_step_batch_high<L, float, __half, LBM_NSE>);
    return fn(k_step_batch_high<L, float, __half, LBM_NCDE>);
  }
  if (store == LBM_BF16_DEV) {
    if (eq == LBM_NSE) return fn(k_step_batch_high<L, float, __nv_bfloat16, LBM_NSE>);
    return fn(k_step_batch_high<L, float, __nv_bfloat16, LBM_NCDE>);
  }
  return set_error(LBM_ERR_NOT_IMPLEMENTED, "batched execution supports F32, F16_DEV and BF16_DEV storage");
}

template <class L, class F>
lbm_status batch_kernel(int store, int eq, int block, F&& fn) {
  if (store == LBM_F32) {
    if (eq == LBM_NSE) return batch_by_block<L, float, float, LBM_NSE>(block, fn);
    return batch_by_block<L, float, float, LBM_NCDE>(block, fn);
  }
  if (store == LBM_F16_DEV) {
    if (eq == LBM_NSE) return batch_by_block<L, float, __half, LBM_NSE>(block, fn);
    return batch_by_block<L, float, __half, LBM_NCDE>(block, fn);
  }
  if (store == LBM_BF16_DEV) {
    if (eq == LBM_NSE) return batch_by_block<L, float, __nv_bfloat16, LBM_NSE>(block, fn);
    return batch_by_block<L, float, __nv_bfloat16, LBM_NCDE>(block, fn);
  }
  return set_error(LBM_ERR_NOT_IMPLEMENTED, "batched execution supports F32, F16_DEV and BF16_DEV storage");
}

template <int KIND>
lbm_status BatchLaunch<KIND>::launch(const BatchGroup& g, int parity, cudaStream_t stream) {
  using L = Lat<KIND>;
  if (g.high) {
    return batch_kernel_high<L>(g.store, g.eq, [&](auto kernel) -> lbm_status {
      const BatchTables<float>& t = *static_cast<const BatchTables<float>*>(g.tables);
      kernel<<<g.grid, kBlock, 0, stream>>>(t, static_cast<const SolveDesc<float>*>(g.d_desc),
                                            static_cast<const HighParams<float>*>(g.d_high), g.d_tiles, g.ntiles,
                                            parity);
      cudaError_t err = cudaGetLastError();
      return err == cudaSuccess ? LBM_OK : cuda_error(err, "batched step launch");
    });
  }
  return batch_kernel<L>(g.store, g.eq, g.block, [&](auto kernel) -> lbm_status {
    using Kern = decltype(kernel);
    (void)sizeof(Kern);
    const BatchTables<float>& t = *static_cast<const BatchTables<float>*>(g.tables);
    kernel<<<g.grid, g.block, 0, stream>>>(t, static_cast<const SolveDesc<float>*>(g.d_desc), g.d_tiles, g.ntiles,
                                           parity);
    cudaError_t err = cudaGetLastError();
    return err == cudaSuccess ? LBM_OK : cuda_error(err, "batched step launch");
  });
}

template <int KIND>
lbm_status BatchLaunch<KIND>::occupancy(int store, int eq, int block, int high, int* blocks_per_sm) {
  using L = Lat<KIND>;
  if (high) {
    return batch_kernel_high<L>(store, eq, [&](auto kernel) -> lbm_status {
      cudaError_t err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, kernel, kBlock, 0);
      return err == cudaSuccess ? LBM_OK : cuda_error(err, "occupancy query");
    });
  }
  return batch_kernel<L>(store, eq, block, [&](auto kernel) -> lbm_status {
    cudaError_t err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, kernel, block, 0);
    return err == cudaSuccess ? LBM_OK : cuda_error(err, "occupancy query");
  });
}

// Host launchers for one lattice kind (instantiated in k_<lattice>.cu).
template <class L, class CT, class ST>
lbm_status launch_step_typed(lbm_model* m, int64_t nsteps, bool collide_on) {
  StepParams<CT> p;
  make_step_params<CT>(m, &p);
  const int grid = (m->ncells + kBlock - 1) / kBlock;
  CT* phi = static_cast<CT*>(m->phi_prev);
  const bool high = collide_on && has_high_rates(m);
  HighParams<CT> hp;
  if (high) make_high_params<CT>(m, &hp);
  // tcgen05 when asked for, and by default with per-order rates (where the dense higher rows make
  // it the faster kernel); on FP32 storage only the higher rows go to the tensor cores
  [[maybe_unused]] const bool tensor = collide_on && (m->tensor_cores || (m->tc_auto && high));
  [[maybe_unused]] const bool tensor32 = std::is_same<ST, float>::value && tensor && high;
  TcParams tp;
  [[maybe_unused]] Tc32Params tp32;
  int tgrid = 0;
  size_t tsmem = 0;
  [[maybe_unused]] auto tc_kernel = [&](auto hi_tag, auto eq_tag) {
    return k_step_tc<L, ST, decltype(eq_tag)::value, decltype(hi_tag)::value>;
  };
  if constexpr (is_deviation_storage<ST>()) {
    if (tensor) {
      make_tc_params(m, &tp);
      using NSE_ = std::integral_constant<int, LBM_NSE>;
      using NCDE_ = std::integral_constant<int, LBM_NCDE>;
      const void* k = nullptr;
      if (high) {
        tsmem = sizeof(TcSmem<L, true>);
        k = m->eq == LBM_NSE ? reinterpret_cast<const void*>(tc_kernel(std::true_type{}, NSE_{}))
                             : reinterpret_cast<const void*>(tc_kernel(std::true_type{}, NCDE_{}));
        tgrid = tc_grid(m, tp.ntiles, k, TcShape<L, true>::CTAS, tsmem);
      } else {
        tsmem = sizeof(TcSmem<L, false>);
        k = m->eq == LBM_NSE ? reinterpret_cast<const void*>(tc_kernel(std::false_type{}, NSE_{}))
                             : reinterpret_cast<const void*>(tc_kernel(std::false_type{}, NCDE_{}));
        tgrid = tc_grid(m, tp.ntiles, k, TcShape<L, false>::CTAS, tsmem);
      }
    }
  }
  if constexpr (std::is_same<ST, float>::value) {
    if (tensor32) {
      make_tc32_params(m, &tp32);
      tsmem = sizeof(Tc32Smem<L>);
      const void* k = m->eq == LBM_NSE ? reinterpret_cast<const void*>(k_step_tc32_high<L, LBM_NSE>)
                                       : reinterpret_cast<const void*>(k_step_tc32_high<L, LBM_NCDE>);
      tgrid = tc_grid(m, tp32.ntiles, k, Tc32Shape<L>::CTAS, tsmem);
    }
  }
  // 16-bit storage: the row-staged gather where it applies (or is forced), with the contractions
  // on the CUDA cores or, when the tensor cores are selected, on tcgen05
  [[maybe_unused]] RowPlan rplan;
  bool rows = false;
  if constexpr (is_deviation_storage<ST>()) {
    if (m->gather == LBM_GATHER_ROWS && high && !tensor)
      return set_error(LBM_ERR_NOT_IMPLEMENTED,
                       "the row-staged gather runs per-order rates on the tensor cores only");
    if (m->gather != LBM_GATHER_THREADS && (!high || tensor)) {
      rows = RowLaunch<L::KIND>::plan(m, &rplan, tensor, high);
      if (!rows && m->gather == LBM_GATHER_ROWS) return set_error(LBM_ERR_ARG, "the row-staged gather does not apply");
      if (rows && nsteps > 0) {
        const lbm_status st = RowLaunch<L::KIND>::configure(m, rplan, collide_on);
        if (st != LBM_OK) return st;
      }
    }
  }
  const bool hist = collide_on && m->m2g_aniso;
  p.grad_on = collide_on && p.grad_on;
  for (int64_t s = 0; s < nsteps; ++s) {
    const ST* fin = static_cast<const ST*>(m->f[m->cur]);
    ST* fout = static_cast<ST*>(m->f[m->cur ^ 1]);
    if (hist) {
      p.grad_in = static_cast<const CT*>(m->rho_hist[m->hist_cur]);
      p.rho_out = static_cast<CT*>(m->rho_hist[m->hist_cur ^ 1]);
    }
    bool done = false;
    if constexpr (is_deviation_storage<ST>()) {
      if (rows) {
        const lbm_status st = RowLaunch<L::KIND>::launch(m, rplan, p, fin, fout, phi, collide_on);
        if (st != LBM_OK) return st;
        done = true;
      } else if (tensor) {
        if (high) {
          if (m->eq == LBM_NSE)
            k_step_tc<L, ST, LBM_NSE, true><<<tgrid, 128, tsmem, m->stream>>>(p, tp, fin, fout, phi);
          else
            k_step_tc<L, ST, LBM_NCDE, true><<<tgrid, 128, tsmem, m->stream>>>(p, tp, fin, fout, phi);
        } else {
          if (m->eq == LBM_NSE)
            k_step_tc<L, ST, LBM_NSE, false><<<tgrid, 128, tsmem, m->stream>>>(p, tp, fin, fout, phi);
          else
            k_step_tc<L, ST, LBM_NCDE, false><<<tgrid, 128, tsmem, m->stream>>>(p, tp, fin, fout, phi);
        }
        done = true;
      }
    }
    if constexpr (std::is_same<ST, float>::value) {
      if (tensor32) {
        if (m->eq == LBM_NSE)
          k_step_tc32_high<L, LBM_NSE><<<tgrid, 128, tsmem, m->stream>>>(p, tp32, fin, fout, phi);
        else
          k_step_tc32_high<L, LBM_NCDE><<<tgrid, 128, tsmem, m->stream>>>(p, tp32, fin, fout, phi);
        done = true;
      }
    }
    if (done) {
    } else if (high) {
      if (m->eq == LBM_NSE)
        k_step_high<L, CT, ST, LBM_NSE><<<grid, kBlock, 0, m->stream>>>(p, hp, fin, fout, phi);
      else
        k_step_high<L, CT, ST, LBM_NCDE><<<grid, kBlock, 0, m->stream>>>(p, hp, fin, fout, phi);
    } else if (!collide_on) {
      k_step<L, CT, ST, LBM_NSE, false><<<grid, kBlock, 0, m->stream>>>(p, fin, fout, phi);
    } else if (m->eq == LBM_NSE) {
      k_step<L, CT, ST, LBM_NSE, true><<<grid, kBlock, 0, m->stream>>>(p, fin, fout, phi);
    } else {
      k_step<L, CT, ST, LBM_NCDE, true><<<grid, kBlock, 0, m->stream>>>(p, fin, fout, phi);
    }
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return cuda_error(err, "collide-stream launch");
    m->cur ^= 1;
    if (hist) m->hist_cur ^= 1;
    m->launches += 1;
    if (collide_on) m->steps += 1;
  }
  return LBM_OK;
}

template <class L, class CT, class ST>
lbm_status launch_init_typed(lbm_model* m, const double* rho_or_phi, const double* u) {
  StepParams<CT> p;
  make_step_params<CT>(m, &p);
  const int grid = (m->ncells + kBlock - 1) / kBlock;
  ST* fout = static_cast<ST*>(m->f[m->cur]);
  CT* phi = static_cast<CT*>(m->eq == LBM_NSE ? m->rho_hist[m->hist_cur] : m->phi_prev);
  if (m->eq == LBM_NSE)
    k_init<L, CT, ST, LBM_NSE><<<grid, kBlock, 0, m->stream>>>(p, rho_or_phi, u, fout, phi);
  else
    k_init<L, CT, ST, LBM_NCDE><<<grid, kBlock, 0, m->stream>>>(p, rho_or_phi, u, fout, phi);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return cuda_error(err, "init launch");
  m->launches += 1;
  return LBM_OK;
}

template <int KIND>
lbm_status Launch<KIND>::step(lbm_model* m, int64_t nsteps, bool collide_on) {
  using L = Lat<KIND>;
  switch (m->store) {
    case LBM_F64: return launch_step_typed<L, double, double>(m, nsteps, collide_on);
    case LBM_F32: return launch_step_typed<L, float, float>(m, nsteps, collide_on);
    case LBM_BF16_DEV: return launch_step_typed<L, float, __nv_bfloat16>(m, nsteps, collide_on);
    case LBM_F16_DEV: return launch_step_typed<L, float, __half>(m, nsteps, collide_on);
  }
  return set_error(LBM_ERR_ARG, "unknown storage dtype");
}

template <int KIND>
lbm_status Launch<KIND>::init(lbm_model* m, const double* rho_or_phi, const double* u) {
  using L = Lat<KIND>;
  switch (m->store) {
    case LBM_F64: return launch_init_typed<L, double, double>(m, rho_or_phi, u);
    case LBM_F32: return launch_init_typed<L, float, float>(m, rho_or_phi, u);
    case LBM_BF16_DEV: return launch_init_typed<L, float, __nv_bfloat16>(m, rho_or_phi, u);
    case LBM_F16_DEV: return launch_init_typed<L, float, __half>(m, rho_or_phi, u);
  }
  return set_error(LBM_ERR_ARG, "unknown storage dtype");
}

}  // namespace lbm

#define LBM_INSTANTIATE_LATTICE(KIND) \
  template struct lbm::Launch<KIND>;     \
  template struct lbm::BatchLaunch<KIND>;
