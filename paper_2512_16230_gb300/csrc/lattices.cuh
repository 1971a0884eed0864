// Compile-time descriptions of the multispeed rectangular lattices (Sec. 5, App. C/D of
// arXiv 2512.16230): integer velocity components e_j in the paper's column order, the
// monomials of order <= 3 in the paper's Hermite-row order, and small constexpr helpers.
//
// Every kernel that walks populations or moments does so with static_for, so the velocity
// components, monomial values and parity pairs are integer constants folded by the compiler:
// structurally zero products never generate an instruction.
#pragma once

#include <cstdint>
#include <type_traits>
#include <utility>

#include "lbm_mrt.h"

namespace lbm {

struct Vel {
  int x, y, z;
};
struct Mono {
  int a, b, c;  // exponents of c_x, c_y, c_z
};

// Eq. (3-1): rD2Q25; rD2Q21/17/13 are its first 21/17/13 columns (Sec. 5 (i)-(iii)).
inline constexpr Vel kQ25[25] = {
    {0, 0, 0},  {1, 0, 0},  {0, 1, 0},  {-1, 0, 0}, {0, -1, 0}, {1, 1, 0},   {-1, 1, 0},
    {-1, -1, 0}, {1, -1, 0}, {2, 0, 0},  {0, 2, 0},  {-2, 0, 0}, {0, -2, 0},  {2, 2, 0},
    {-2, 2, 0}, {-2, -2, 0}, {2, -2, 0}, {3, 0, 0},  {0, 3, 0},  {-3, 0, 0},  {0, -3, 0},
    {3, 3, 0},  {-3, 3, 0}, {-3, -3, 0}, {3, -3, 0}};

// App. D: rD3Q53 = 27 single-speed vectors then the 26 doubled non-zero ones; rD3Q33 and
// rD3Q45 are its first 33 and 45 columns.
inline constexpr Vel kQ27[27] = {
    {0, 0, 0},   {1, 0, 0},   {-1, 0, 0},  {0, 1, 0},  {0, -1, 0},  {0, 0, 1},   {0, 0, -1},
    {1, 1, 0},   {-1, -1, 0}, {-1, 1, 0},  {1, -1, 0}, {1, 0, 1},   {-1, 0, -1}, {-1, 0, 1},
    {1, 0, -1},  {0, 1, 1},   {0, -1, -1}, {0, -1, 1}, {0, 1, -1},  {1, 1, 1},   {-1, -1, -1},
    {1, 1, -1},  {-1, -1, 1}, {1, -1, 1},  {-1, 1, -1}, {-1, 1, 1}, {1, -1, -1}};

constexpr Vel q53(int j) {
  return j < 27 ? kQ27[j] : Vel{2 * kQ27[j - 26].x, 2 * kQ27[j - 26].y, 2 * kQ27[j - 26].z};
}

// Hermite rows / monomials in the paper's order. 2D (App. C): 1, x, y, xx, xy, yy, xyy, xxy,
// xxx, yyy. 3D (App. D, M1..M20): 1, x, y, z, xx, yy, zz, xy, zx, yz, xyy, zzx, xxy, yzz, zxx,
// yyz, xyz, xxx, yyy, zzz.
inline constexpr Mono kMono2[10] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {2, 0, 0}, {1, 1, 0},
                                    {0, 2, 0}, {1, 2, 0}, {2, 1, 0}, {3, 0, 0}, {0, 3, 0}};
inline constexpr Mono kMono3[20] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {2, 0, 0},
                                    {0, 2, 0}, {0, 0, 2}, {1, 1, 0}, {1, 0, 1}, {0, 1, 1},
                                    {1, 2, 0}, {1, 0, 2}, {2, 1, 0}, {0, 1, 2}, {2, 0, 1},
                                    {0, 2, 1}, {1, 1, 1}, {3, 0, 0}, {0, 3, 0}, {0, 0, 3}};

constexpr int ipow(int b, int e) { return e == 0 ? 1 : b * ipow(b, e - 1); }

template <int D>
constexpr Mono mono(int k) {
  return D == 2 ? kMono2[k] : kMono3[k];
}
constexpr int degree(Mono m) { return m.a + m.b + m.c; }
constexpr int mono_value(Vel v, Mono m) {
  return ipow(v.x, m.a) * ipow(v.y, m.b) * ipow(v.z, m.c);
}
// Parity class of a monomial: reflections of a symmetric lattice only couple monomials whose
// exponents have the same parities (Sec. 5: odd lattice moments vanish).
constexpr int parity_class(Mono m) {
  return (m.a & 1) | ((m.b & 1) << 1) | ((m.c & 1) << 2);
}

template <int KIND>
struct Lat;

// SINGLE: the single-speed lattices (components in {0, +-1}), where c_a^3 = c_a^2 c_a makes the
// pure-cube rows (the last D of the paper's list) dependent: they keep the first R - D rows, and
// their equilibrium takes M30 = 0 (the standard-lattice case, k = 1).
template <int Q_>
struct Lat2D {
  static constexpr bool SINGLE = Q_ == 9;
  static constexpr int D = 2, Q = Q_, R = SINGLE ? 8 : 10;
  static constexpr int RMAX = SINGLE ? 1 : (Q_ >= 17 ? 3 : 2);
  static constexpr Vel e(int j) { return kQ25[j]; }
};
template <int Q_>
struct Lat3D {
  static constexpr bool SINGLE = Q_ == 27;
  static constexpr int D = 3, Q = Q_, R = SINGLE ? 17 : 20, RMAX = SINGLE ? 1 : 2;
  static constexpr Vel e(int j) { return q53(j); }
};

template <> struct Lat<LBM_RD2Q13> : Lat2D<13> { static constexpr int KIND = LBM_RD2Q13; };
template <> struct Lat<LBM_RD2Q17> : Lat2D<17> { static constexpr int KIND = LBM_RD2Q17; };
template <> struct Lat<LBM_RD2Q21> : Lat2D<21> { static constexpr int KIND = LBM_RD2Q21; };
template <> struct Lat<LBM_RD2Q25> : Lat2D<25> { static constexpr int KIND = LBM_RD2Q25; };
template <> struct Lat<LBM_RD3Q33> : Lat3D<33> { static constexpr int KIND = LBM_RD3Q33; };
template <> struct Lat<LBM_RD3Q45> : Lat3D<45> { static constexpr int KIND = LBM_RD3Q45; };
template <> struct Lat<LBM_RD3Q53> : Lat3D<53> { static constexpr int KIND = LBM_RD3Q53; };
template <> struct Lat<LBM_RD2Q9> : Lat2D<9> { static constexpr int KIND = LBM_RD2Q9; };
template <> struct Lat<LBM_RD3Q27> : Lat3D<27> { static constexpr int KIND = LBM_RD3Q27; };

// Index of the velocity opposite to j (every lattice here is symmetric under e -> -e).
template <class L>
constexpr int opposite(int j) {
  int found = -1;
  for (int i = 0; i < L::Q; ++i) {
    const Vel a = L::e(i), b = L::e(j);
    if (a.x == -b.x && a.y == -b.y && a.z == -b.z) found = i;
  }
  return found;
}

// Largest |component| of the velocity set.
template <class L>
constexpr int max_component() {
  int m = 0;
  for (int i = 0; i < L::Q; ++i) {
    const Vel v = L::e(i);
    m = v.x > m ? v.x : m;
    m = v.y > m ? v.y : m;
    m = v.z > m ? v.z : m;
  }
  return m;
}

// Index (axis) of a normal second-order row c_a^2 - c_sa^2 among the d normal rows, or -1.
template <int D>
constexpr int normal_index(int r) {
  const Mono m = mono<D>(r);
  return (degree(m) == 2 && (m.a == 2 || m.b == 2 || m.c == 2)) ? (m.a == 2 ? 0 : (m.b == 2 ? 1 : 2)) : -1;
}
// Row of the normal second moment along axis a (2D: rows 3, 5; 3D: rows 4, 5, 6).
template <int D>
constexpr int normal_row(int a) {
  int found = -1;
  for (int r = 0; r < (D == 2 ? 10 : 20); ++r)
    if (normal_index<D>(r) == a) found = r;
  return found;
}

// Primitive directions: every velocity is e = m d with d primitive (components coprime, first
// non-zero component positive) and m in {+-1, +-2, +-3}. Since mono_k(m d) = m^deg(k) mono_k(d),
// the populations of one direction can be combined per degree before the monomial products.
constexpr int iabs(int v) { return v < 0 ? -v : v; }
constexpr int gcd2(int a, int b) { return b == 0 ? a : gcd2(b, a % b); }
constexpr Vel primitive(Vel v) {
  const int g = gcd2(gcd2(iabs(v.x), iabs(v.y)), iabs(v.z));
  const Vel p{v.x / g, v.y / g, v.z / g};
  const int lead = p.x != 0 ? p.x : (p.y != 0 ? p.y : p.z);
  return lead < 0 ? Vel{-p.x, -p.y, -p.z} : p;
}
constexpr bool same_vel(Vel a, Vel b) { return a.x == b.x && a.y == b.y && a.z == b.z; }

template <class L>
constexpr int num_directions() {
  int n = 0;
  for (int i = 1; i < L::Q; ++i) {
    bool seen = false;
    for (int j = 1; j < i; ++j) seen = seen || same_vel(primitive(L::e(j)), primitive(L::e(i)));
    n += seen ? 0 : 1;
  }
  return n;
}
// k-th primitive direction, in order of first appearance in the velocity table
template <class L>
constexpr Vel direction(int k) {
  int n = 0;
  for (int i = 1; i < L::Q; ++i) {
    bool seen = false;
    for (int j = 1; j < i; ++j) seen = seen || same_vel(primitive(L::e(j)), primitive(L::e(i)));
    if (!seen) {
      if (n == k) return primitive(L::e(i));
      ++n;
    }
  }
  return Vel{0, 0, 0};
}
// index of the velocity m d, or -1 if the lattice does not have it
template <class L>
constexpr int velocity_index(Vel d, int m) {
  for (int i = 0; i < L::Q; ++i)
    if (same_vel(L::e(i), Vel{m * d.x, m * d.y, m * d.z})) return i;
  return -1;
}

// +-e pairs: the p-th pair is (pair_plus(p), opposite(pair_plus(p))), pair_plus(p) being the p-th
// velocity i >= 1 (in table order) whose opposite has a larger index.
template <class L>
constexpr int num_pairs() {
  return (L::Q - 1) / 2;
}
template <class L>
constexpr int pair_plus(int p) {
  int n = 0;
  for (int i = 1; i < L::Q; ++i)
    if (opposite<L>(i) > i) {
      if (n == p) return i;
      ++n;
    }
  return -1;
}
// Rows of order >= 4 of the complete Q x Q Hermite matrix, split by parity under e -> -e: the
// even lattice functions span the rest velocity and one function per pair (num_pairs + 1), the
// odd ones one per pair; the orders <= 3 take the even rows of degree 0, 2 and the odd ones of
// degree 1, 3.
template <class L>
constexpr int low_rows_even() {
  int n = 0;
  for (int r = 0; r < L::R; ++r) n += (degree(mono<L::D>(r)) % 2 == 0) ? 1 : 0;
  return n;
}
template <class L>
constexpr int high_even() {
  return num_pairs<L>() + 1 - low_rows_even<L>();
}
template <class L>
constexpr int high_odd() {
  return num_pairs<L>() - (L::R - low_rows_even<L>());
}

// static_for<N>(f) calls f(std::integral_constant<int, 0>) ... f(integral_constant<int, N-1>).
// Inside nested lambdas, read a captured index as decltype(i)::value (a constant expression
// whatever the capture); the constexpr helpers above are evaluated at compile time only.
template <class F, int... I>
__host__ __device__ __forceinline__ void static_for_impl(F&& f, std::integer_sequence<int, I...>) {
  (f(std::integral_constant<int, I>{}), ...);
}
template <int N, class F>
__host__ __device__ __forceinline__ void static_for(F&& f) {
  static_for_impl(f, std::make_integer_sequence<int, N>{});
}

// Host-side view of a lattice's velocity table (for generic, non-hot kernels and set-up).
inline int lattice_dims(int kind) { return (kind <= LBM_RD2Q25 || kind == LBM_RD2Q9) ? 2 : 3; }
inline bool lattice_single(int kind) { return kind == LBM_RD2Q9 || kind == LBM_RD3Q27; }
// rows of order <= 3: the paper's 10 (2D) or 20 (3D), without the d pure cubes on single-speed sets
inline int lattice_r(int kind) {
  const int d = lattice_dims(kind);
  return (d == 2 ? 10 : 20) - (lattice_single(kind) ? d : 0);
}
inline int lattice_q(int kind) {
  switch (kind) {
    case LBM_RD2Q13: return 13;
    case LBM_RD2Q17: return 17;
    case LBM_RD2Q21: return 21;
    case LBM_RD2Q25: return 25;
    case LBM_RD3Q33: return 33;
    case LBM_RD3Q45: return 45;
    case LBM_RD3Q53: return 53;
    case LBM_RD2Q9: return 9;
    case LBM_RD3Q27: return 27;
  }
  return 0;
}
inline Vel lattice_e(int kind, int j) { return lattice_dims(kind) == 2 ? kQ25[j] : q53(j); }
// Host view of the pair order above: plus[p] for p < (Q - 1) / 2.
inline void lattice_pairs(int kind, int* plus) {
  const int Q = lattice_q(kind);
  int n = 0;
  for (int i = 1; i < Q; ++i) {
    const Vel a = lattice_e(kind, i);
    int opp = -1;
    for (int j = 0; j < Q; ++j) {
      const Vel b = lattice_e(kind, j);
      if (a.x == -b.x && a.y == -b.y && a.z == -b.z) opp = j;
    }
    if (opp > i) plus[n++] = i;
  }
}
inline int lattice_rmax(int kind) {
  if (lattice_single(kind)) return 1;
  return (kind == LBM_RD2Q17 || kind == LBM_RD2Q21 || kind == LBM_RD2Q25) ? 3 : 2;
}

constexpr int kMaxQ = 53;
constexpr int kMaxR = 20;
constexpr int kMaxPairs = 26;  // rD3Q53
constexpr int kMaxHighEven = 20;
constexpr int kMaxHighOdd = 13;
constexpr int kMaxOrder = 12;  // highest monomial degree tried when completing the Hermite matrix

}  // namespace lbm
