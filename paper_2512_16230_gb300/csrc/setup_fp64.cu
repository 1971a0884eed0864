// FP64 lattice set-up on the GPU (one thread block).
//
// 1. Weights. Sec. 5 determines the weights of a symmetric lattice by its even-order moments:
//    sum w = 1 (Eq. (new11a)), Delta2_aa = c_sa^2 (Eq. (Cont1-5a)), Delta4_aabb = Delta2_aa
//    Delta2_bb (Eq. (Cont1-5b)), Delta4_aaaa = 3 Delta2_aa^2 (Eq. (Cont1-5c)) and, in 3D,
//    Delta6_xxyyzz = Delta2_xx Delta2_yy Delta2_zz (Eq. (Cont1-5e)); the rD3Q53/rD3Q45 weight
//    list of App. D also imposes Eq. (Cont1-5d) for the axis pairs a < b. Velocities related by
//    axis reflections share a weight (Eq. (3-1-2), App. D), so the unknowns are one weight per
//    reflection class |e| = (|e_x|, |e_y|, |e_z|); the free weights of the paper (App. D:
//    w45; Eq. (WeightQ25): w13, w17, w18, w21) are given, and the remaining square linear
//    system is solved by Gaussian elimination with partial pivoting. This reproduces the
//    printed closed forms (Eq. (WeightQ25), Eq. (Q13lattice), App. D) without transcribing them.
// 2. Hermite rows. Weighted (W-inner-product) modified Gram-Schmidt of the monomials in the
//    paper's row order, restricted to monomials of the same parity class (reflection symmetry
//    makes every cross-class inner product vanish). In that order the projections of the
//    third-order rows onto x(y^2 - c_sy^2) etc. are exactly the rectangular-cell correction of
//    Eq. (CorrectQ25) and App. D. The result is kept as the monic lower-triangular factor T
//    (H_r = sum_k T_rk mono_k) together with H on the lattice and the norms N_r.
// 3. Checks: N_r > 0 and |<H_r, H_s>_W| <= 1e-12 sqrt(N_r N_s) for r != s.
// 4. Rows of order >= 4 (the paper leaves them to the designer): monomials of degree 4, 5, ...
//    are tried in graded order and kept when they raise the rank of the rows so far (Euclidean
//    test against an orthonormal basis of their span); each kept one is W-orthogonalised against
//    every earlier row, lower orders and its own, so that the order-k rows span the W-orthogonal
//    complement of the orders < k within the monomials of degree <= k, a block that can carry
//    one rate per order.
#include <cmath>
#include <cstring>

#include "lbm_internal.cuh"

namespace lbm {

namespace {

struct SetupIn {
  int kind, d, Q, R;
  int8_t e[kMaxQ][3];
  int mono[kMaxR][3];
  double c[3], cs2[3];
  double free_w[4];
};

struct SetupOut {
  double w[kMaxQ];
  double H[kMaxR][kMaxQ];
  double N[kMaxR];
  double T[kMaxR][kMaxR];
  double max_offdiag;
  int status;  // 0 ok, 1 singular weight system, 2 non-positive norm, 3 not orthogonal
};

constexpr int kSetupThreads = 64;

__device__ double block_sum64(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  const double s = sh[0] + sh[1];
  __syncthreads();
  return s;
}

// Reflection class key of a velocity: (|e_x|, |e_y|, |e_z|) packed in base 4.
__device__ int class_key(const int8_t* e) {
  return abs(e[0]) + 4 * abs(e[1]) + 16 * abs(e[2]);
}

// Solve the weight system on one thread. Returns false if singular.
__device__ bool solve_weights(const SetupIn& in, double* w) {
  const int d = in.d;
  double d0[3];
  for (int a = 0; a < 3; ++a) d0[a] = a < d ? in.cs2[a] / (in.c[a] * in.c[a]) : 0.0;
  // distinct classes present in the lattice, in order of first appearance
  int keys[kMaxQ], nk = 0, cls_of[kMaxQ];
  for (int j = 0; j < in.Q; ++j) {
    const int k = class_key(in.e[j]);
    int found = -1;
    for (int t = 0; t < nk; ++t)
      if (keys[t] == k) found = t;
    if (found < 0) {
      keys[nk] = k;
      found = nk++;
    }
    cls_of[j] = found;
  }
  // given (free) class weights
  double given[kMaxQ];
  bool is_given[kMaxQ];
  for (int t = 0; t < nk; ++t) {
    is_given[t] = false;
    given[t] = 0.0;
  }
  auto give = [&](int ax, int ay, int az, double v) {
    const int k = ax + 4 * ay + 16 * az;
    for (int t = 0; t < nk; ++t)
      if (keys[t] == k) {
        is_given[t] = true;
        given[t] = v;
      }
  };
  switch (in.kind) {
    case LBM_RD2Q25: give(3, 3, 0, in.free_w[3]);  // fallthrough
    case LBM_RD2Q21: give(3, 0, 0, in.free_w[1]); give(0, 3, 0, in.free_w[2]);  // fallthrough
    case LBM_RD2Q17: give(2, 2, 0, in.free_w[0]); break;
    case LBM_RD3Q53: give(2, 2, 2, in.free_w[0]); break;
    default: break;
  }
  // moment equations: sum_classes W_t * g_t = rhs, g_t = sum_{j in class t} g(e_j)
  double A[16][17];
  int neq = 0;
  auto add_eq = [&](int px, int py, int pz, double rhs) {
    for (int t = 0; t < nk; ++t) A[neq][t] = 0.0;
    for (int j = 0; j < in.Q; ++j) {
      double g = 1.0;
      for (int q = 0; q < px; ++q) g *= in.e[j][0];
      for (int q = 0; q < py; ++q) g *= in.e[j][1];
      for (int q = 0; q < pz; ++q) g *= in.e[j][2];
      A[neq][cls_of[j]] += g;
    }
    A[neq][16] = rhs;
    ++neq;
  };
  add_eq(0, 0, 0, 1.0);
  for (int a = 0; a < d; ++a) add_eq(a == 0 ? 2 : 0, a == 1 ? 2 : 0, a == 2 ? 2 : 0, d0[a]);
  // the axis fourth moments: a single-speed set cannot meet them (c^4 = c^2), its defect is the
  // delta^(4) of k = 1
  const bool single = in.kind == LBM_RD2Q9 || in.kind == LBM_RD3Q27;
  if (!single)
    for (int a = 0; a < d; ++a) add_eq(a == 0 ? 4 : 0, a == 1 ? 4 : 0, a == 2 ? 4 : 0, 3.0 * d0[a] * d0[a]);
  for (int a = 0; a < d; ++a)
    for (int b = a + 1; b < d; ++b)
      add_eq((a == 0) * 2 + (b == 0) * 2, (a == 1) * 2 + (b == 1) * 2, (a == 2) * 2 + (b == 2) * 2,
             d0[a] * d0[b]);
  if (d == 3) {
    add_eq(2, 2, 2, d0[0] * d0[1] * d0[2]);
    if (in.kind == LBM_RD3Q53 || in.kind == LBM_RD3Q45) {
      for (int a = 0; a < 3; ++a)
        for (int b = a + 1; b < 3; ++b)
          add_eq((a == 0) * 4 + (b == 0) * 2, (a == 1) * 4 + (b == 1) * 2, (a == 2) * 4 + (b == 2) * 2,
                 3.0 * d0[a] * d0[a] * d0[b]);
    }
  }
  // move given classes to the right-hand side, compress unknown columns
  int unk[16], nu = 0;
  for (int t = 0; t < nk; ++t)
    if (!is_given[t]) unk[nu++] = t;
  if (nu != neq) return false;
  double M[16][17];
  for (int r = 0; r < neq; ++r) {
    double rhs = A[r][16];
    for (int t = 0; t < nk; ++t)
      if (is_given[t]) rhs -= A[r][t] * given[t];
    for (int u = 0; u < nu; ++u) M[r][u] = A[r][unk[u]];
    M[r][nu] = rhs;
  }
  for (int col = 0; col < nu; ++col) {
    int piv = col;
    for (int r = col + 1; r < nu; ++r)
      if (fabs(M[r][col]) > fabs(M[piv][col])) piv = r;
    if (fabs(M[piv][col]) < 1e-300) return false;
    if (piv != col)
      for (int q = 0; q <= nu; ++q) {
        const double t = M[col][q];
        M[col][q] = M[piv][q];
        M[piv][q] = t;
      }
    for (int r = 0; r < nu; ++r) {
      if (r == col) continue;
      const double f = M[r][col] / M[col][col];
      for (int q = col; q <= nu; ++q) M[r][q] -= f * M[col][q];
    }
  }
  double cw[kMaxQ];
  for (int t = 0; t < nk; ++t) cw[t] = given[t];
  for (int u = 0; u < nu; ++u) cw[unk[u]] = M[u][nu] / M[u][u];
  for (int j = 0; j < in.Q; ++j) w[j] = cw[cls_of[j]];
  return true;
}

__global__ void __launch_bounds__(kSetupThreads) k_setup(const SetupIn in, SetupOut* out) {
  __shared__ double w[kMaxQ];
  __shared__ double H[kMaxR][kMaxQ];
  __shared__ double T[kMaxR][kMaxR];
  __shared__ double N[kMaxR];
  __shared__ double red[2];
  __shared__ int ok;
  const int tid = threadIdx.x;
  if (tid == 0) ok = solve_weights(in, w) ? 0 : 1;
  __syncthreads();
  if (ok != 0) {
    if (tid == 0) out->status = ok;
    return;
  }
  const int Q = in.Q, R = in.R;
  // monomials mono_k(c_j) = prod_a (c_a e_ja)^{p_ka}
  for (int r = 0; r < R; ++r) {
    if (tid < Q) {
      double v = 1.0;
      for (int a = 0; a < 3; ++a)
        for (int q = 0; q < in.mono[r][a]; ++q) v *= in.c[a] * double(in.e[tid][a]);
      H[r][tid] = v;
    }
    if (tid < R) T[r][tid] = (r == tid) ? 1.0 : 0.0;
  }
  __syncthreads();
  auto cls = [&](int r) {
    return (in.mono[r][0] & 1) | ((in.mono[r][1] & 1) << 1) | ((in.mono[r][2] & 1) << 2);
  };
  for (int r = 0; r < R; ++r) {
    for (int s = 0; s < r; ++s) {
      if (cls(s) != cls(r)) continue;
      const double ip = block_sum64(tid < Q ? w[tid] * H[r][tid] * H[s][tid] : 0.0, red);
      const double coef = ip / N[s];
      if (tid < Q) H[r][tid] -= coef * H[s][tid];
      if (tid < R) T[r][tid] -= coef * T[s][tid];
      __syncthreads();
    }
    const double nr = block_sum64(tid < Q ? w[tid] * H[r][tid] * H[r][tid] : 0.0, red);
    if (tid == 0) N[r] = nr;
    __syncthreads();
  }
  // checks
  int status = 0;
  double maxoff = 0.0;
  for (int r = 0; r < R; ++r) {
    if (!(N[r] > 0.0)) status = 2;
    for (int s = 0; s < r; ++s) {
      const double ip = block_sum64(tid < Q ? w[tid] * H[r][tid] * H[s][tid] : 0.0, red);
      const double rel = fabs(ip) / sqrt(fabs(N[r] * N[s]));
      maxoff = rel > maxoff ? rel : maxoff;
    }
  }
  if (status == 0 && !(maxoff <= 1e-12)) status = 3;
  if (tid < Q) {
    out->w[tid] = w[tid];
    for (int r = 0; r < R; ++r) out->H[r][tid] = H[r][tid];
  }
  if (tid < R) {
    out->N[tid] = N[tid];
    for (int k = 0; k < R; ++k) out->T[tid][k] = T[tid][k];
  }
  if (tid == 0) {
    out->status = status;
    out->max_offdiag = maxoff;
  }
}

// Completion of the Hermite matrix by rows of order >= 4 (one block, global scratch).
struct HighWork {
  double U[kMaxQ][kMaxQ];   // Euclidean orthonormal basis of the span of the rows so far
  double Hh[kMaxQ][kMaxQ];  // W-orthogonal rows (H0..H3 first, then the higher ones)
  double N[kMaxQ];
  int order[kMaxQ];
  int nrows, status;
};

__global__ void __launch_bounds__(kSetupThreads) k_setup_high(const SetupIn in, const SetupOut* low,
                                                              HighWork* hw) {
  __shared__ double v[kMaxQ], coef[kMaxQ];
  __shared__ double red[2];
  __shared__ int nu;
  const int tid = threadIdx.x;
  const int Q = in.Q, R = in.R;
  auto euclid_project_out = [&](int count) {  // v -= U U^T v over the first count basis vectors
    for (int pass = 0; pass < 2; ++pass) {
      if (tid < count) {
        double dot = 0.0;
        for (int i = 0; i < Q; ++i) dot += hw->U[tid][i] * v[i];
        coef[tid] = dot;
      }
      __syncthreads();
      if (tid < Q) {
        double acc = v[tid];
        for (int j = 0; j < count; ++j) acc -= coef[j] * hw->U[j][tid];
        v[tid] = acc;
      }
      __syncthreads();
    }
  };
  auto w_project_out = [&](int count) {  // v -= sum_j <v, H_j>_W / N_j H_j
    for (int pass = 0; pass < 2; ++pass) {
      if (tid < count) {
        double dot = 0.0;
        for (int i = 0; i < Q; ++i) dot += low->w[i] * hw->Hh[tid][i] * v[i];
        coef[tid] = dot / hw->N[tid];
      }
      __syncthreads();
      if (tid < Q) {
        double acc = v[tid];
        for (int j = 0; j < count; ++j) acc -= coef[j] * hw->Hh[j][tid];
        v[tid] = acc;
      }
      __syncthreads();
    }
  };
  auto append_basis = [&](int slot) {  // U[slot] = v / |v| (v already orthogonal to U[0..slot))
    const double nrm = sqrt(block_sum64(tid < Q ? v[tid] * v[tid] : 0.0, red));
    if (tid < Q) hw->U[slot][tid] = v[tid] / nrm;
    __syncthreads();
  };
  // H0..H3 seed both bases
  if (tid == 0) {
    nu = 0;
    hw->status = 0;
  }
  __syncthreads();
  for (int r = 0; r < R; ++r) {
    if (tid < Q) {
      v[tid] = low->H[r][tid];
      hw->Hh[r][tid] = low->H[r][tid];
    }
    if (tid == 0) {
      hw->N[r] = low->N[r];
      hw->order[r] = in.mono[r][0] + in.mono[r][1] + in.mono[r][2];
    }
    __syncthreads();
    euclid_project_out(r);
    append_basis(r);
  }
  int n = R;
  for (int deg = 4; deg <= kMaxOrder && n < Q; ++deg) {
    for (int a = deg; a >= 0 && n < Q; --a) {
      for (int b = deg - a; b >= 0 && n < Q; --b) {
        const int c = deg - a - b;
        if (in.d == 2 && c != 0) continue;
        if (tid < Q) {
          double x = 1.0;
          for (int q = 0; q < a; ++q) x *= in.c[0] * double(in.e[tid][0]);
          for (int q = 0; q < b; ++q) x *= in.c[1] * double(in.e[tid][1]);
          for (int q = 0; q < c; ++q) x *= in.c[2] * double(in.e[tid][2]);
          v[tid] = x;
        }
        __syncthreads();
        const double n0 = sqrt(block_sum64(tid < Q ? v[tid] * v[tid] : 0.0, red));
        euclid_project_out(n);
        const double n1 = sqrt(block_sum64(tid < Q ? v[tid] * v[tid] : 0.0, red));
        if (!(n1 > 1e-9 * n0)) continue;  // already in the span
        append_basis(n);
        // the new row: the monomial, W-orthogonal to every earlier row, scaled to unit max
        if (tid < Q) {
          double x = 1.0;
          for (int q = 0; q < a; ++q) x *= in.c[0] * double(in.e[tid][0]);
          for (int q = 0; q < b; ++q) x *= in.c[1] * double(in.e[tid][1]);
          for (int q = 0; q < c; ++q) x *= in.c[2] * double(in.e[tid][2]);
          v[tid] = x;
        }
        __syncthreads();
        w_project_out(n);
        if (tid == 0) {
          double m = 0.0;
          for (int i = 0; i < Q; ++i) m = fabs(v[i]) > m ? fabs(v[i]) : m;
          coef[0] = m;
        }
        __syncthreads();
        const double scale = coef[0];
        __syncthreads();
        if (tid < Q) hw->Hh[n][tid] = v[tid] / scale;
        __syncthreads();
        // a row whose W-norm vanishes on the scale of the largest weight lives on zero-weight
        // velocities only (the Euclidean norm of a unit-max row is at least 1)
        const double nn = block_sum64(tid < Q ? low->w[tid] * hw->Hh[n][tid] * hw->Hh[n][tid] : 0.0, red);
        const double ne = block_sum64(tid < Q ? hw->Hh[n][tid] * hw->Hh[n][tid] : 0.0, red);
        if (tid == 0) {
          double wmax = 0.0;
          for (int i = 0; i < Q; ++i) wmax = fabs(low->w[i]) > wmax ? fabs(low->w[i]) : wmax;
          hw->N[n] = nn;
          hw->order[n] = deg;
          if (!(fabs(nn) > 1e-10 * wmax * ne)) hw->status = 2;
        }
        __syncthreads();
        ++n;
      }
    }
  }
  if (tid == 0) {
    hw->nrows = n;
    if (n < Q && hw->status == 0) hw->status = 1;
  }
}

}  // namespace

lbm_status setup_lattice_fp64(lbm_lattice* lat) {
  SetupIn in;
  std::memset(&in, 0, sizeof(in));
  in.kind = lat->kind;
  in.d = lat->d;
  in.Q = lat->Q;
  in.R = lat->R;
  for (int j = 0; j < lat->Q; ++j)
    for (int a = 0; a < 3; ++a) in.e[j][a] = lat->e[j * 3 + a];
  for (int r = 0; r < lat->R; ++r) {
    const Mono m = lat->d == 2 ? kMono2[r] : kMono3[r];
    in.mono[r][0] = m.a;
    in.mono[r][1] = m.b;
    in.mono[r][2] = m.c;
  }
  for (int a = 0; a < 3; ++a) {
    in.c[a] = lat->c[a];
    in.cs2[a] = lat->cs2[a];
  }
  for (int k = 0; k < 4; ++k) in.free_w[k] = lat->free_w[k];
  SetupOut* dout = nullptr;
  HighWork* dhigh = nullptr;
  cudaError_t err = cudaMalloc(&dout, sizeof(SetupOut));
  if (err == cudaSuccess) err = cudaMalloc(&dhigh, sizeof(HighWork));
  if (err != cudaSuccess) {
    cudaFree(dout);
    return cuda_error(err, "set-up allocation");
  }
  k_setup<<<1, kSetupThreads>>>(in, dout);
  err = cudaGetLastError();
  SetupOut out;
  if (err == cudaSuccess) err = cudaMemcpy(&out, dout, sizeof(SetupOut), cudaMemcpyDeviceToHost);
  if (err == cudaSuccess && out.status == 0) {
    k_setup_high<<<1, kSetupThreads>>>(in, dout, dhigh);
    err = cudaGetLastError();
  }
  HighWork* high = nullptr;
  if (err == cudaSuccess && out.status == 0) {
    high = new HighWork;
    err = cudaMemcpy(high, dhigh, sizeof(HighWork), cudaMemcpyDeviceToHost);
  }
  cudaFree(dout);
  cudaFree(dhigh);
  if (err != cudaSuccess) {
    delete high;
    return cuda_error(err, "set-up kernel");
  }
  if (out.status == 1) return set_error(LBM_ERR_LATTICE_INFEASIBLE, "weight moment system is singular");
  if (out.status == 2) return set_error(LBM_ERR_LATTICE_INFEASIBLE, "a Hermite norm N_r is not positive");
  if (out.status == 3)
    return set_error(LBM_ERR_LATTICE_INFEASIBLE,
                     "H W H^T is not diagonal (max relative off-diagonal " + std::to_string(out.max_offdiag) + ")");
  for (int j = 0; j < lat->Q; ++j) lat->w[j] = out.w[j];
  for (int r = 0; r < lat->R; ++r) {
    for (int j = 0; j < lat->Q; ++j) lat->H[r * lat->Q + j] = out.H[r][j];
    lat->N[r] = out.N[r];
    for (int k = 0; k < lat->R; ++k) lat->T[r * lat->R + k] = out.T[r][k];
  }
  // higher rows: even degrees first, then odd, each by order (stable)
  lat->high_status = high->status;
  lat->nhigh = 0;
  for (int odd = 0; odd < 2; ++odd)
    for (int r = lat->R; r < high->nrows; ++r) {
      if ((high->order[r] & 1) != odd) continue;
      const int t = lat->nhigh++;
      lat->h_order[t] = high->order[r];
      lat->Nh[t] = high->N[r];
      for (int j = 0; j < lat->Q; ++j) lat->Hh[t * lat->Q + j] = high->Hh[r][j];
    }
  delete high;
  return LBM_OK;
}

}  // namespace lbm
