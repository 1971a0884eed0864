// The extern "C" entry points of include/lbm_mrt.h: argument validation, device memory layout,
// parameter marshalling and dispatch to the kernels. No exception crosses the ABI.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "lbm_internal.cuh"

namespace lbm {

namespace {
thread_local std::string g_last_error;
}

lbm_status set_error(lbm_status st, const std::string& msg) {
  g_last_error = msg;
  return st;
}

lbm_status cuda_error(cudaError_t err, const char* what) {
  return set_error(err == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA,
                   std::string(what) + ": " + cudaGetErrorName(err) + " (" + cudaGetErrorString(err) + ")");
}

template <class CT>
void make_step_params(const lbm_model* m, StepParams<CT>* p) {
  const lbm_lattice* L = m->lat;
  std::memset(p, 0, sizeof(*p));
  const int R = L->R;
  for (int r = 0; r < R; ++r) {
    for (int k = 0; k < R; ++k) p->T[r][k] = CT(L->T[r * R + k]);
    const Mono mk = L->d == 2 ? kMono2[r] : kMono3[r];
    double Dk = 1.0;
    for (int q = 0; q < mk.a; ++q) Dk *= L->c[0];
    for (int q = 0; q < mk.b; ++q) Dk *= L->c[1];
    for (int q = 0; q < mk.c; ++q) Dk *= L->c[2];
    p->D[r] = CT(Dk);
    p->invN[r] = CT(1.0 / L->N[r]);
    p->sd[r] = CT(m->s[r] - m->s_high);
    p->half[r] = CT(1.0 - 0.5 * m->s[r]);
  }
  // normal second-order block: S_n = inverse of diag(1/s_sa) + a 1^T / d, a_a = 1/s_b - 1/s_sa
  // (Eq. (4-27) with k = 0), or diag(s_sa) without a bulk rate
  {
    const int d = L->d;
    int rows[3] = {0, 0, 0};
    for (int r = 0, k = 0; r < R; ++r) {
      const Mono mk = d == 2 ? kMono2[r] : kMono3[r];
      if (mk.a + mk.b + mk.c == 2 && (mk.a == 2 || mk.b == 2 || mk.c == 2)) rows[k++] = r;
    }
    double Sn[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    if (m->s_bulk > 0.0 && m->eq == LBM_NSE) {
      // k = 1 (single-speed lattices): a_a = (1/s_b - 1/s_sa)(c_a^2 - c_s^2), b_b = 1/(c_b^2 - c_s^2)
      double Dk[3] = {1.0, 1.0, 1.0};
      if (lattice_single(L->kind))
        for (int a = 0; a < d; ++a) Dk[a] = L->c[a] * L->c[a] - m->cs2_eq;
      double A[3][6];  // [M | I] Gauss-Jordan
      for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) {
          A[i][j] = (i == j ? 1.0 / m->s[rows[i]] : 0.0) +
                    (1.0 / m->s_bulk - 1.0 / m->s[rows[i]]) * Dk[i] / Dk[j] / d;
          A[i][d + j] = i == j ? 1.0 : 0.0;
        }
      for (int c = 0; c < d; ++c) {
        int piv = c;
        for (int r = c + 1; r < d; ++r)
          if (std::fabs(A[r][c]) > std::fabs(A[piv][c])) piv = r;
        for (int q = 0; q < 2 * d; ++q) std::swap(A[c][q], A[piv][q]);
        const double inv = 1.0 / A[c][c];
        for (int q = 0; q < 2 * d; ++q) A[c][q] *= inv;
        for (int r = 0; r < d; ++r)
          if (r != c) {
            const double f = A[r][c];
            for (int q = 0; q < 2 * d; ++q) A[r][q] -= f * A[c][q];
          }
      }
      for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) Sn[i][j] = A[i][d + j];
    } else {
      for (int i = 0; i < d; ++i) Sn[i][i] = m->s[rows[i]];
    }
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        p->sdn[i][j] = CT(Sn[i][j] - (i == j && i < d ? m->s_high : 0.0));
        p->halfn[i][j] = CT((i == j && i < d ? 1.0 : 0.0) - 0.5 * Sn[i][j]);
      }
  }
  const bool dev = m->store == LBM_BF16_DEV || m->store == LBM_F16_DEV;
  for (int i = 0; i < L->Q; ++i) {
    p->w[i] = CT(L->w[i]);
    p->wref[i] = dev ? CT(L->w[i] * m->rho_ref) : CT(0);
  }
  const double rho_ref = dev ? m->rho_ref : 0.0;
  for (int r = 0; r < R; ++r) {
    const Mono mk = L->d == 2 ? kMono2[r] : kMono3[r];
    double acc = 0.0;
    for (int i = 0; i < L->Q; ++i) {
      double v = L->w[i];
      for (int q = 0; q < mk.a; ++q) v *= L->e[i * 3 + 0];
      for (int q = 0; q < mk.b; ++q) v *= L->e[i * 3 + 1];
      for (int q = 0; q < mk.c; ++q) v *= L->e[i * 3 + 2];
      acc += v;
    }
    p->wmom_ref[r] = CT(rho_ref * acc);
  }
  // NCDE variants (App. A): a1 folds into the first-order factor of M1G (moment variant);
  // the rate variant takes its per-cell factors in the kernel; the CDE has no M1 and no M1G
  p->ncde_variant = m->eq == LBM_NCDE ? m->ncde_variant : LBM_NCDE_MOMENT;
  if (m->eq == LBM_NCDE) {
    for (int a = 0; a < L->d; ++a) {
      const double s1 = m->s[1 + a];
      p->half[1 + a] = CT(1.0 - 0.5 * s1 - s1 * m->a1);
      p->kfac[a] = CT(1.0 / s1 - 0.5);
      p->cde_coef[a] = m->ncde_variant == LBM_NCDE_CDE ? CT(m->u_const[a] * s1 / m->cs2_eq) : CT(0);
    }
    p->nonlin_rate = m->ncde_variant == LBM_NCDE_RATE ? CT(m->nonlin) : CT(0);
    p->a1 = CT(m->a1);
    p->half0 = CT(1.0 - 0.5 * m->s[0]);
  }
  // (delta4 . u) . grad rho of Eq. (M2Ga) on the single-speed lattices: delta4_aaaa = c_a^2 - 3 c_s^2,
  // d_a rho by the central difference over the cell spacing c_a (dt = 1)
  // (the step launcher points grad_in / rho_out at the density history); the cross diffusion of
  // the NCDE, -S1 A2 grad psi in M1G with A2 = a2 I (Eq. (M-NCDE-6)), from the prescribed psi
  if (m->eq == LBM_NSE && m->m2g_aniso) {
    p->grad_on = 1;
    for (int a = 0; a < L->d; ++a) p->gscale[a] = CT((L->c[a] * L->c[a] - 3.0 * m->cs2_eq) / (2.0 * L->c[a]));
  } else if (m->eq == LBM_NCDE && m->a2 != 0.0) {
    p->grad_on = 1;
    for (int a = 0; a < L->d; ++a) p->gscale[a] = CT(m->a2 / (2.0 * L->c[a]));
    p->grad_in = static_cast<const CT*>(m->psi);
  }
  p->sh_rho_ref = CT(m->s_high * rho_ref);
  p->s_high = CT(m->s_high);
  p->one_minus_sh = CT(1.0 - m->s_high);
  p->cs2_eq = CT(m->cs2_eq);
  p->nonlin_third = CT(m->ncde_variant == LBM_NCDE_MOMENT ? m->nonlin / 3.0 : 0.0);
  for (int a = 0; a < 3; ++a) {
    p->u_const[a] = CT(m->ncde_variant == LBM_NCDE_CDE ? 0.0 : m->u_const[a]);
    p->n[a] = a < L->d ? int(m->n[a]) : 1;
  }
  p->ncells = m->ncells;
  for (int a = 0; a < 2; ++a) division_magic(unsigned(p->n[a] > 1 ? p->n[a] : 2), &p->div_m[a], &p->div_s[a]);
  const bool force = m->eq == LBM_NSE && m->force_A != 0.0;
  p->force_a = force ? m->force_a : 0;
  p->force_b = force ? m->force_b : -1;
  p->force_tab = static_cast<const CT*>(m->force_tab);
}

template void make_step_params<float>(const lbm_model*, StepParams<float>*);
template void make_step_params<double>(const lbm_model*, StepParams<double>*);

double high_rate(const lbm_model* m, int order) {
  const double s = order <= kMaxOrder ? m->s_order[order] : 0.0;
  return s > 0.0 ? s : m->s_high;
}

bool has_high_rates(const lbm_model* m) {
  const lbm_lattice* L = m->lat;
  for (int r = 0; r < L->nhigh; ++r)
    if (high_rate(m, L->h_order[r]) != m->s_high) return true;
  return false;
}

template <class CT>
void make_high_params(const lbm_model* m, HighParams<CT>* hp) {
  const lbm_lattice* L = m->lat;
  std::memset(hp, 0, sizeof(*hp));
  int plus[kMaxPairs];
  lattice_pairs(L->kind, plus);
  const int np = (L->Q - 1) / 2;
  int ne = 0, no = 0;
  for (int r = 0; r < L->nhigh; ++r) {
    const double* h = L->Hh + size_t(r) * L->Q;
    const double a = -(high_rate(m, L->h_order[r]) - m->s_high) / L->Nh[r];
    if ((L->h_order[r] & 1) == 0) {
      hp->he[ne][0] = CT(h[0]);
      for (int q = 0; q < np; ++q) hp->he[ne][q + 1] = CT(h[plus[q]]);
      hp->ae[ne++] = CT(a);
    } else {
      for (int q = 0; q < np; ++q) hp->ho[no][q] = CT(h[plus[q]]);
      hp->ao[no++] = CT(a);
    }
  }
}

void make_tc_params(const lbm_model* m, TcParams* tp) {
  const lbm_lattice* L = m->lat;
  std::memset(tp, 0, sizeof(*tp));
  for (int i = 0; i < L->Q; ++i)
    for (int r = 0; r < L->R; ++r) {
      const Mono mk = L->d == 2 ? kMono2[r] : kMono3[r];
      int v = 1;
      for (int q = 0; q < mk.a; ++q) v *= L->e[i * 3 + 0];
      for (int q = 0; q < mk.b; ++q) v *= L->e[i * 3 + 1];
      for (int q = 0; q < mk.c; ++q) v *= L->e[i * 3 + 2];
      tp->mono[i][r] = int8_t(v);
    }
  if (has_high_rates(m))
    for (int r = 0; r < L->nhigh; ++r) {
      for (int i = 0; i < L->Q; ++i) tp->hrow[r][i] = float(L->Hh[size_t(r) * L->Q + i]);
      tp->ah[r] = float(-(high_rate(m, L->h_order[r]) - m->s_high) / L->Nh[r]);
    }
  tp->ntiles = (m->ncells + 127) / 128;
  tp->status = m->status;
  tp->no_issue = m->tc_no_issue ? 1 : 0;
  tp->wait_limit = m->tc_no_issue ? (1u << 10) : (1u << 22);
}

void make_tc32_params(const lbm_model* m, Tc32Params* tp) {
  const lbm_lattice* L = m->lat;
  const int Q = L->Q;
  std::memset(tp, 0, sizeof(*tp));
  // G_ij = sum_r a_r H_r(c_i) H_r(c_j), a_r = -(s_r - s_high) / N_r, in FP64
  std::vector<double> G(size_t(Q) * Q, 0.0);
  if (has_high_rates(m))
    for (int r = 0; r < L->nhigh; ++r) {
      const double a = -(high_rate(m, L->h_order[r]) - m->s_high) / L->Nh[r];
      if (a == 0.0) continue;
      const double* h = L->Hh + size_t(r) * Q;
      for (int i = 0; i < Q; ++i)
        for (int j = 0; j < Q; ++j) G[size_t(i) * Q + j] += a * h[i] * h[j];
    }
  // row i scaled by the power of two 2^-k_i that brings its max |G_ij| into [1, 2) (the high/low
  // split then keeps about 22 bits of each row's large entries), undone in wg_i = 2^k_i w_i
  for (int i = 0; i < Q; ++i) {
    double gmax = 0.0;
    for (int j = 0; j < Q; ++j) gmax = std::max(gmax, std::fabs(G[size_t(i) * Q + j]));
    int e = 1;
    if (gmax > 0.0) std::frexp(gmax, &e);  // gmax = m 2^e, m in [0.5, 1)
    const int k = e - 1;
    for (int j = 0; j < Q; ++j) tp->g[i][j] = float(std::ldexp(G[size_t(i) * Q + j], -k));
    tp->wg[i] = float(std::ldexp(L->w[i], k));
  }
  tp->ntiles = (m->ncells + 127) / 128;
  tp->status = m->status;
  tp->no_issue = m->tc_no_issue ? 1 : 0;
  tp->wait_limit = m->tc_no_issue ? (1u << 10) : (1u << 22);
}

// Persistent grid of the tensor-core kernel: ctas_per_sm CTAs per SM (their 128 TMEM columns
// each fit the SM's 512; __launch_bounds__ caps the registers so that they are resident) times
// the SM count, capped by the tile count. The operand tiles are dynamic shared memory.
int tc_grid(const lbm_model* m, int ntiles, const void* kernel, int ctas_per_sm, size_t smem_bytes) {
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, m->device);
  if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem_bytes)) != cudaSuccess ||
      cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                           int(cudaSharedmemCarveoutMaxShared)) != cudaSuccess)
    cudaGetLastError();
  const int g = (sms > 0 ? sms : 1) * ctas_per_sm;
  return ntiles < g ? ntiles : g;
}

template void make_high_params<float>(const lbm_model*, HighParams<float>*);
template void make_high_params<double>(const lbm_model*, HighParams<double>*);

namespace {

constexpr size_t kAlign = 256;
size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

struct Layout {
  size_t f_bytes, phi_off, force_off, part_off, sums_off, status_off, total;
};

Layout layout(const lbm_lattice* L, int eq, const int64_t* n, int store) {
  int64_t ncells = 1, nmax = 1;
  for (int a = 0; a < L->d; ++a) {
    ncells *= n[a];
    nmax = n[a] > nmax ? n[a] : nmax;
  }
  const size_t cbytes = store == LBM_F64 ? 8 : 4;
  Layout lo;
  lo.f_bytes = align_up(size_t(L->Q) * size_t(ncells) * dtype_bytes(store));
  lo.phi_off = 2 * lo.f_bytes;
  // NCDE: phi of the previous step and psi of the cross diffusion; single-speed NSE: two density
  // fields for the M2G gradient
  const size_t fields = eq == LBM_NCDE || lattice_single(L->kind) ? 2 : 0;
  const size_t phi_bytes = fields * align_up(size_t(ncells) * cbytes);
  lo.force_off = lo.phi_off + phi_bytes;
  lo.part_off = lo.force_off + align_up(size_t(nmax) * cbytes);
  lo.sums_off = lo.part_off + align_up(size_t(kRedBlocks) * 4 * sizeof(double));
  lo.status_off = lo.sums_off + align_up(4 * sizeof(double));
  lo.total = lo.status_off + align_up(sizeof(int));
  return lo;
}

lbm_status check_grid(const lbm_lattice* L, const int64_t* n) {
  if (!n) return set_error(LBM_ERR_ARG, "grid size pointer is NULL");
  int64_t ncells = 1;
  for (int a = 0; a < L->d; ++a) {
    if (n[a] < L->rmax)
      return set_error(LBM_ERR_ARG, "every grid extent must be at least " + std::to_string(L->rmax) +
                                        " (the largest velocity component)");
    if (n[a] > (int64_t(1) << 30)) return set_error(LBM_ERR_ARG, "grid extent too large");
    ncells *= n[a];
    if (ncells > kMaxCells)
      return set_error(LBM_ERR_ARG, "cell count must be at most 2^31 - 2^21 (" + std::to_string(kMaxCells) + ")");
  }
  return LBM_OK;
}

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

lbm_status upload_force(lbm_model* m) {
  if (m->eq != LBM_NSE || m->force_A == 0.0) return LBM_OK;
  const int nb = int(m->n[m->force_b]);
  const double Lb = double(nb);  // L_b / c_b in cells: x_b / L_b = i_b / n_b
  std::vector<double> tab(nb);
  const double kTwoPi = 6.283185307179586476925286766559;
  for (int i = 0; i < nb; ++i) tab[i] = m->force_A * std::sin(kTwoPi * m->force_k * i / Lb + m->force_phase);
  cudaError_t err;
  if (m->store == LBM_F64) {
    err = cudaMemcpyAsync(m->force_tab, tab.data(), nb * sizeof(double), cudaMemcpyHostToDevice, m->stream);
  } else {
    std::vector<float> tf(tab.begin(), tab.end());
    err = cudaMemcpyAsync(m->force_tab, tf.data(), nb * sizeof(float), cudaMemcpyHostToDevice, m->stream);
    if (err == cudaSuccess) err = cudaStreamSynchronize(m->stream);  // tf is about to go out of scope
  }
  if (err == cudaSuccess) err = cudaStreamSynchronize(m->stream);
  return err == cudaSuccess ? LBM_OK : cuda_error(err, "force upload");
}

// Read and clear the model's device status word (the stream must allow a synchronisation).
lbm_status take_status(lbm_model* m) {
  int s = 0;
  cudaError_t err = cudaMemcpyAsync(&s, m->status, sizeof(int), cudaMemcpyDeviceToHost, m->stream);
  if (err == cudaSuccess) err = cudaStreamSynchronize(m->stream);
  if (err != cudaSuccess) return cuda_error(err, "status word");
  if (s == 0) return LBM_OK;
  err = cudaMemsetAsync(m->status, 0, sizeof(int), m->stream);
  if (err == cudaSuccess) err = cudaStreamSynchronize(m->stream);
  if (err != cudaSuccess) return cuda_error(err, "status word");
  return set_error(LBM_ERR_TIMEOUT,
                   "a step gave up waiting on the device (tensor-core products or row copies); the populations "
                   "are invalid");
}

template <class F>
lbm_status dispatch_kind(int kind, F&& f) {
  switch (kind) {
    case LBM_RD2Q13: return f(std::integral_constant<int, LBM_RD2Q13>{});
    case LBM_RD2Q17: return f(std::integral_constant<int, LBM_RD2Q17>{});
    case LBM_RD2Q21: return f(std::integral_constant<int, LBM_RD2Q21>{});
    case LBM_RD2Q25: return f(std::integral_constant<int, LBM_RD2Q25>{});
    case LBM_RD3Q33: return f(std::integral_constant<int, LBM_RD3Q33>{});
    case LBM_RD3Q45: return f(std::integral_constant<int, LBM_RD3Q45>{});
    case LBM_RD3Q53: return f(std::integral_constant<int, LBM_RD3Q53>{});
    case LBM_RD2Q9: return f(std::integral_constant<int, LBM_RD2Q9>{});
    case LBM_RD3Q27: return f(std::integral_constant<int, LBM_RD3Q27>{});
  }
  return set_error(LBM_ERR_ARG, "unknown lattice kind");
}

// Run fn with a device staging buffer of `bytes` when the user buffer is in host memory.
template <class F>
lbm_status with_staging(lbm_model* m, size_t bytes, bool need, F&& fn) {
  if (!need) return fn(nullptr);
  void* tmp = nullptr;
  cudaError_t err = cudaMallocAsync(&tmp, bytes, m->stream);
  if (err != cudaSuccess) return cuda_error(err, "staging allocation");
  lbm_status st = fn(tmp);
  err = cudaFreeAsync(tmp, m->stream);
  if (st == LBM_OK && err != cudaSuccess) st = cuda_error(err, "staging free");
  return st;
}

}  // namespace
}  // namespace lbm

using namespace lbm;

extern "C" {

int lbm_abi_version(void) { return LBM_ABI_VERSION; }

const char* lbm_last_error(void) { return g_last_error.c_str(); }

lbm_status lbm_lattice_create(lbm_kind kind, const double* c, const double* cs2, const double* free_w,
                              int n_free, lbm_lattice** out) {
  try {
    if (!out || !c || !cs2) return set_error(LBM_ERR_ARG, "NULL argument");
    *out = nullptr;
    if (int(kind) < LBM_RD2Q13 || int(kind) > LBM_RD3Q27) return set_error(LBM_ERR_ARG, "unknown lattice kind");
    static const int kFree[9] = {0, 1, 3, 4, 0, 0, 1, 0, 0};
    if (n_free != kFree[kind])
      return set_error(LBM_ERR_ARG, "lattice kind " + std::to_string(int(kind)) + " takes " +
                                        std::to_string(kFree[kind]) + " free weights");
    if (n_free > 0 && !free_w) return set_error(LBM_ERR_ARG, "free_w is NULL");
    auto* L = new (std::nothrow) lbm_lattice;
    if (!L) return set_error(LBM_ERR_OOM, "host allocation failed");
    std::memset(L, 0, sizeof(*L));
    L->kind = kind;
    L->d = lattice_dims(kind);
    L->Q = lattice_q(kind);
    L->R = lattice_r(kind);
    L->rmax = lattice_rmax(kind);
    for (int a = 0; a < L->d; ++a) {
      if (!(c[a] > 0.0) || !(cs2[a] > 0.0) || !std::isfinite(c[a]) || !std::isfinite(cs2[a])) {
        delete L;
        return set_error(LBM_ERR_ARG, "c and cs2 must be positive and finite");
      }
      L->c[a] = c[a];
      L->cs2[a] = cs2[a];
    }
    for (int k = 0; k < n_free; ++k) L->free_w[k] = free_w[k];
    for (int j = 0; j < L->Q; ++j) {
      const Vel v = lattice_e(kind, j);
      L->e[j * 3 + 0] = int8_t(v.x);
      L->e[j * 3 + 1] = int8_t(v.y);
      L->e[j * 3 + 2] = int8_t(v.z);
    }
    cudaGetDevice(&L->device);
    lbm_status st = setup_lattice_fp64(L);
    if (st != LBM_OK) {
      delete L;
      return st;
    }
    *out = L;
    return LBM_OK;
  } catch (...) {
    return set_error(LBM_ERR_ARG, "unexpected exception in lbm_lattice_create");
  }
}

lbm_status lbm_lattice_query(const lbm_lattice* L, int* d, int* Q, int* R, int8_t* e, double* w, double* H,
                             double* N, double* T) {
  if (!L) return set_error(LBM_ERR_ARG, "NULL lattice");
  if (d) *d = L->d;
  if (Q) *Q = L->Q;
  if (R) *R = L->R;
  if (e)
    for (int j = 0; j < L->Q; ++j)
      for (int a = 0; a < L->d; ++a) e[j * L->d + a] = L->e[j * 3 + a];
  if (w) std::memcpy(w, L->w, sizeof(double) * L->Q);
  if (H) std::memcpy(H, L->H, sizeof(double) * L->Q * L->R);
  if (N) std::memcpy(N, L->N, sizeof(double) * L->R);
  if (T) std::memcpy(T, L->T, sizeof(double) * L->R * L->R);
  return LBM_OK;
}

lbm_status lbm_lattice_query_high(const lbm_lattice* L, int* n_high, int* orders, double* H, double* N) {
  if (!L) return set_error(LBM_ERR_ARG, "NULL lattice");
  if (L->high_status == 1)
    return set_error(LBM_ERR_LATTICE_INFEASIBLE, "the graded monomials do not complete the Hermite matrix");
  if (L->high_status == 2)
    return set_error(LBM_ERR_LATTICE_INFEASIBLE, "a higher-order row has zero W-norm (zero weights)");
  if (n_high) *n_high = L->nhigh;
  if (orders) std::memcpy(orders, L->h_order, sizeof(int) * L->nhigh);
  if (H) std::memcpy(H, L->Hh, sizeof(double) * L->nhigh * L->Q);
  if (N) std::memcpy(N, L->Nh, sizeof(double) * L->nhigh);
  return LBM_OK;
}

lbm_status lbm_lattice_destroy(lbm_lattice* L) {
  delete L;
  return LBM_OK;
}

lbm_status lbm_model_workspace_bytes(const lbm_lattice* L, lbm_eq eq, const int64_t* n, lbm_dtype store,
                                     size_t* bytes) {
  if (!L || !bytes) return set_error(LBM_ERR_ARG, "NULL argument");
  if (int(store) < LBM_F64 || int(store) > LBM_F16_DEV) return set_error(LBM_ERR_ARG, "unknown storage dtype");
  if (eq != LBM_NSE && eq != LBM_NCDE) return set_error(LBM_ERR_ARG, "unknown equation");
  lbm_status st = check_grid(L, n);
  if (st != LBM_OK) return st;
  *bytes = layout(L, eq, n, store).total;
  return LBM_OK;
}

lbm_status lbm_model_create(const lbm_lattice* L, lbm_eq eq, const int64_t* n, lbm_dtype store, lbm_dtype compute,
                            void* stream, void* workspace, size_t workspace_bytes, lbm_model** out) {
  try {
    if (!L || !out) return set_error(LBM_ERR_ARG, "NULL argument");
    *out = nullptr;
    if (eq != LBM_NSE && eq != LBM_NCDE) return set_error(LBM_ERR_ARG, "unknown equation");
    const bool ok_types = (store == LBM_F64 && compute == LBM_F64) || (store == LBM_F32 && compute == LBM_F32) ||
                          ((store == LBM_BF16_DEV || store == LBM_F16_DEV) && compute == LBM_F32);
    if (!ok_types)
      return set_error(LBM_ERR_ARG, "supported (store, compute): (F64,F64), (F32,F32), (BF16_DEV,F32), (F16_DEV,F32)");
    lbm_status st = check_grid(L, n);
    if (st != LBM_OK) return st;
    const Layout lo = layout(L, eq, n, store);
    if (workspace && (workspace_bytes < lo.total || (reinterpret_cast<uintptr_t>(workspace) % kAlign) != 0))
      return set_error(LBM_ERR_OOM, "workspace must hold " + std::to_string(lo.total) + " bytes, 256-byte aligned");
    DeviceGuard guard(L->device);
    auto* m = new (std::nothrow) lbm_model;
    if (!m) return set_error(LBM_ERR_OOM, "host allocation failed");
    std::memset(m, 0, sizeof(*m));
    m->lat = L;
    m->eq = eq;
    m->ncells = 1;
    for (int a = 0; a < 3; ++a) m->n[a] = a < L->d ? n[a] : 1;
    for (int a = 0; a < L->d; ++a) m->ncells *= int(n[a]);
    m->store = store;
    m->compute = compute;
    m->stream = static_cast<cudaStream_t>(stream);
    m->device = L->device;
    if (workspace) {
      m->ws = workspace;
      m->owns_ws = false;
    } else {
      cudaError_t err = cudaMalloc(&m->ws, lo.total);
      if (err != cudaSuccess) {
        delete m;
        return cuda_error(err, "model allocation");
      }
      m->owns_ws = true;
    }
    m->ws_bytes = lo.total;
    char* base = static_cast<char*>(m->ws);
    m->f[0] = base;
    m->f[1] = base + lo.f_bytes;
    m->phi_prev = eq == LBM_NCDE ? base + lo.phi_off : nullptr;
    const size_t field_bytes = align_up(size_t(m->ncells) * (store == LBM_F64 ? 8 : 4));
    if (eq == LBM_NCDE) m->psi = base + lo.phi_off + field_bytes;
    if (eq == LBM_NSE && lattice_single(L->kind)) {
      m->rho_hist[0] = base + lo.phi_off;
      m->rho_hist[1] = base + lo.phi_off + field_bytes;
    }
    m->force_tab = base + lo.force_off;
    m->partials = reinterpret_cast<double*>(base + lo.part_off);
    m->sums = reinterpret_cast<double*>(base + lo.sums_off);
    m->status = reinterpret_cast<int*>(base + lo.status_off);
    cudaError_t err = cudaMemsetAsync(m->ws, 0, lo.total, m->stream);
    if (err != cudaSuccess) {
      if (m->owns_ws) cudaFree(m->ws);
      delete m;
      return cuda_error(err, "workspace clear");
    }
    for (int r = 0; r < lbm::kMaxR; ++r) m->s[r] = 1.0;
    m->s_high = 1.0;
    m->cs2_eq = L->cs2[0];
    m->rho_ref = eq == LBM_NSE ? 1.0 : 0.0;
    m->force_b = -1;
    m->tc_auto = store != LBM_F64;
    *out = m;
    return LBM_OK;
  } catch (...) {
    return set_error(LBM_ERR_ARG, "unexpected exception in lbm_model_create");
  }
}

lbm_status lbm_model_set_relaxation(lbm_model* m, const double* s, double s_high) {
  if (!m || !s) return set_error(LBM_ERR_ARG, "NULL argument");
  for (int r = 0; r < m->lat->R; ++r)
    if (!(s[r] > 0.0 && s[r] <= 2.0)) return set_error(LBM_ERR_ARG, "rates must lie in (0, 2]");
  if (!(s_high > 0.0 && s_high <= 2.0)) return set_error(LBM_ERR_ARG, "rates must lie in (0, 2]");
  for (int r = 0; r < m->lat->R; ++r) m->s[r] = s[r];
  m->s_high = s_high;
  batch_mark_dirty(m->batch);
  return LBM_OK;
}

lbm_status lbm_model_set_bulk(lbm_model* m, double s_bulk) {
  if (!m) return set_error(LBM_ERR_ARG, "NULL model");
  if (m->eq != LBM_NSE) return set_error(LBM_ERR_ARG, "the bulk rate applies to the NSE model");
  if (!(s_bulk <= 2.0) || !std::isfinite(s_bulk)) return set_error(LBM_ERR_ARG, "bulk rate must be <= 2");
  m->s_bulk = s_bulk;
  batch_mark_dirty(m->batch);
  return LBM_OK;
}

lbm_status lbm_model_set_high_rates(lbm_model* m, const double* s_order, int n_orders) {
  if (!m) return set_error(LBM_ERR_ARG, "NULL model");
  if (n_orders < 0 || n_orders > kMaxOrder - 3 || (n_orders > 0 && !s_order))
    return set_error(LBM_ERR_ARG, "n_orders must lie in [0, " + std::to_string(kMaxOrder - 3) + "]");
  for (int k = 0; k < n_orders; ++k)
    if (!(s_order[k] > 0.0 && s_order[k] <= 2.0)) return set_error(LBM_ERR_ARG, "rates must lie in (0, 2]");
  double next[kMaxOrder + 1] = {};
  for (int k = 0; k < n_orders; ++k) next[4 + k] = s_order[k];
  bool differ = false;
  for (int r = 0; r < m->lat->nhigh; ++r) {
    const double s = next[m->lat->h_order[r]];
    differ = differ || (s > 0.0 && s != m->s_high);
  }
  if (differ && m->lat->high_status != 0)
    return set_error(LBM_ERR_LATTICE_INFEASIBLE, m->lat->high_status == 1
                                                     ? "the graded monomials do not complete the Hermite matrix"
                                                     : "a higher-order row has zero W-norm (zero weights)");
  for (int k = 0; k <= kMaxOrder; ++k) m->s_order[k] = next[k];
  batch_mark_dirty(m->batch);
  return LBM_OK;
}

lbm_status lbm_model_set_tensor_cores(lbm_model* m, int enable) {
  if (!m) return set_error(LBM_ERR_ARG, "NULL model");
  if (enable < 0 || enable > 2) return set_error(LBM_ERR_ARG, "enable must be 0, 1 or 2");
  if (enable && m->store == LBM_F64)
    return set_error(LBM_ERR_ARG, "the tensor-core collision needs FP32 or 16-bit deviation storage");
  m->tensor_cores = enable != 0;
  m->tc_no_issue = enable == 2;
  m->tc_auto = false;
  return LBM_OK;
}

lbm_status lbm_model_set_gather(lbm_model* m, lbm_gather mode) {
  if (!m) return set_error(LBM_ERR_ARG, "NULL model");
  const bool no_copy = int(mode) == 3;  // test hook: rows without copies (every wait runs out)
  if (mode != LBM_GATHER_AUTO && mode != LBM_GATHER_THREADS && mode != LBM_GATHER_ROWS && !no_copy)
    return set_error(LBM_ERR_ARG, "gather must be LBM_GATHER_AUTO, _THREADS or _ROWS");
  if (no_copy) mode = LBM_GATHER_ROWS;
  if (mode == LBM_GATHER_ROWS) {
    RowPlan plan;
    DeviceGuard guard(m->device);
    bool ok = false;
    lbm_status st = dispatch_kind(m->lat->kind, [&](auto kind) -> lbm_status {
      ok = RowLaunch<decltype(kind)::value>::plan(m, &plan);
      return LBM_OK;
    });
    if (st != LBM_OK) return st;
    if (!ok)
      return set_error(LBM_ERR_ARG, "the row-staged gather needs 16-bit deviation storage and n_x a multiple of 8, "
                                    "at most 256 cells");
  }
  m->gather = int(mode);
  m->row_no_copy = no_copy;
  return LBM_OK;
}

lbm_status lbm_model_set_eos(lbm_model* m, double cs2_eq) {
  if (!m) return set_error(LBM_ERR_ARG, "NULL model");
  if (!(cs2_eq > 0.0) || !std::isfinite(cs2_eq)) return set_error(LBM_ERR_ARG, "cs2_eq must be positive");
  m->cs2_eq = cs2_eq;
  batch_mark_dirty(m->batch);
  return LBM_OK;
}

lbm_status lbm_model_set_force(lbm_model* m, int axis_a, int axis_b, double A, int k, double phase) {
  if (!m) return set_error(LBM_ERR_ARG, "NULL model");
  if (m->eq != LBM_NSE) return set_error(LBM_ERR_ARG, "body force applies to the NSE model");
  const int d = m->lat->d;
  if (axis_a < 0 || axis_a >= d || axis_b < 0 || axis_b >= d) return set_error(LBM_ERR_ARG, "axis out of range");
  if (!std::isfinite(A) || !std::isfinite(phase)) return set_error(LBM_ERR_ARG, "non-finite force parameter");
  DeviceGuard guard(m->device);
  m->force_a = axis_a;
  m->force_b = axis_b;
  m->force_A = A;
  m->force_k = k;
  m->force_phase = phase;
  batch_mark_dirty(m->batch);
  return upload_force(m);
}

lbm_status lbm_model_set_ncde(lbm_model* m, const double* u_const, double nonlin) {
  if (!m || !u_const) return set_error(LBM_ERR_ARG, "NULL argument");
  if (m->eq != LBM_NCDE) return set_error(LBM_ERR_ARG, "convection velocity applies to the NCDE model");
  for (int a = 0; a < 3; ++a) m->u_const[a] = a < m->lat->d ? u_const[a] : 0.0;
  m->nonlin = nonlin;
  batch_mark_dirty(m->batch);
  return LBM_OK;
}

lbm_status lbm_model_set_ncde_variant(lbm_model* m, lbm_ncde_variant variant, double a1) {
  if (!m) return set_error(LBM_ERR_ARG, "NULL model");
  if (m->eq != LBM_NCDE) return set_error(LBM_ERR_ARG, "the variants apply to the NCDE model");
  if (int(variant) < LBM_NCDE_MOMENT || int(variant) > LBM_NCDE_CDE) return set_error(LBM_ERR_ARG, "unknown NCDE variant");
  if (!std::isfinite(a1)) return set_error(LBM_ERR_ARG, "a1 must be finite");
  if (variant == LBM_NCDE_CDE && a1 != 0.0) return set_error(LBM_ERR_ARG, "the CDE variant has no mixed-derivative term");
  if (variant == LBM_NCDE_CDE && m->a2 != 0.0) return set_error(LBM_ERR_ARG, "the CDE variant has no cross-diffusion term");
  m->ncde_variant = variant;
  m->a1 = a1;
  batch_mark_dirty(m->batch);
  return LBM_OK;
}

lbm_status lbm_model_set_ncde_cross_diffusion(lbm_model* m, double a2, const double* psi, int on_device) {
  if (!m) return set_error(LBM_ERR_ARG, "NULL model");
  if (m->eq != LBM_NCDE) return set_error(LBM_ERR_ARG, "the cross-diffusion term applies to the NCDE model");
  if (!std::isfinite(a2)) return set_error(LBM_ERR_ARG, "a2 must be finite");
  if (a2 == 0.0) {
    m->a2 = 0.0;
    batch_mark_dirty(m->batch);
    return LBM_OK;
  }
  if (!psi) return set_error(LBM_ERR_ARG, "psi is NULL");
  if (m->ncde_variant == LBM_NCDE_CDE) return set_error(LBM_ERR_ARG, "the CDE variant has no cross-diffusion term");
  DeviceGuard guard(m->device);
  const size_t bytes = size_t(m->ncells) * sizeof(double);
  lbm_status st = with_staging(m, bytes, !on_device, [&](void* tmp) -> lbm_status {
    const double* src = psi;
    if (tmp) {
      cudaError_t err = cudaMemcpyAsync(tmp, psi, bytes, cudaMemcpyHostToDevice, m->stream);
      if (err != cudaSuccess) return cuda_error(err, "psi upload");
      src = static_cast<const double*>(tmp);
    }
    return launch_to_compute(m, src, m->psi);
  });
  if (st != LBM_OK) return st;
  if (!on_device) {
    cudaError_t err = cudaStreamSynchronize(m->stream);
    if (err != cudaSuccess) return cuda_error(err, "psi upload");
  }
  m->a2 = a2;
  batch_mark_dirty(m->batch);
  return LBM_OK;
}

lbm_status lbm_model_set_m2g_anisotropy(lbm_model* m, int enable) {
  if (!m) return set_error(LBM_ERR_ARG, "NULL model");
  if (m->eq != LBM_NSE || !lattice_single(m->lat->kind))
    return set_error(LBM_ERR_ARG, "the delta4 term of M2G applies to the NSE on rD2Q9 / rD3Q27");
  if (enable != 0 && enable != 1) return set_error(LBM_ERR_ARG, "enable must be 0 or 1");
  DeviceGuard guard(m->device);
  if (enable && !m->m2g_aniso) {
    // the previous-step density starts as the density of the current state
    lbm_status st = launch_density_history(m);
    if (st != LBM_OK) return st;
  }
  m->m2g_aniso = enable != 0;
  batch_mark_dirty(m->batch);
  return LBM_OK;
}

lbm_status lbm_model_init_fields(lbm_model* m, const double* rho_or_phi, const double* u, int on_device) {
  if (!m || !rho_or_phi) return set_error(LBM_ERR_ARG, "NULL argument");
  if (m->eq == LBM_NSE && !u) return set_error(LBM_ERR_ARG, "the NSE model needs a velocity field");
  DeviceGuard guard(m->device);
  const size_t N = size_t(m->ncells);
  const int d = m->lat->d;
  const size_t nval = m->eq == LBM_NSE ? (1 + d) * N : N;
  lbm_status st = with_staging(m, nval * sizeof(double), !on_device, [&](void* tmp) -> lbm_status {
    const double* r = rho_or_phi;
    const double* uu = u;
    if (tmp) {
      double* t = static_cast<double*>(tmp);
      cudaError_t err = cudaMemcpyAsync(t, rho_or_phi, N * sizeof(double), cudaMemcpyHostToDevice, m->stream);
      if (err == cudaSuccess && m->eq == LBM_NSE)
        err = cudaMemcpyAsync(t + N, u, d * N * sizeof(double), cudaMemcpyHostToDevice, m->stream);
      if (err != cudaSuccess) return cuda_error(err, "field upload");
      r = t;
      uu = m->eq == LBM_NSE ? t + N : nullptr;
    }
    return dispatch_kind(m->lat->kind, [&](auto kc) { return Launch<decltype(kc)::value>::init(m, r, uu); });
  });
  if (st != LBM_OK) return st;
  if (!on_device) {
    cudaError_t err = cudaStreamSynchronize(m->stream);
    if (err != cudaSuccess) return cuda_error(err, "field upload");
  }
  m->steps = 0;
  return LBM_OK;
}

lbm_status lbm_model_set_populations(lbm_model* m, const double* f, int on_device) {
  if (!m || !f) return set_error(LBM_ERR_ARG, "NULL argument");
  DeviceGuard guard(m->device);
  const size_t bytes = size_t(m->lat->Q) * m->ncells * sizeof(double);
  lbm_status st = with_staging(m, bytes, !on_device, [&](void* tmp) -> lbm_status {
    const double* src = f;
    if (tmp) {
      cudaError_t err = cudaMemcpyAsync(tmp, f, bytes, cudaMemcpyHostToDevice, m->stream);
      if (err != cudaSuccess) return cuda_error(err, "population upload");
      src = static_cast<const double*>(tmp);
    }
    lbm_status s2 = launch_scatter(m, src);
    if (s2 == LBM_OK && m->eq == LBM_NCDE) s2 = launch_phi_from_populations(m);
    if (s2 == LBM_OK && m->rho_hist[0]) s2 = launch_density_history(m);
    return s2;
  });
  if (st != LBM_OK) return st;
  if (!on_device) {
    cudaError_t err = cudaStreamSynchronize(m->stream);
    if (err != cudaSuccess) return cuda_error(err, "population upload");
  }
  m->steps = 0;
  return LBM_OK;
}

lbm_status lbm_model_get_populations(lbm_model* m, double* f, int on_device) {
  if (!m || !f) return set_error(LBM_ERR_ARG, "NULL argument");
  DeviceGuard guard(m->device);
  const size_t bytes = size_t(m->lat->Q) * m->ncells * sizeof(double);
  lbm_status st = with_staging(m, bytes, !on_device, [&](void* tmp) -> lbm_status {
    double* dst = tmp ? static_cast<double*>(tmp) : f;
    lbm_status s2 = launch_gather(m, dst);
    if (s2 != LBM_OK) return s2;
    if (tmp) {
      cudaError_t err = cudaMemcpyAsync(f, tmp, bytes, cudaMemcpyDeviceToHost, m->stream);
      if (err != cudaSuccess) return cuda_error(err, "population download");
    }
    return LBM_OK;
  });
  if (st != LBM_OK) return st;
  if (!on_device) {
    cudaError_t err = cudaStreamSynchronize(m->stream);
    if (err != cudaSuccess) return cuda_error(err, "population download");
    return take_status(m);
  }
  return LBM_OK;
}

lbm_status lbm_model_step(lbm_model* m, int64_t nsteps) {
  if (!m) return set_error(LBM_ERR_ARG, "NULL model");
  if (m->batch) return set_error(LBM_ERR_ARG, "the model is in a batch: advance it with lbm_batch_step");
  if (nsteps < 0) return set_error(LBM_ERR_ARG, "nsteps must be non-negative");
  DeviceGuard guard(m->device);
  return dispatch_kind(m->lat->kind, [&](auto kc) { return Launch<decltype(kc)::value>::step(m, nsteps, true); });
}

lbm_status lbm_model_stream_only(lbm_model* m, int64_t nsteps) {
  if (!m) return set_error(LBM_ERR_ARG, "NULL model");
  if (m->batch) return set_error(LBM_ERR_ARG, "the model is in a batch: advance it with lbm_batch_step");
  if (nsteps < 0) return set_error(LBM_ERR_ARG, "nsteps must be non-negative");
  DeviceGuard guard(m->device);
  return dispatch_kind(m->lat->kind, [&](auto kc) { return Launch<decltype(kc)::value>::step(m, nsteps, false); });
}

lbm_status lbm_model_read_fields(lbm_model* m, double* rho_or_phi, double* u, int on_device) {
  if (!m || !rho_or_phi) return set_error(LBM_ERR_ARG, "NULL argument");
  DeviceGuard guard(m->device);
  const size_t N = size_t(m->ncells);
  const int d = m->lat->d;
  const bool want_u = m->eq == LBM_NSE && u != nullptr;
  const size_t nval = want_u ? (1 + d) * N : N;
  lbm_status st = with_staging(m, nval * sizeof(double), !on_device, [&](void* tmp) -> lbm_status {
    double* r = tmp ? static_cast<double*>(tmp) : rho_or_phi;
    double* uu = want_u ? (tmp ? static_cast<double*>(tmp) + N : u) : nullptr;
    lbm_status s2 = launch_fields(m, r, uu);
    if (s2 != LBM_OK) return s2;
    if (tmp) {
      cudaError_t err = cudaMemcpyAsync(rho_or_phi, r, N * sizeof(double), cudaMemcpyDeviceToHost, m->stream);
      if (err == cudaSuccess && want_u)
        err = cudaMemcpyAsync(u, uu, d * N * sizeof(double), cudaMemcpyDeviceToHost, m->stream);
      if (err != cudaSuccess) return cuda_error(err, "field download");
    }
    return LBM_OK;
  });
  if (st != LBM_OK) return st;
  if (!on_device) {
    cudaError_t err = cudaStreamSynchronize(m->stream);
    if (err != cudaSuccess) return cuda_error(err, "field download");
    return take_status(m);
  }
  return LBM_OK;
}

lbm_status lbm_model_conserved_sums(lbm_model* m, double* out_host) {
  if (!m || !out_host) return set_error(LBM_ERR_ARG, "NULL argument");
  DeviceGuard guard(m->device);
  lbm_status st = launch_sums(m);
  if (st != LBM_OK) return st;
  double s[4];
  cudaError_t err = cudaMemcpyAsync(s, m->sums, sizeof(s), cudaMemcpyDeviceToHost, m->stream);
  if (err == cudaSuccess) err = cudaStreamSynchronize(m->stream);
  if (err != cudaSuccess) return cuda_error(err, "conservation sums");
  st = take_status(m);
  if (st != LBM_OK) return st;
  const int d = m->lat->d;
  bool finite = true;
  for (int q = 0; q <= d; ++q) {
    out_host[q] = s[q];
    finite = finite && std::isfinite(s[q]);
  }
  if (!finite) return set_error(LBM_ERR_NONFINITE, "a conservation sum is not finite");
  return LBM_OK;
}

lbm_status lbm_model_counters(const lbm_model* m, int64_t* steps, int64_t* launches) {
  if (!m) return set_error(LBM_ERR_ARG, "NULL model");
  if (steps) *steps = m->steps;
  if (launches) *launches = m->launches;
  return LBM_OK;
}

lbm_status lbm_model_synchronize(lbm_model* m) {
  if (!m) return set_error(LBM_ERR_ARG, "NULL model");
  DeviceGuard guard(m->device);
  cudaError_t err = cudaStreamSynchronize(m->stream);
  if (err != cudaSuccess) return cuda_error(err, "synchronize");
  return take_status(m);
}

lbm_status lbm_model_destroy(lbm_model* m) {
  if (!m) return LBM_OK;
  if (m->batch) lbm_batch_remove(m->batch, m);
  DeviceGuard guard(m->device);
  cudaStreamSynchronize(m->stream);
  if (m->owns_ws) cudaFree(m->ws);
  delete m;
  return LBM_OK;
}

}  // extern "C"
