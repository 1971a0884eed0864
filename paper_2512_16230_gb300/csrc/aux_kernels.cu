// Lattice-agnostic kernels around the time step: population gather/scatter for I/O, the
// macroscopic-field readout (Eq. (2-4-2) / (2-4-1)) and the FP64 conservation sums.
// None of these is on the per-step path; the velocity table is read from the kernel
// parameters with a runtime index.
#include "lbm_internal.cuh"

namespace lbm {

namespace {

// Periodic wrap of a coordinate displaced by at most one grid extent (every extent is at least
// the largest velocity component, checked at model creation).
__device__ __forceinline__ int wrap(int v, int n) {
  v += v < 0 ? n : 0;
  return v >= n ? v - n : v;
}

__device__ __forceinline__ void coords(const GenParams& p, int cell, int& x, int& y, int& z) {
  const int nx = p.n[0], ny = p.n[1];
  const int t = cell / nx;
  x = cell - t * nx;
  if (p.d == 2) {
    y = t;
    z = 0;
  } else {
    z = t / ny;
    y = t - z * ny;
  }
}

// cell index of (x + s e_i) for s = +1 / -1
__device__ __forceinline__ int shifted(const GenParams& p, int x, int y, int z, int i, int s) {
  const int xs = wrap(x + s * p.e[i][0], p.n[0]);
  const int ys = wrap(y + s * p.e[i][1], p.n[1]);
  const int zs = p.d == 3 ? wrap(z + s * p.e[i][2], p.n[2]) : 0;
  return (zs * p.n[1] + ys) * p.n[0] + xs;
}

// f-bar_i(x) = A_i(x - e_i): the pre-collision populations from the stored array.
template <class ST, class CT>
__global__ void k_gather(const GenParams p, const GenTables<CT> t, const ST* __restrict__ A,
                         double* __restrict__ out) {
  const int cell = blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= p.ncells) return;
  int x, y, z;
  coords(p, cell, x, y, z);
  const size_t N = size_t(p.ncells);
  for (int i = 0; i < p.Q; ++i) {
    const int src = shifted(p, x, y, z, i, -1);
    out[size_t(i) * N + cell] = double(Codec<ST>::template dec<CT>(A[size_t(i) * N + src], t.wref[i]));
  }
}

// A_i(x - e_i) = f-bar_i(x)
template <class ST, class CT>
__global__ void k_scatter(const GenParams p, const GenTables<CT> t, const double* __restrict__ in,
                          ST* __restrict__ A) {
  const int cell = blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= p.ncells) return;
  int x, y, z;
  coords(p, cell, x, y, z);
  const size_t N = size_t(p.ncells);
  for (int i = 0; i < p.Q; ++i) {
    const int dst = shifted(p, x, y, z, i, -1);
    A[size_t(i) * N + dst] = Codec<ST>::template enc<CT>(CT(in[size_t(i) * N + cell]), t.wref[i]);
  }
}

// Eq. (2-4-2): rho = sum f, u = (sum c f + F/2) / rho; Eq. (2-4-1): phi = sum f (+ S_G / 2 for
// the CDE variant).
// Computed in the model's compute dtype from the gathered f-bar.
template <class ST, class CT>
__global__ void k_fields(const GenParams p, const GenTables<CT> t, const ST* __restrict__ A, int nse,
                         double* __restrict__ rho_out, double* __restrict__ u_out) {
  const int cell = blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= p.ncells) return;
  int x, y, z;
  coords(p, cell, x, y, z);
  const size_t N = size_t(p.ncells);
  CT rho = CT(0), j[3] = {CT(0), CT(0), CT(0)};
  for (int i = 0; i < p.Q; ++i) {
    const int src = shifted(p, x, y, z, i, -1);
    const CT f = Codec<ST>::template dec<CT>(A[size_t(i) * N + src], t.wref[i]);
    rho += f;
    j[0] = fma(t.ce[i][0], f, j[0]);
    j[1] = fma(t.ce[i][1], f, j[1]);
    j[2] = fma(t.ce[i][2], f, j[2]);
  }
  if (!nse) {
    // Eq. (2-4-1) with lambda = 1 for the CDE variant: phi = sum f + S_G / 2 (zero otherwise)
    for (int a = 0; a < 3; ++a) rho = fma(CT(p.cde_half[a]), j[a], rho);
  }
  rho_out[cell] = double(rho);
  if (!nse || u_out == nullptr) return;
  CT F[3] = {CT(0), CT(0), CT(0)};
  if (p.force_b >= 0) {
    const int ib = p.force_b == 0 ? x : (p.force_b == 1 ? y : z);
    F[p.force_a] = static_cast<const CT*>(p.force_tab)[ib];
  }
  for (int a = 0; a < p.d; ++a) u_out[size_t(a) * N + cell] = double(fma(CT(0.5), F[a], j[a]) / rho);
}

// NCDE: phi_prev(x) = sum_i f-bar_i(x); for the NSE (S = 0) the same sum is the density
template <class ST, class CT>
__global__ void k_phi(const GenParams p, const GenTables<CT> t, const ST* __restrict__ A, CT* __restrict__ phi) {
  const int cell = blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= p.ncells) return;
  int x, y, z;
  coords(p, cell, x, y, z);
  const size_t N = size_t(p.ncells);
  CT s = CT(0);
  for (int i = 0; i < p.Q; ++i)
    s += Codec<ST>::template dec<CT>(A[size_t(i) * N + shifted(p, x, y, z, i, -1)], t.wref[i]);
  phi[cell] = s;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Conservation sums, pass 1: each thread sums whole cells (per-cell sums in the compute dtype,
// cross-cell accumulation in FP64) over a fixed grid-stride; each block reduces in a fixed
// order and writes its four partial sums. Streaming is a permutation, so the stored array has
// the same totals as f-bar and needs no gather.
template <class ST, class CT>
__global__ void __launch_bounds__(256) k_sums_partial(const GenParams p, const GenTables<CT> t,
                                                      const ST* __restrict__ A, double* __restrict__ partials) {
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  const size_t N = size_t(p.ncells);
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t cell = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; cell < p.ncells; cell += stride) {
    CT m = CT(0), j[3] = {CT(0), CT(0), CT(0)};
    for (int i = 0; i < p.Q; ++i) {
      const CT f = Codec<ST>::template dec<CT>(A[size_t(i) * N + cell], t.wref[i]);
      m += f;
      j[0] = fma(t.ce[i][0], f, j[0]);
      j[1] = fma(t.ce[i][1], f, j[1]);
      j[2] = fma(t.ce[i][2], f, j[2]);
    }
    acc[0] += double(m);
    for (int a = 0; a < 3; ++a) acc[1 + a] += double(j[a]);
  }
  __shared__ double red[4][256 / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int q = 0; q < 4; ++q) {
    const double v = warp_sum(acc[q]);
    if (lane == 0) red[q][wid] = v;
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double s = 0.0;
    for (int w = 0; w < int(blockDim.x / 32); ++w) s += red[threadIdx.x][w];
    partials[size_t(blockIdx.x) * 4 + threadIdx.x] = s;
  }
}

// Pass 2: one warp per quantity sums the block partials in a fixed order.
__global__ void k_sums_final(const double* __restrict__ partials, int nblocks, double* __restrict__ out) {
  const int q = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double s = 0.0;
  for (int b = lane; b < nblocks; b += 32) s += partials[size_t(b) * 4 + q];
  s = warp_sum(s);
  if (lane == 0) out[q] = s;
}

template <class F>
lbm_status dispatch_store(const lbm_model* m, F&& f) {
  switch (m->store) {
    case LBM_F64: return f(double(), double());
    case LBM_F32: return f(float(), float());
    case LBM_BF16_DEV: return f(__nv_bfloat16(), float());
    case LBM_F16_DEV: return f(__half(), float());
  }
  return set_error(LBM_ERR_ARG, "unknown storage dtype");
}

template <class CT>
GenTables<CT> gen_tables(const GenParams& p) {
  GenTables<CT> t{};
  for (int i = 0; i < p.Q; ++i) {
    for (int a = 0; a < 3; ++a) t.ce[i][a] = a < p.d ? CT(p.c[a] * p.e[i][a]) : CT(0);
    t.wref[i] = CT(p.wref[i]);
  }
  return t;
}

lbm_status after_launch(lbm_model* m, const char* what) {
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return cuda_error(err, what);
  m->launches += 1;
  return LBM_OK;
}

}  // namespace

lbm_status gen_params(const lbm_model* m, GenParams* gp) {
  const lbm_lattice* L = m->lat;
  *gp = GenParams{};
  gp->Q = L->Q;
  gp->d = L->d;
  for (int a = 0; a < 3; ++a) gp->n[a] = a < L->d ? int(m->n[a]) : 1;
  gp->ncells = m->ncells;
  for (int i = 0; i < L->Q; ++i) {
    for (int a = 0; a < 3; ++a) gp->e[i][a] = L->e[i * 3 + a];
    gp->wref[i] = (m->store == LBM_BF16_DEV || m->store == LBM_F16_DEV) ? L->w[i] * m->rho_ref : 0.0;
  }
  for (int a = 0; a < 3; ++a) gp->c[a] = a < L->d ? L->c[a] : 0.0;
  for (int a = 0; a < 3; ++a)
    gp->cde_half[a] = (m->eq == LBM_NCDE && m->ncde_variant == LBM_NCDE_CDE && a < L->d)
                          ? 0.5 * m->u_const[a] * m->s[1 + a] / m->cs2_eq
                          : 0.0;
  gp->force_a = m->force_a;
  gp->force_b = (m->eq == LBM_NSE && m->force_A != 0.0) ? m->force_b : -1;
  gp->force_tab = m->force_tab;
  return LBM_OK;
}

lbm_status launch_gather(lbm_model* m, double* out) {
  GenParams p;
  gen_params(m, &p);
  const int grid = (m->ncells + 127) / 128;
  return dispatch_store(m, [&](auto st, auto ct) {
    using ST = decltype(st);
    using CT = decltype(ct);
    k_gather<ST, CT><<<grid, 128, 0, m->stream>>>(p, gen_tables<CT>(p), static_cast<const ST*>(m->f[m->cur]), out);
    return after_launch(m, "gather launch");
  });
}

lbm_status launch_scatter(lbm_model* m, const double* in) {
  GenParams p;
  gen_params(m, &p);
  const int grid = (m->ncells + 127) / 128;
  return dispatch_store(m, [&](auto st, auto ct) {
    using ST = decltype(st);
    using CT = decltype(ct);
    k_scatter<ST, CT><<<grid, 128, 0, m->stream>>>(p, gen_tables<CT>(p), in, static_cast<ST*>(m->f[m->cur]));
    return after_launch(m, "scatter launch");
  });
}

lbm_status launch_fields(lbm_model* m, double* rho, double* u) {
  GenParams p;
  gen_params(m, &p);
  const int grid = (m->ncells + 127) / 128;
  return dispatch_store(m, [&](auto st, auto ct) {
    using ST = decltype(st);
    using CT = decltype(ct);
    k_fields<ST, CT><<<grid, 128, 0, m->stream>>>(p, gen_tables<CT>(p), static_cast<const ST*>(m->f[m->cur]),
                                                    m->eq == LBM_NSE ? 1 : 0, rho, u);
    return after_launch(m, "fields launch");
  });
}

lbm_status launch_phi_from_populations(lbm_model* m) {
  GenParams p;
  gen_params(m, &p);
  const int grid = (m->ncells + 127) / 128;
  return dispatch_store(m, [&](auto st, auto ct) {
    using ST = decltype(st);
    using CT = decltype(ct);
    k_phi<ST, CT><<<grid, 128, 0, m->stream>>>(p, gen_tables<CT>(p), static_cast<const ST*>(m->f[m->cur]),
                                                 static_cast<CT*>(m->phi_prev));
    return after_launch(m, "phi launch");
  });
}

template <class CT>
__global__ void k_to_compute(const double* __restrict__ src, CT* __restrict__ dst, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = CT(src[i]);
}

lbm_status launch_to_compute(lbm_model* m, const double* src, void* dst) {
  const int grid = (m->ncells + 127) / 128;
  if (m->store == LBM_F64)
    k_to_compute<double><<<grid, 128, 0, m->stream>>>(src, static_cast<double*>(dst), m->ncells);
  else
    k_to_compute<float><<<grid, 128, 0, m->stream>>>(src, static_cast<float*>(dst), m->ncells);
  return after_launch(m, "field conversion launch");
}

lbm_status launch_density_history(lbm_model* m) {
  GenParams p;
  gen_params(m, &p);
  const int grid = (m->ncells + 127) / 128;
  return dispatch_store(m, [&](auto st, auto ct) {
    using ST = decltype(st);
    using CT = decltype(ct);
    k_phi<ST, CT><<<grid, 128, 0, m->stream>>>(p, gen_tables<CT>(p), static_cast<const ST*>(m->f[m->cur]),
                                                 static_cast<CT*>(m->rho_hist[m->hist_cur]));
    return after_launch(m, "density history launch");
  });
}

lbm_status launch_sums(lbm_model* m) {
  GenParams p;
  gen_params(m, &p);
  return dispatch_store(m, [&](auto st, auto ct) {
    using ST = decltype(st);
    using CT = decltype(ct);
    k_sums_partial<ST, CT><<<kRedBlocks, 256, 0, m->stream>>>(
        p, gen_tables<CT>(p), static_cast<const ST*>(m->f[m->cur]), m->partials);
    lbm_status s = after_launch(m, "sums launch");
    if (s != LBM_OK) return s;
    k_sums_final<<<1, 128, 0, m->stream>>>(m->partials, kRedBlocks, m->sums);
    return after_launch(m, "sums final launch");
  });
}

lbm_status launch_sums_into(lbm_model* m, double* partials, int partial_slots, double* out) {
  if (partial_slots < kRedBlocks) return set_error(LBM_ERR_ARG, "reduction scratch too small");
  GenParams p;
  gen_params(m, &p);
  return dispatch_store(m, [&](auto st, auto ct) {
    using ST = decltype(st);
    using CT = decltype(ct);
    k_sums_partial<ST, CT><<<kRedBlocks, 256, 0, m->stream>>>(p, gen_tables<CT>(p), static_cast<const ST*>(m->f[m->cur]), partials);
    lbm_status s = after_launch(m, "sums launch");
    if (s != LBM_OK) return s;
    k_sums_final<<<1, 128, 0, m->stream>>>(partials, kRedBlocks, out);
    return after_launch(m, "sums final launch");
  });
}

}  // namespace lbm
