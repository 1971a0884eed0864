// Row-staged collide-stream kernel for 16-bit deviation storage (FP16 or BF16 deviations
// f_i - w_i rho_ref, collision arithmetic in FP32).
//
// The per-thread pull gather and store of k_step move 64 bytes per warp access when a population
// takes 2 bytes, too little per memory request to keep HBM busy. Here a CTA works on whole x-rows
// of the grid, one cell per thread, and moves memory in 512-byte warp accesses. For the row (y, z)
// the pull sources of population i (Eq. (2-2b)) are the cells (x - e_ix, y - e_iy, z - e_iz): the
// x-row (y - e_iy, z - e_iz) of array i, read with a periodic shift along x. The warps copy these
// Q source rows into a shared-memory row buffer with 16-byte cp.async copies (one warp instruction
// per population row, completing on the buffer's mbarrier); the periodic wraps in y and z are the
// choice of source row, the wrap in x an index wrap: every thread reads its sources at
// (x - e_ix) mod n_x. After a CTA barrier (every source read) the threads write their
// post-collision populations back into the buffer at their own x; after the next row's barrier
// the warps store the Q rows with 16-byte stores. A ring of row buffers keeps the following rows
// in flight while the current one is collided. The collision is the code of k_step on the same
// inputs, so the results are bitwise the same.
//
// The wait for a row's copies is bounded: on timeout (decided for the whole CTA at the next
// barrier) the CTA records an error in the model's status word, waits for its own copies and
// returns.
#pragma once

#include <algorithm>

#include "bulk.cuh"

namespace lbm {

// 16-bit shared-memory accesses at a register address plus a compile-time byte offset, and the
// conversions of one value between the storage format and FP32.
template <int OFF>
__device__ __forceinline__ uint16_t lds16(uint32_t addr) {
  uint16_t v;
  asm volatile("ld.shared.b16 %0, [%1+%2];" : "=h"(v) : "r"(addr), "n"(OFF));
  return v;
}
template <int OFF>
__device__ __forceinline__ void sts16(uint32_t addr, uint16_t v) {
  asm volatile("st.shared.b16 [%0+%1], %2;" ::"r"(addr), "n"(OFF), "h"(v) : "memory");
}
template <class ST>
__device__ __forceinline__ float dec16(uint16_t b) {
  if constexpr (std::is_same<ST, __half>::value) return __half2float(__ushort_as_half(b));
  else return __uint_as_float(uint32_t(b) << 16);
}
template <class ST>
__device__ __forceinline__ uint16_t enc16(float v) {
  uint16_t b;
  if constexpr (std::is_same<ST, __half>::value) asm("cvt.rn.f16.f32 %0, %1;" : "=h"(b) : "f"(v));
  else asm("cvt.rn.bf16.f32 %0, %1;" : "=h"(b) : "f"(v));
  return b;
}

template <class L, class ST, int EQ, bool COLLIDE, bool FULL>
__global__ void __launch_bounds__(kRowThreads, 2)
    k_step_rows(const StepParams<float> p, const RowParams rp, const ST* __restrict__ fin, ST* __restrict__ fout,
                float* __restrict__ phi) {
  constexpr int Q = L::Q, RM = L::RMAX, PITCH = kRowPitch, WARPS = kRowThreads / 32;
  constexpr uint32_t ROWB = PITCH * sizeof(ST);  // bytes of one population's row in a buffer
  static_assert(ROWB == 32 * 16, "a row of the buffer is one 16-byte chunk per lane");
  extern __shared__ __align__(128) uint8_t row_smem[];
  uint64_t* full = reinterpret_cast<uint64_t*>(row_smem);  // every thread's copies of the row landed
  ST* rows = reinterpret_cast<ST*>(row_smem + kRowBarBytes);
  const uint32_t rows_s = tc::smem_addr(row_smem + kRowBarBytes);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nx = p.n[0], ny = p.n[1], nz = L::D == 3 ? p.n[2] : 1;
  const int G = int(gridDim.x);
  const int K = (rp.nrows - int(blockIdx.x) + G - 1) / G;  // rows of this CTA (the grid is <= nrows)
  const int NS = rp.stages;
  const uint32_t stage_elems = rp.stage_bytes / uint32_t(sizeof(ST));
  const size_t N = size_t(p.ncells);
  const size_t pop_bytes = N * sizeof(ST);
  const int x = tid;
  // FULL: n_x equals the pitch, every thread has a cell and every lane a 16-byte chunk of a row
  const bool live = FULL || x < nx;
  const bool lane_chunk = FULL || lane * 8 < nx;
  // rows of this CTA are r = blockIdx.x + k G: (y, z) advance by (G mod n_y, G div n_y) with a carry
  const int gy = G % ny, gz = G / ny;
  auto advance = [&](int& y, int& z) {
    y += gy;
    z += gz;
    if (y >= ny) {
      y -= ny;
      z += 1;
    }
  };
  if (tid == 0) {
    for (int s = 0; s < NS; ++s) tc::mbar_init(&full[s], kRowThreads);
    tc::mbar_fence_init();
  }
  __syncthreads();

  // every thread: its chunks of the Q source rows of row (y, z) into buffer s (warp w takes the
  // populations w, w + 8, ...), then one arrival on the buffer's mbarrier when they have landed
  auto load_row = [&](int y, int z, int s) {
    if (lane_chunk) {
      const size_t r = size_t(z) * ny + y;
      const uint8_t* base = reinterpret_cast<const uint8_t*>(fin) + (r * nx + lane * 8) * sizeof(ST);
      const uint32_t dst = rows_s + uint32_t(s) * rp.stage_bytes + uint32_t(lane * 16);
      const bool inner = y >= RM && y < ny - RM && (L::D == 2 || (z >= RM && z < nz - RM));
      if (inner) {
        static_for<(Q + WARPS - 1) / WARPS>([&](auto m) {
          const int i = warp + WARPS * decltype(m)::value;
          if (i < Q) bulk::cp_async16(dst + uint32_t(i) * ROWB, base + rp.src_off[i]);
        });
      } else {
        const uint8_t* b0 = reinterpret_cast<const uint8_t*>(fin) + size_t(lane * 8) * sizeof(ST);
        for (int i = warp; i < Q; i += WARPS) {
          int ys = y - rp.ey[i];
          ys += ys < 0 ? ny : 0;
          ys -= ys >= ny ? ny : 0;
          int zs = 0;
          if constexpr (L::D == 3) {
            zs = z - rp.ez[i];
            zs += zs < 0 ? nz : 0;
            zs -= zs >= nz ? nz : 0;
          }
          bulk::cp_async16(dst + uint32_t(i) * ROWB,
                           b0 + size_t(i) * pop_bytes + (size_t(zs) * ny + ys) * nx * sizeof(ST));
        }
      }
    }
    bulk::cp_async_arrive(&full[s]);
  };

  int ly = int(blockIdx.x) % ny, lz = int(blockIdx.x) / ny;  // next row to load
  int y = ly, z = lz;                                          // row being collided
  // one warp-wide 16-byte store per population row of buffer sb to row (sy, sz) of the output
  auto store_row = [&](int sy, int sz, int sb) {
    if (lane_chunk) {
      const size_t sr = size_t(sz) * ny + sy;
      const uint8_t* src = reinterpret_cast<const uint8_t*>(rows + size_t(sb) * stage_elems) + warp * ROWB + lane * 16;
      uint8_t* dst = reinterpret_cast<uint8_t*>(fout) + (sr * nx + lane * 8) * sizeof(ST) + warp * pop_bytes;
      static_for<(Q + WARPS - 1) / WARPS>([&](auto m) {
        constexpr int M = decltype(m)::value;
        if (warp + WARPS * M < Q)
          *reinterpret_cast<uint4*>(dst + M * WARPS * pop_bytes) = *reinterpret_cast<const uint4*>(src + M * WARPS * ROWB);
      });
    }
  };

  // Ring of NS buffers: while row k is collided (in its buffer), row k - 1 is stored from its
  // buffer and rows k + 1 .. k + NS - 2 are in flight; one CTA barrier per row separates the reads
  // of row k from the in-place writes, and the writes of row k - 1 from its store.
  for (int j = 0; j < K && j < NS - 2; ++j) {
    load_row(ly, lz, j);
    advance(ly, lz);
  }
  bool failed = false;
  int py = y, pz = z;  // row k - 1
  for (int k = 0; k < K; ++k) {
    const int s = k % NS;
    const bool landed = tc::mbar_wait_bounded(&full[s], uint32_t(k / NS) & 1u, rp.wait_limit);
    const int r = z * ny + y;
    const uint32_t st_s = rows_s + uint32_t(s) * rp.stage_bytes;
    float f[Q];
    if (live && landed) {
      uint32_t xa[2 * RM + 1];  // address of (x - sh) mod n_x in row 0 of the buffer, sh = -RM..RM
#pragma unroll
      for (int sh = -RM; sh <= RM; ++sh) {
        int v = x - sh;
        if (sh > 0) v += v < 0 ? nx : 0;
        if (sh < 0) v -= v >= nx ? nx : 0;
        xa[sh + RM] = st_s + uint32_t(v) * uint32_t(sizeof(ST));
      }
      static_for<Q>([&](auto i) {
        constexpr int I = decltype(i)::value;
        f[I] = dec16<ST>(lds16<I * int(ROWB)>(xa[RM + L::e(I).x]));
      });
    }
    // every source of row k read, row k - 1 collided into its buffer, row k - 2 stored
    if (__syncthreads_or(!landed)) {
      failed = true;
      break;
    }
    if (k >= 1) store_row(py, pz, (k - 1) % NS);
    if (k + NS - 2 < K) {  // into the buffer of row k - 2
      load_row(ly, lz, (k + NS - 2) % NS);
      advance(ly, lz);
    }
    if (live) {
      if constexpr (COLLIDE) {
        const int cell = r * nx + x;
        float F[3];
        body_force(p.force_a, p.force_b, p.force_tab, x, y, z, F);
        float phi_prev = 0.f, phi_now = 0.f;
        if constexpr (EQ == LBM_NCDE) phi_prev = phi[cell];
        constexpr bool AG = GradTerm<L, EQ>::kOn;
        float gr[3];
        if constexpr (AG) cell_field_gradient<L>(p, cell, x, y, z, gr);
        collide<L, float, EQ, true>(f, p, F, phi_prev, phi_now, static_cast<NoHigh*>(nullptr), AG ? gr : nullptr);
        if constexpr (EQ == LBM_NCDE) phi[cell] = phi_now;
        if constexpr (AG && EQ == LBM_NSE) {
          if (p.grad_on) p.rho_out[cell] = phi_now;
        }
      }
      const uint32_t xs = st_s + uint32_t(x) * uint32_t(sizeof(ST));
      static_for<Q>([&](auto i) {
        constexpr int I = decltype(i)::value;
        sts16<I * int(ROWB)>(xs, enc16<ST>(f[I]));
      });
    }
    py = y;
    pz = z;
    advance(y, z);
  }
  if (!failed && K > 0) {
    __syncthreads();  // the last row is complete in its buffer
    store_row(py, pz, (K - 1) % NS);
  }
  if (failed && tid == 0) atomicExch(rp.status, 1);
  bulk::cp_async_wait_all();  // no copy of this thread is still writing the CTA's shared memory
}

// Launch plan: the kernel applies to 16-bit storage with n_x a multiple of 8 (16-byte rows) and
// at most the row pitch (256 cells). Two CTAs per SM when three row buffers each fit, otherwise
// one; as many buffers (up to kRowMaxStages) as the shared memory of a CTA holds.
template <int KIND>
bool RowLaunch<KIND>::plan(const lbm_model* m, RowPlan* out) {
  using L = Lat<KIND>;
  if (m->store != LBM_F16_DEV && m->store != LBM_BF16_DEV) return false;
  const int64_t nx = m->n[0];
  if (nx % 8 != 0 || nx > kRowPitch) return false;
  int sms = 0, per_sm = 0, per_block = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, m->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, m->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&per_block, cudaDevAttrMaxSharedMemoryPerBlockOptin, m->device) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  const size_t stage_bytes = size_t(L::Q) * kRowPitch * 2;
  RowPlan p{};
  int ctas = 0, stages = 0;
  for (int c = 2; c >= 1 && ctas == 0; --c) {
    const size_t avail = std::min<size_t>(size_t(per_block), size_t(per_sm) / c - 1024);  // 1 KB reserved per CTA
    const int ns = int(std::min<size_t>(kRowMaxStages, (avail - kRowBarBytes) / stage_bytes));
    if (ns >= 3) {  // the row being collided, the row being stored, at least one in flight
      ctas = c;
      stages = ns;
    }
  }
  if (ctas == 0) return false;
  const int64_t nrows = m->n[1] * m->n[2];
  p.rp.nrows = int(nrows);
  p.rp.stages = stages;
  p.rp.stage_bytes = uint32_t(stage_bytes);
  p.rp.status = m->status;
  p.rp.wait_limit = 1u << 22;
  const int64_t N = m->n[0] * m->n[1] * m->n[2];
  for (int i = 0; i < L::Q; ++i) {
    p.rp.ey[i] = int8_t(L::e(i).y);
    p.rp.ez[i] = int8_t(L::e(i).z);
    p.rp.src_off[i] = 2 * (int64_t(i) * N - (int64_t(L::e(i).y) + int64_t(L::e(i).z) * m->n[1]) * nx);
  }
  p.grid = int(std::min<int64_t>(nrows, int64_t(sms) * ctas));
  p.smem = kRowBarBytes + size_t(stages) * stage_bytes;
  *out = p;
  return true;
}

// The kernel of a model: storage type, equation, collision on / off (stream only).
template <class L, class ST, bool FULL, class F>
lbm_status row_kernel_full(int eq, bool collide, F&& fn) {
  if (!collide) return fn(k_step_rows<L, ST, LBM_NSE, false, FULL>);
  if (eq == LBM_NSE) return fn(k_step_rows<L, ST, LBM_NSE, true, FULL>);
  return fn(k_step_rows<L, ST, LBM_NCDE, true, FULL>);
}
template <class L, class ST, class F>
lbm_status row_kernel(int eq, bool collide, bool full, F&& fn) {
  if (full) return row_kernel_full<L, ST, true>(eq, collide, fn);
  return row_kernel_full<L, ST, false>(eq, collide, fn);
}

template <int KIND>
lbm_status RowLaunch<KIND>::configure(const lbm_model* m, const RowPlan& plan, bool collide) {
  using L = Lat<KIND>;
  auto set = [&](auto kernel) -> lbm_status {
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(plan.smem)) != cudaSuccess ||
        cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                             int(cudaSharedmemCarveoutMaxShared)) != cudaSuccess)
      return cuda_error(cudaGetLastError(), "row-staged kernel attributes");
    return LBM_OK;
  };
  const bool full = m->n[0] == kRowPitch;
  if (m->store == LBM_F16_DEV) return row_kernel<L, __half>(m->eq, collide, full, set);
  return row_kernel<L, __nv_bfloat16>(m->eq, collide, full, set);
}

template <int KIND>
lbm_status RowLaunch<KIND>::launch(const lbm_model* m, const RowPlan& plan, const StepParams<float>& p,
                                   const void* fin, void* fout, float* phi, bool collide) {
  using L = Lat<KIND>;
  auto go = [&](auto kernel, auto tag) -> lbm_status {
    using ST = decltype(tag);
    kernel<<<plan.grid, kRowThreads, plan.smem, m->stream>>>(p, plan.rp, static_cast<const ST*>(fin),
                                                              static_cast<ST*>(fout), phi);
    cudaError_t err = cudaGetLastError();
    return err == cudaSuccess ? LBM_OK : cuda_error(err, "row-staged collide-stream launch");
  };
  const bool full = m->n[0] == kRowPitch;
  if (m->store == LBM_F16_DEV)
    return row_kernel<L, __half>(m->eq, collide, full, [&](auto kernel) { return go(kernel, __half()); });
  return row_kernel<L, __nv_bfloat16>(m->eq, collide, full,
                                      [&](auto kernel) { return go(kernel, __nv_bfloat16()); });
}

}  // namespace lbm

#define LBM_INSTANTIATE_ROWS(KIND) template struct lbm::RowLaunch<KIND>;
