// Row-staged collide-stream kernel for 16-bit deviation storage (FP16 or BF16 deviations
// f_i - w_i rho_ref, collision arithmetic in FP32).
//
// The per-thread pull gather of k_step moves 64 bytes per warp access when a population takes
// 2 bytes, too little per memory request to keep HBM busy. Here a CTA works on whole x-rows of
// the grid instead. For the row (y, z) the pull sources of population i (Eq. (2-2b)) are the
// cells (x - e_ix, y - e_iy, z - e_iz): the x-row (y - e_iy, z - e_iz) of array i, read with a
// periodic shift along x. Warp 0 brings these Q source rows into shared memory with one bulk
// copy each (n_x * 2 bytes, 16-byte aligned, completing on the stage's mbarrier), the periodic
// wraps in y and z being the choice of source row. Every thread then reads its cell's
// populations at (x - e_ix) mod n_x, so the wrap in x is an index wrap. A ring of row buffers
// keeps the next rows in flight while the current one is collided; a buffer is refilled once
// every warp has arrived on its `empty` mbarrier. The collision and the aligned per-cell stores
// are those of k_step (same code, same inputs), so the results are bitwise the same.
//
// Every mbarrier wait is bounded: on timeout the CTA records an error in the model's status word,
// waits (bounded again) for the copies it still has in flight and returns.
#pragma once

#include <algorithm>

#include "bulk.cuh"

namespace lbm {

template <class L>
struct RowShape {
  static constexpr int PITCH = L::D == 3 ? kRowPitch3 : kRowPitch2;  // largest n_x (cells per row buffer)
  static constexpr int THREADS = kRowThreads;
  static constexpr int WARPS = THREADS / 32;
};

template <class L, class ST, int EQ, bool COLLIDE>
__global__ void __launch_bounds__(kRowThreads, 2)
    k_step_rows(const StepParams<float> p, const RowParams rp, const ST* __restrict__ fin, ST* __restrict__ fout,
                float* __restrict__ phi) {
  using S = RowShape<L>;
  constexpr int Q = L::Q, RM = L::RMAX, PITCH = S::PITCH;
  extern __shared__ __align__(128) uint8_t row_smem[];
  uint64_t* full = reinterpret_cast<uint64_t*>(row_smem);
  uint64_t* empty = full + kRowMaxStages;
  const ST* rows = reinterpret_cast<const ST*>(row_smem + kRowBarBytes);
  const uint32_t rows_s = tc::smem_addr(row_smem + kRowBarBytes);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nx = p.n[0], ny = p.n[1];
  const int G = int(gridDim.x);
  const int K = (rp.nrows - int(blockIdx.x) + G - 1) / G;  // rows of this CTA (the grid is <= nrows)
  const int NS = rp.stages;
  const uint32_t stage_elems = rp.stage_bytes / uint32_t(sizeof(ST));
  const size_t N = size_t(p.ncells);
  if (tid == 0) {
    for (int s = 0; s < NS; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], S::WARPS);
    }
    tc::mbar_fence_init();
  }
  __syncthreads();

  // warp 0: the Q source rows of local row j into stage j % NS
  auto issue = [&](int j) {
    const int r = int(blockIdx.x) + j * G;
    const int y = r % ny, z = r / ny;
    const int s = j % NS;
    if (lane == 0) bulk::arrive_expect_tx(&full[s], uint32_t(Q) * rp.row_bytes);
    __syncwarp();
    for (int i = lane; i < Q; i += 32) {
      int ys = y - rp.ey[i];
      ys += ys < 0 ? ny : 0;
      ys -= ys >= ny ? ny : 0;
      int zs = 0;
      if constexpr (L::D == 3) {
        zs = z - rp.ez[i];
        zs += zs < 0 ? p.n[2] : 0;
        zs -= zs >= p.n[2] ? p.n[2] : 0;
      }
      const ST* src = fin + size_t(i) * N + (size_t(zs) * size_t(ny) + size_t(ys)) * size_t(nx);
      bulk::copy_g2s(rows_s + uint32_t(s) * rp.stage_bytes + uint32_t(i * PITCH * int(sizeof(ST))), src,
                     rp.row_bytes, &full[s]);
    }
  };

  int issued = 0;  // warp 0: local rows whose copies have been issued
  bool failed = false;
  if (warp == 0)
    for (; issued < K && issued < NS; ++issued) issue(issued);
  int k = 0;
  for (; k < K; ++k) {
    const int s = k % NS;
    // warp 0 refills the buffer of the previous row once every warp has read it
    if (warp == 0 && k >= 1 && issued < K) {
      const int sp = (k - 1) % NS;
      bool ok = true;
      if (lane == 0) ok = tc::mbar_wait_bounded(&empty[sp], uint32_t((k - 1) / NS) & 1u, rp.wait_limit);
      if (!__shfl_sync(0xffffffffu, ok ? 1 : 0, 0)) {
        failed = true;
        break;
      }
      issue(issued++);
    }
    const bool landed = tc::mbar_wait_bounded(&full[s], uint32_t(k / NS) & 1u, rp.wait_limit);
    if (!__all_sync(0xffffffffu, landed)) {
      failed = true;
      break;
    }
    const int r = int(blockIdx.x) + k * G;
    const int y = r % ny, z = r / ny;  // z = 0 in 2D
    const ST* st = rows + size_t(s) * stage_elems;
    for (int x0 = 0; x0 < nx; x0 += S::THREADS) {
      const int x = x0 + tid;
      const bool live = x < nx;
      float f[Q];
      if (live) {
        int xo[2 * RM + 1];  // (x - sh) mod n_x for the x-shifts sh = -RM..RM
#pragma unroll
        for (int sh = -RM; sh <= RM; ++sh) {
          int v = x - sh;
          if (sh > 0) v += v < 0 ? nx : 0;
          if (sh < 0) v -= v >= nx ? nx : 0;
          xo[sh + RM] = v;
        }
        static_for<Q>([&](auto i) {
          constexpr int I = decltype(i)::value;
          f[I] = RawCodec<ST>::dec(st[I * PITCH + xo[RM + L::e(I).x]]);
        });
      }
      if (x0 + S::THREADS >= nx) {  // this warp's last read of the buffer
        __syncwarp();
        if (lane == 0) bulk::arrive(&empty[s]);
      }
      if (live) {
        const int cell = r * nx + x;
        if constexpr (COLLIDE) {
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
        static_for<Q>([&](auto i) {
          constexpr int I = decltype(i)::value;
          k1_store(fout + size_t(I) * N + cell, RawCodec<ST>::enc(f[I]));
        });
      }
    }
  }
  if (failed && lane == 0) atomicExch(rp.status, 1);
  // copies still in flight into this CTA's shared memory land before it exits
  if (warp == 0 && lane == 0)
    for (int j = k; j < issued; ++j) tc::mbar_wait_bounded(&full[j % NS], uint32_t(j / NS) & 1u, rp.wait_limit);
}

// Launch plan: the kernel applies to 16-bit storage with n_x a multiple of 8 (16-byte rows) and
// at most the row pitch. Two CTAs per SM when two row buffers each fit, otherwise one; as many
// buffers (up to kRowMaxStages) as the shared memory of a CTA holds.
template <int KIND>
bool RowLaunch<KIND>::plan(const lbm_model* m, RowPlan* out) {
  using L = Lat<KIND>;
  using S = RowShape<L>;
  if (m->store != LBM_F16_DEV && m->store != LBM_BF16_DEV) return false;
  const int64_t nx = m->n[0];
  if (nx % 8 != 0 || nx > S::PITCH) return false;
  int sms = 0, per_sm = 0, per_block = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, m->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, m->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&per_block, cudaDevAttrMaxSharedMemoryPerBlockOptin, m->device) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  const size_t stage_bytes = size_t(L::Q) * S::PITCH * 2;
  RowPlan p{};
  int ctas = 0, stages = 0;
  for (int c = 2; c >= 1 && ctas == 0; --c) {
    const size_t avail = std::min<size_t>(size_t(per_block), size_t(per_sm) / c - 1024);  // 1 KB reserved per CTA
    const int ns = int(std::min<size_t>(kRowMaxStages, (avail - kRowBarBytes) / stage_bytes));
    if (ns >= 2) {
      ctas = c;
      stages = ns;
    }
  }
  if (ctas == 0) return false;
  const int64_t nrows = m->n[1] * m->n[2];
  p.rp.nrows = int(nrows);
  p.rp.stages = stages;
  p.rp.stage_bytes = uint32_t(stage_bytes);
  p.rp.row_bytes = uint32_t(nx * 2);
  p.rp.status = m->status;
  p.rp.wait_limit = 1u << 22;
  for (int i = 0; i < L::Q; ++i) {
    p.rp.ey[i] = int8_t(L::e(i).y);
    p.rp.ez[i] = int8_t(L::e(i).z);
  }
  p.grid = int(std::min<int64_t>(nrows, int64_t(sms) * ctas));
  p.smem = kRowBarBytes + size_t(stages) * stage_bytes;
  *out = p;
  return true;
}

// The kernel of a model: storage type, equation, collision on / off (stream only).
template <class L, class ST, class F>
lbm_status row_kernel(int eq, bool collide, F&& fn) {
  if (!collide) return fn(k_step_rows<L, ST, LBM_NSE, false>);
  if (eq == LBM_NSE) return fn(k_step_rows<L, ST, LBM_NSE, true>);
  return fn(k_step_rows<L, ST, LBM_NCDE, true>);
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
  if (m->store == LBM_F16_DEV) return row_kernel<L, __half>(m->eq, collide, set);
  return row_kernel<L, __nv_bfloat16>(m->eq, collide, set);
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
  if (m->store == LBM_F16_DEV)
    return row_kernel<L, __half>(m->eq, collide, [&](auto kernel) { return go(kernel, __half()); });
  return row_kernel<L, __nv_bfloat16>(m->eq, collide, [&](auto kernel) { return go(kernel, __nv_bfloat16()); });
}

}  // namespace lbm

#define LBM_INSTANTIATE_ROWS(KIND) template struct lbm::RowLaunch<KIND>;
