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
    if (rp.no_copy) return;  // test hook: nothing lands, every wait on the buffer runs out
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

// The same row-staged step with the two contractions of the collision on the tensor cores. A CTA
// is two tiles of 128 cells (warps 0-3: cells 0..127 of the row, warps 4-7: 128..255), each with
// its own 128 TMEM columns. Per row and tile:
//   forward  mu (128 x RP) = D (128 x QP) . M^T, D the stored 16-bit deviations, written by each
//            thread into its own TMEM lane (A from tensor memory), M_ki = mono_k(e_i) in shared
//            memory (exact in 16 bits); HI (one rate per order >= 4): the higher rows H_r(c_i) join
//            M as NH more columns, y_r = sum_i H_r(c_i) d_i;
//   back     Delta (128 x QP) = [h_high | h_low | z] . [M; M; H], h the monomial coefficients of the
//            collision in moment space (FP32, collide_moments) and z_r = a_r y_r, scaled per cell by
//            a power of two, h split into a 16-bit high and low part;
//   then     f*_i = (1 - s_h) d_i + w_i Delta_i / scale, written back into the row buffer.
// TMEM columns of a tile: without HI D1 [0, RP), A [32, ..), D2 [64, 64 + QP); with HI D1 [0, N1),
// the forward A at [N1, N1 + QP / 2), the back A at [64, 64 + K2 / 2) (over the read columns of D1)
// and D2 [0, QP).
// One thread per tile issues the products after a named barrier of the tile's 128 threads; every
// thread waits for their completion on the tile's mbarriers (bounded: a timeout is carried to the
// next row barrier, where the whole CTA stops, waits for what it has in flight and frees its TMEM).
template <class L, class ST, int EQ, bool HI>
__global__ void __launch_bounds__(kRowThreads, 2)
    k_step_rows_tc(const StepParams<float> p, const RowParams rp, const TcParams tp, const ST* __restrict__ fin,
                   ST* __restrict__ fout, float* __restrict__ phi) {
  using Sh = TcShape<L, HI>;
  constexpr int Q = L::Q, R = L::R, RM = L::RMAX, PITCH = kRowPitch, WARPS = kRowThreads / 32;
  constexpr int QP = Sh::QP, RP = Sh::RP, NH = Sh::NH, NHP = Sh::NHP, N1 = Sh::N1, K2 = Sh::K2;
  constexpr uint32_t ROWB = PITCH * sizeof(ST);
  constexpr bool BF = std::is_same<ST, __nv_bfloat16>::value;
  constexpr uint32_t TILE_COLS = 128;
  constexpr uint32_t CA = HI ? N1 : 32, CA2 = HI ? 64 : 32, CD2 = HI ? 0 : 64;
  static_assert(QP % 16 == 0 && K2 % 16 == 0 && N1 % 16 == 0, "product shapes");
  static_assert(HI ? (CA + QP / 2 <= TILE_COLS && CA2 + K2 / 2 <= TILE_COLS && CA2 >= QP)
                   : (N1 <= int(CA) && CA + QP / 2 <= CD2 && CA2 + K2 / 2 <= CD2 && CD2 + QP <= TILE_COLS),
                "TMEM column plan");
  static_assert(NH <= kMaxHigh, "higher-row table");
  extern __shared__ __align__(128) uint8_t row_smem[];
  uint64_t* full = reinterpret_cast<uint64_t*>(row_smem);
  uint64_t* mbar = full + kRowMaxStages;                     // [tile][0: forward, 1: back]
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 4);  // TMEM base address
  uint8_t* b1 = row_smem + kRowBarBytes;                     // N1 x QP, K-major: mono_n(e_i), H_r(c_i)
  uint8_t* b2 = b1 + N1 * QP * 2;                            // QP x K2, K-major: mono_k(e_i) twice, H_r(c_i)
  uint8_t* rows_b = b2 + QP * K2 * 2;
  ST* rows = reinterpret_cast<ST*>(rows_b);
  const uint32_t rows_s = tc::smem_addr(rows_b);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, tile = warp >> 2;
  const int nx = p.n[0], ny = p.n[1], nz = L::D == 3 ? p.n[2] : 1;
  const int G = int(gridDim.x);
  const int K = (rp.nrows - int(blockIdx.x) + G - 1) / G;
  const int NS = rp.stages;
  const uint32_t stage_elems = rp.stage_bytes / uint32_t(sizeof(ST));
  const size_t N = size_t(p.ncells);
  const size_t pop_bytes = N * sizeof(ST);
  const int x = tid;
  const bool live = x < nx;
  const bool lane_chunk = lane * 8 < nx;
  const int gy = G % ny, gz = G / ny;
  auto advance = [&](int& y, int& z) {
    y += gy;
    z += gz;
    if (y >= ny) {
      y -= ny;
      z += 1;
    }
  };
  // operand tables, once per CTA
  for (int idx = tid; idx < N1 * QP; idx += kRowThreads) {
    const int n = idx / QP, k = idx % QP;
    float v = 0.f;
    if (k < Q) {
      if (n < R) v = float(tp.mono[k][n]);
      else if (n >= RP && n - RP < NH) v = tp.hrow[n - RP][k];
    }
    *reinterpret_cast<uint16_t*>(b1 + kmajor_off(n, k, QP)) = round16<ST>(v);
  }
  for (int idx = tid; idx < QP * K2; idx += kRowThreads) {
    const int i = idx / K2, k = idx % K2;
    float v = 0.f;
    if (i < Q) {
      if (k < 2 * RP && k % RP < R) v = float(tp.mono[i][k % RP]);
      else if (k >= 2 * RP && k - 2 * RP < NH) v = tp.hrow[k - 2 * RP][i];
    }
    *reinterpret_cast<uint16_t*>(b2 + kmajor_off(i, k, K2)) = round16<ST>(v);
  }
  if (tid == 0) {
    for (int s = 0; s < NS; ++s) tc::mbar_init(&full[s], kRowThreads);
    for (int b = 0; b < 4; ++b) tc::mbar_init(&mbar[b], 1);
    tc::mbar_fence_init();
  }
  if (warp == 0) {
    tc::alloc(tslot, 2 * TILE_COLS);
    tc::relinquish();
  }
  tc::fence_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = *tslot + uint32_t(tile) * TILE_COLS;
  const uint32_t lane_off = uint32_t((warp & 3) * 32) << 16;  // this warp's 32 TMEM lanes
  const uint32_t b1_s = tc::smem_addr(b1), b2_s = tc::smem_addr(b2);
  constexpr uint32_t idesc1 = tc::idesc_f16<BF>(128, N1);
  constexpr uint32_t idesc2 = tc::idesc_f16<BF>(128, QP);
  const bool issuer = (tid & 127) == 0;

  auto load_row = [&](int y, int z, int s) {
    if (rp.no_copy) return;  // test hook: nothing lands, every wait on the buffer runs out
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

  int ly = int(blockIdx.x) % ny, lz = int(blockIdx.x) / ny;
  int y = ly, z = lz;
  for (int j = 0; j < K && j < NS - 2; ++j) {
    load_row(ly, lz, j);
    advance(ly, lz);
  }
  bool failed = false, bad = false;
  int issued = 0, waited = 0;  // products this tile's issuer committed / that every thread waited for
  int py = y, pz = z;
  uint32_t phase = 0;
  for (int k = 0; k < K; ++k) {
    const int s = k % NS;
    const bool landed = tc::mbar_wait_bounded(&full[s], uint32_t(k / NS) & 1u, rp.wait_limit);
    const int r = z * ny + y;
    const uint32_t st_s = rows_s + uint32_t(s) * rp.stage_bytes;
    // the stored deviations of this cell's sources, packed in pairs (zero past Q or past the row)
    uint32_t a[QP / 2];
    static_for<QP / 2>([&](auto j) { a[decltype(j)::value] = 0u; });
    if (live && landed) {
      uint32_t xa[2 * RM + 1];
#pragma unroll
      for (int sh = -RM; sh <= RM; ++sh) {
        int v = x - sh;
        if (sh > 0) v += v < 0 ? nx : 0;
        if (sh < 0) v -= v >= nx ? nx : 0;
        xa[sh + RM] = st_s + uint32_t(v) * uint32_t(sizeof(ST));
      }
      static_for<Q>([&](auto i) {
        constexpr int I = decltype(i)::value;
        const uint32_t b = lds16<I * int(ROWB)>(xa[RM + L::e(I).x]);
        a[I / 2] |= (I & 1) ? (b << 16) : b;
      });
    }
    if (__syncthreads_or(!landed || bad)) {
      failed = true;
      break;
    }
    if (k >= 1) store_row(py, pz, (k - 1) % NS);
    if (k + NS - 2 < K) {
      load_row(ly, lz, (k + NS - 2) % NS);
      advance(ly, lz);
    }
    // forward product: the moments of the row's 128 cells of this tile (QP / 2 columns of A: 16 at
    // a time, then a remainder of 8)
    static_for<QP / 32>([&](auto c) {
      uint32_t w[16];
      static_for<16>([&](auto j) { w[decltype(j)::value] = a[16 * decltype(c)::value + decltype(j)::value]; });
      tc::st16(tbase + lane_off + CA + 16 * decltype(c)::value, w);
    });
    if constexpr ((QP / 2) % 16 == 8) {
      uint32_t w[8];
      static_for<8>([&](auto j) { w[decltype(j)::value] = a[QP / 2 - 8 + decltype(j)::value]; });
      tc::st8(tbase + lane_off + CA + QP / 2 - 8, w);
    }
    tc::wait_st();
    tc::fence_before_sync();
    if (tile == 0) tc::named_barrier<1, 128>(); else tc::named_barrier<2, 128>();
    if (issuer && !tp.no_issue) {
      tc::fence_after_sync();
      static_for<QP / 16>([&](auto kk) {
        constexpr int KK = decltype(kk)::value;
        tc::mma_f16_tmem_a(tbase, tbase + CA + 8 * KK, tc::smem_desc(b1_s + KK * 256, 128, QP * 16), idesc1,
                           KK > 0 ? 1u : 0u);
      });
      tc::commit(&mbar[2 * tile]);
      ++issued;
    }
    bool ok = tc::mbar_wait_bounded(&mbar[2 * tile], phase, tp.wait_limit);
    bad = bad || !ok;
    if (ok) ++waited;
    tc::fence_after_sync();
    float mu[R];
    static_for<RP / 16>([&](auto c) {
      constexpr int C = decltype(c)::value;
      float v[16];
      tc::ld16(tbase + lane_off + 16 * C, v);
      tc::wait_ld();
      static_for<16>([&](auto j) {
        constexpr int KX = 16 * C + decltype(j)::value;
        if constexpr (KX < R) mu[KX] = v[decltype(j)::value];
      });
    });
    // HI: z_r = a_r y_r from the higher-row columns of the forward product
    float zr[NH > 0 ? NH : 1];
    if constexpr (HI) {
      static_for<NHP / 16>([&](auto c) {
        constexpr int C = decltype(c)::value;
        float v[16];
        tc::ld16(tbase + lane_off + RP + 16 * C, v);
        tc::wait_ld();
        static_for<16>([&](auto j) {
          constexpr int KX = 16 * C + decltype(j)::value;
          if constexpr (KX < NH) zr[KX] = tp.ah[KX] * v[decltype(j)::value];
        });
      });
    }
    // the collision in moment space, in FP32 (the CUDA-core kernel's code)
    const int cell = r * nx + x;
    float F[3] = {0.f, 0.f, 0.f};
    body_force(p.force_a, p.force_b, p.force_tab, x, y, z, F);
    float phi_prev = 0.f, phi_now = 0.f;
    if constexpr (EQ == LBM_NCDE) phi_prev = live ? phi[cell] : 0.f;
    constexpr bool AG = GradTerm<L, EQ>::kOn;
    float gr[3] = {0.f, 0.f, 0.f};
    if constexpr (AG) {
      if (live) cell_field_gradient<L>(p, cell, x, y, z, gr);
    }
    float h[R];
    collide_moments<L, float, EQ, true>(mu, p, F, phi_prev, phi_now, h, AG ? gr : nullptr);
    if constexpr (EQ == LBM_NCDE) {
      if (live) phi[cell] = phi_now;
    }
    if constexpr (AG && EQ == LBM_NSE) {
      if (live && p.grad_on) p.rho_out[cell] = phi_now;
    }
    // back projection: h (and z) scaled by a power of two, h in 16-bit high and low parts
    float hmax = 0.f;
    static_for<R>([&](auto kx) { hmax = fmaxf(hmax, fabsf(h[decltype(kx)::value])); });
    if constexpr (HI) static_for<NH>([&](auto kx) { hmax = fmaxf(hmax, fabsf(zr[decltype(kx)::value])); });
    const uint32_t ex = (__float_as_uint(hmax) >> 23) & 0xFFu;
    const float sc = (live && hmax > 0.f && ex >= 1u && ex <= 252u) ? __uint_as_float((254u - ex) << 23) : 1.f;
    uint32_t hp[K2 / 2];
    static_for<RP / 2>([&](auto kx) {
      constexpr int KX = 2 * decltype(kx)::value;
      const float u0 = (KX < R && live) ? h[KX < R ? KX : 0] * sc : 0.f;
      const float u1 = (KX + 1 < R && live) ? h[KX + 1 < R ? KX + 1 : 0] * sc : 0.f;
      split16x2<ST>(u0, u1, hp[KX / 2], hp[(RP + KX) / 2]);
    });
    if constexpr (HI) {
      static_for<NHP / 2>([&](auto kx) {
        constexpr int KX = 2 * decltype(kx)::value;
        const float u0 = (KX < NH && live) ? zr[KX < NH ? KX : 0] * sc : 0.f;
        const float u1 = (KX + 1 < NH && live) ? zr[KX + 1 < NH ? KX + 1 : 0] * sc : 0.f;
        hp[(2 * RP + KX) / 2] = pack16x2<ST>(u0, u1);
      });
    }
    static_for<K2 / 32>([&](auto c) {
      uint32_t w[16];
      static_for<16>([&](auto j) { w[decltype(j)::value] = hp[16 * decltype(c)::value + decltype(j)::value]; });
      tc::st16(tbase + lane_off + CA2 + 16 * decltype(c)::value, w);
    });
    if constexpr ((K2 / 2) % 16 == 8) {
      uint32_t w[8];
      static_for<8>([&](auto j) { w[decltype(j)::value] = hp[K2 / 2 - 8 + decltype(j)::value]; });
      tc::st8(tbase + lane_off + CA2 + K2 / 2 - 8, w);
    }
    tc::wait_st();
    tc::fence_before_sync();
    if (tile == 0) tc::named_barrier<1, 128>(); else tc::named_barrier<2, 128>();
    if (issuer && !tp.no_issue) {
      tc::fence_after_sync();
      static_for<K2 / 16>([&](auto kk) {
        constexpr int KK = decltype(kk)::value;
        tc::mma_f16_tmem_a(tbase + CD2, tbase + CA2 + 8 * KK, tc::smem_desc(b2_s + KK * 256, 128, K2 * 16),
                           idesc2, KK > 0 ? 1u : 0u);
      });
      tc::commit(&mbar[2 * tile + 1]);
      ++issued;
    }
    ok = tc::mbar_wait_bounded(&mbar[2 * tile + 1], phase, tp.wait_limit);
    bad = bad || !ok;
    if (ok) ++waited;
    tc::fence_after_sync();
    phase ^= 1u;
    // f*_i = (1 - s_h) d_i + w_i Delta_i / sc, back into the row buffer at x
    const float inv = 1.f / sc;
    const uint32_t xs = st_s + uint32_t(x) * uint32_t(sizeof(ST));
    static_for<QP / 16>([&](auto c) {
      constexpr int C = decltype(c)::value;
      float v[16];
      tc::ld16(tbase + lane_off + CD2 + 16 * C, v);
      tc::wait_ld();
      static_for<16>([&](auto j) {
        constexpr int J = decltype(j)::value;
        constexpr int I = 16 * C + J;
        if constexpr (I < Q) {
          if (live) {
            const uint16_t bits = uint16_t((I & 1) ? (a[I / 2] >> 16) : (a[I / 2] & 0xFFFFu));
            const float fs = fmaf(p.one_minus_sh, dec16<ST>(bits), p.w[I] * (v[J] * inv));
            sts16<I * int(ROWB)>(xs, enc16<ST>(fs));
          }
        }
      });
    });
    py = y;
    pz = z;
    advance(y, z);
  }
  // a wait that ran out in the last row is seen here by the whole CTA
  if (!failed && __syncthreads_or(bad)) failed = true;
  if (!failed && K > 0) store_row(py, pz, (K - 1) % NS);
  if (failed) {
    // products that were committed but not seen complete may still write this tile's TMEM: give
    // them one more bounded wait before the columns are released
    if (issued > waited) {  // (the row that failed flipped the phase after its products)
      tc::mbar_wait_bounded(&mbar[2 * tile], phase ^ 1u, tp.wait_limit);
      tc::mbar_wait_bounded(&mbar[2 * tile + 1], phase ^ 1u, tp.wait_limit);
    }
    if (tid == 0) atomicExch(tp.status, 1);
  }
  bulk::cp_async_wait_all();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::dealloc(*tslot, 2 * TILE_COLS);
}

// Launch plan: the kernel applies to 16-bit storage with n_x a multiple of 8 (16-byte rows) and
// at most the row pitch (256 cells). Two CTAs per SM when three row buffers each fit, otherwise
// one; as many buffers (up to kRowMaxStages) as the shared memory of a CTA holds.
template <int KIND>
bool RowLaunch<KIND>::plan(const lbm_model* m, RowPlan* out, bool tensor, bool high) {
  using L = Lat<KIND>;
  if (high && !tensor) return false;  // the higher rows are row-staged on the tensor cores only
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
  // the tensor-core kernel keeps its two operand tables ahead of the row buffers
  auto table_bytes = [](auto shape) {
    using Sh = decltype(shape);
    return size_t(Sh::N1) * Sh::QP * 2 + size_t(Sh::QP) * Sh::K2 * 2;
  };
  const size_t tables = !tensor ? 0 : high ? table_bytes(TcShape<L, true>{}) : table_bytes(TcShape<L, false>{});
  RowPlan p{};
  int ctas = 0, stages = 0;
  for (int c = 2; c >= 1 && ctas == 0; --c) {
    const size_t avail = std::min<size_t>(size_t(per_block), size_t(per_sm) / c - 1024);  // 1 KB reserved per CTA
    const int ns = int(std::min<size_t>(kRowMaxStages, (avail - kRowBarBytes - tables) / stage_bytes));
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
  p.rp.no_copy = m->row_no_copy ? 1 : 0;
  p.rp.wait_limit = m->row_no_copy ? (1u << 10) : (1u << 22);
  const int64_t N = m->n[0] * m->n[1] * m->n[2];
  for (int i = 0; i < L::Q; ++i) {
    p.rp.ey[i] = int8_t(L::e(i).y);
    p.rp.ez[i] = int8_t(L::e(i).z);
    p.rp.src_off[i] = 2 * (int64_t(i) * N - (int64_t(L::e(i).y) + int64_t(L::e(i).z) * m->n[1]) * nx);
  }
  p.grid = int(std::min<int64_t>(nrows, int64_t(sms) * ctas));
  p.smem = kRowBarBytes + tables + size_t(stages) * stage_bytes;
  p.tensor = tensor;
  p.high = high;
  if (tensor) make_tc_params(m, &p.tp);
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

// The tensor-core kernel of a model: fn(kernel, storage tag).
template <class L, class F>
lbm_status row_tc_kernel(int store, int eq, bool high, F&& fn) {
  auto by_eq = [&](auto tag, auto hi) -> lbm_status {
    using ST = decltype(tag);
    constexpr bool H = decltype(hi)::value;
    if (eq == LBM_NSE) return fn(k_step_rows_tc<L, ST, LBM_NSE, H>, tag);
    return fn(k_step_rows_tc<L, ST, LBM_NCDE, H>, tag);
  };
  auto by_hi = [&](auto tag) -> lbm_status {
    if (high) return by_eq(tag, std::true_type{});
    return by_eq(tag, std::false_type{});
  };
  if (store == LBM_F16_DEV) return by_hi(__half());
  return by_hi(__nv_bfloat16());
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
  if (plan.tensor && collide) return row_tc_kernel<L>(m->store, m->eq, plan.high, [&](auto k, auto) { return set(k); });
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
  if (plan.tensor && collide) {
    auto go_tc = [&](auto kernel, auto tag) -> lbm_status {
      using ST = decltype(tag);
      kernel<<<plan.grid, kRowThreads, plan.smem, m->stream>>>(p, plan.rp, plan.tp, static_cast<const ST*>(fin),
                                                                static_cast<ST*>(fout), phi);
      cudaError_t err = cudaGetLastError();
      return err == cudaSuccess ? LBM_OK : cuda_error(err, "row-staged tensor-core collide-stream launch");
    };
    return row_tc_kernel<L>(m->store, m->eq, plan.high, go_tc);
  }
  const bool full = m->n[0] == kRowPitch;
  if (m->store == LBM_F16_DEV)
    return row_kernel<L, __half>(m->eq, collide, full, [&](auto kernel) { return go(kernel, __half()); });
  return row_kernel<L, __nv_bfloat16>(m->eq, collide, full,
                                      [&](auto kernel) { return go(kernel, __nv_bfloat16()); });
}

}  // namespace lbm

#define LBM_INSTANTIATE_ROWS(KIND) template struct lbm::RowLaunch<KIND>;
