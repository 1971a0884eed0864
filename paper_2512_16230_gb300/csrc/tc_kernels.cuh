// Tensor-core collide-stream kernel for 16-bit deviation storage (FP16 or BF16 deviations
// f_i - w_i rho_ref, collision arithmetic in FP32).
//
// The two contractions of the collision with the lattice are dense products over one tile of
// 128 cells, with integer coefficients mono_k(e_i) that are exact in FP16/BF16:
//   forward   mu (128 x R)  = D (128 x Q) . M^T (Q x R),   D the stored deviations (exact operands)
//   backward  Delta (128 x Q) = h (128 x R) . M (R x Q),    f*_i = (1 - s_h) d_i + w_i Delta_i
// with M_ki = mono_k(e_i). Both run on tcgen05 (kind::f16, M = 128, FP32 accumulation in TMEM);
// one thread of the CTA issues them, and every thread reads its own cell's row back with a
// 32x32b tensor-memory load. h, computed per cell in FP32 by the same moment-space collision as
// the CUDA-core kernel (collide_moments), is scaled per cell by a power of two and split into a
// 16-bit high and low part (K = 2R), so the back projection keeps about 22 bits of h.
// HI (one rate per order >= 4): the Q - R higher rows join both products as dense 16-bit
// operands, y_r = sum_i H_r(c_i) d_i in the forward product and sum_r H_r(c_i) z_r (z_r = a_r y_r,
// a_r = -(s_r - s_h) / N_r) in the back projection, which is the full Q x Q collision.
// Operands sit in shared memory in the K-major, non-swizzled canonical layout (core matrices of
// 8 rows x 16 bytes). Every mbarrier wait is bounded: on timeout the CTA issues no further
// product, waits (bounded again) for the one in flight, records an error in the model's status
// word, frees its tensor memory and returns.
#pragma once

#include "tcgen05.cuh"

namespace lbm {

template <class L, bool HI>
struct TcShape {
  static constexpr int QP = (L::Q + 15) / 16 * 16;    // K of the forward product, N of the backward
  static constexpr int RP = (L::R + 15) / 16 * 16;    // moment columns of the forward product
  static constexpr int NH = HI ? L::Q - L::R : 0;     // higher rows (HI)
  static constexpr int NHP = (NH + 15) / 16 * 16;
  static constexpr int N1 = RP + NHP;                 // N of the forward product
  static constexpr int K2 = 2 * RP + NHP;             // K of the backward: h high | h low | z
  static constexpr int CTAS = HI ? 3 : 4;             // resident CTAs per SM (shared memory)
};

// Byte offset of element (r, k) of a K-major tile of 16-bit values with KP values per row.
__host__ __device__ constexpr uint32_t kmajor_off(int r, int k, int KP) {
  return uint32_t((r >> 3) * (KP * 16) + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

template <class L, bool HI>
struct __align__(1024) TcSmem {
  using S = TcShape<L, HI>;
  uint8_t a[128 * S::QP * 2];     // deviations: row = cell, k = population
  uint8_t b1[S::N1 * S::QP * 2];  // row n < R: mono_n(e_i); row RP + r: H_r(c_i) of the higher rows
  uint8_t a2[128 * S::K2 * 2];    // per cell: h high parts, h low parts, z
  uint8_t b2[S::QP * S::K2 * 2];  // row = population i: mono_k(e_i) twice, then H_r(c_i)
  uint64_t mbar;
  uint32_t tmem;
};

template <class ST>
__device__ __forceinline__ uint16_t bits16(ST v);
template <>
__device__ __forceinline__ uint16_t bits16(__half v) { return __half_as_ushort(v); }
template <>
__device__ __forceinline__ uint16_t bits16(__nv_bfloat16 v) { return __bfloat16_as_ushort(v); }

template <class ST>
__device__ __forceinline__ ST from_bits16(uint16_t b);
template <>
__device__ __forceinline__ __half from_bits16(uint16_t b) { return __ushort_as_half(b); }
template <>
__device__ __forceinline__ __nv_bfloat16 from_bits16(uint16_t b) { return __ushort_as_bfloat16(b); }

template <class ST>
__device__ __forceinline__ uint16_t round16(float v) {
  if constexpr (std::is_same<ST, __half>::value) return __half_as_ushort(__float2half_rn(v));
  else return __bfloat16_as_ushort(__float2bfloat16_rn(v));
}

// Two values rounded to 16 bits in one packed conversion (a in the low half, b in the high half),
// each rounded to nearest as round16 does; split16x2 adds the low parts v - high (also rounded).
template <class ST>
__device__ __forceinline__ uint32_t pack16x2(float a, float b) {
  if constexpr (std::is_same<ST, __half>::value) {
    const __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&h);
  } else {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&h);
  }
}
template <class ST>
__device__ __forceinline__ void split16x2(float a, float b, uint32_t& hi, uint32_t& lo) {
  float2 hf;
  if constexpr (std::is_same<ST, __half>::value) {
    const __half2 h = __floats2half2_rn(a, b);
    hi = *reinterpret_cast<const uint32_t*>(&h);
    hf = __half22float2(h);
  } else {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    hi = *reinterpret_cast<const uint32_t*>(&h);
    hf = __bfloat1622float2(h);
  }
  lo = pack16x2<ST>(a - hf.x, b - hf.y);
}

constexpr int kTcCols = 128;  // TMEM columns per CTA: D1 in [0, N1), then D2 in [0, QP)

template <class L, class ST, int EQ, bool HI>
__global__ void __launch_bounds__(128, TcShape<L, HI>::CTAS)
    k_step_tc(const StepParams<float> p, const TcParams tp, const ST* __restrict__ fin, ST* __restrict__ fout,
              float* __restrict__ phi) {
  using S = TcShape<L, HI>;
  constexpr int Q = L::Q, R = L::R, QP = S::QP, RP = S::RP, NH = S::NH, NHP = S::NHP, N1 = S::N1, K2 = S::K2;
  constexpr bool BF = std::is_same<ST, __nv_bfloat16>::value;
  static_assert(QP <= kTcCols && N1 <= kTcCols, "TMEM column plan");
  static_assert(NH <= kMaxHigh, "higher-row table");
  extern __shared__ __align__(1024) uint8_t tc_smem_raw[];
  TcSmem<L, HI>& sm = *reinterpret_cast<TcSmem<L, HI>*>(tc_smem_raw);
  const int tid = threadIdx.x;

  // operand tables, once per CTA
  for (int idx = tid; idx < N1 * QP; idx += 128) {
    const int n = idx / QP, k = idx % QP;
    float v = 0.f;
    if (k < Q) {
      if (n < R) v = float(tp.mono[k][n]);
      else if (n >= RP && n - RP < NH) v = tp.hrow[n - RP][k];
    }
    *reinterpret_cast<uint16_t*>(sm.b1 + kmajor_off(n, k, QP)) = round16<ST>(v);
  }
  for (int idx = tid; idx < QP * K2; idx += 128) {
    const int i = idx / K2, k = idx % K2;
    float v = 0.f;
    if (i < Q) {
      if (k < 2 * RP && k % RP < R) v = float(tp.mono[i][k % RP]);
      else if (k >= 2 * RP && k - 2 * RP < NH) v = tp.hrow[k - 2 * RP][i];
    }
    *reinterpret_cast<uint16_t*>(sm.b2 + kmajor_off(i, k, K2)) = round16<ST>(v);
  }
  if (tid == 0) {
    tc::mbar_init(&sm.mbar, 1);
    tc::mbar_fence_init();
  }
  if (tid < 32) {
    tc::alloc(&sm.tmem, kTcCols);
    tc::relinquish();
  }
  tc::fence_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = sm.tmem;
  const uint32_t row_lane = uint32_t(tid & ~31) << 16;  // this warp's 32 TMEM lanes
  const uint32_t d1 = tmem, d2 = tmem;  // D2 reuses D1's columns once every row has been read
  const uint32_t a_s = tc::smem_addr(sm.a), b1_s = tc::smem_addr(sm.b1);
  const uint32_t a2_s = tc::smem_addr(sm.a2), b2_s = tc::smem_addr(sm.b2);
  constexpr uint32_t idesc1 = tc::idesc_f16<BF>(128, N1);
  constexpr uint32_t idesc2 = tc::idesc_f16<BF>(128, QP);
  const size_t N = size_t(p.ncells);
  uint32_t phase = 0;
  bool failed = false;

  // Software pipeline: the gather loads of the next tile are issued before this tile's collision
  // and consumed only when that tile is written to shared memory, so their latency overlaps the
  // matrix products and the moment-space arithmetic.
  auto gather = [&](int tile, uint16_t (&raw)[Q]) {
    const int cell = tile * 128 + tid;
    if (tile < tp.ntiles && cell < p.ncells) {
      const Neigh<L> nb(cell, p);
      static_for<Q>([&](auto i) {
        constexpr int I = decltype(i)::value;
        raw[I] = bits16(k1_load(fin + size_t(I) * N + nb.template src<I>()));
      });
    } else {
      static_for<Q>([&](auto i) { raw[decltype(i)::value] = 0; });
    }
  };
  auto stage = [&](const uint16_t (&raw)[Q]) {  // row tid of A, then the forward product
    static_for<QP / 8>([&](auto c) {
      constexpr int C = decltype(c)::value;
      uint32_t w4[4];
      static_for<4>([&](auto j) {
        constexpr int I0 = 8 * C + 2 * decltype(j)::value;
        const uint32_t lo = I0 < Q ? uint32_t(raw[I0 < Q ? I0 : 0]) : 0u;
        const uint32_t hi = I0 + 1 < Q ? uint32_t(raw[I0 + 1 < Q ? I0 + 1 : 0]) : 0u;
        w4[decltype(j)::value] = lo | (hi << 16);
      });
      *reinterpret_cast<uint4*>(sm.a + kmajor_off(tid, 8 * C, QP)) = make_uint4(w4[0], w4[1], w4[2], w4[3]);
    });
    tc::fence_async_smem();
    __syncthreads();
    if (tid == 0 && !tp.no_issue) {
      tc::fence_after_sync();
      static_for<QP / 16>([&](auto kk) {
        constexpr int KK = decltype(kk)::value;
        tc::mma_f16(d1, tc::smem_desc(a_s + KK * 256, 128, QP * 16), tc::smem_desc(b1_s + KK * 256, 128, QP * 16),
                    idesc1, KK > 0 ? 1u : 0u);
      });
      tc::commit(&sm.mbar);
    }
  };
  if (int(blockIdx.x) < tp.ntiles) {
    uint16_t raw[Q];
    gather(blockIdx.x, raw);
    stage(raw);
  }
  for (int tile = blockIdx.x; tile < tp.ntiles; tile += gridDim.x) {
    const int cell = tile * 128 + tid;
    const bool live = cell < p.ncells;
    const int next = tile + int(gridDim.x);
    uint16_t nraw[Q];
    gather(next, nraw);
    bool ok = tc::mbar_wait_bounded(&sm.mbar, phase, tp.wait_limit);
    phase ^= 1u;
    if (__syncthreads_or(!ok)) {
      failed = true;
      break;
    }
    tc::fence_after_sync();

    // moments of this cell's row, then the moment-space collision in FP32
    float mu[R];
    static_for<RP / 16>([&](auto c) {
      constexpr int C = decltype(c)::value;
      float v[16];
      tc::ld16(d1 + row_lane + 16 * C, v);
      tc::wait_ld();
      static_for<16>([&](auto j) {
        constexpr int K = 16 * C + decltype(j)::value;
        if constexpr (K < R) mu[K] = v[decltype(j)::value];
      });
    });
    int x = 0, y = 0, z = 0;
    if (live) {
      const Neigh<L> nb(cell, p);
      x = nb.x;
      y = nb.y;
      z = nb.z;
    }
    float F[3] = {0.f, 0.f, 0.f};
    body_force(p.force_a, p.force_b, p.force_tab, x, y, z, F);
    float phi_prev = 0.f, phi_now = 0.f;
    if constexpr (EQ == LBM_NCDE) phi_prev = live ? phi[cell] : 0.f;
    // HI: z_r = a_r y_r from the higher-row columns of the forward product
    float zr[NH > 0 ? NH : 1];
    if constexpr (HI) {
      static_for<NHP / 16>([&](auto c) {
        constexpr int C = decltype(c)::value;
        float v[16];
        tc::ld16(d1 + row_lane + RP + 16 * C, v);
        tc::wait_ld();
        static_for<16>([&](auto j) {
          constexpr int K = 16 * C + decltype(j)::value;
          if constexpr (K < NH) zr[K] = tp.ah[K] * v[decltype(j)::value];
        });
      });
    }
    float h[R];
    constexpr bool AG = GradTerm<L, EQ>::kOn;
    float gr[3] = {0.f, 0.f, 0.f};
    if constexpr (AG) {
      if (live) cell_field_gradient<L>(p, cell, x, y, z, gr);
    }
    collide_moments<L, float, EQ, true>(mu, p, F, phi_prev, phi_now, h, AG ? gr : nullptr);
    if constexpr (EQ == LBM_NCDE) {
      if (live) phi[cell] = phi_now;
    }
    if constexpr (AG && EQ == LBM_NSE) {
      if (live && p.grad_on) p.rho_out[cell] = phi_now;
    }
    // per-cell power-of-two scale, then h = high + low in 16 bits each (z rides with h's scale)
    float hmax = 0.f;
    static_for<R>([&](auto k) { hmax = fmaxf(hmax, fabsf(h[decltype(k)::value])); });
    if constexpr (HI) static_for<NH>([&](auto k) { hmax = fmaxf(hmax, fabsf(zr[decltype(k)::value])); });
    const uint32_t ex = (__float_as_uint(hmax) >> 23) & 0xFFu;
    const float sc = (live && hmax > 0.f && ex >= 1u && ex <= 252u) ? __uint_as_float((254u - ex) << 23) : 1.f;
    uint32_t hp[K2 / 2];
    static_for<K2 / 2>([&](auto j) { hp[decltype(j)::value] = 0u; });
    static_for<RP / 2>([&](auto k) {  // h in pairs (K, K + 1): high parts, then low parts
      constexpr int K = 2 * decltype(k)::value;
      const float a = (K < R && live) ? h[K < R ? K : 0] * sc : 0.f;
      const float b = (K + 1 < R && live) ? h[K + 1 < R ? K + 1 : 0] * sc : 0.f;
      split16x2<ST>(a, b, hp[K / 2], hp[(RP + K) / 2]);
    });
    if constexpr (HI) {
      static_for<NHP / 2>([&](auto k) {
        constexpr int K = 2 * decltype(k)::value;
        const float a = (K < NH && live) ? zr[K < NH ? K : 0] * sc : 0.f;
        const float b = (K + 1 < NH && live) ? zr[K + 1 < NH ? K + 1 : 0] * sc : 0.f;
        hp[(2 * RP + K) / 2] = pack16x2<ST>(a, b);
      });
    }
    static_for<K2 / 8>([&](auto c) {
      constexpr int C = decltype(c)::value;
      *reinterpret_cast<uint4*>(sm.a2 + kmajor_off(tid, 8 * C, K2)) =
          make_uint4(hp[4 * C], hp[4 * C + 1], hp[4 * C + 2], hp[4 * C + 3]);
    });
    tc::fence_before_sync();
    tc::fence_async_smem();
    __syncthreads();
    if (tid == 0 && !tp.no_issue) {
      tc::fence_after_sync();
      static_for<K2 / 16>([&](auto kk) {
        constexpr int KK = decltype(kk)::value;
        tc::mma_f16(d2, tc::smem_desc(a2_s + KK * 256, 128, K2 * 16), tc::smem_desc(b2_s + KK * 256, 128, K2 * 16),
                    idesc2, KK > 0 ? 1u : 0u);
      });
      tc::commit(&sm.mbar);
    }
    ok = tc::mbar_wait_bounded(&sm.mbar, phase, tp.wait_limit);
    phase ^= 1u;
    if (__syncthreads_or(!ok)) {
      failed = true;
      break;
    }
    tc::fence_after_sync();

    // f*_i = (1 - s_h) d_i + w_i Delta_i / sc, stored at the cell itself; d_i from row tid of A
    const float inv = 1.f / sc;
    static_for<QP / 16>([&](auto c) {
      constexpr int C = decltype(c)::value;
      float v[16];
      tc::ld16(d2 + row_lane + 16 * C, v);
      const uint4 q0 = *reinterpret_cast<const uint4*>(sm.a + kmajor_off(tid, 16 * C, QP));
      const uint4 q1 = *reinterpret_cast<const uint4*>(sm.a + kmajor_off(tid, 16 * C + 8, QP));
      const uint32_t dw[8] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w};
      tc::wait_ld();
      static_for<16>([&](auto j) {
        constexpr int J = decltype(j)::value;
        constexpr int I = 16 * C + J;
        if constexpr (I < Q) {
          if (live) {
            const uint16_t b = uint16_t((J & 1) ? (dw[J / 2] >> 16) : (dw[J / 2] & 0xFFFFu));
            const float d = RawCodec<ST>::dec(from_bits16<ST>(b));
            const float fs = fmaf(p.one_minus_sh, d, p.w[I] * (v[J] * inv));
            k1_store(fout + size_t(I) * N + cell, RawCodec<ST>::enc(fs));
          }
        }
      });
    });
    tc::fence_before_sync();
    __syncthreads();
    if (next < tp.ntiles) stage(nraw);
  }
  if (failed) {
    // the product whose wait ran out may still be writing this CTA's TMEM columns: give its
    // commit one more bounded wait before the columns are released (and issue nothing more)
    if (!tp.no_issue) tc::mbar_wait_bounded(&sm.mbar, phase ^ 1u, tp.wait_limit);
    if (tid == 0) atomicExch(tp.status, 1);
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (tid < 32) tc::dealloc(tmem, kTcCols);
}


// FP32 storage with one rate per order >= 4: the low-order collision runs on the CUDA cores (the
// reduced form of collide, exact FP32), and only the correction of the higher rows goes to
// tcgen05. That correction is linear in the pre-collision populations,
//   Delta_i = w_i sum_r a_r H_r(c_i) y_r,  y_r = sum_j H_r(c_j) f_j,
// so it is applied as one dense Q x Q operator G_ij = sum_r a_r H_r(c_i) H_r(c_j) (built in FP64
// with the rates): Delta (128 x Q) = f (128 x Q) . G^T (Q x Q), one product per 128-cell tile,
// issued before the CUDA cores collide the same cells and read back after. Both operands are
// FP32 values, so each is scaled by a power of two (G row by row on the host, the populations per
// cell) and split into an FP16 high and low part; the product takes three kind::f16 chains into
// one accumulator, hi.hi + hi.lo + lo.hi (about 22 bits). One CTA-wide barrier per tile orders
// the operand stores before the product and the previous tile's tensor-memory reads before it is
// overwritten. The gather of the next tile is issued before this tile's collision, so its latency
// overlaps the CUDA-core work.
//
// Resident CTAs per SM of k_step_tc32_high (128 threads each). 3 leaves 168 registers, room for
// the next tile's populations, which are loaded while the current tile collides: 1.30 ms per step
// on rD3Q53 256x256x192 against 1.35 ms with 4 CTAs and no prefetch (128 registers) and 1.41 ms
// with 3 CTAs and no prefetch (GB300).
#ifndef LBM_TC32_CTAS
#define LBM_TC32_CTAS 3
#endif

template <class L>
struct Tc32Shape {
  static constexpr int QP = (L::Q + 15) / 16 * 16;  // K and N of the product
  static constexpr int CTAS = LBM_TC32_CTAS;        // resident CTAs per SM
};

template <class L>
struct __align__(1024) Tc32Smem {
  using S = Tc32Shape<L>;
  uint8_t a_hi[128 * S::QP * 2];  // scaled pre-collision f, high parts: row = cell, k = population j
  uint8_t a_lo[128 * S::QP * 2];
  uint8_t b_hi[S::QP * S::QP * 2];  // row = population i, column = population j: g_ij
  uint8_t b_lo[S::QP * S::QP * 2];
  uint64_t mbar;
  uint32_t tmem;
};

constexpr int kTc32Cols = 64;  // TMEM columns per CTA: Delta in [0, QP)

// power of two that brings max |v| into [1, 2) (1 for zero or out-of-range values)
__device__ __forceinline__ float pow2_scale(float vmax) {
  const uint32_t ex = (__float_as_uint(vmax) >> 23) & 0xFFu;
  return (vmax > 0.f && ex >= 1u && ex <= 252u) ? __uint_as_float((254u - ex) << 23) : 1.f;
}

__device__ __forceinline__ void split16(float v, uint16_t& hi, uint16_t& lo) {
  const __half h = __float2half_rn(v);
  hi = __half_as_ushort(h);
  lo = __half_as_ushort(__float2half_rn(v - __half2float(h)));
}

template <class L, int EQ>
__global__ void __launch_bounds__(128, Tc32Shape<L>::CTAS)
    k_step_tc32_high(const StepParams<float> p, const Tc32Params tp, const float* __restrict__ fin,
                     float* __restrict__ fout, float* __restrict__ phi) {
  using S = Tc32Shape<L>;
  constexpr int Q = L::Q, QP = S::QP;
  static_assert(QP <= kTc32Cols, "TMEM column plan");
  extern __shared__ __align__(1024) uint8_t tc_smem_raw[];
  Tc32Smem<L>& sm = *reinterpret_cast<Tc32Smem<L>*>(tc_smem_raw);
  const int tid = threadIdx.x;

  // the operator, once per CTA (each row of g is scaled to unit max on the host)
  for (int idx = tid; idx < QP * QP; idx += 128) {
    const int i = idx / QP, j = idx % QP;
    const float v = (i < Q && j < Q) ? tp.g[i][j] : 0.f;
    uint16_t hi, lo;
    split16(v, hi, lo);
    *reinterpret_cast<uint16_t*>(sm.b_hi + kmajor_off(i, j, QP)) = hi;
    *reinterpret_cast<uint16_t*>(sm.b_lo + kmajor_off(i, j, QP)) = lo;
  }
  if (tid == 0) {
    tc::mbar_init(&sm.mbar, 1);
    tc::mbar_fence_init();
  }
  if (tid < 32) {
    tc::alloc(&sm.tmem, kTc32Cols);
    tc::relinquish();
  }
  tc::fence_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = sm.tmem;
  const uint32_t row_lane = uint32_t(tid & ~31) << 16;
  const uint32_t ah_s = tc::smem_addr(sm.a_hi), al_s = tc::smem_addr(sm.a_lo);
  const uint32_t bh_s = tc::smem_addr(sm.b_hi), bl_s = tc::smem_addr(sm.b_lo);
  constexpr uint32_t idesc = tc::idesc_f16<false>(128, QP);
  const size_t N = size_t(p.ncells);
  uint32_t phase = 0;
  bool failed = false;

  auto load_tile = [&](int tile, float (&g)[Q], int& gx, int& gy, int& gz) {
    const int cell = tile * 128 + tid;
    gx = gy = gz = 0;
    if (tile < tp.ntiles && cell < p.ncells) {
      const Neigh<L> nb(cell, p);
      gx = nb.x;
      gy = nb.y;
      gz = nb.z;
      static_for<Q>([&](auto i) {
        constexpr int I = decltype(i)::value;
        g[I] = k1_load(fin + size_t(I) * N + nb.template src<I>());
      });
    } else {
      static_for<Q>([&](auto i) { g[decltype(i)::value] = 0.f; });
    }
  };
  float f[Q];
  int x, y, z;
  load_tile(blockIdx.x, f, x, y, z);
  for (int tile = blockIdx.x; tile < tp.ntiles; tile += gridDim.x) {
    const int cell = tile * 128 + tid;
    const bool live = cell < p.ncells;
    // A = scaled pre-collision populations, high and low parts. The previous tile's product has
    // completed (this thread saw its barrier phase) unless a wait ran out, and then no thread
    // stores: one that did see the phase knows the product is done.
    float fmax = 0.f;
    static_for<Q>([&](auto i) { fmax = fmaxf(fmax, fabsf(f[decltype(i)::value])); });
    const float sa = pow2_scale(fmax);
    if (!failed) {
      static_for<QP / 8>([&](auto c) {
        constexpr int C = decltype(c)::value;
        uint32_t wh[4], wl[4];
        static_for<4>([&](auto j) {
          constexpr int I0 = 8 * C + 2 * decltype(j)::value;
          const float a = I0 < Q ? f[I0 < Q ? I0 : 0] * sa : 0.f;
          const float b = I0 + 1 < Q ? f[I0 + 1 < Q ? I0 + 1 : 0] * sa : 0.f;
          split16x2<__half>(a, b, wh[decltype(j)::value], wl[decltype(j)::value]);
        });
        *reinterpret_cast<uint4*>(sm.a_hi + kmajor_off(tid, 8 * C, QP)) = make_uint4(wh[0], wh[1], wh[2], wh[3]);
        *reinterpret_cast<uint4*>(sm.a_lo + kmajor_off(tid, 8 * C, QP)) = make_uint4(wl[0], wl[1], wl[2], wl[3]);
      });
    }
    tc::fence_async_smem();
    tc::fence_before_sync();  // this thread's reads of the previous tile's Delta are complete
    if (__syncthreads_or(failed)) {
      failed = true;
      break;
    }
    tc::fence_after_sync();
    if (tid == 0 && !tp.no_issue) {
      // Delta = A_hi G_hi + A_hi G_lo + A_lo G_hi
      static_for<3 * (QP / 16)>([&](auto q) {
        constexpr int Kc = decltype(q)::value % (QP / 16), part = decltype(q)::value / (QP / 16);
        const uint32_t a = (part == 2 ? al_s : ah_s) + Kc * 256, b = (part == 1 ? bl_s : bh_s) + Kc * 256;
        tc::mma_f16(tmem, tc::smem_desc(a, 128, QP * 16), tc::smem_desc(b, 128, QP * 16), idesc,
                    decltype(q)::value > 0 ? 1u : 0u);
      });
      tc::commit(&sm.mbar);
    }
    // the next tile's populations are loaded while this one collides
    float fn[Q];
    int xn, yn, zn;
    load_tile(tile + int(gridDim.x), fn, xn, yn, zn);
    // the low-order collision on the CUDA cores meanwhile
    float F[3] = {0.f, 0.f, 0.f};
    body_force(p.force_a, p.force_b, p.force_tab, x, y, z, F);
    float phi_prev = 0.f, phi_now = 0.f;
    if constexpr (EQ == LBM_NCDE) phi_prev = live ? phi[cell] : 0.f;
    constexpr bool AG = GradTerm<L, EQ>::kOn;
    float gr[3] = {0.f, 0.f, 0.f};
    if constexpr (AG) {
      if (live) cell_field_gradient<L>(p, cell, x, y, z, gr);
    }
    collide<L, float, EQ, false>(f, p, F, phi_prev, phi_now, static_cast<NoHigh*>(nullptr), AG ? gr : nullptr);
    if constexpr (EQ == LBM_NCDE) {
      if (live) phi[cell] = phi_now;
    }
    if constexpr (AG && EQ == LBM_NSE) {
      if (live && p.grad_on) p.rho_out[cell] = phi_now;
    }
    const bool ok = tc::mbar_wait_bounded(&sm.mbar, phase, tp.wait_limit);
    phase ^= 1u;
    if (!ok) {
      failed = true;  // the CTA stops at the next barrier; this tile's populations are not written
      static_for<Q>([&](auto i) { f[decltype(i)::value] = fn[decltype(i)::value]; });
      x = xn; y = yn; z = zn;
      continue;
    }
    tc::fence_after_sync();
    // f*_i = collided f_i + w_i Delta_i, Delta = D / sa (sa a power of two: exact reciprocal)
    const float inv = 1.f / sa;
    static_for<QP / 16>([&](auto c) {
      constexpr int C = decltype(c)::value;
      float v[16];
      tc::ld16(tmem + row_lane + 16 * C, v);
      tc::wait_ld();
      static_for<16>([&](auto j) {
        constexpr int I = 16 * C + decltype(j)::value;
        if constexpr (I < Q) {
          if (live) k1_store(fout + size_t(I) * N + cell, fmaf(tp.wg[I], v[decltype(j)::value] * inv, f[I]));
        }
      });
    });
    static_for<Q>([&](auto i) { f[decltype(i)::value] = fn[decltype(i)::value]; });
    x = xn; y = yn; z = zn;
  }
  // a wait that ran out on the CTA's last tile: every thread learns of it here
  tc::fence_before_sync();
  failed = __syncthreads_or(failed);
  tc::fence_after_sync();
  if (failed) {
    // the product in flight, if any, completes before its tensor memory is freed (bounded again)
    if (!tp.no_issue) tc::mbar_wait_bounded(&sm.mbar, phase ^ 1u, tp.wait_limit);
    if (tid == 0) atomicExch(tp.status, 1);
  }
  __syncthreads();
  if (tid < 32) tc::dealloc(tmem, kTc32Cols);
}

}  // namespace lbm
