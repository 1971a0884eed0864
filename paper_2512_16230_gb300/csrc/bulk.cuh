// Inline-PTX wrappers for the bulk-copy (TMA) engine: untiled global -> shared copies that
// complete on an mbarrier through its transaction count, and the mbarrier arrivals that go with
// them (PTX ISA: cp.async.bulk, mbarrier.arrive, mbarrier.expect_tx).
//
// Rules the callers keep: both addresses of a copy are 16-byte aligned and its size is a multiple
// of 16 bytes; the destination is this CTA's own shared memory (no cluster, no multicast); the
// arrive.expect_tx of a phase comes before the copies that complete it.
#pragma once

#include <cstdint>

#include "tcgen05.cuh"

namespace lbm {
namespace bulk {

// Arrive once on the mbarrier and add `bytes` to the transaction count of its current phase.
__device__ __forceinline__ void arrive_expect_tx(uint64_t* mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc::smem_addr(mbar)), "r"(bytes)
               : "memory");
}

// Plain arrival (release semantics: this thread's earlier shared-memory reads are performed
// before the arrival is observed).
__device__ __forceinline__ void arrive(uint64_t* mbar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_addr(mbar)) : "memory");
}

// Copy `bytes` from global memory to this CTA's shared memory; the mbarrier's transaction count
// drops by `bytes` when the data has landed.
__device__ __forceinline__ void copy_g2s(uint32_t dst_smem, const void* src, uint32_t bytes, uint64_t* mbar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst_smem),
      "l"(src), "r"(bytes), "r"(tc::smem_addr(mbar))
      : "memory");
}

}  // namespace bulk
}  // namespace lbm
