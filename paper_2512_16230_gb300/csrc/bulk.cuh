// Inline-PTX wrappers for the per-thread asynchronous copies of the row-staged kernels: 16-byte
// global -> shared copies through L2 that bypass the registers (cp.async.cg), whose completion is
// counted on an mbarrier (cp.async.mbarrier.arrive.noinc), and the wait for a thread's own copies.
//
// Rules the callers keep: both addresses of a copy are 16-byte aligned; the destination is this
// CTA's own shared memory; the mbarrier is initialised with the number of arriving threads.
#pragma once

#include <cstdint>

#include "tcgen05.cuh"

namespace lbm {
namespace bulk {

// 16-byte asynchronous copy global -> shared through L2 (cp.async.cg, no register staging).
__device__ __forceinline__ void cp_async16(uint32_t dst_smem, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst_smem), "l"(src) : "memory");
}

// One arrival on the mbarrier once every cp.async this thread has issued so far has completed (the
// barrier's expected count is not incremented: it counts the arriving threads).
__device__ __forceinline__ void cp_async_arrive(uint64_t* mbar) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(tc::smem_addr(mbar)) : "memory");
}

// Wait until every cp.async of this thread has completed.
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

}  // namespace bulk
}  // namespace lbm
