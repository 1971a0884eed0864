// Inline-PTX wrappers for the bulk-copy (TMA) engine: untiled global -> shared copies that
// complete on an mbarrier through its transaction count, shared -> global copies tracked by bulk
// groups, and the mbarrier arrivals and fences that go with them (PTX ISA: cp.async.bulk,
// cp.async.bulk.commit_group / wait_group, mbarrier.arrive, mbarrier.expect_tx, fence.proxy.async),
// and the per-thread 16-byte cp.async copies that can complete on an mbarrier as well.
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

// Copy `bytes` from this CTA's shared memory to global memory, in the thread's current bulk group.
__device__ __forceinline__ void copy_s2g(void* dst, uint32_t src_smem, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(src_smem), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void commit_group() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// Wait until this thread's bulk groups have finished reading their shared-memory sources.
__device__ __forceinline__ void wait_groups_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// Wait until this thread's bulk groups have completed (their writes performed).
__device__ __forceinline__ void wait_groups() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
// Order this thread's generic-proxy shared-memory writes before later async-proxy (bulk) accesses.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 16-byte asynchronous copy global -> shared through L2 (cp.async.cg, no register staging).
__device__ __forceinline__ void cp_async16(uint32_t dst_smem, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst_smem), "l"(src) : "memory");
}
// One arrival on the mbarrier once every cp.async this thread has issued so far has completed (the
// barrier's expected count is not incremented: it counts the arriving threads).
__device__ __forceinline__ void cp_async_arrive(uint64_t* mbar) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(tc::smem_addr(mbar)) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

}  // namespace bulk
}  // namespace lbm
