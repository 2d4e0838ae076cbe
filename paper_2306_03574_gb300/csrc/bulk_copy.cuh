// Bulk asynchronous copies (the TMA engine's untiled form) and mbarriers, written as
// inline PTX for sm_100-class GPUs.
//
// cp.async.bulk moves a contiguous run of bytes between global and shared memory
// without occupying the issuing thread: both addresses must be 16-byte aligned and the
// size a multiple of 16.  A load signals completion on an mbarrier in shared memory
// (complete_tx: the barrier's phase completes when the expected byte count has arrived
// and the expected arrivals have been made); a store is tracked by bulk async-groups.
//
// Every wait here is bounded: after a fixed number of polls it gives up, counts the
// event in a device-global counter (read on the host by aao_wait_timeouts) and returns
// false, so a lost completion can never hang the GPU.
#pragma once

#include <cstdint>

namespace aao {

// polls of a bounded mbarrier wait (each try_wait may also suspend the thread for an
// implementation-defined time), far beyond any legitimate copy time
constexpr long long MBAR_POLLS = 1LL << 24;

// bounded waits that gave up, per translation unit that includes this header (each
// such unit exports a host reader)
static __device__ unsigned int g_wait_timeouts = 0;

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(count) : "memory");
  // make the initialised barrier visible to the async proxy (the bulk-copy engine)
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}

// one arrival that also raises the expected transaction count by `bytes`
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for phase `parity` of the barrier; false (and the timeout counted) if it
// did not complete within MBAR_POLLS polls.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (long long i = 0; i < MBAR_POLLS; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  atomicAdd(&g_wait_timeouts, 1u);
  return false;
}

// global -> shared, `bytes` (multiple of 16) from 16-byte aligned addresses; completion
// counted on `bar`
__device__ __forceinline__ void bulk_load(void* dst_smem, const void* src_gmem, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
          smem_addr(dst_smem)),
      "l"(src_gmem), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// shared -> global, `bytes` (multiple of 16) from 16-byte aligned addresses, in the
// issuing thread's current bulk async-group
__device__ __forceinline__ void bulk_store(void* dst_gmem, const void* src_smem, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;\n" ::"l"(dst_gmem),
               "r"(smem_addr(src_smem)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;\n" ::: "memory"); }

// wait until every committed bulk store of this thread has finished reading shared memory
__device__ __forceinline__ void bulk_wait_read_all() {
  asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory");
}

// order this thread's generic-proxy shared-memory writes before later async-proxy reads
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}

}  // namespace aao
