// Bulk copies global -> shared memory by the TMA engine (cp.async.bulk),
// completed on a shared-memory mbarrier, with a bounded wait.
//
// Use (one block): thread 0 calls mbar_init, the block synchronises, thread 0
// calls bulk_load (after mbar_expect_tx for the total byte count), every
// thread later calls mbar_wait before reading the destination.  Addresses and
// sizes of a bulk copy are multiples of 16 bytes.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace esplit {

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// one expected arrival (the expect_tx below); the phase completes when that
// arrival and all announced bytes have landed
__device__ __forceinline__ void mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void bulk_load(void* dst_smem, const void* src_gmem, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst_smem)),
      "l"(src_gmem), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// waits for phase `parity` of the barrier; false after max_tries unsuccessful
// probes (each probe may suspend the thread for a short, hardware-bounded time)
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int max_tries = 1 << 20) {
  const uint32_t a = smem_addr(bar);
  for (int it = 0; it < max_tries; ++it) {
    uint32_t done;
    asm volatile(
        "{\n"
        " .reg .pred p;\n"
        " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

}  // namespace esplit
