// rk_tma.cuh -- tensor-memory-accelerator (TMA) tile loads with mbarrier
// completion, as inline PTX for sm_103a, and the tensor maps a strided pass reads
// its input tiles with.
//
// One thread arms the block's mbarrier with the expected byte count and issues
// cp.async.bulk.tensor; every thread then waits on the barrier's phase.  Waits are
// bounded: after kWaitLimit polls the wait reports failure, the kernel records it
// in an error word the host reads, waits (bounded again) for the copy in flight
// and returns instead of hanging.
#pragma once

#include <cuda.h>
#include <stdint.h>

namespace rk {

constexpr unsigned kWaitLimit = 1u << 26;  // polls (seconds) before giving up
constexpr int kMaxTma = 10;                // inputs of one strided pass served by TMA

// Tensor maps of the inputs of one strided pass, in the order of PassArgs::in.
struct TileMaps {
  CUtensorMap m[kMaxTma];
};

RK_DEV uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

RK_DEV void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// make the barrier initialisation visible to the async (TMA) proxy
RK_DEV void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// order this thread's earlier shared-memory accesses before later async-proxy writes
RK_DEV void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

RK_DEV void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

RK_DEV void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1, int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];" ::
          "r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2)
      : "memory");
}

RK_DEV bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for the phase `parity` of bar: at most `limit` polls; false if the
// limit ran out.
RK_DEV bool mbar_wait(uint64_t* bar, uint32_t parity, unsigned limit = kWaitLimit) {
  for (unsigned i = 0; i < limit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// Record that a bounded wait gave up: the error word is a mapped host word or a
// device word; storing 1 is idempotent, so no atomic is needed.
RK_DEV void flag_wait_error(int* err) {
  if (err) {
    *(volatile int*)err = 1;
    __threadfence_system();
  }
}

}  // namespace rk
