// Tensor-memory-accelerator (TMA) tile loads and shared-memory mbarriers
// for sm_103a, as inline PTX.
//
// A tile load (cp.async.bulk.tensor) copies a box of a tensor in global
// memory into shared memory without passing through registers; the copy
// signals completion on an mbarrier by transaction bytes.  One thread arms
// the barrier with the bytes it expects and issues the copies; every thread
// that reads the tile waits on the barrier's phase.  Waits are bounded: a
// wait that gives up reports it to the caller, which raises an error flag
// instead of spinning for ever.
#pragma once

#include <cuda.h>
#include <stdint.h>

namespace glemur {

// Tensor maps of the fields a mixed-precision mimetic stage reads as tiles:
// the ping-pong displacements (stage 1 input), the two stage-input buffers
// and B0s.  Passed as a __grid_constant__ kernel parameter.
struct TmaMaps {
  CUtensorMap d[2];
  CUtensorMap ys[2];
  CUtensorMap b0;
};

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}

// Make initialised barriers visible to the async (TMA) proxy.
__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}

// Arrive once and add `bytes` to the transaction count the current phase
// waits for (0: the phase completes with this arrival).
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n"
      ".reg .pred p;\n"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      "selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
  return t;
}

// A tile wait gives up after this long (a completed load is seen within
// microseconds).
constexpr uint64_t TMA_WAIT_NS = 500000000ull;

// Wait for the phase of the given parity to complete; false if it has not
// after TMA_WAIT_NS nanoseconds of polling.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer_ns();
  for (int i = 0; i < (1 << 26); ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if (globaltimer_ns() - t0 > TMA_WAIT_NS) return false;
  }
  return false;
}

// 4-D tile load: box at coordinates (c0, c1, c2, c3) of `map` into `dst`
// (128-byte aligned shared memory), completing on `bar`.  c0 times the
// element size must be a multiple of 16 bytes; out-of-range elements are
// filled with zeros.
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int c0, int c1,
                                            int c2, int c3, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];\n" ::"r"(smem_u32(dst)),
      "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
      : "memory");
}

}  // namespace glemur
