// Bounded mbarrier waits shared by the kernels that wait on asynchronous
// copies or tensor-core work.  Every wait gives up after a cycle budget (the
// process-wide limit set by sable_set_wait_limit, read at each launch), so a
// wait that is never satisfied ends with an error status instead of a hang.
#pragma once

#include <cstdint>

namespace sable {

__device__ __forceinline__ unsigned smem_u32(const void *p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t *bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// true once the phase of the given parity has completed; false after `limit`
// clock cycles without it
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity, long long limit) {
  if (mbar_try(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try(bar, parity))
    if (clock64() - t0 > limit) return false;
  return true;
}

// After a wait ran out, a kernel still waits for its own copies or
// tensor-core work in flight before it leaves: with at least this budget
// (about 2 s), whatever the caller's limit, since such work normally ends in
// microseconds.
__device__ __forceinline__ long long drain_limit(long long limit) {
  const long long floor_cycles = 4000000000LL;
  return limit > floor_cycles ? limit : floor_cycles;
}

// Host: the current wait budget in clock cycles (sable_set_wait_limit).
long long wait_limit_cycles();

}  // namespace sable
