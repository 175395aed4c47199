// Index checks of the debug build (compiled with SABLE_CHECKS): before each
// gather whose index comes from the plan's tables (a CSR column, a block
// column), the hot kernels test it against the matrix's column count.  A bad
// index is recorded in the plan's device error word — SABLE_ERR_KERNEL, then
// the check's tag, the index and its bound; the first one recorded stays —
// and the access is skipped (the entry contributes nothing).  Without
// SABLE_CHECKS every test is the constant true and the kernels are the
// release kernels.
#pragma once

#include <cstdint>

namespace sable {

enum CheckTag : int32_t {
  kCheckSpmvCsr = 1,    // SpMV, CSR remainder column
  kCheckSpmvBlock = 2,  // SpMV, VBR block column
  kCheckSpmmCsr = 3,    // SpMM row kernel, CSR remainder column
  kCheckSpmmBlock = 4   // SpMM row kernel, FP32 block column
};

#ifdef SABLE_CHECKS
__device__ __forceinline__ bool index_ok(int32_t *err, int32_t tag, long long idx, long long bound) {
  if (idx >= 0 && idx < bound) return true;
  if (err != nullptr && atomicCAS(err, 0, 7) == 0) {   // 7 = SABLE_ERR_KERNEL
    err[1] = tag;
    err[2] = (int32_t)idx;
    err[3] = (int32_t)bound;
  }
  return false;
}
#else
__device__ __forceinline__ constexpr bool index_ok(int32_t *, int32_t, long long, long long) { return true; }
#endif

}  // namespace sable
