// Accuracy check on the device: the error of an FP32 result against an FP64
// reference, reduced in FP64 (the only FP64 arithmetic on the device).  The
// grid is fixed and both reduction stages run in a fixed order, so the sums
// do not depend on the GPU or on scheduling.
#include <cuda_runtime.h>

#include <cmath>

#include "sable_internal.h"

namespace sable {
namespace {

constexpr int kBlocks = 512, kThreads = 256;

struct Acc {
  double emax, rmax, e2, r2;
};

// maximum in which a NaN wins, so that a NaN in the result shows in the error
__device__ __forceinline__ double nanmax(double a, double b) { return (b > a || b != b) && a == a ? b : a; }

__device__ __forceinline__ Acc combine(Acc a, const Acc &b) {
  a.emax = nanmax(a.emax, b.emax);
  a.rmax = nanmax(a.rmax, b.rmax);
  a.e2 += b.e2;
  a.r2 += b.r2;
  return a;
}

// tree over the block's threads, lowest index first at every level
__device__ Acc block_reduce(Acc a, Acc *sh) {
  const int t = threadIdx.x;
  sh[t] = a;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (t < s) sh[t] = combine(sh[t], sh[t + s]);
    __syncthreads();
  }
  return sh[0];
}

__global__ void __launch_bounds__(kThreads) err_partial(const float *__restrict__ y, const double *__restrict__ ref,
                                                        int64_t count, Acc *__restrict__ part) {
  __shared__ Acc sh[kThreads];
  Acc a{0.0, 0.0, 0.0, 0.0};
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < count; i += (int64_t)kBlocks * kThreads) {
    const double r = ref[i], e = (double)y[i] - r;
    a.emax = nanmax(a.emax, fabs(e));
    a.rmax = nanmax(a.rmax, fabs(r));
    a.e2 = fma(e, e, a.e2);
    a.r2 = fma(r, r, a.r2);
  }
  const Acc b = block_reduce(a, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = b;
}

__global__ void __launch_bounds__(kBlocks) err_final(const Acc *__restrict__ part, double *__restrict__ out) {
  __shared__ Acc sh[kBlocks];
  const Acc b = block_reduce(part[threadIdx.x], sh);
  if (threadIdx.x == 0) {
    out[0] = b.emax;
    out[1] = b.rmax;
    out[2] = b.e2;
    out[3] = b.r2;
  }
}

}  // namespace
}  // namespace sable

using namespace sable;

extern "C" {

int64_t sable_error_workspace_bytes(void) { return (int64_t)(kBlocks * sizeof(Acc)); }

sable_status sable_error_norms(const float *y, const double *ref, int64_t count, double *out, void *work,
                               int64_t work_bytes, void *stream) {
  if (count < 0 || !out || !work || (count > 0 && (!y || !ref)) || work_bytes < sable_error_workspace_bytes())
    return SABLE_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  Acc *part = static_cast<Acc *>(work);
  err_partial<<<kBlocks, kThreads, 0, st>>>(y, ref, count, part);
  err_final<<<1, kBlocks, 0, st>>>(part, out);
  return cudaGetLastError() == cudaSuccess ? SABLE_OK : SABLE_ERR_CUDA;
}

}  // extern "C"
