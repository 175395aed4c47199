// Calibration kernels: throughput of random 4-byte gathers from a vector, and
// of random row gathers from a dense row-major matrix.
// The CSR part of SpMV reads x at random columns; each such read moves one
// 32-byte L2 sector to an SM, and on GB300 the rate of those sector moves,
// not HBM bandwidth, bounds SpMV on matrices with scattered entries.  This
// kernel measures that rate on the device at hand so that reports can quote
// it beside the HBM figure.  Indices come from a fixed integer hash of the
// gather number, reduced modulo n (never out of range).  The CSR part of SpMM
// reads, per entry, one whole row of the dense operand B; the row probe
// measures the rate of those reads (a warp per row, 8 rows in flight).
#include <cuda_runtime.h>

#include <cstdint>

#include "sable_internal.h"

namespace {

__device__ __forceinline__ unsigned mix32(unsigned a) {
  a ^= a >> 16;
  a *= 0x7feb352du;
  a ^= a >> 15;
  a *= 0x846ca68bu;
  a ^= a >> 16;
  return a;
}

__global__ void __launch_bounds__(256) gather_probe_kernel(const float *__restrict__ x, unsigned n,
                                                           long long count, float *out) {
  const long long stride = (long long)gridDim.x * blockDim.x * 8;
  float acc = 0.f;
  for (long long i = ((long long)blockIdx.x * blockDim.x + threadIdx.x) * 8; i < count; i += stride) {
#pragma unroll
    for (int e = 0; e < 8; ++e)
      if (i + e < count) acc += __ldg(x + mix32((unsigned)(i + e)) % n);
  }
  if (acc == 1.2345e-30f) out[0] = acc;   // keeps the loads; practically never taken
}

// count random rows of B (row-major, leading dimension ld floats), N <= 128
// columns each, N and ld multiples of 4, B 16-byte aligned: lane l reads the
// float4 at column 4l when 4l < N.  As in the SpMM kernel, each lane computes
// one of the warp's next 32 row indices and the warp walks them by shuffles,
// 8 rows in flight.
__global__ void __launch_bounds__(256, 5) row_gather_probe_kernel(const float *__restrict__ B, unsigned n,
                                                               long long ld, int N, long long count,
                                                               float *out) {
  const int lane = threadIdx.x & 31;
  const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
  const long long w = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const bool on = 4 * lane < N;
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  for (long long i = w * 32; i < count; i += warps * 32) {
    const unsigned mine = i + lane < count ? mix32((unsigned)(i + lane)) % n : 0u;
    const int cnt = (int)(count - i < 32 ? count - i : 32);
    for (int j = 0; j < cnt; j += 8) {
      float4 v[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const unsigned r = __shfl_sync(0xffffffffu, mine, j + e);
        v[e] = (on && j + e < cnt) ? __ldg(reinterpret_cast<const float4 *>(B + (long long)r * ld) + lane)
                                   : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        acc.x += v[e].x;
        acc.y += v[e].y;
        acc.z += v[e].z;
        acc.w += v[e].w;
      }
    }
  }
  if (acc.x + acc.y + acc.z + acc.w == 1.2345e-30f) out[0] = acc.x;   // keeps the loads
}

}  // namespace

extern "C" sable_status sable_probe_row_gather(const float *B, int64_t n, int64_t ld, int32_t N, int64_t count,
                                               float *out, void *stream) {
  if (!B || !out || n < 1 || n > 0xffffffffLL || N < 4 || N > 128 || N % 4 || ld < N || ld % 4 ||
      (reinterpret_cast<uintptr_t>(B) & 15) || count < 0)
    return SABLE_ERR_INVALID;
  int dev = 0, sms = 1;
  if (cudaGetDevice(&dev) != cudaSuccess) return SABLE_ERR_CUDA;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int per_sm = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, row_gather_probe_kernel, 256, 0) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  row_gather_probe_kernel<<<sms * per_sm, 256, 0, (cudaStream_t)stream>>>(B, (unsigned)n, ld, N, count, out);
  return cudaGetLastError() == cudaSuccess ? SABLE_OK : SABLE_ERR_CUDA;
}

extern "C" sable_status sable_probe_gather(const float *x, int64_t n, int64_t count, float *out,
                                           void *stream) {
  if (!x || !out || n < 1 || n > 0xffffffffLL || count < 0) return SABLE_ERR_INVALID;
  int dev = 0, sms = 1;
  if (cudaGetDevice(&dev) != cudaSuccess) return SABLE_ERR_CUDA;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  gather_probe_kernel<<<sms * 8, 256, 0, (cudaStream_t)stream>>>(x, (unsigned)n, count, out);
  return cudaGetLastError() == cudaSuccess ? SABLE_OK : SABLE_ERR_CUDA;
}
