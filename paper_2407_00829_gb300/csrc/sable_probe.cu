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

#include <atomic>
#include <cstdint>

#include "sable_internal.h"
#include "sable_wait.cuh"

namespace sable {
namespace {
std::atomic<long long> g_wait_limit{4000000000LL};   // ~2 s at 2 GHz
}
long long wait_limit_cycles() { return g_wait_limit.load(std::memory_order_relaxed); }
}  // namespace sable

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

// Random 16-byte chunks of x copied to shared memory by the bulk-copy
// (TMA) unit instead of the load path: chunk mix32(i) % nchunks of x (16-byte
// aligned, nchunks = n / 4), 256 copies per round per CTA, two rounds in
// flight on two mbarriers.  Every wait is bounded; a wait that runs out
// records SABLE_ERR_TIMEOUT in *status, and the CTA still waits (bounded,
// sable::drain_limit) for the copies it issued before it exits.
constexpr int kBulkThreads = 128, kBulkPer = 2, kBulkRound = kBulkThreads * kBulkPer;

__global__ void __launch_bounds__(kBulkThreads) bulk_gather_probe_kernel(const float *__restrict__ x, unsigned nchunks,
                                                                        long long count, long long limit,
                                                                        float *out, int *status) {
  __shared__ __align__(128) float4 buf[2][kBulkRound];
  __shared__ __align__(8) uint64_t bar[2];
  const int tid = threadIdx.x;
  if (tid == 0) {
    sable::mbar_init(&bar[0], 1);
    sable::mbar_init(&bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const long long rounds = (count + kBulkRound - 1) / kBulkRound;
  unsigned ph[2] = {0u, 0u};
  bool pend[2] = {false, false};
  float acc = 0.f;
  bool ok = true;
  int k = 0;
  for (long long r = blockIdx.x; r < rounds; r += gridDim.x, ++k) {
    const int s = k & 1;
    if (pend[s]) {   // the round issued two rounds ago into this slot
      const bool got = sable::mbar_wait(&bar[s], ph[s], limit);
      if (got) {
        ph[s] ^= 1u;
        pend[s] = false;
        acc += buf[s][tid].x + buf[s][tid + kBulkThreads].x;
      }
      ok = __syncthreads_and(got) != 0;
      if (!ok) break;
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic reads before async writes
    }
    const long long base = r * kBulkRound;
    const int nvalid = (int)(count - base < kBulkRound ? count - base : kBulkRound);
    if (tid == 0)
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(sable::smem_u32(&bar[s])),
                   "r"((unsigned)(16 * nvalid))
                   : "memory");
    __syncthreads();   // the byte count is expected before any copy lands
    pend[s] = true;
#pragma unroll
    for (int e = 0; e < kBulkPer; ++e) {
      const int idx = tid + e * kBulkThreads;
      if (idx < nvalid) {
        const float *src = x + 4ull * (mix32((unsigned)(base + idx)) % nchunks);
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], 16, [%2];" ::"r"(
                sable::smem_u32(&buf[s][idx])),
            "l"(src), "r"(sable::smem_u32(&bar[s]))
            : "memory");
      }
    }
  }
  // every issued copy lands before the CTA leaves (bounded again, longer)
  for (int s = 0; s < 2; ++s)
    if (pend[s] && !sable::mbar_wait(&bar[s], ph[s], sable::drain_limit(limit))) ok = false;
  if (!ok && tid == 0) atomicExch(status, (int)SABLE_ERR_TIMEOUT);
  if (acc == 1.2345e-30f) out[0] = acc;   // keeps the copies' results live
}

// A wait nothing satisfies: an mbarrier expecting one arrival that never
// comes, waited on with the given budget.  Writes SABLE_ERR_TIMEOUT to
// *status when the budget runs out (always, unless the budget is huge), 0
// otherwise.  No copy or tensor-core work is in flight.
__global__ void wait_limit_probe_kernel(long long limit, int *status) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    sable::mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const bool got = sable::mbar_wait(&bar, 0u, limit);
  if (threadIdx.x == 0) *status = got ? 0 : (int)SABLE_ERR_TIMEOUT;
}

}  // namespace

extern "C" sable_status sable_set_wait_limit(int64_t cycles) {
  if (cycles < 1000 || cycles > (int64_t)1 << 40) return SABLE_ERR_INVALID;
  sable::g_wait_limit.store(cycles, std::memory_order_relaxed);
  return SABLE_OK;
}

extern "C" int64_t sable_get_wait_limit(void) { return sable::wait_limit_cycles(); }

extern "C" sable_status sable_probe_wait_limit(int32_t *status, void *stream) {
  if (!status) return SABLE_ERR_INVALID;
  wait_limit_probe_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(sable::wait_limit_cycles(), status);
  return cudaGetLastError() == cudaSuccess ? SABLE_OK : SABLE_ERR_CUDA;
}

extern "C" sable_status sable_probe_bulk_gather(const float *x, int64_t n, int64_t count, float *out, int32_t *status,
                                                void *stream) {
  if (!x || !out || !status || n < 4 || n > 0xffffffffLL || count < 0 || (reinterpret_cast<uintptr_t>(x) & 15))
    return SABLE_ERR_INVALID;
  int dev = 0, sms = 1;
  if (cudaGetDevice(&dev) != cudaSuccess) return SABLE_ERR_CUDA;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int per_sm = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bulk_gather_probe_kernel, kBulkThreads, 0) !=
          cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  if (cudaMemsetAsync(status, 0, sizeof(int32_t), (cudaStream_t)stream) != cudaSuccess) return SABLE_ERR_CUDA;
  bulk_gather_probe_kernel<<<sms * per_sm, kBulkThreads, 0, (cudaStream_t)stream>>>(
      x, (unsigned)(n / 4), count, sable::wait_limit_cycles(), out, status);
  return cudaGetLastError() == cudaSuccess ? SABLE_OK : SABLE_ERR_CUDA;
}

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
