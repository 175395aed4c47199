// FindBlock (Section 4.1, Algorithm 2) on the device: the inspector's most
// expensive step, for the large candidate regions of big matrices.
//
// One warp per outer start o0.  The warp keeps the histogram H of Algorithm 2
// (entries of the lines o0 .. o1 per inner position) in shared memory: each
// line's entries inside the inner range are added by the lanes (shared
// atomics), and warp reductions keep the tallest bin, the total and the
// occupied range.  The host's exact span prunings are applied as on the host
// (a span whose every window density is below delta, or whose best possible
// score cannot exceed the warp's best), plus one more: a span whose best
// possible score is below the best score any warp has recorded so far (a
// global maximum, strict margin) cannot hold the region's answer.  Lane 0
// then runs Algorithm 2's window scan over H exactly as the host does, with
// the score compared through its square (nnz - delta a)^3 / a in explicitly
// rounded IEEE operations, so host and device choose the same window.  The
// host merges the per-o0 results: highest score, then lowest o0.
//
// Measured on GB300 against the host search (16 threads of the Grace host) on
// the 200k x 200k block workload: same 820 blocks, 32.7 s against 7.2 s.  The
// window scan is sequential per start and a region offers only a few hundred
// starts, so the device search stays an option (device_search = 1), off by
// default.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <stdexcept>

#include "sable_internal.h"

namespace sable {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kWarpsPerBlock = 4;
constexpr int kMaxInner = 4096;          // histogram bins per warp (shared memory)

struct DevFound {
  double sc;
  int32_t o1, i0, i1, pad;
};

__device__ __forceinline__ double score2_dev(long long nnz, long long a, double delta) {
  double t = __dsub_rn((double)nnz, __dmul_rn(delta, (double)a));
  if (t < 0.0) t = 0.0;
  return __ddiv_rn(__dmul_rn(__dmul_rn(t, t), t), (double)a);
}

__global__ void __launch_bounds__(32 * kWarpsPerBlock)
find_block_kernel(const int32_t *__restrict__ rp, const int32_t *__restrict__ ci, int O0, int O1, int I0, int I1,
                  int max_span, int s_min, long long a_min, double delta, double ub_unit, DevFound *out,
                  unsigned long long *gbest) {
  extern __shared__ int hsm[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int L = I1 - I0;
  int *H = hsm + wib * L;
  const int o0 = O0 + blockIdx.x * kWarpsPerBlock + wib;
  if (o0 >= O1) return;   // the whole warp leaves; no block-wide barrier follows
  for (int i = lane; i < L; i += 32) H[i] = 0;
  __syncwarp();
  double bsc = -1.0;      // lane 0's record
  int bo1 = 0, bi0 = 0, bi1 = 0;
  int hmax = 0, tmin = INT_MAX, tmax = -1;
  long long total = 0;
  const int oend = min(O1, o0 + max_span);
  for (int o1 = o0; o1 < oend; ++o1) {
    const int b = rp[o1], e = rp[o1 + 1];
    int lb = b;
    if (lane == 0) {        // first entry of the line at or after I0
      int lo = b, hi = e;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (ci[mid] < I0) lo = mid + 1;
        else hi = mid;
      }
      lb = lo;
    }
    lb = __shfl_sync(kFull, lb, 0);
    int lh = 0, lmin = INT_MAX, lmax = -1, lcnt = 0;
    for (int q = lb + lane; q < e; q += 32) {
      const int c = ci[q];
      if (c >= I1) break;   // the line is sorted: this lane's later entries are past I1 too
      const int rel = c - I0;
      const int h = atomicAdd(&H[rel], 1) + 1;
      lh = max(lh, h);
      lmin = min(lmin, rel);
      lmax = max(lmax, rel);
      ++lcnt;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      lh = max(lh, __shfl_xor_sync(kFull, lh, o));
      lmin = min(lmin, __shfl_xor_sync(kFull, lmin, o));
      lmax = max(lmax, __shfl_xor_sync(kFull, lmax, o));
      lcnt += __shfl_xor_sync(kFull, lcnt, o);
    }
    __syncwarp();           // every lane's shared-memory additions are visible below
    hmax = max(hmax, lh);
    tmin = min(tmin, lmin);
    tmax = max(tmax, lmax);
    total += lcnt;
    const int s = o1 - o0 + 1;
    if (s < s_min || tmax < 0) continue;
    if ((double)hmax < __dmul_rn(delta, (double)s)) continue;
    double ub;
    if (total >= a_min) ub = __dmul_rn(__dmul_rn((double)total, (double)total), ub_unit);
    else if ((double)total >= __dmul_rn(delta, (double)a_min)) ub = score2_dev(total, a_min, delta);
    else continue;
    const double mine = __shfl_sync(kFull, bsc, 0);
    if (mine >= 0.0 && ub * (1.0 + 1e-9) <= mine) continue;
    double g = 0.0;         // one read, broadcast: the branch must be the same in every lane
    if (lane == 0) g = __longlong_as_double((long long)atomicAdd(gbest, 0ull));
    g = __shfl_sync(kFull, g, 0);
    if (g > 0.0 && ub * (1.0 + 1e-9) < g) continue;
    if (lane == 0) {
      const long long w_small = (a_min + s - 1) / s - 1;   // widest window with area < a_min
      int i0 = tmin - (int)min((long long)tmin, w_small);
      long long nnz = 0;
      for (int i1 = tmin; i1 < L; ++i1) {
        nnz += H[i1];
        while (i0 <= i1) {
          const long long a = (long long)s * (i1 - i0 + 1);
          if (a < a_min) break;
          if (__ddiv_rn((double)nnz, (double)a) >= delta) {
            const double sc = score2_dev(nnz, a, delta);
            if (sc > bsc) {
              bsc = sc;
              bo1 = o1 + 1;
              bi0 = I0 + i0;
              bi1 = I0 + i1 + 1;
            }
            break;
          }
          nnz -= H[i0];
          ++i0;
        }
        if (i1 >= tmax && nnz == 0) break;
      }
    }
    __syncwarp();
  }
  if (lane == 0) {
    DevFound f;
    f.sc = bsc;
    f.o1 = bo1;
    f.i0 = bi0;
    f.i1 = bi1;
    f.pad = 0;
    out[o0 - O0] = f;
    if (bsc > 0.0) atomicMax(gbest, (unsigned long long)__double_as_longlong(bsc));
  }
}

void check(cudaError_t e) {
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    throw std::runtime_error(cudaGetErrorString(e));
  }
}

}  // namespace

struct DeviceLines {
  int32_t *rp = nullptr, *ci = nullptr;
  int64_t m = 0;
  DevFound *out = nullptr, *h_out = nullptr;
  int64_t cap = 0;
  unsigned long long *gbest = nullptr;
  cudaStream_t st = nullptr;
};

DeviceLines *device_lines(const Csr &M) {
  DeviceLines *D = new DeviceLines();
  try {
    D->m = M.m;
    std::vector<int32_t> rp32(M.rp.begin(), M.rp.end());
    check(cudaStreamCreateWithFlags(&D->st, cudaStreamNonBlocking));
    check(cudaMalloc(&D->rp, rp32.size() * 4));
    check(cudaMalloc(&D->ci, std::max<size_t>(M.ci.size(), 1) * 4));
    check(cudaMalloc(&D->gbest, 8));
    check(cudaMemcpy(D->rp, rp32.data(), rp32.size() * 4, cudaMemcpyHostToDevice));
    if (!M.ci.empty()) check(cudaMemcpy(D->ci, M.ci.data(), M.ci.size() * 4, cudaMemcpyHostToDevice));
  } catch (...) {
    device_lines_free(D);
    throw;
  }
  return D;
}

void device_lines_free(DeviceLines *D) {
  if (!D) return;
  cudaFree(D->rp);
  cudaFree(D->ci);
  cudaFree(D->out);
  cudaFree(D->gbest);
  cudaFreeHost(D->h_out);
  if (D->st) cudaStreamDestroy(D->st);
  (void)cudaGetLastError();
  delete D;
}

bool find_block_device(DeviceLines *D, int64_t O0, int64_t O1, int64_t I0, int64_t I1,
                       const sable_extract_params &p, int64_t s_min, FindBest &best) {
  const int64_t count = O1 - O0, L = I1 - I0;
  if (!D || count < 128 || L < 1 || L > kMaxInner || O1 > D->m || O1 >= INT32_MAX || I1 >= INT32_MAX) return false;
  if (count > D->cap) {
    cudaFree(D->out);
    cudaFreeHost(D->h_out);
    D->out = nullptr;
    D->h_out = nullptr;
    D->cap = 0;
    check(cudaMalloc(&D->out, count * sizeof(DevFound)));
    check(cudaMallocHost(&D->h_out, count * sizeof(DevFound)));
    D->cap = count;
  }
  const double omd = 1.0 - p.delta;
  const size_t smem = (size_t)kWarpsPerBlock * L * sizeof(int);
  check(cudaFuncSetAttribute(find_block_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  check(cudaMemsetAsync(D->gbest, 0, 8, D->st));
  const int grid = (int)((count + kWarpsPerBlock - 1) / kWarpsPerBlock);   // one warp per start
  find_block_kernel<<<grid, 32 * kWarpsPerBlock, smem, D->st>>>(
      D->rp, D->ci, (int)O0, (int)O1, (int)I0, (int)I1, p.max_span, (int)s_min, (long long)p.a_min, p.delta,
      omd * omd * omd, D->out, D->gbest);
  check(cudaGetLastError());
  check(cudaMemcpyAsync(D->h_out, D->out, count * sizeof(DevFound), cudaMemcpyDeviceToHost, D->st));
  check(cudaStreamSynchronize(D->st));
  FindBest b;
  for (int64_t k = 0; k < count; ++k) {      // highest score, then lowest o0
    const DevFound &f = D->h_out[k];
    if (f.sc >= 0.0 && f.sc > b.sc) b = FindBest{f.sc, O0 + k, f.o1, f.i0, f.i1};
  }
  best = b;
  return true;
}

}  // namespace sable
