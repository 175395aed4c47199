// Device inspector: the counting steps of the band and block extractors on
// the GPU (the host keeps the sequential steps: candidate order, GrowSegments,
// acceptance, FindBlock and Trim).
//  * diag_count_kernel: the diagonal histogram M[d] of Algorithm 3 (residual
//    entries on diagonal d = j - i, |d| <= d_max), a warp per row, atomics.
//  * fit_ribbon_kernel: FitRibbon (Section 4.2, Algorithm 3) for every
//    residual entry on a candidate diagonal at once (the ribbon of row i and
//    offset d starts at the entry (i, i + d)), a warp per row.
//  * hot_cells_kernel: the candidate-region pre-pass of the block extractor:
//    the entries of every tile x tile cell, counted in shared memory one tile
//    row and one column chunk at a time; cells that reach the density floor
//    are appended to a key list.
// Integer arithmetic only.  Each density test the host takes in FP64
// ((z + 1) / w < delta in FitRibbon, c >= delta * area for a hot cell) is a
// comparison of an integer numerator with a threshold that the host computes
// per denominator with the same FP64 expression (the FP64 quotient and product
// are monotone in the numerator), so the device takes the host's decisions.
#include <cuda_runtime.h>

#include <algorithm>

#include "sable_internal.h"
#include "sable_trace.h"

namespace sable {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kThreads = 256;
constexpr int kCellChunk = 16384;   // cell counters per tile row and pass (64 KB)

__global__ void __launch_bounds__(kThreads)
diag_count_kernel(const int64_t *__restrict__ rp, const int32_t *__restrict__ ci, int64_t m, int64_t d_max,
                  unsigned *__restrict__ M) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * (kThreads / 32);
  for (int64_t i = ((int64_t)blockIdx.x * kThreads + threadIdx.x) >> 5; i < m; i += nw) {
    const int64_t e = rp[i + 1];
    for (int64_t k = rp[i] + lane; k < e; k += 32) {
      const int64_t d = (int64_t)ci[k] - i;
      if (d <= d_max && -d <= d_max) atomicAdd(M + (d + m), 1u);
    }
  }
}

// FitRibbon of every residual entry on a candidate diagonal: entry k of row i
// sits at column j = i + d; when cand[d + m] is set, the ribbon of (i, d)
// starts at that entry, so no search is needed.  ext[k] = l | u << 10 |
// z << 20 (z = entries in the final ribbon), 0 for other entries.  zt[w] is
// the least numerator q with q / w >= delta in FP64 (w + 1 if none), so
// "(z + 1) / w < delta" is "z + 1 < zt[w]".  l, u <= w_max <= 512 and
// z <= 2 w_max + 1.  A warp per row, lanes over its entries.
__global__ void __launch_bounds__(kThreads)
fit_ribbon_kernel(const int64_t *__restrict__ rp, const int32_t *__restrict__ ci, int64_t m, int64_t d_max,
                  const unsigned char *__restrict__ cand, int w_max, const int32_t *__restrict__ zt,
                  unsigned *__restrict__ ext) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * (kThreads / 32);
  for (int64_t i = ((int64_t)blockIdx.x * kThreads + threadIdx.x) >> 5; i < m; i += nw) {
    const int64_t b = rp[i], e = rp[i + 1];
    for (int64_t k = b + lane; k < e; k += 32) {
      const int64_t col = ci[k], d = col - i;
      unsigned out = 0;
      if (d <= d_max && -d <= d_max && cand[d + m]) {
        int64_t pl = k, ph = k;                     // first and last entry of the ribbon
        int l = 0, u = 0, z = 1;
        for (;;) {
          int wb = -1, wa = -1, nl = 0, nu = 0;
          if (pl > b && col - ci[pl - 1] <= w_max) {
            nl = (int)(col - ci[pl - 1]);
            wb = nl + u + 1;
          }
          if (ph + 1 < e && ci[ph + 1] - col <= w_max) {
            nu = (int)(ci[ph + 1] - col);
            wa = l + nu + 1;
          }
          if (wb < 0 && wa < 0) break;
          const bool below = wb >= 0 && (wa < 0 || wb <= wa);
          const int w = below ? wb : wa;
          if (z + 1 < zt[w]) break;
          ++z;
          if (below) {
            l = nl;
            --pl;
          } else {
            u = nu;
            ++ph;
          }
        }
        out = (unsigned)l | ((unsigned)u << 10) | ((unsigned)z << 20);
      }
      ext[k] = out;
    }
  }
}

// Tile row I (rows [I g, I g + g)) per CTA iteration.  Rows are sorted by
// column, so each row's entries of a column chunk form a prefix of what is
// left of the row: a per-row cursor walks every entry once.  A chunk starts at
// the cell of the smallest column left in the tile row (empty stretches are
// skipped) and spans kCellChunk cells.  thr[a] is the least count c with
// c >= delta * a in FP64 for a cell of area a.  Keys are I * TJ + J, appended in
// no particular order; `cap` bounds the list (every key has an entry, so
// cap = nnz is never reached).
__global__ void __launch_bounds__(kThreads)
hot_cells_kernel(const int64_t *__restrict__ rp, const int32_t *__restrict__ ci, int64_t m, int64_t n, int g,
                 int64_t TI, int64_t TJ, const int32_t *__restrict__ thr, unsigned long long *__restrict__ keys,
                 unsigned long long *__restrict__ nkeys, int64_t cap) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned *cnt = reinterpret_cast<unsigned *>(smem_raw);
  long long *cur = reinterpret_cast<long long *>(cnt + kCellChunk);   // g cursors
  int *next_col = reinterpret_cast<int *>(cur + g);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int64_t I = blockIdx.x; I < TI; I += gridDim.x) {
    const int64_t r0 = I * g;
    const int R = (int)(m - r0 < g ? m - r0 : g);
    for (int t = threadIdx.x; t < R; t += kThreads) cur[t] = rp[r0 + t];
    for (;;) {
      if (threadIdx.x == 0) *next_col = (int)n;
      __syncthreads();
      for (int t = threadIdx.x; t < R; t += kThreads)
        if (cur[t] < rp[r0 + t + 1]) atomicMin(next_col, ci[cur[t]]);
      for (int t = threadIdx.x; t < kCellChunk; t += kThreads) cnt[t] = 0u;
      __syncthreads();
      const int64_t nc = *next_col;
      if (nc >= n) break;                                      // every row is done (uniform)
      const int64_t J0 = nc / g;
      const int64_t Jn = TJ - J0 < kCellChunk ? TJ - J0 : kCellChunk;   // cells of this chunk
      const int64_t cend = (J0 + Jn) * g < n ? (J0 + Jn) * g : n;   // first column past the chunk
      for (int rr = warp; rr < R; rr += kThreads / 32) {
        long long k = cur[rr];
        const long long e = rp[r0 + rr + 1];
        for (;;) {
          const long long q = k + lane;
          const bool in = q < e && ci[q] < cend;
          if (in) atomicAdd(&cnt[ci[q] / g - J0], 1u);
          const unsigned bal = __ballot_sync(kFull, in);
          if (bal != kFull) {
            k += __popc(bal);
            break;
          }
          k += 32;
        }
        if (lane == 0) cur[rr] = k;
      }
      __syncthreads();
      const int64_t rows_area = R;
      for (int64_t t0 = (int64_t)warp * 32; t0 < Jn; t0 += kThreads) {
        const int64_t t = t0 + lane;
        bool hot = false;
        if (t < Jn) {
          const unsigned v = cnt[t];
          if (v > 0u) {
            const int64_t J = J0 + t;
            const int64_t area = rows_area * (n - J * g < g ? n - J * g : g);
            hot = (int64_t)v >= (int64_t)thr[area];
          }
        }
        const unsigned bal = __ballot_sync(kFull, hot);
        if (bal) {
          unsigned long long base = 0;
          if (lane == 0) base = atomicAdd(nkeys, (unsigned long long)__popc(bal));
          base = __shfl_sync(kFull, base, 0);
          const unsigned long long at = base + __popc(bal & ((1u << lane) - 1u));
          if (hot && (int64_t)at < cap) keys[at] = (unsigned long long)(I * TJ + J0 + t);
        }
      }
      __syncthreads();
    }
  }
}

sable_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return SABLE_OK;
  (void)cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? SABLE_ERR_OOM : SABLE_ERR_CUDA;
}

}  // namespace

struct DevResidual {
  int64_t m = 0, n = 0, nnz = 0;
  int64_t *rp = nullptr;
  int32_t *ci = nullptr;
  cudaStream_t st = nullptr;
  int sm_count = 1;
};

void dev_residual_close(DevResidual *D) {
  if (!D) return;
  if (D->st) (void)cudaStreamSynchronize(D->st);
  cudaFree(D->rp);
  cudaFree(D->ci);
  if (D->st) cudaStreamDestroy(D->st);
  (void)cudaGetLastError();
  delete D;
}

sable_status dev_residual_open(const Csr &R, DevResidual **out) {
  *out = nullptr;
  DevResidual *D = new DevResidual;
  D->m = R.m;
  D->n = R.n;
  D->nnz = R.nnz();
  int dev = 0;
  sable_status s = cuda_status(cudaGetDevice(&dev));
  if (!s) s = cuda_status(cudaDeviceGetAttribute(&D->sm_count, cudaDevAttrMultiProcessorCount, dev));
  if (!s) s = cuda_status(cudaStreamCreateWithFlags(&D->st, cudaStreamNonBlocking));
  if (!s && alloc_fails()) s = SABLE_ERR_OOM;
  if (!s) s = cuda_status(cudaMalloc(&D->rp, (size_t)(D->m + 1) * sizeof(int64_t)));
  if (!s) s = cuda_status(cudaMalloc(&D->ci, (size_t)std::max<int64_t>(D->nnz, 1) * sizeof(int32_t)));
  if (!s)
    s = cuda_status(cudaMemcpyAsync(D->rp, R.rp.data(), (size_t)(D->m + 1) * sizeof(int64_t),
                                    cudaMemcpyHostToDevice, D->st));
  if (!s && D->nnz > 0)
    s = cuda_status(cudaMemcpyAsync(D->ci, R.ci.data(), (size_t)D->nnz * sizeof(int32_t), cudaMemcpyHostToDevice,
                                    D->st));
  if (!s) s = cuda_status(cudaStreamSynchronize(D->st));
  if (s) {
    dev_residual_close(D);
    return s;
  }
  *out = D;
  return SABLE_OK;
}

sable_status dev_diag_counts(DevResidual *D, int64_t d_max, std::vector<int64_t> &M) {
  sable::TraceRange trace_("inspect_diag_counts");
  const int64_t span = D->m + D->n;
  unsigned *dM = nullptr;
  sable_status s = alloc_fails() ? SABLE_ERR_OOM : SABLE_OK;
  if (!s) s = cuda_status(cudaMalloc(&dM, (size_t)(span + 1) * sizeof(unsigned)));
  if (!s) s = cuda_status(cudaMemsetAsync(dM, 0, (size_t)(span + 1) * sizeof(unsigned), D->st));
  if (!s && D->m > 0) {
    const int64_t want = (D->m + kThreads / 32 - 1) / (kThreads / 32);
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)D->sm_count * 8));
    diag_count_kernel<<<grid, kThreads, 0, D->st>>>(D->rp, D->ci, D->m, d_max, dM);
    s = cuda_status(cudaGetLastError());
  }
  std::vector<unsigned> h;
  if (!s) {
    h.resize((size_t)span + 1);
    s = cuda_status(cudaMemcpyAsync(h.data(), dM, h.size() * sizeof(unsigned), cudaMemcpyDeviceToHost, D->st));
  }
  if (!s) s = cuda_status(cudaStreamSynchronize(D->st));
  cudaFree(dM);
  if (s) return s;
  M.assign(h.begin(), h.end());
  return SABLE_OK;
}

sable_status dev_fit_ribbons(DevResidual *D, int64_t d_max, const std::vector<unsigned char> &cand, int w_max,
                             const std::vector<int32_t> &zt, std::vector<uint32_t> &ext) {
  sable::TraceRange trace_("inspect_fit_ribbons");
  ext.assign((size_t)D->nnz, 0u);
  if (D->m == 0 || D->nnz == 0) return SABLE_OK;
  if (w_max < 0 || w_max > 512 || (int64_t)zt.size() < 2 * (int64_t)w_max + 2 ||
      (int64_t)cand.size() < D->m + D->n + 1)
    return SABLE_ERR_INVALID;
  unsigned char *dcand = nullptr;
  int32_t *dzt = nullptr;
  unsigned *dext = nullptr;
  sable_status s = alloc_fails() ? SABLE_ERR_OOM : SABLE_OK;
  if (!s) s = cuda_status(cudaMalloc(&dcand, cand.size()));
  if (!s) s = cuda_status(cudaMalloc(&dzt, zt.size() * sizeof(int32_t)));
  if (!s) s = cuda_status(cudaMalloc(&dext, (size_t)D->nnz * sizeof(unsigned)));
  if (!s) s = cuda_status(cudaMemcpyAsync(dcand, cand.data(), cand.size(), cudaMemcpyHostToDevice, D->st));
  if (!s)
    s = cuda_status(cudaMemcpyAsync(dzt, zt.data(), zt.size() * sizeof(int32_t), cudaMemcpyHostToDevice, D->st));
  if (!s) {
    const int64_t want = (D->m + kThreads / 32 - 1) / (kThreads / 32);
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)D->sm_count * 8));
    fit_ribbon_kernel<<<grid, kThreads, 0, D->st>>>(D->rp, D->ci, D->m, d_max, dcand, w_max, dzt, dext);
    s = cuda_status(cudaGetLastError());
  }
  if (!s)
    s = cuda_status(cudaMemcpyAsync(ext.data(), dext, (size_t)D->nnz * sizeof(unsigned), cudaMemcpyDeviceToHost,
                                    D->st));
  if (!s) s = cuda_status(cudaStreamSynchronize(D->st));
  cudaFree(dcand);
  cudaFree(dzt);
  cudaFree(dext);
  return s;
}

sable_status dev_hot_cells(DevResidual *D, int g, const std::vector<int32_t> &thr, std::vector<int64_t> &hot) {
  sable::TraceRange trace_("inspect_hot_cells");
  hot.clear();
  if (g < 1 || g > 64 || (int64_t)thr.size() < (int64_t)g * g + 1) return SABLE_ERR_INVALID;
  if (D->m == 0 || D->n == 0 || D->nnz == 0) return SABLE_OK;
  const int64_t TI = (D->m + g - 1) / g, TJ = (D->n + g - 1) / g;
  int32_t *dthr = nullptr;
  unsigned long long *dkeys = nullptr, *dcount = nullptr;
  const int64_t cap = D->nnz;
  const size_t smem = (size_t)kCellChunk * sizeof(unsigned) + (size_t)g * sizeof(long long) + 16;
  sable_status s = alloc_fails() ? SABLE_ERR_OOM : SABLE_OK;
  if (!s) s = cuda_status(cudaMalloc(&dthr, thr.size() * sizeof(int32_t)));
  if (!s) s = cuda_status(cudaMalloc(&dkeys, (size_t)cap * sizeof(unsigned long long)));
  if (!s) s = cuda_status(cudaMalloc(&dcount, sizeof(unsigned long long)));
  if (!s)
    s = cuda_status(cudaMemcpyAsync(dthr, thr.data(), thr.size() * sizeof(int32_t), cudaMemcpyHostToDevice, D->st));
  if (!s) s = cuda_status(cudaMemsetAsync(dcount, 0, sizeof(unsigned long long), D->st));
  if (!s)
    s = cuda_status(cudaFuncSetAttribute(hot_cells_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  if (!s) {
    int per_sm = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, hot_cells_kernel, kThreads, smem) != cudaSuccess ||
        per_sm < 1)
      per_sm = 1;
    (void)cudaGetLastError();
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(TI, (int64_t)per_sm * D->sm_count));
    hot_cells_kernel<<<grid, kThreads, smem, D->st>>>(D->rp, D->ci, D->m, D->n, g, TI, TJ, dthr, dkeys, dcount,
                                                       cap);
    s = cuda_status(cudaGetLastError());
  }
  unsigned long long count = 0;
  if (!s) s = cuda_status(cudaMemcpyAsync(&count, dcount, sizeof(count), cudaMemcpyDeviceToHost, D->st));
  if (!s) s = cuda_status(cudaStreamSynchronize(D->st));
  if (!s && (int64_t)count > cap) s = SABLE_ERR_KERNEL;
  std::vector<unsigned long long> h;
  if (!s && count > 0) {
    h.resize((size_t)count);
    s = cuda_status(cudaMemcpyAsync(h.data(), dkeys, (size_t)count * sizeof(unsigned long long),
                                    cudaMemcpyDeviceToHost, D->st));
    if (!s) s = cuda_status(cudaStreamSynchronize(D->st));
  }
  cudaFree(dthr);
  cudaFree(dkeys);
  cudaFree(dcount);
  if (s) return s;
  hot.assign(h.begin(), h.end());
  std::sort(hot.begin(), hot.end());
  return SABLE_OK;
}

}  // namespace sable
