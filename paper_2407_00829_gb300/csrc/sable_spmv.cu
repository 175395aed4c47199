// Hybrid VDIA+VBR+CSR SpMV: one launch over a table of row tiles.
//
// A CTA owns a row tile [r0, r1) (at most 4 x kThreads rows) and writes each
// of its rows of y exactly once (row ownership; the paper instead accumulates
// every dispatch into a shared output, Section 3.4).  Per tile:
//   A. VDIA: every segment piece touching the rows (Section 4.2.1 layout:
//      diagonal-major runs, padded to 16-byte alignment); a thread owns 4
//      consecutive rows, so each diagonal's values arrive as one float4 and x
//      is read as 4 consecutive words.  Sums stay in registers, then seed the
//      tile's row accumulators in shared memory.
//   B. VBR: every block touching the rows (column-major, Appendix B); lanes
//      own rows, warps split the columns, partial sums go in with shared
//      atomics.
//   C. CSR remainder: the tile's entries are one contiguous range, streamed
//      4 per thread with vector loads; a thread finds the row of its first
//      entry by binary search in the tile's row pointers (shared memory),
//      sums runs of equal rows, and a warp segmented scan merges partial sums
//      across lanes before the shared atomics.
// Eight CTAs per SM work on different tiles, so one tile's VDIA phase
// overlaps other tiles' gathers.  On GB300 the CSR gathers of x (random 4-byte
// reads, one 32-byte L2 sector each) and the streamed arrays share the
// L2-to-SM sector bandwidth, which bounds this kernel (see the bench report).
#include <cuda_runtime.h>

#include <algorithm>

#include "sable_checks.cuh"
#include "sable_internal.h"

namespace sable {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kThreads = 256;

// Streamed operands (VDIA values, CSR values and columns) are read once: they
// bypass L1 allocation, which leaves L1 to the x gathers that hit it.
__device__ __forceinline__ float4 ld_stream_f4(const float *p) {
  float4 r;
  asm("ld.global.nc.L1::no_allocate.v4.f32 {%0,%1,%2,%3}, [%4];"
      : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w)
      : "l"(p));
  return r;
}
__device__ __forceinline__ int4 ld_stream_i4(const int *p) {
  int4 r;
  asm("ld.global.nc.L1::no_allocate.v4.s32 {%0,%1,%2,%3}, [%4];"
      : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
      : "l"(p));
  return r;
}

// CUT: the launch's tile table may hold partial tiles (single-plan launches;
// a batch refuses plans with cut tiles)
template <bool PLAIN, bool CUT>
__device__ __forceinline__ void spmv_tile(const DevHybrid &A, const DevItems &T, const DevItem &I, int it,
                                          const float *__restrict__ x, float *__restrict__ y, float *ys,
                                          int *rps) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int NW = kThreads / 32;
  const unsigned n = (unsigned)A.n;
  {
    const int r0 = I.r0, R = I.r1 - I.r0;
    // row pointers clamped to the tile's CSR range: a no-op for a whole tile;
    // for a cut tile (its first chunk, or a partial tile) only the chunk's
    // entries remain, each in its own row
    for (int i = tid; i <= R; i += kThreads) rps[i] = min(max(__ldg(A.rp + r0 + i), I.pb), I.pe);

    // ---- A. VDIA: a quad of 4 consecutive rows; when the tile has fewer
    // quads than threads, S threads (adjacent lanes) split the quad's
    // diagonals and their partial sums meet by warp shuffles
    const int Q = (R + 3) >> 2;
    int S = 1;
    while (S < 32 && 2 * S * Q <= kThreads) S *= 2;
    const int q4 = tid / S, jj = tid & (S - 1);
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
    const int my = r0 + 4 * q4;
    if (!PLAIN && q4 < Q)
      for (int q = I.seg_lo; q < I.seg_hi; ++q) {
        const DevSeg s = T.pseg[q];
        const int ra = max(r0, s.row0), rb = min(I.r1, s.row0 + s.nrows);
        if (my + 3 < ra || my >= rb) continue;
        const bool g0 = my >= ra && my < rb, g1 = my + 1 >= ra && my + 1 < rb;
        const bool g2 = my + 2 >= ra && my + 2 < rb, g3 = my + 3 >= ra && my + 3 < rb;
        const float *vp = A.vdia + s.val_off + (my - s.base);
        const int c0 = my + s.off_lo;
#pragma unroll 1
        for (int k = jj; k < s.ndiag; k += S) {
          const float4 v = ld_stream_f4(vp + (size_t)k * s.ld);
          const int c = c0 + k;
          const float x0 = (g0 && (unsigned)c < n) ? __ldg(x + c) : 0.f;
          const float x1 = (g1 && (unsigned)(c + 1) < n) ? __ldg(x + c + 1) : 0.f;
          const float x2 = (g2 && (unsigned)(c + 2) < n) ? __ldg(x + c + 2) : 0.f;
          const float x3 = (g3 && (unsigned)(c + 3) < n) ? __ldg(x + c + 3) : 0.f;
          a0 = fmaf(v.x, x0, a0);
          a1 = fmaf(v.y, x1, a1);
          a2 = fmaf(v.z, x2, a2);
          a3 = fmaf(v.w, x3, a3);
        }
      }
    for (int o = S >> 1; o > 0; o >>= 1) {   // S is uniform over the CTA: every lane takes part
      a0 += __shfl_xor_sync(kFull, a0, o);
      a1 += __shfl_xor_sync(kFull, a1, o);
      a2 += __shfl_xor_sync(kFull, a2, o);
      a3 += __shfl_xor_sync(kFull, a3, o);
    }
    if (jj == 0 && q4 < Q) {
      const int i = 4 * q4;
      ys[i] = a0;
      if (i + 1 < R) ys[i + 1] = a1;
      if (i + 2 < R) ys[i + 2] = a2;
      if (i + 3 < R) ys[i + 3] = a3;
    }
    __syncthreads();

    // ---- B. VBR: lanes over rows, warps over columns
    if (!PLAIN)
      for (int q = I.blk_lo; q < I.blk_hi; ++q) {
        const DevBlk b = T.pblk[q];
        const int ra = max(r0, b.r0), rb = min(I.r1, b.r0 + b.nr);
        for (int rr = ra + lane; rr < rb; rr += 32) {
          const float *bp = A.vbr + b.val_off + (rr - b.r0);
          const float *xp = x + b.c0;
          float acc = 0.f;
          for (int c = warp; c < b.nc; c += NW)
            if (index_ok(A.err, kCheckSpmvBlock, (long long)b.c0 + c, n))
              acc = fmaf(__ldg(bp + (size_t)c * b.nr), __ldg(xp + c), acc);
          atomicAdd(&ys[rr - r0], acc);
        }
      }

    // ---- C. CSR remainder: 4 entries per thread, warp segmented scan
    const int pb = rps[0], pe = rps[R];
    for (int base = pb & ~3; base < pe; base += 4 * kThreads) {
      const int p0 = base + 4 * tid;
      int row = -1 - lane;
      float run = 0.f;
      if (p0 < pe && p0 + 4 > pb) {
        const float4 v = ld_stream_f4(A.cv + p0);
        const int4 c = ld_stream_i4(A.ci + p0);
        const int pf = max(p0, pb);
        int lo = 0, hi = R;                 // rps[lo] <= pf < rps[hi]
        while (hi - lo > 1) {
          const int mid = (lo + hi) >> 1;
          if (rps[mid] <= pf) lo = mid;
          else hi = mid;
        }
        int cur = lo, nxt = rps[lo + 1], cnt = 0;
        float vv[4] = {v.x, v.y, v.z, v.w};
        int cc[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
        for (int e = 0; e < 4; ++e)   // debug build: a column outside the matrix contributes nothing
          if (p0 + e >= pb && p0 + e < pe && !index_ok(A.err, kCheckSpmvCsr, cc[e], n)) {
            cc[e] = 0;
            vv[e] = 0.f;
          }
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int pp = p0 + e;
          if (pp >= pb && pp < pe) {
            while (pp >= nxt) {
              if (cnt) atomicAdd(&ys[cur], run);
              run = 0.f;
              cnt = 0;
              ++cur;
              nxt = rps[cur + 1];
            }
            run = fmaf(vv[e], __ldg(x + cc[e]), run);
            ++cnt;
          }
        }
        row = cur;
      }
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const float s2 = __shfl_up_sync(kFull, run, d);
        const int r2 = __shfl_up_sync(kFull, row, d);
        if (lane >= d && r2 == row) run += s2;
      }
      const int rn = __shfl_down_sync(kFull, row, 1);
      if (row >= 0 && (lane == 31 || rn != row)) atomicAdd(&ys[row], run);
    }
    __syncthreads();
    const int part = CUT ? __ldg(&T.items[it].part) : 0;   // read again here, not held through the phases
    if (part == 0)
      for (int i = tid; i < R; i += kThreads) y[r0 + i] = ys[i];
    else   // a partial tile: its row sums go to the part slots, added to y by spmv_fixup_kernel
      for (int i = tid; i < R; i += kThreads) T.part[part - 1 + i] = ys[i];
    __syncthreads();
  }
}

// One matrix: tiles A.spmv.items[blockIdx.x + k gridDim.x].
template <bool PLAIN>
__global__ void __launch_bounds__(kThreads, 8)
spmv_hybrid_kernel(const __grid_constant__ DevHybrid A, const float *__restrict__ x, float *__restrict__ y) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float *ys = reinterpret_cast<float *>(smem_raw);
  int *rps = reinterpret_cast<int *>(ys + A.spmv.rows_max);
  for (int it = blockIdx.x; it < A.spmv.n; it += gridDim.x) {
    const DevItem I = A.spmv.items[it];
    spmv_tile<PLAIN, true>(A, A.spmv, I, it, x, y, ys, rps);
  }
}

// Many matrices in one launch: the grouped tile table carries each tile's
// matrix index; xs / ys hold one device pointer per matrix.
__global__ void __launch_bounds__(kThreads, 8)
spmv_grouped_kernel(const DevHybrid *__restrict__ mats, const DevItem *__restrict__ items, int n_items,
                    int rows_max, const float *const *__restrict__ xs, float *const *__restrict__ yv) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float *ys = reinterpret_cast<float *>(smem_raw);
  int *rps = reinterpret_cast<int *>(ys + rows_max);
  for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
    const DevItem I = items[it];
    const DevHybrid &A = mats[I.mat];
    spmv_tile<false, false>(A, A.spmv, I, it, xs[I.mat], yv[I.mat], ys, rps);
  }
}

// y[r] += the partial row sums of the cut tiles, in partial-tile order: a warp
// per cut tile, lanes over its rows.  Runs after spmv_hybrid_kernel on the
// same stream (the owning tiles have stored their rows by then).
__global__ void __launch_bounds__(kThreads)
spmv_fixup_kernel(const int32_t *__restrict__ fix, int n_fix, const float *__restrict__ part,
                  float *__restrict__ y) {
  const int lane = threadIdx.x & 31;
  const int nw = gridDim.x * (kThreads / 32);
  for (int f = (blockIdx.x * kThreads + threadIdx.x) >> 5; f < n_fix; f += nw) {
    const int r0 = fix[4 * f], R = fix[4 * f + 1], first = fix[4 * f + 2], np = fix[4 * f + 3];
    for (int i = lane; i < R; i += 32) {
      float acc = 0.f;
      for (int k = 0; k < np; ++k) acc += part[first + k * R + i];
      y[r0 + i] += acc;
    }
  }
}

int spmv_resident_ctas(int rows_max) {
  const size_t smem = (size_t)rows_max * 4 + ((size_t)rows_max + 1) * 4;
  int per_sm = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, spmv_hybrid_kernel<false>, kThreads, smem) !=
          cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  (void)cudaGetLastError();
  return per_sm;
}

sable_status launch_spmv(sable_plan_t P, const DevHybrid &D, bool plain, const float *x, float *y,
                         cudaStream_t_ st) {
  if (D.m == 0) return SABLE_OK;
  if (!y || (D.n > 0 && !x)) return SABLE_ERR_INVALID;
  if (D.spmv.rows_max > 4 * kThreads) return fail(P, SABLE_ERR_INVALID);
  const size_t smem = (size_t)D.spmv.rows_max * 4 + ((size_t)D.spmv.rows_max + 1) * 4;
  auto k = plain ? spmv_hybrid_kernel<true> : spmv_hybrid_kernel<false>;
  // resident CTAs per SM for this shared-memory size, queried once per plan
  // and size (the query costs host time on every call of a small matrix)
  const int which = plain ? 1 : 0;
  int per_sm = P->spmv_occ[which];
  if (per_sm < 1 || P->spmv_occ_smem[which] != smem) {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kThreads, smem) != cudaSuccess || per_sm < 1)
      per_sm = 1;
    (void)cudaGetLastError();
    P->spmv_occ[which] = per_sm;
    P->spmv_occ_smem[which] = smem;
  }
  const int grid = std::max(1, std::min(D.spmv.n, per_sm * std::max(P->sm_count, 1)));
  k<<<grid, kThreads, smem, st>>>(D, x, y);
  if (D.spmv.n_fix > 0) {
    const int fgrid = std::max(1, std::min((D.spmv.n_fix + kThreads / 32 - 1) / (kThreads / 32), 4 * P->sm_count));
    spmv_fixup_kernel<<<fgrid, kThreads, 0, st>>>(D.spmv.fix, D.spmv.n_fix, D.spmv.part, y);
  }
  if (cudaGetLastError() != cudaSuccess) {
    (void)cudaGetLastError();
    return fail(P, SABLE_ERR_CUDA);
  }
  return SABLE_OK;
}

}  // namespace sable

namespace sable {

sable_status launch_spmv_grouped(const DevHybrid *mats, const DevItem *items, int n_items, int rows_max,
                                 const float *const *xs, float *const *ys, int sm_count, cudaStream_t_ st) {
  if (n_items == 0) return SABLE_OK;
  if (rows_max > 4 * kThreads) return SABLE_ERR_INVALID;
  const size_t smem = (size_t)rows_max * 4 + ((size_t)rows_max + 1) * 4;
  int per_sm = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, spmv_grouped_kernel, kThreads, smem) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  const int grid = std::max(1, std::min(n_items, per_sm * std::max(sm_count, 1)));
  spmv_grouped_kernel<<<grid, kThreads, smem, st>>>(mats, items, n_items, rows_max, xs, ys);
  if (cudaGetLastError() != cudaSuccess) {
    (void)cudaGetLastError();
    return SABLE_ERR_CUDA;
  }
  return SABLE_OK;
}

}  // namespace sable
