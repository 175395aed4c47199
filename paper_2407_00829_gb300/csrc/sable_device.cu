// Device side of libsable: table upload, the row-split SpMM kernels (FP32
// arithmetic) and the C-ABI compute entry points.  (The SpMV kernel is in
// sable_spmv.cu, the tensor-core block kernel in sable_tc.cu.)
//
// SpMM C = A B is row split: a group of lanes owns one row of C (a panel of
// its columns) and sums, in registers, one stream of entries: the row's VDIA
// diagonals (Section 4.2.1 layout), its FP32 VBR block columns (column-major,
// Appendix B) and its CSR remainder entries, one B row per entry, then stores
// the row once, instead of the paper's sequence of dispatches that each
// accumulate into a shared output (Section 3.4).  VBR blocks whose rows no
// other block shares are instead multiplied first, either on the tensor cores
// (sable_tc.cu) or FP32 in groups of 8 block rows that share each B row
// read, and their rows of C stored; the row-split launch adds the rest.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>

#include "sable_checks.cuh"
#include "sable_internal.h"
#include "sable_trace.h"

using namespace sable;

namespace sable {

constexpr unsigned kFull = 0xffffffffu;

// ------------------------------------------------------------------ SpMM (FP32)
template <int V> struct VecT;
template <> struct VecT<4> {
  using T = float4;
  __device__ static T zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
  __device__ static T load(const float *p) { return __ldg(reinterpret_cast<const float4 *>(p)); }
  __device__ static T load_once(const float *p) { return __ldcs(reinterpret_cast<const float4 *>(p)); }
  __device__ static void store_once(float *p, const T &a) { __stcs(reinterpret_cast<float4 *>(p), a); }
  __device__ static void fma(T &a, float s, const T &b) {
    a.x = fmaf(s, b.x, a.x); a.y = fmaf(s, b.y, a.y); a.z = fmaf(s, b.z, a.z); a.w = fmaf(s, b.w, a.w);
  }
  __device__ static void add_to(float *p, const T &a) {
    p[0] += a.x; p[1] += a.y; p[2] += a.z; p[3] += a.w;
  }
  __device__ static void atomic_add_to(float *p, const T &a) {
    atomicAdd(p, a.x); atomicAdd(p + 1, a.y); atomicAdd(p + 2, a.z); atomicAdd(p + 3, a.w);
  }
};
template <> struct VecT<2> {
  using T = float2;
  __device__ static T zero() { return make_float2(0.f, 0.f); }
  __device__ static T load(const float *p) { return __ldg(reinterpret_cast<const float2 *>(p)); }
  __device__ static T load_once(const float *p) { return __ldcs(reinterpret_cast<const float2 *>(p)); }
  __device__ static void store_once(float *p, const T &a) { __stcs(reinterpret_cast<float2 *>(p), a); }
  __device__ static void fma(T &a, float s, const T &b) {
    a.x = fmaf(s, b.x, a.x); a.y = fmaf(s, b.y, a.y);
  }
  __device__ static void add_to(float *p, const T &a) {
    p[0] += a.x; p[1] += a.y;
  }
  __device__ static void atomic_add_to(float *p, const T &a) {
    atomicAdd(p, a.x); atomicAdd(p + 1, a.y);
  }
};
template <> struct VecT<1> {
  using T = float;
  __device__ static T zero() { return 0.f; }
  __device__ static T load(const float *p) { return __ldg(p); }
  __device__ static T load_once(const float *p) { return __ldcs(p); }
  __device__ static void store_once(float *p, const T &a) { __stcs(p, a); }
  __device__ static void fma(T &a, float s, const T &b) { a = fmaf(s, b, a); }
  __device__ static void add_to(float *p, const T &a) { p[0] += a; }
  __device__ static void atomic_add_to(float *p, const T &a) { atomicAdd(p, a); }
};

// Row-split SpMM works on lane groups: a group of L lanes (8, 16 or 32) owns
// one row of C and V columns per lane, so a warp holds 32 / L rows at once
// and a CTA panel covers L V columns.  Small N (32 or 64 columns at V = 4)
// uses L = 8 or 16: a warp then keeps 32 / L rows' B-row reads in flight
// instead of idling three quarters of its lanes on one row.  mask: the
// group's lanes; shuffles use width L, so lane numbers are group-relative.
template <int L>
__device__ __forceinline__ unsigned group_mask() {
  if constexpr (L == 32) return 0xffffffffu;
  else return ((1u << L) - 1u) << (((threadIdx.x & 31) / L) * L);
}

// acc += sum over the cnt (1..L) entries held by the group's lanes 0..cnt-1
// (value v, column c; the lanes past cnt hold c = 0, a row that always
// exists) of v x the lane's columns of B row c, U rows of B in flight.  Whole
// groups of U run unchecked; the last group leaves its missing entries out of
// the sum by a group-uniform test.
template <int V, int L, int U>
__device__ __forceinline__ void rows_chunk(typename VecT<V>::T &acc, float v, int c, int cnt,
                                           const float *__restrict__ Bl, int ldb, bool lane_ok, unsigned mask) {
  using Vt = VecT<V>;
  using T = typename Vt::T;
  int j = 0;
  for (; j + U <= cnt; j += U) {
    T bj[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int cu = __shfl_sync(mask, c, j + u, L);
      bj[u] = lane_ok ? Vt::load(Bl + (int64_t)cu * ldb) : Vt::zero();
    }
#pragma unroll
    for (int u = 0; u < U; ++u) Vt::fma(acc, __shfl_sync(mask, v, j + u, L), bj[u]);
  }
  if (j < cnt) {   // source lanes past L wrap inside the group: a held entry or c = 0, left out below
    T bj[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int cu = __shfl_sync(mask, c, j + u, L);
      bj[u] = lane_ok ? Vt::load(Bl + (int64_t)cu * ldb) : Vt::zero();
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const float vu = __shfl_sync(mask, v, j + u, L);
      if (j + u < cnt) Vt::fma(acc, vu, bj[u]);
    }
  }
}

// The sum of one row of A B over the row's covering parts: its VDIA
// diagonals (columns r + off_lo + k, values strided by the segment's run
// length) and its FP32 block columns (columns c0 + k, values strided by the
// block's height), into acc.  tc: the matrix's blocks were stored first (on
// the tensor cores, or FP32 in row groups), so a block sets pre (the row adds
// the stored sum) instead.  own: some segment or block summed here covers the
// row.  A matrix with neither segments nor blocks has no per-row list
// (srp == nullptr): nothing covers its rows.  t: the lane within its group.
template <int V, int L, int U>
__device__ __forceinline__ void row_parts(const DevHybrid &A, int r, const float *__restrict__ Bl, int ldb,
                                          bool lane_ok, bool tc, typename VecT<V>::T &acc, bool &pre, bool &own,
                                          int t, unsigned mask) {
  const int n = A.n;
  if (A.srp == nullptr) return;
  const int q1 = __ldg(A.srp + r + 1);
  for (int q = __ldg(A.srp + r); q < q1; ++q) {   // the segments and blocks covering the row
    const int ref = __ldg(A.sref + q);
    const float *vp;
    int stride, cb, kb, k1;   // entries kb .. k1 - 1: value vp[k * stride], column cb + k
    if (ref & 1) {
      if (tc) {
        pre = true;
        continue;
      }
      const DevBlk b = A.blks[ref >> 1];
      vp = A.vbr + b.val_off + (r - b.r0);
      stride = b.nr;
      cb = b.c0;
      kb = 0;
      k1 = b.nc;
    } else {
      const DevSeg sg = A.segs[ref >> 1];
      vp = A.vdia + sg.val_off + (r - sg.base);
      stride = sg.ld;
      cb = r + sg.off_lo;   // columns kept inside [0, n)
      kb = max(0, -cb);
      k1 = min(sg.ndiag, n - cb);
    }
    own = true;
    for (; kb < k1; kb += L) {
      const int k = kb + t;
      float v = 0.f;
      int c = 0;
      if (k < k1) {
        v = __ldg(vp + (int64_t)k * stride);
        c = cb + k;
        if (!index_ok(A.err, kCheckSpmmBlock, c, n)) {   // debug build: contributes nothing
          c = 0;
          v = 0.f;
        }
      }
      rows_chunk<V, L, U>(acc, v, c, min(L, k1 - kb), Bl, ldb, lane_ok, mask);
    }
  }
}

// acc += the row's CSR remainder entries (values and columns streamed once).
template <int V, int L, int U>
__device__ __forceinline__ void row_csr(const DevHybrid &A, int r, const float *__restrict__ Bl, int ldb,
                                        bool lane_ok, typename VecT<V>::T &acc, int t, unsigned mask) {
  const int p0 = __ldg(A.rp + r), p1 = __ldg(A.rp + r + 1);
  for (int base = p0; base < p1; base += L) {
    const int p = base + t;
    float v = 0.f;
    int c = 0;
    if (p < p1) {
      v = __ldcs(A.cv + p);
      c = __ldcs(A.ci + p);
      if (!index_ok(A.err, kCheckSpmmCsr, c, A.n)) {   // debug build: contributes nothing
        c = 0;
        v = 0.f;
      }
    }
    rows_chunk<V, L, U>(acc, v, c, min(L, p1 - base), Bl, ldb, lane_ok, mask);
  }
}

// SpMM, row split: lane group gamma of the grid owns rows gamma, gamma + G, ...
// (consecutive rows on the groups of a warp and the warps of a CTA) and sums
// each row in registers from one stream of entries: the row's covering parts
// (row_parts), then its CSR entries; it stores the row once.  Neighbouring
// groups walk neighbouring rows of a segment or block at about the same time,
// so their B rows and strided values are shared in L1.  tc: the blocks'
// rows of C were stored first (tensor cores, or FP32 row groups); the row
// adds that stored sum instead of the block's entries.  No shared memory and
// no barriers (the tiled form's per-tile barriers held its B-row gathers to
// ~60 % of the device's row-gather rate).  FULL: N is a multiple of the panel
// width L V (no per-lane column test).  GEN: the matrix has VDIA segments, or
// blocks summed here; without it every covering part is a stored block and
// the row only tests whether it has one.
template <int V, int L, int U, bool FULL, bool GEN>
__global__ void __launch_bounds__(256, U == 8 ? 4 : 5)
spmm_rows_kernel(const __grid_constant__ DevHybrid A, const float *__restrict__ B, int ldb,
                 float *__restrict__ C, int ldc, int N, int tc) {
  using Vt = VecT<V>;
  using T = typename Vt::T;
  constexpr int G = 32 / L;
  const int t = (threadIdx.x & 31) % L;
  const unsigned mask = group_mask<L>();
  const int n0 = blockIdx.y * L * V;
  const int lc = V * t;
  const bool lane_ok = FULL || n0 + lc < N;
  const float *Bl = B + n0 + lc;
  const int W = gridDim.x * (blockDim.x >> 5) * G;
  for (int r = (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * G + (threadIdx.x & 31) / L; r < A.m;
       r += W) {
    T acc = Vt::zero();
    bool pre = false;   // C holds the row's stored block sum
    if constexpr (GEN) {
      bool own = false;
      row_parts<V, L, U>(A, r, Bl, ldb, lane_ok, tc != 0, acc, pre, own, t, mask);
      if (pre && !own && __ldg(A.rp + r) == __ldg(A.rp + r + 1)) continue;   // stored whole already
    } else {
      // every covering part is a stored block: a row with one and no CSR
      // entries is already stored whole
      if (A.srp != nullptr && __ldg(A.srp + r) < __ldg(A.srp + r + 1) && __ldg(A.rp + r) == __ldg(A.rp + r + 1))
        continue;
    }
    row_csr<V, L, U>(A, r, Bl, ldb, lane_ok, acc, t, mask);
    if (lane_ok) {
      float *dst = C + (int64_t)r * ldc + n0 + lc;
      if constexpr (!GEN) pre = A.srp != nullptr && __ldg(A.srp + r) < __ldg(A.srp + r + 1);
      if (pre) Vt::fma(acc, 1.0f, Vt::load_once(dst));   // exact add of the stored block sum
      Vt::store_once(dst, acc);
    }
  }
}

// FP32 VBR blocks of SpMM, a group of kGroupRows consecutive rows of one block
// per lane group: each B row c0 + c that the group needs is loaded once and
// multiplied by the group's kGroupRows values of block column c, so a block
// cell costs 1 / kGroupRows of a B-row read instead of one.  Four block
// columns per step: their 8 x 4 values (column-major, Appendix B: each
// column's 8 rows consecutive in memory) arrive in one coalesced load per
// lane (32 / L registers) and reach every lane of the group by shuffles; the
// next step's values and B rows are loaded before this step's products.  The
// group's rows of C are stored; the row-split launch then adds each row's
// other parts to that stored sum, as after the tensor cores.  Work items:
// (matrix, block, group) triples; Bs / Cs per matrix (leading dimension N) or
// B0 / C0 for a single matrix.  Only matrices whose blocks share no rows.
constexpr int kGroupRows = 8;

template <int V, int L, bool FULL>
__global__ void __launch_bounds__(256, 2)
vbr_rows_kernel(const DevHybrid *__restrict__ mats, const int32_t *__restrict__ trip, int n_items,
                const float *__restrict__ B0, int ldb0, float *__restrict__ C0, int ldc0,
                const float *const *__restrict__ Bs, float *const *__restrict__ Cs, int N) {
  using Vt = VecT<V>;
  using T = typename Vt::T;
  constexpr int G = 32 / L, R = 32 / L;   // groups per warp; value registers per lane per step
  const int t = (threadIdx.x & 31) % L;
  const unsigned mask = group_mask<L>();
  const int n0 = blockIdx.y * L * V;
  const int lc = V * t;
  const bool lane_ok = FULL || n0 + lc < N;
  const int W = gridDim.x * (blockDim.x >> 5) * G;
  for (int it = (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * G + (threadIdx.x & 31) / L; it < n_items;
       it += W) {
    const int mat = __ldg(trip + 3 * it), bi = __ldg(trip + 3 * it + 1), g = __ldg(trip + 3 * it + 2);
    const DevHybrid &A = mats[mat];
    const DevBlk b = A.blks[bi];
    const float *B = Bs ? Bs[mat] : B0;
    float *C = Cs ? Cs[mat] : C0;
    const int ldb = Bs ? N : ldb0, ldc = Cs ? N : ldc0;
    const int rr0 = g * kGroupRows, nrow = min(kGroupRows, b.nr - rr0);   // 1 .. kGroupRows rows
    const float *ap = A.vbr + b.val_off + rr0;                           // value (rr0 + j, c) at ap[c nr + j]
    const float *bp = B + (int64_t)b.c0 * ldb + n0 + lc;
    // value q = 8 u + j of a step (row j, column c + u) is held by lane q % L, register q / L
    auto load_step = [&](int c, float (&w)[R], T (&bv)[4]) {
#pragma unroll
      for (int s = 0; s < R; ++s) {
        const int q = s * L + t, u = q >> 3, j = q & 7;
        w[s] = (j < nrow && c + u < b.nc) ? __ldg(ap + (int64_t)(c + u) * b.nr + j) : 0.f;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
        bv[u] = (lane_ok && c + u < b.nc) ? Vt::load(bp + (int64_t)(c + u) * ldb) : Vt::zero();
    };
    T acc[kGroupRows];
#pragma unroll
    for (int j = 0; j < kGroupRows; ++j) acc[j] = Vt::zero();
    float w[R], wn[R];
    T bv[4], bn[4];
    load_step(0, w, bv);
    for (int c = 0; c < b.nc; c += 4) {
      if (c + 4 < b.nc) load_step(c + 4, wn, bn);   // next step in flight during this one
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int j = 0; j < kGroupRows; ++j) {
          const int q = 8 * u + j;
          Vt::fma(acc[j], __shfl_sync(mask, w[q / L], q % L, L), bv[u]);
        }
#pragma unroll
      for (int s = 0; s < R; ++s) w[s] = wn[s];
#pragma unroll
      for (int u = 0; u < 4; ++u) bv[u] = bn[u];
    }
    if (lane_ok) {
#pragma unroll
      for (int j = 0; j < kGroupRows; ++j)
        if (j < nrow) Vt::store_once(C + (int64_t)(b.r0 + rr0 + j) * ldc + n0 + lc, acc[j]);
    }
  }
}

// Many matrices in one row-split launch: the rows of every matrix numbered one
// after another (row_base[i] = rows of the matrices before i, row_base[count]
// = all rows); B_i is n_i x N and C_i is m_i x N, leading dimension N.  A
// group's rows only grow, so the matrix it looks up only moves forward.
// vbrc: the block launch stored the block rows of every matrix whose blocks
// share no rows (n_tc > 0); other matrices sum their blocks here.
template <int V, int L, int U, bool FULL>
__global__ void __launch_bounds__(256, U == 8 ? 4 : 5)
spmm_rows_grouped_kernel(const DevHybrid *__restrict__ mats, const int64_t *__restrict__ row_base, int count,
                         const float *const *__restrict__ Bs, float *const *__restrict__ Cs, int N, int vbrc) {
  using Vt = VecT<V>;
  using T = typename Vt::T;
  constexpr int G = 32 / L;
  const int t = (threadIdx.x & 31) % L;
  const unsigned mask = group_mask<L>();
  const int n0 = blockIdx.y * L * V;
  const int lc = V * t;
  const bool lane_ok = FULL || n0 + lc < N;
  const int64_t total = row_base[count];
  const int64_t W = (int64_t)gridDim.x * (blockDim.x >> 5) * G;
  int mat = 0;
  for (int64_t gr = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * G + (threadIdx.x & 31) / L;
       gr < total; gr += W) {
    while (row_base[mat + 1] <= gr) ++mat;   // gr < total = row_base[count], so mat < count
    const DevHybrid &A = mats[mat];
    const int r = (int)(gr - row_base[mat]);
    const float *Bl = Bs[mat] + n0 + lc;
    T acc = Vt::zero();
    bool pre = false, own = false;
    row_parts<V, L, U>(A, r, Bl, N, lane_ok, vbrc != 0 && A.n_tc > 0, acc, pre, own, t, mask);
    if (pre && !own && __ldg(A.rp + r) == __ldg(A.rp + r + 1)) continue;   // stored whole already
    row_csr<V, L, U>(A, r, Bl, N, lane_ok, acc, t, mask);
    if (lane_ok) {
      float *dst = Cs[mat] + (int64_t)r * N + n0 + lc;
      if (pre) Vt::fma(acc, 1.0f, Vt::load_once(dst));
      Vt::store_once(dst, acc);
    }
  }
}

// ------------------------------------------------------------------ host helpers
struct HostItems {
  std::vector<DevItem> items;
  std::vector<int32_t> iseg, iblk;
  std::vector<DevSeg> pseg;
  std::vector<DevBlk> pblk;
  int32_t rows_max = 0;
  std::vector<int32_t> fix;   // 4 per cut tile: first row, rows, first part slot, partial tiles
  int64_t n_slots = 0;        // partial row sums
};

// A tile's CSR range longer than two chunks (a few long rows) is cut: the tile
// keeps its first chunk, partial tiles take the rest; a chunk is the entries a
// tile of the byte target holds, at least this many.
constexpr int64_t kSplitMinEntries = 4096;

// Cut rows into SpMV tiles of at most rows_max rows (multiples of 4) whose
// summed per-row algorithmic bytes stay near `target`; list the
// segments/blocks touching each.  A tile of one 4-row group whose CSR range
// exceeds two chunks (rows of tens of thousands of entries) keeps its first
// chunk and hands the rest to partial tiles of one chunk each, run by other
// CTAs; their row sums are added to y by a second launch.
static HostItems build_items(int64_t m, const std::vector<Segment> &segs,
                             const std::vector<Block> &blks, const std::vector<int64_t> &rp,
                             int rows_max, int64_t target) {
  std::vector<int64_t> vd(m + 1, 0), vb(m + 1, 0);
  for (auto &s : segs) {
    vd[s.row0] += s.ndiag;
    vd[s.row0 + s.nrows] -= s.ndiag;
  }
  for (auto &b : blks) {
    vb[b.r0] += b.nc;
    vb[b.r0 + b.nr] -= b.nc;
  }
  for (int64_t i = 1; i <= m; ++i) {
    vd[i] += vd[i - 1];
    vb[i] += vb[i - 1];
  }
  auto cost = [&](int64_t i) -> int64_t {
    const int64_t c = rp[i + 1] - rp[i];
    return 8 + 4 * vd[i] + 4 * vb[i] + 8 * c;
  };
  HostItems H;
  size_t sp = 0, bp = 0;
  std::vector<int32_t> as, ab;
  int64_t r = 0;
  while (r < m) {
    const int64_t a = r;
    int64_t acc = 0;
    while (r < m && r - a < rows_max) {
      const int64_t e = std::min<int64_t>(m, r + 4);
      int64_t q = 0;
      for (int64_t i = r; i < e; ++i) q += cost(i);
      if (r > a && acc + q > target) break;
      acc += q;
      r = e;
    }
    const int64_t b = r;
    DevItem it{};
    it.r0 = (int32_t)a;
    it.r1 = (int32_t)b;
    while (sp < segs.size() && segs[sp].row0 < b) as.push_back((int32_t)sp++);
    while (bp < blks.size() && blks[bp].r0 < b) ab.push_back((int32_t)bp++);
    as.erase(std::remove_if(as.begin(), as.end(),
                            [&](int32_t s) { return segs[s].row0 + segs[s].nrows <= a; }),
             as.end());
    ab.erase(std::remove_if(ab.begin(), ab.end(), [&](int32_t s) { return blks[s].r0 + blks[s].nr <= a; }),
             ab.end());
    it.seg_lo = (int32_t)H.iseg.size();
    H.iseg.insert(H.iseg.end(), as.begin(), as.end());
    it.seg_hi = (int32_t)H.iseg.size();
    it.blk_lo = (int32_t)H.iblk.size();
    H.iblk.insert(H.iblk.end(), ab.begin(), ab.end());
    it.blk_hi = (int32_t)H.iblk.size();
    it.pb = (int32_t)rp[a];
    it.pe = (int32_t)rp[b];
    int64_t vc = 0;
    for (int32_t q : as) vc += (std::min(b, segs[q].row0 + segs[q].nrows) - std::max(a, segs[q].row0)) * segs[q].ndiag;
    for (int32_t q : ab) vc += (std::min(b, blks[q].r0 + blks[q].nr) - std::max(a, blks[q].r0)) * blks[q].nc;
    it.vcells = (int32_t)std::min<int64_t>(vc, INT32_MAX);
    const int64_t chunk = std::max<int64_t>(kSplitMinEntries, target / 8);
    if (rp[b] - rp[a] > 2 * chunk) {
      it.pe = (int32_t)(rp[a] + chunk);
      H.items.push_back(it);
      const int64_t first = H.n_slots;
      int64_t nparts = 0;
      for (int64_t p = rp[a] + chunk; p < rp[b]; p += chunk) {
        DevItem pt{};
        pt.r0 = (int32_t)a;
        pt.r1 = (int32_t)b;
        pt.seg_lo = pt.seg_hi = (int32_t)H.iseg.size();
        pt.blk_lo = pt.blk_hi = (int32_t)H.iblk.size();
        pt.pb = (int32_t)p;
        pt.pe = (int32_t)std::min<int64_t>(rp[b], p + chunk);
        pt.part = (int32_t)(H.n_slots + 1);
        H.n_slots += b - a;
        H.items.push_back(pt);
        ++nparts;
      }
      H.fix.insert(H.fix.end(), {(int32_t)a, (int32_t)(b - a), (int32_t)first, (int32_t)nparts});
    } else {
      H.items.push_back(it);
    }
    H.rows_max = std::max<int32_t>(H.rows_max, (int32_t)(b - a));
  }
  return H;
}

struct Piece {
  size_t off;
  const void *src;
  size_t bytes;
};

struct Arena {
  size_t off = 0;
  std::vector<Piece> pieces;
  size_t add(const void *src, size_t bytes) {
    const size_t o = off;
    off = (off + bytes + 255) & ~(size_t)255;
    if (bytes) pieces.push_back({o, src, bytes});
    return o;
  }
  size_t reserve(size_t bytes) { return add(nullptr, bytes); }
};

// Host staging kept alive by the plan until destroy (uploads are async).
struct Staging {
  std::vector<DevSeg> segs;
  std::vector<float> vdia;
  std::vector<DevBlk> blks;
  std::vector<int32_t> rp, ci, prp, pci, tc_pairs, fg_pairs;
  std::vector<uint16_t> vbr_bf16, vbr_bf16_mid, vbr_bf16_lo;
  std::vector<float> vbr_scale;
  std::vector<float> cv, pcv;
  std::vector<int32_t> srp, sref;
  HostItems it_v, pit_v;
};

}  // namespace sable

static sable_status cuda_fail(sable_plan_t P, cudaError_t e) {
  (void)cudaGetLastError();
  return fail(P, e == cudaErrorMemoryAllocation ? SABLE_ERR_OOM : SABLE_ERR_CUDA);
}

extern "C" {

sable_status sable_plan_upload(sable_plan_t P, void *stream) {
  sable::TraceRange trace_("sable_plan_upload");
  if (!P) return SABLE_ERR_INVALID;
  if (P->sticky) return P->sticky;
  if (!P->extracted) return SABLE_ERR_ORDER;
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(P, e);
  if (P->dev_blob) {                       // re-upload (new tiling): release first
    cudaFree(P->dev_blob);
    P->dev_blob = nullptr;
  }
  Staging *S = nullptr;
  try {
    alloc_point();
    S = new Staging();
    const Hybrid &H = P->hyb;
    const Csr &Cn = P->canon;
    // VDIA, padded runs
    std::vector<int64_t> sptr(H.segs.size() + 1, 0);
    for (size_t s = 0; s < H.segs.size(); ++s) sptr[s + 1] = sptr[s] + H.segs[s].nrows * H.segs[s].ndiag;
    int64_t voff = 0;
    for (size_t s = 0; s < H.segs.size(); ++s) {
      const Segment &g = H.segs[s];
      DevSeg d{};
      d.row0 = (int32_t)g.row0;
      d.nrows = (int32_t)g.nrows;
      d.off_lo = (int32_t)g.off_lo;
      d.ndiag = (int32_t)g.ndiag;
      d.base = (int32_t)(g.row0 & ~(int64_t)3);
      d.ld = (int32_t)(((g.row0 + g.nrows + 3) & ~(int64_t)3) - d.base);
      d.val_off = voff;
      S->segs.push_back(d);
      voff += (int64_t)d.ld * d.ndiag;
    }
    S->vdia.assign(std::max<int64_t>(voff, 4), 0.0f);
    for (size_t s = 0; s < H.segs.size(); ++s) {
      const DevSeg &d = S->segs[s];
      for (int64_t k = 0; k < d.ndiag; ++k)
        for (int64_t r = 0; r < d.nrows; ++r)
          S->vdia[d.val_off + k * d.ld + (d.row0 - d.base) + r] = H.vdia_canon[sptr[s] + k * d.nrows + r];
    }
    int64_t boff = 0;
    for (const Block &b : H.blks) {
      DevBlk d{};
      d.r0 = (int32_t)b.r0;
      d.nr = (int32_t)b.nr;
      d.c0 = (int32_t)b.c0;
      d.nc = (int32_t)b.nc;
      d.val_off = boff;
      d.bf_off = 0;
      S->blks.push_back(d);
      boff += b.nr * b.nc;
    }
    {
      std::vector<int64_t> offs;
      pack_vbr_bf16(H.blks, H.vbr_canon, S->vbr_bf16, S->vbr_scale, offs, &S->vbr_bf16_mid, &S->vbr_bf16_lo);
      for (size_t b = 0; b < S->blks.size(); ++b) S->blks[b].bf_off = offs[b];
      S->tc_pairs.clear();
      // the tensor-core kernel stores its blocks' rows of C: blocks that share
      // rows (two VBR stages) stay on the FP32 path
      bool shared_rows = false;
      int64_t end = -1;
      for (const Block &b : H.blks) {
        shared_rows = shared_rows || b.r0 < end;
        end = std::max(end, b.r0 + b.nr);
      }
      S->fg_pairs.clear();
      if (!shared_rows) {
        vbr_tc_pairs(H.blks, 0, S->tc_pairs);
        vbr_group_pairs(H.blks, 0, S->fg_pairs);
      }
    }
    if (!H.segs.empty() || !H.blks.empty()) {   // per row: the segments and blocks covering it
      S->srp.assign(P->m + 1, 0);
      for (const Segment &g : H.segs)
        for (int64_t r = g.row0; r < g.row0 + g.nrows; ++r) ++S->srp[r + 1];
      for (const Block &b : H.blks)
        for (int64_t r = b.r0; r < b.r0 + b.nr; ++r) ++S->srp[r + 1];
      for (int64_t r = 0; r < P->m; ++r) S->srp[r + 1] += S->srp[r];
      S->sref.resize(S->srp[P->m]);
      std::vector<int32_t> at(S->srp.begin(), S->srp.end() - 1);
      for (size_t i = 0; i < H.segs.size(); ++i)
        for (int64_t r = H.segs[i].row0; r < H.segs[i].row0 + H.segs[i].nrows; ++r)
          S->sref[at[r]++] = (int32_t)(i << 1);
      for (size_t i = 0; i < H.blks.size(); ++i)
        for (int64_t r = H.blks[i].r0; r < H.blks[i].r0 + H.blks[i].nr; ++r)
          S->sref[at[r]++] = (int32_t)((i << 1) | 1);
    }
    S->rp.assign(H.crp.begin(), H.crp.end());
    S->ci.assign(H.cci.begin(), H.cci.end());
    S->cv.assign(H.ccv.begin(), H.ccv.end());
    S->ci.resize(S->ci.size() + kCsrPad, 0);
    S->cv.resize(S->cv.size() + kCsrPad, 0.0f);
    S->prp.assign(Cn.rp.begin(), Cn.rp.end());
    S->pci.assign(Cn.ci.begin(), Cn.ci.end());
    S->pcv.assign(P->cval.begin(), P->cval.end());
    S->pci.resize(S->pci.size() + kCsrPad, 0);
    S->pcv.resize(S->pcv.size() + kCsrPad, 0.0f);
    const Tiling &T = P->tiling;
    S->it_v = build_items(P->m, H.segs, H.blks, H.crp, T.rows_per_item, T.item_bytes);
    const std::vector<Segment> no_s;
    const std::vector<Block> no_b;
    S->pit_v = build_items(P->m, no_s, no_b, Cn.rp, T.rows_per_item, T.item_bytes);
  } catch (const std::bad_alloc &) {
    delete S;
    return fail(P, SABLE_ERR_OOM);
  }
  Arena ar;
  auto vec_bytes = [](const auto &v) { return v.size() * sizeof(v[0]); };
  const size_t o_err = ar.reserve(256);
  const size_t o_segs = ar.add(S->segs.data(), vec_bytes(S->segs));
  const size_t o_vdia = ar.add(S->vdia.data(), vec_bytes(S->vdia));
  const size_t o_blks = ar.add(S->blks.data(), vec_bytes(S->blks));
  const size_t o_vbr = ar.add(P->hyb.vbr_canon.data(), vec_bytes(P->hyb.vbr_canon));
  const size_t o_bf16 = ar.add(S->vbr_bf16.data(), vec_bytes(S->vbr_bf16));
  const size_t o_bf16_mid = ar.add(S->vbr_bf16_mid.data(), vec_bytes(S->vbr_bf16_mid));
  const size_t o_bf16_lo = ar.add(S->vbr_bf16_lo.data(), vec_bytes(S->vbr_bf16_lo));
  const size_t o_scale = ar.add(S->vbr_scale.data(), vec_bytes(S->vbr_scale));
  const size_t o_pairs = ar.add(S->tc_pairs.data(), vec_bytes(S->tc_pairs));
  const size_t o_fg = ar.add(S->fg_pairs.data(), vec_bytes(S->fg_pairs));
  const size_t o_self = ar.reserve(sizeof(DevHybrid));
  const size_t o_rp = ar.add(S->rp.data(), vec_bytes(S->rp));
  const size_t o_ci = ar.add(S->ci.data(), vec_bytes(S->ci));
  const size_t o_cv = ar.add(S->cv.data(), vec_bytes(S->cv));
  const size_t o_prp = ar.add(S->prp.data(), vec_bytes(S->prp));
  const size_t o_pci = ar.add(S->pci.data(), vec_bytes(S->pci));
  const size_t o_pcv = ar.add(S->pcv.data(), vec_bytes(S->pcv));
  const size_t o_srp = ar.add(S->srp.data(), vec_bytes(S->srp));
  const size_t o_sref = ar.add(S->sref.data(), vec_bytes(S->sref));
  size_t o_it[2][8];
  HostItems *its[2] = {&S->it_v, &S->pit_v};
  for (int k = 0; k < 2; ++k) {
    for (int32_t q : its[k]->iseg) its[k]->pseg.push_back(S->segs[q]);
    for (int32_t q : its[k]->iblk) its[k]->pblk.push_back(S->blks[q]);
    o_it[k][4] = ar.add(its[k]->pseg.data(), vec_bytes(its[k]->pseg));
    o_it[k][5] = ar.add(its[k]->pblk.data(), vec_bytes(its[k]->pblk));
    o_it[k][0] = ar.add(its[k]->items.data(), vec_bytes(its[k]->items));
    o_it[k][1] = ar.add(its[k]->iseg.data(), vec_bytes(its[k]->iseg));
    o_it[k][2] = ar.add(its[k]->iblk.data(), vec_bytes(its[k]->iblk));
    o_it[k][6] = ar.add(its[k]->fix.data(), vec_bytes(its[k]->fix));
    o_it[k][7] = ar.reserve((size_t)its[k]->n_slots * sizeof(float));
  }
  char *blob = nullptr;
  e = alloc_fails() ? cudaErrorMemoryAllocation : cudaMalloc(&blob, ar.off);
  if (e != cudaSuccess) {
    delete S;
    return cuda_fail(P, e);
  }
  e = cudaMemsetAsync(blob, 0, 256, st);
  for (const Piece &pc : ar.pieces)
    if (e == cudaSuccess && pc.src) e = cudaMemcpyAsync(blob + pc.off, pc.src, pc.bytes, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    delete S;
    cudaFree(blob);
    return cuda_fail(P, e);
  }
  auto items_of = [&](int k, const HostItems *h) {
    DevItems d;
    d.items = reinterpret_cast<const DevItem *>(blob + o_it[k][0]);
    d.iseg = reinterpret_cast<const int32_t *>(blob + o_it[k][1]);
    d.iblk = reinterpret_cast<const int32_t *>(blob + o_it[k][2]);
    d.pseg = reinterpret_cast<const DevSeg *>(blob + o_it[k][4]);
    d.pblk = reinterpret_cast<const DevBlk *>(blob + o_it[k][5]);
    d.n = (int32_t)h->items.size();
    d.rows_max = h->rows_max;
    d.fix = reinterpret_cast<const int32_t *>(blob + o_it[k][6]);
    d.n_fix = (int32_t)(h->fix.size() / 4);
    d.part = reinterpret_cast<float *>(blob + o_it[k][7]);
    return d;
  };
  DevHybrid &D = P->dev;
  D = DevHybrid{};
  D.m = (int32_t)P->m;
  D.n = (int32_t)P->n;
  D.segs = reinterpret_cast<const DevSeg *>(blob + o_segs);
  D.vdia = reinterpret_cast<const float *>(blob + o_vdia);
  D.blks = reinterpret_cast<const DevBlk *>(blob + o_blks);
  D.vbr = reinterpret_cast<const float *>(blob + o_vbr);
  D.vbr_bf16 = reinterpret_cast<const uint16_t *>(blob + o_bf16);
  D.vbr_bf16_mid = reinterpret_cast<const uint16_t *>(blob + o_bf16_mid);
  D.vbr_bf16_lo = reinterpret_cast<const uint16_t *>(blob + o_bf16_lo);
  D.vbr_scale = reinterpret_cast<const float *>(blob + o_scale);
  D.n_tc = (int32_t)(S->tc_pairs.size() / 3);
  P->dev_trip = reinterpret_cast<const int32_t *>(blob + o_pairs);
  D.n_fg = (int32_t)(S->fg_pairs.size() / 3);
  P->dev_fg = reinterpret_cast<const int32_t *>(blob + o_fg);
  P->dev_self = reinterpret_cast<DevHybrid *>(blob + o_self);
  D.rp = reinterpret_cast<const int32_t *>(blob + o_rp);
  D.ci = reinterpret_cast<const int32_t *>(blob + o_ci);
  D.cv = reinterpret_cast<const float *>(blob + o_cv);
  D.err = reinterpret_cast<int32_t *>(blob + o_err);
  D.n_segs = (int32_t)S->segs.size();
  D.n_blks = (int32_t)S->blks.size();
  D.srp = S->srp.empty() ? nullptr : reinterpret_cast<const int32_t *>(blob + o_srp);
  D.sref = S->srp.empty() ? nullptr : reinterpret_cast<const int32_t *>(blob + o_sref);
  D.spmv = items_of(0, its[0]);
  DevHybrid &Q = P->dev_plain;
  Q = DevHybrid{};
  Q.m = D.m;
  Q.n = D.n;
  Q.rp = reinterpret_cast<const int32_t *>(blob + o_prp);
  Q.ci = reinterpret_cast<const int32_t *>(blob + o_pci);
  Q.cv = reinterpret_cast<const float *>(blob + o_pcv);
  Q.err = D.err;
  Q.spmv = items_of(1, its[1]);
  P->stats.n_items = D.spmv.n;
  P->h_items_v = S->it_v.items;
  P->h_trip = S->tc_pairs;
  P->h_fg = S->fg_pairs;
  P->h_segs = S->segs;
  P->o_vdia = o_vdia;
  P->o_vbr = o_vbr;
  P->o_bf16 = o_bf16;
  P->o_bf16_mid = o_bf16_mid;
  P->o_bf16_lo = o_bf16_lo;
  P->o_scale = o_scale;
  P->o_cv = o_cv;
  P->o_pcv = o_pcv;
  delete S;
  e = cudaMemcpy(P->dev_self, &P->dev, sizeof(DevHybrid), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(blob);
    P->dev_blob = nullptr;
    return cuda_fail(P, e);
  }
  P->dev_blob = blob;
  P->dev_bytes = ar.off;
  P->device = dev;
  cudaDeviceGetAttribute(&P->sm_count, cudaDevAttrMultiProcessorCount, dev);
  P->uploaded = true;
  return SABLE_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ launches
namespace {

template <class K>
int grid_for(K kernel, int threads, size_t smem, int items, int sm_count) {
  int per_sm = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  (void)cudaGetLastError();
  const int g = per_sm * std::max(sm_count, 1);
  return std::max(1, std::min(items, g));
}

}  // namespace

namespace sable {
// Column panel of the row-split SpMM kernels: V columns per lane and L lanes
// per row (panel width L V).  cols is the tiling knob (0 = widest the
// operands allow, 32, 64 or 128 columns); vec: N, the leading dimensions and
// the operands allow float4 lanes (16-byte aligned), vec2 float2 lanes.
Panel spmm_panel(int cols, int64_t N, bool vec, bool vec2) {
  if (vec) {
    const int L = cols == 32 ? 8 : cols == 64 ? 16 : cols == 128 ? 32 : N <= 32 ? 8 : N <= 64 ? 16 : 32;
    return {4, L};
  }
  if (vec2 && cols != 32) return {2, 32};
  return {1, 32};
}
}  // namespace sable

namespace {

sable_status check_ready(sable_plan_t P) {
  if (!P) return SABLE_ERR_INVALID;
  if (P->sticky) return P->sticky;
  if (!P->uploaded) return SABLE_ERR_ORDER;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return cuda_fail(P, cudaErrorInvalidDevice);
  if (dev != P->device) return SABLE_ERR_INVALID;
  return SABLE_OK;
}

template <int V, int L, int U>
void launch_rows(const DevHybrid &D, const float *B, int64_t ldb, float *C, int64_t ldc, int N, int sms, bool tc,
                 cudaStream_t st) {
  const bool full = N % (L * V) == 0, gen = D.n_segs > 0 || (D.n_blks > 0 && !tc);
  auto k = gen ? (full ? spmm_rows_kernel<V, L, U, true, true> : spmm_rows_kernel<V, L, U, false, true>)
               : (full ? spmm_rows_kernel<V, L, U, true, false> : spmm_rows_kernel<V, L, U, false, false>);
  const int gy = (N + L * V - 1) / (L * V);
  dim3 grid(grid_for(k, 256, 0, (D.m + 8 * (32 / L) - 1) / (8 * (32 / L)), sms), gy);
  k<<<grid, 256, 0, st>>>(D, B, (int)ldb, C, (int)ldc, N, tc ? 1 : 0);
}

// C = A B in one row-split launch (after the tensor-core blocks when vbrc:
// their rows of C are stored).
sable_status launch_spmm(sable_plan_t P, const DevHybrid &D, const float *B, int64_t N, int64_t ldb,
                         float *C, int64_t ldc, bool vbrc, cudaStream_t st) {
  if (N < 1 || ldb < N || ldc < N || N > (int64_t)65535 * 32 || ldb > INT32_MAX || ldc > INT32_MAX)
    return SABLE_ERR_INVALID;
  if (D.m == 0) return SABLE_OK;
  if (!C || (D.n > 0 && !B)) return SABLE_ERR_INVALID;
  const bool vec = N % 4 == 0 && ldb % 4 == 0 && ldc % 4 == 0 &&
                   ((uintptr_t)B & 15) == 0 && ((uintptr_t)C & 15) == 0;
  const bool vec2 = N % 2 == 0 && ldb % 2 == 0 && ldc % 2 == 0 &&
                    ((uintptr_t)B & 7) == 0 && ((uintptr_t)C & 7) == 0;
  // column panel per CTA: 128, 64 or 32 columns (float4 lanes, 32, 16 or 8
  // lanes per row), or float2 / scalar lanes when the operands are not aligned
  const Panel pn = spmm_panel(P->tiling.spmm_cols, N, vec, vec2);
  const int sms = P->sm_count;
  const bool deep = P->tiling.spmm_depth == 8;   // 8 B rows in flight per lane group
  const int n = (int)N;
  if (pn.V == 4) {
    if (pn.L == 8) deep ? launch_rows<4, 8, 8>(D, B, ldb, C, ldc, n, sms, vbrc, st)
                        : launch_rows<4, 8, 4>(D, B, ldb, C, ldc, n, sms, vbrc, st);
    else if (pn.L == 16) deep ? launch_rows<4, 16, 8>(D, B, ldb, C, ldc, n, sms, vbrc, st)
                              : launch_rows<4, 16, 4>(D, B, ldb, C, ldc, n, sms, vbrc, st);
    else deep ? launch_rows<4, 32, 8>(D, B, ldb, C, ldc, n, sms, vbrc, st)
              : launch_rows<4, 32, 4>(D, B, ldb, C, ldc, n, sms, vbrc, st);
  } else if (pn.V == 2) {
    deep ? launch_rows<2, 32, 8>(D, B, ldb, C, ldc, n, sms, vbrc, st)
         : launch_rows<2, 32, 4>(D, B, ldb, C, ldc, n, sms, vbrc, st);
  } else {
    launch_rows<1, 32, 4>(D, B, ldb, C, ldc, n, sms, vbrc, st);
  }
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SABLE_OK : cuda_fail(P, e);
}

}  // namespace

extern "C" {

sable_status sable_spmv(sable_plan_t P, const float *x, float *y, void *stream) {
  sable::TraceRange trace_("sable_spmv");
  const sable_status s = check_ready(P);
  if (s) return s;
  return launch_spmv(P, P->dev, false, x, y, (cudaStream_t)stream);
}

sable_status sable_csr_spmv(sable_plan_t P, const float *x, float *y, void *stream) {
  sable::TraceRange trace_("sable_csr_spmv");
  const sable_status s = check_ready(P);
  if (s) return s;
  return launch_spmv(P, P->dev_plain, true, x, y, (cudaStream_t)stream);
}

sable_status sable_spmm(sable_plan_t P, const float *B, int64_t N, int64_t ldb, float *C, int64_t ldc,
                        sable_precision prec, void *stream) {
  sable::TraceRange trace_("sable_spmm");
  const sable_status s = check_ready(P);
  if (s) return s;
  if (prec != SABLE_FP32 && prec != SABLE_BF16_BLOCKS && prec != SABLE_FP32_SPLIT) return SABLE_ERR_INVALID;
  // blocks first, storing their rows of C: on the tensor cores, or FP32 in
  // groups of rows; the row-split launch adds the other parts
  const bool first = P->dev.n_tc > 0;
  if (first) {
    if (N < 1 || ldb < N || ldc < N || !B || !C || N > (int64_t)65535 * 32 || ldb > INT32_MAX || ldc > INT32_MAX)
      return SABLE_ERR_INVALID;
    const sable_status s2 =
        prec == SABLE_FP32
            ? launch_vbr_rows(P->dev_self, P->dev_fg, P->dev.n_fg, B, ldb, C, ldc, nullptr, nullptr, (int)N,
                              P->tiling.spmm_cols, P->sm_count, (cudaStream_t)stream)
            : launch_vbr_tc(P->dev_self, P->dev_trip, P->dev.n_tc, B, ldb, C, ldc, nullptr, nullptr, (int)N,
                            P->sm_count, P->dev.err, (cudaStream_t)stream, prec == SABLE_FP32_SPLIT ? 3 : 1);
    if (s2) return fail(P, s2);
  }
  return launch_spmm(P, P->dev, B, N, ldb, C, ldc, first, (cudaStream_t)stream);
}

sable_status sable_csr_spmm(sable_plan_t P, const float *B, int64_t N, int64_t ldb, float *C, int64_t ldc,
                            void *stream) {
  sable::TraceRange trace_("sable_csr_spmm");
  const sable_status s = check_ready(P);
  if (s) return s;
  return launch_spmm(P, P->dev_plain, B, N, ldb, C, ldc, false, (cudaStream_t)stream);
}

sable_status sable_plan_update_values(sable_plan_t P, const float *val, void *stream) {
  if (!P || (!val && !P->canon_of.empty())) return SABLE_ERR_INVALID;
  if (P->sticky) return P->sticky;
  if (!P->extracted) return SABLE_ERR_ORDER;
  if (P->uploaded) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != P->device) return SABLE_ERR_INVALID;
  }
  cudaStream_t st = (cudaStream_t)stream;
  Hybrid &H = P->hyb;
  std::vector<float> vdia, cv, pcv, scales;
  std::vector<uint16_t> bf16, bf16_mid, bf16_lo;
  try {
    // duplicates summed in FP64 in input order, rounded once: as at create
    std::vector<double> sum(P->cval.size(), 0.0);
    for (size_t k = 0; k < P->canon_of.size(); ++k) sum[P->canon_of[k]] += (double)val[k];
    for (size_t c = 0; c < sum.size(); ++c) {
      const float v = (float)sum[c];
      P->cval[c] = v;
      if (P->owner[c] == OWN_VDIA) H.vdia_canon[P->dest[c]] = v;
      else if (P->owner[c] == OWN_VBR) H.vbr_canon[P->dest[c]] = v;
      else H.ccv[P->dest[c]] = v;
    }
    if (!P->uploaded) return SABLE_OK;
    int64_t cells = 4;
    for (const DevSeg &d : P->h_segs) cells = std::max<int64_t>(cells, d.val_off + (int64_t)d.ld * d.ndiag);
    vdia.assign(cells, 0.0f);
    int64_t sp = 0;
    for (const DevSeg &d : P->h_segs) {
      for (int64_t k = 0; k < d.ndiag; ++k)
        for (int64_t r = 0; r < d.nrows; ++r) vdia[d.val_off + k * d.ld + (d.row0 - d.base) + r] = H.vdia_canon[sp + k * d.nrows + r];
      sp += (int64_t)d.nrows * d.ndiag;
    }
    std::vector<int64_t> offs;
    pack_vbr_bf16(H.blks, H.vbr_canon, bf16, scales, offs, &bf16_mid, &bf16_lo);
    cv.assign(H.ccv.begin(), H.ccv.end());
    cv.resize(cv.size() + kCsrPad, 0.0f);
    pcv.assign(P->cval.begin(), P->cval.end());
    pcv.resize(pcv.size() + kCsrPad, 0.0f);
  } catch (const std::bad_alloc &) {
    return fail(P, SABLE_ERR_OOM);
  }
  char *blob = static_cast<char *>(P->dev_blob);
  const struct { size_t off; const void *src; size_t bytes; } parts[] = {
      {P->o_vdia, vdia.data(), H.segs.empty() ? 0 : vdia.size() * 4},
      {P->o_vbr, H.vbr_canon.data(), H.vbr_canon.size() * 4},
      {P->o_bf16, bf16.data(), bf16.size() * 2},
      {P->o_bf16_mid, bf16_mid.data(), bf16_mid.size() * 2},
      {P->o_bf16_lo, bf16_lo.data(), bf16_lo.size() * 2},
      {P->o_scale, scales.data(), scales.size() * 4},
      {P->o_cv, cv.data(), cv.size() * 4},
      {P->o_pcv, pcv.data(), pcv.size() * 4}};
  cudaError_t e = cudaSuccess;
  for (const auto &pt : parts)
    if (e == cudaSuccess && pt.bytes) e = cudaMemcpyAsync(blob + pt.off, pt.src, pt.bytes, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);   // the staging vectors die here
  return e == cudaSuccess ? SABLE_OK : cuda_fail(P, e);
}

sable_status sable_debug_set_csr_column(sable_plan_t P, int64_t entry, int32_t value) {
#ifndef SABLE_CHECKS
  (void)P;
  (void)entry;
  (void)value;
  return SABLE_ERR_UNSUPPORTED;   // only the checked build may hold a column outside the matrix
#else
  if (!P) return SABLE_ERR_INVALID;
  if (!P->uploaded) return SABLE_ERR_ORDER;
  if (entry < 0 || entry >= P->stats.nnz_csr) return SABLE_ERR_INVALID;
  const cudaError_t e =
      cudaMemcpy(const_cast<int32_t *>(P->dev.ci) + entry, &value, sizeof(int32_t), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return SABLE_ERR_CUDA;
  }
  return SABLE_OK;
#endif
}

sable_status sable_plan_device_error(sable_plan_t P, int32_t *out) {
  if (!P || !out) return SABLE_ERR_INVALID;
  if (!P->uploaded) return SABLE_ERR_ORDER;
  const cudaError_t e = cudaMemcpy(out, P->dev.err, 4 * sizeof(int32_t), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return SABLE_ERR_CUDA;
  }
  return SABLE_OK;
}

sable_status sable_plan_reset(sable_plan_t P) {
  if (!P) return SABLE_ERR_INVALID;
  if (P->dev_blob) {
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != P->device) cudaSetDevice(P->device);
    const cudaError_t e = cudaFree(P->dev_blob);
    if (cur >= 0 && cur != P->device) cudaSetDevice(cur);
    P->dev_blob = nullptr;
    if (e != cudaSuccess) {
      (void)cudaGetLastError();
      return fail(P, SABLE_ERR_CUDA);
    }
  }
  P->dev_bytes = 0;
  P->dev = DevHybrid{};
  P->dev_plain = DevHybrid{};
  P->dev_self = nullptr;
  P->dev_trip = nullptr;
  P->dev_fg = nullptr;
  P->dev_err = nullptr;
  P->h_items_v.clear();
  P->h_trip.clear();
  P->h_fg.clear();
  P->extractors.clear();
  P->stage_regions.clear();
  P->stage_fixed.clear();
  P->seg_stage.clear();
  P->blk_stage.clear();
  P->dest.clear();
  P->h_segs.clear();
  P->o_vdia = P->o_vbr = P->o_bf16 = P->o_scale = P->o_cv = P->o_pcv = 0;
  P->o_bf16_mid = P->o_bf16_lo = 0;
  P->owner.assign(P->canon.ci.size(), OWN_NONE);
  P->hyb = Hybrid{};
  P->stats = sable_plan_stats{};
  P->extracted = P->uploaded = false;
  P->sticky = SABLE_OK;
  return SABLE_OK;
}

sable_status sable_plan_destroy(sable_plan_t P) {
  if (!P) return SABLE_OK;
  if (P->dev_blob) {
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != P->device) cudaSetDevice(P->device);
    cudaFree(P->dev_blob);
    if (cur >= 0 && cur != P->device) cudaSetDevice(cur);
    (void)cudaGetLastError();
  }
  delete P;
  return SABLE_OK;
}

}  // extern "C"

namespace sable {

void vbr_group_pairs(const std::vector<Block> &blks, int32_t mat, std::vector<int32_t> &trip) {
  for (size_t bi = 0; bi < blks.size(); ++bi)
    for (int64_t g = 0; g * kGroupRows < blks[bi].nr; ++g) {
      trip.push_back(mat);
      trip.push_back((int32_t)bi);
      trip.push_back((int32_t)g);
    }
}

sable_status launch_vbr_rows(const DevHybrid *mats, const int32_t *trip, int n_items, const float *B, int64_t ldb,
                             float *C, int64_t ldc, const float *const *Bs, float *const *Cs, int N, int cols,
                             int sm_count, cudaStream_t_ st) {
  if (n_items == 0) return SABLE_OK;
  if (N < 1 || N > 65535 * 32) return SABLE_ERR_INVALID;
  // float4 lanes need N, ldb, ldc multiples of 4 and 16-byte aligned B, C
  // (batches: every B_i, C_i, documented); float2 lanes even sizes, 8 bytes
  const bool one = Bs == nullptr;
  const bool vec4 = N % 4 == 0 && (!one || (ldb % 4 == 0 && ldc % 4 == 0 && ((uintptr_t)B & 15) == 0 &&
                                             ((uintptr_t)C & 15) == 0));
  const bool vec2 = N % 2 == 0 && (!one || (ldb % 2 == 0 && ldc % 2 == 0 && ((uintptr_t)B & 7) == 0 &&
                                             ((uintptr_t)C & 7) == 0));
  const Panel pn = spmm_panel(cols, N, vec4, vec2);
  const int gy = (N + pn.L * pn.V - 1) / (pn.L * pn.V);
  const bool full = N % (pn.L * pn.V) == 0;
  const int per = 8 * (32 / pn.L);   // items one CTA takes at once
  auto go = [&](auto k) {
    dim3 grid(grid_for(k, 256, 0, (n_items + per - 1) / per, sm_count), gy);
    k<<<grid, 256, 0, st>>>(mats, trip, n_items, B, (int)ldb, C, (int)ldc, Bs, Cs, N);
  };
  if (pn.V == 4 && pn.L == 8) full ? go(vbr_rows_kernel<4, 8, true>) : go(vbr_rows_kernel<4, 8, false>);
  else if (pn.V == 4 && pn.L == 16) full ? go(vbr_rows_kernel<4, 16, true>) : go(vbr_rows_kernel<4, 16, false>);
  else if (pn.V == 4) full ? go(vbr_rows_kernel<4, 32, true>) : go(vbr_rows_kernel<4, 32, false>);
  else if (pn.V == 2) full ? go(vbr_rows_kernel<2, 32, true>) : go(vbr_rows_kernel<2, 32, false>);
  else full ? go(vbr_rows_kernel<1, 32, true>) : go(vbr_rows_kernel<1, 32, false>);
  if (cudaGetLastError() != cudaSuccess) {
    (void)cudaGetLastError();
    return SABLE_ERR_CUDA;
  }
  return SABLE_OK;
}

sable_status launch_spmm_rows_grouped(const DevHybrid *mats, const int64_t *row_base, int count, int64_t rows,
                                      const float *const *Bs, float *const *Cs, int N, bool vbrc, int cols, int depth,
                                      int sm_count, cudaStream_t_ st) {
  if (count == 0 || rows == 0) return SABLE_OK;
  if (N < 1 || N > 65535 * 32) return SABLE_ERR_INVALID;
  // B_i, C_i are 16-byte aligned when N is a multiple of 4 (documented), 8-byte when even
  const Panel pn = spmm_panel(cols, N, N % 4 == 0, N % 2 == 0);
  const int gy = (N + pn.L * pn.V - 1) / (pn.L * pn.V);
  const bool deep = depth == 8;
  const int64_t per = 8 * (32 / pn.L);   // rows one CTA takes at once
  auto go = [&](auto k) {
    dim3 grid(grid_for(k, 256, 0, (int)std::min<int64_t>(INT32_MAX, (rows + per - 1) / per), sm_count), gy);
    k<<<grid, 256, 0, st>>>(mats, row_base, count, Bs, Cs, N, vbrc ? 1 : 0);
  };
  const bool full = N % (pn.L * pn.V) == 0;
#define SABLE_GROUPED(V_, L_)                                                                             \
  (deep ? (full ? go(spmm_rows_grouped_kernel<V_, L_, 8, true>) : go(spmm_rows_grouped_kernel<V_, L_, 8, false>)) \
        : (full ? go(spmm_rows_grouped_kernel<V_, L_, 4, true>) : go(spmm_rows_grouped_kernel<V_, L_, 4, false>)))
  if (pn.V == 4 && pn.L == 8) SABLE_GROUPED(4, 8);
  else if (pn.V == 4 && pn.L == 16) SABLE_GROUPED(4, 16);
  else if (pn.V == 4) SABLE_GROUPED(4, 32);
  else if (pn.V == 2) SABLE_GROUPED(2, 32);
  else SABLE_GROUPED(1, 32);
#undef SABLE_GROUPED
  if (cudaGetLastError() != cudaSuccess) {
    (void)cudaGetLastError();
    return SABLE_ERR_CUDA;
  }
  return SABLE_OK;
}

}  // namespace sable
