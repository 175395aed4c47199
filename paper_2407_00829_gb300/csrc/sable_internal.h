// Internal declarations shared by the host C++ and CUDA translation units of
// libsable.  Nothing here is part of the public ABI (include/sable.h).
#pragma once

#include <cstdint>
#include <vector>

#include "../../include/sable.h"

struct CUstream_st;
typedef CUstream_st *cudaStream_t_;   // cudaStream_t without including the runtime header

namespace sable {

// Owner tags of canonical entries.
enum : int8_t { OWN_NONE = -1, OWN_VDIA = 0, OWN_VBR = 1, OWN_CSR = 2 };

// Canonical matrix / residual in compressed-row form.  `id` maps each stored
// entry back to its canonical index.
struct Csr {
  int64_t m = 0, n = 0;
  std::vector<int64_t> rp;   // m + 1
  std::vector<int32_t> ci;   // column (or row, for the transposed form)
  std::vector<int64_t> id;   // canonical entry index
  int64_t nnz() const { return rp.empty() ? 0 : rp.back(); }
  // entries of line i with inner index in [lo, hi]
  int64_t count(int64_t i, int64_t lo, int64_t hi) const;
};

// One VDIA segment: rows [row0, row0 + nrows), diagonals off_lo .. off_lo + ndiag - 1.
struct Segment {
  int64_t row0, nrows, off_lo, ndiag;
};

// One VBR block: rows [r0, r0 + nr), columns [c0, c0 + nc).
struct Block {
  int64_t r0, nr, c0, nc;
};

// ---- device-side tables (plain structs shared with the kernels) -------------
struct DevSeg {          // 32 bytes
  int32_t row0, nrows;   // segment rows
  int32_t off_lo, ndiag; // consecutive offsets off_lo .. off_lo + ndiag - 1
  int32_t base;          // row0 rounded down to a multiple of 4
  int32_t ld;            // padded run length (multiple of 4)
  int64_t val_off;       // start of the segment's runs in the value array (floats)
};

struct DevBlk {          // 32 bytes
  int32_t r0, nr, c0, nc;
  int64_t val_off;       // FP32 values, column-major, leading dimension nr
  int64_t bf_off;        // BF16 tile-packed values (elements)
};

struct DevItem {         // 48 bytes: one row tile of a launch
  int32_t r0, r1;        // rows [r0, r1), r0 a multiple of 4
  int32_t seg_lo, seg_hi;// segments overlapping the rows
  int32_t blk_lo, blk_hi;// blocks overlapping the rows
  int32_t mat;           // matrix index (batched launches), 0 otherwise
  int32_t pb, pe;        // CSR remainder entries of the rows: [pb, pe)
  int32_t vcells;        // VDIA + VBR cells of the tile's rows
  int32_t part;          // 0: the tile stores its rows of y; k + 1: a partial tile (a long
                         // CSR range cut in chunks) that stores its row sums in part[k ..]
  int32_t pad;
};

// Row tiles of one launch: items, and per item the indices of the segments
// (iseg[seg_lo, seg_hi)) and blocks (iblk[blk_lo, blk_hi)) touching its rows.
struct DevItems {
  const DevItem *items = nullptr;
  const int32_t *iseg = nullptr;
  const int32_t *iblk = nullptr;
  const DevSeg *pseg = nullptr;    // copies of segs[iseg[k]] (one load per piece)
  const DevBlk *pblk = nullptr;    // copies of blks[iblk[k]]
  int32_t n = 0;
  int32_t rows_max = 0;          // largest r1 - r0
  // tiles whose CSR range was cut: (first row, rows, first part slot, partial
  // tiles) per cut tile; a second launch adds their partial sums to y
  const int32_t *fix = nullptr;  // 4 int32 per cut tile
  int32_t n_fix = 0;
  float *part = nullptr;         // partial row sums, written by the partial tiles
};

// Device copy of one hybrid matrix.
struct DevHybrid {
  int32_t m = 0, n = 0;
  const DevSeg *segs = nullptr;
  const float *vdia = nullptr;
  const DevBlk *blks = nullptr;
  const float *vbr = nullptr;
  const uint16_t *vbr_bf16 = nullptr;
  const uint16_t *vbr_bf16_mid = nullptr;  // second and third bf16 terms (SABLE_FP32_SPLIT)
  const uint16_t *vbr_bf16_lo = nullptr;
  const float *vbr_scale = nullptr;  // per block power-of-two scale
  int32_t n_tc = 0;                  // (block, 128-row tile) pairs for the tensor-core path
  int32_t n_fg = 0;                  // (block, row group) pairs for the FP32 block kernel
  int32_t n_segs = 0, n_blks = 0;
  // per row, the VDIA segments and VBR blocks covering it: refs srp[r] ..
  // srp[r + 1] - 1 of sref, each (index << 1) | (1 for a block); null when
  // the matrix has neither
  const int32_t *srp = nullptr;
  const int32_t *sref = nullptr;
  const int32_t *rp = nullptr;   // CSR remainder row pointer (m + 1)
  const int32_t *ci = nullptr;   // padded by kCsrPad entries
  const float *cv = nullptr;     // padded by kCsrPad entries
  DevItems spmv;
  int32_t *err = nullptr;        // device error word (0 = ok)
};

// Largest SpMV row tile (one CTA of 256 threads, 4 rows per thread) and the
// zero padding after the CSR arrays that lets vector reads run past the last
// entry.
constexpr int kRangeRows = 1024;
constexpr int kCsrPad = 8;

// Host tiling knobs.
struct Tiling {
  int32_t rows_per_item = 512;   // SpMV row tile (<= kRangeRows, multiple of 4)
  int64_t item_bytes = 48 * 1024;
  int32_t spmm_cols = 0;         // SpMM column panel per CTA: 0 = widest the operands allow, 32, 64, 128
  int32_t spmm_depth = 4;        // SpMM: B rows in flight per lane group (4 or 8)
};

// Host-side extracted hybrid form and its device mirror.
struct Hybrid {
  int64_t m = 0, n = 0;
  std::vector<Segment> segs;          // sorted by row0
  std::vector<float> vdia_canon;      // Fig. 4 layout, no padding
  std::vector<Block> blks;            // sorted by r0
  std::vector<float> vbr_canon;       // column-major per block
  std::vector<int64_t> crp;           // CSR remainder
  std::vector<int32_t> cci;
  std::vector<float> ccv;
};

}  // namespace sable

// The opaque plan.
struct sable_plan_s {
  int64_t m = 0, n = 0;
  sable::Csr canon;                    // canonical matrix (sorted, duplicates summed)
  std::vector<float> cval;             // canonical values
  std::vector<std::pair<sable_extractor, sable_extract_params>> extractors;
  std::vector<std::vector<int64_t>> stage_regions;   // per stage: given regions (4 values each)
  std::vector<uint8_t> stage_fixed;                  // per stage: 1 = given regions, 0 = search
  std::vector<int32_t> seg_stage, blk_stage;         // stage of each segment / block (sorted order)
  std::vector<int32_t> canon_of;                     // input COO entry -> canonical entry
  std::vector<int64_t> dest;                         // canonical entry -> index in its format's value array
  std::vector<sable::DevSeg> h_segs;                 // device segment descriptors (padded VDIA layout)
  size_t o_vdia = 0, o_vbr = 0, o_bf16 = 0, o_scale = 0, o_cv = 0, o_pcv = 0;   // value arrays in the blob
  size_t o_bf16_mid = 0, o_bf16_lo = 0;
  std::vector<int8_t> owner;           // per canonical entry
  sable::Hybrid hyb;
  sable::Tiling tiling;
  bool extracted = false, uploaded = false;
  sable_status sticky = SABLE_OK;
  // device state (owned)
  void *dev_blob = nullptr;            // one allocation holding every table
  size_t dev_bytes = 0;
  sable::DevHybrid dev;                // hybrid tables
  sable::DevHybrid *dev_self = nullptr;// device copy of `dev` (matrix table of one entry)
  const int32_t *dev_trip = nullptr;   // (0, block, row tile) triples for the tensor-core path
  const int32_t *dev_fg = nullptr;     // (0, block, row group) triples for the FP32 block kernel
  std::vector<sable::DevItem> h_items_v;   // host copy of the SpMV tile table
  std::vector<int32_t> h_trip, h_fg;
  sable::DevHybrid dev_plain;          // whole matrix as CSR (comparison kernel)
  int32_t *dev_err = nullptr;
  int device = -1;
  int sm_count = 0;
  int inspector = 0;                   // sable_inspector of sable_extract
  int spmv_occ[2] = {0, 0};            // resident SpMV CTAs per SM (hybrid, plain) at ...
  size_t spmv_occ_smem[2] = {0, 0};    // ... this dynamic shared memory per CTA
  sable_plan_stats stats{};
};

namespace sable {
// host_plan.cpp
sable_status fail(sable_plan_t p, sable_status s);
// Allocation-failure injection (sable_debug_fail_allocations): alloc_point()
// throws std::bad_alloc, and alloc_fails() returns true, when the countdown
// reaches this guarded allocation; both do nothing while injection is off.
void alloc_point();
bool alloc_fails();
// sable_inspect.cu: the device inspector (the extractors' counting steps on the
// GPU, integer arithmetic only).  A residual CSR copied to the current device,
// with a stream of its own; every call is synchronous.
struct DevResidual;
sable_status dev_residual_open(const Csr &R, DevResidual **out);
void dev_residual_close(DevResidual *D);
// M[d + m] = residual entries on diagonal d, |d| <= d_max (size m + n + 1)
sable_status dev_diag_counts(DevResidual *D, int64_t d_max, std::vector<int64_t> &M);
// FitRibbon of every residual entry (i, i + d) with |d| <= d_max and cand[d + m]
// set: ext[k] = l | u << 10 | z << 20 for the entry at CSR position k (0 for
// the others); zt[w] = least q with q / w >= delta in FP64 (w + 1 if none),
// w in [0, 2 w_max + 1]
sable_status dev_fit_ribbons(DevResidual *D, int64_t d_max, const std::vector<unsigned char> &cand, int w_max,
                             const std::vector<int32_t> &zt, std::vector<uint32_t> &ext);
// keys I * TJ + J of the g x g cells whose count c has c >= delta * area in FP64,
// i.e. c >= thr[area] (area in [1, g^2]), ascending
sable_status dev_hot_cells(DevResidual *D, int g, const std::vector<int32_t> &thr, std::vector<int64_t> &hot);
// a failed device inspector call, thrown through the extractors to sable_extract
struct InspectError {
  sable_status status;
};

// host_band.cpp: Algorithms 3 and 4; returns accepted segments (acceptance order)
// as (row0, row_end, d, L, U).  With `dev`, M[d] and FitRibbon come from the
// device inspector (same results).
struct BandSeg { int64_t i0, i1, d, L, U, z; };
std::vector<BandSeg> extract_bands(const Csr &R, const sable_extract_params &p, DevResidual *dev = nullptr);
// host_block.cpp: Algorithms 1 and 2; returns accepted blocks (acceptance order).
// With `dev`, the candidate-region cell counts come from the device inspector.
struct BlockFound { int64_t r0, r1, c0, c1, nnz; };
std::vector<BlockFound> partition_blocks(const Csr &R, const Csr &RT, const sable_extract_params &p,
                                         DevResidual *dev = nullptr);
// threads used by the host extractors
int host_threads();
// sable_tc.cu: BF16 VBR blocks on the tensor cores
void pack_vbr_bf16(const std::vector<Block> &blks, const std::vector<float> &canon,
                   std::vector<uint16_t> &packed, std::vector<float> &scales, std::vector<int64_t> &offs,
                   std::vector<uint16_t> *mid = nullptr, std::vector<uint16_t> *lo = nullptr);
void vbr_tc_pairs(const std::vector<Block> &blks, int32_t mat, std::vector<int32_t> &trip);
// sable_device.cu: column panel of the row-split SpMM kernels (V columns per
// lane, L lanes per row)
struct Panel { int V, L; };
Panel spmm_panel(int cols, int64_t N, bool vec, bool vec2);
// sable_device.cu: FP32 VBR blocks of SpMM in groups of rows (stores their rows of C)
void vbr_group_pairs(const std::vector<Block> &blks, int32_t mat, std::vector<int32_t> &trip);
sable_status launch_vbr_rows(const DevHybrid *mats, const int32_t *trip, int n_items, const float *B, int64_t ldb,
                             float *C, int64_t ldc, const float *const *Bs, float *const *Cs, int N, int cols,
                             int sm_count, cudaStream_t_ st);
sable_status launch_vbr_tc(const DevHybrid *mats, const int32_t *trip, int n_trip, const float *B, int64_t ldb,
                           float *C, int64_t ldc, const float *const *Bs, float *const *Cs, int N, int sm_count,
                           int *err, cudaStream_t_ st, int terms);
sable_status launch_spmv_grouped(const DevHybrid *mats, const DevItem *items, int n_items, int rows_max,
                                 const float *const *xs, float *const *ys, int sm_count, cudaStream_t_ st);
sable_status launch_spmm_rows_grouped(const DevHybrid *mats, const int64_t *row_base, int count, int64_t rows,
                                      const float *const *Bs, float *const *Cs, int N, bool vbrc, int cols, int depth,
                                      int sm_count, cudaStream_t_ st);
// sable_spmv.cu
int spmv_resident_ctas(int rows_max);   // SpMV CTAs one SM holds at this tile height
sable_status launch_spmv(sable_plan_t P, const DevHybrid &D, bool plain, const float *x, float *y,
                         cudaStream_t_ st);
}  // namespace sable
