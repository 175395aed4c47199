/*
 * sable.h -- C ABI of the GB300 hybrid VDIA+VBR+CSR SpMV/SpMM library.
 *
 * The library follows the plan -> extract -> dispatch pipeline of the paper
 * (Section 3, Fig. 2): a plan holds a sparse matrix and an ordered list of
 * extractors; extraction carves the matrix into VDIA diagonal segments
 * (Section 4.2, Algorithms 3 and 4), VBR dense blocks (Section 4.1,
 * Algorithms 1 and 2) and a CSR remainder (Appendix A.1); the SpMV/SpMM
 * entry points then compute y = A x or C = A B (Section 5, "Kernels") with one
 * CUDA kernel launch over a device table of row tiles.  Extraction runs on the
 * host (native C++); every arithmetic step of SpMV/SpMM runs in this
 * library's CUDA kernels.  There is no CPU fallback: without a CUDA device the
 * compute calls return SABLE_ERR_CUDA.
 *
 * Conventions for every call:
 *   - Indices are 0-based.  Matrices are m x n.  Dense operands are row-major.
 *   - Host pointers are read during the call only and copied where kept.
 *   - Device pointers (x, y, B, C, the pointer tables of the batch calls) are
 *     owned by the caller and must stay valid until the stream work ends.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream); compute
 *     calls are asynchronous and ordered on it.
 *   - Errors are reported by status code only; the library never aborts or
 *     prints.  The first error of a plan is kept (sticky) and returned by
 *     every later call on that plan; sable_plan_status() reads it.
 *   - A plan may be used by one host thread at a time.
 */
#ifndef SABLE_H
#define SABLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SABLE_OK = 0,
  SABLE_ERR_INVALID = 1,     /* bad argument: index out of range, size, NULL   */
  SABLE_ERR_OOM = 2,         /* host or device allocation failed               */
  SABLE_ERR_CUDA = 3,        /* a CUDA runtime call failed (or no device)      */
  SABLE_ERR_INCOMPLETE = 4,  /* extractors left entries unclaimed (Section 3)  */
  SABLE_ERR_ORDER = 5,       /* call made in the wrong phase of the plan       */
  SABLE_ERR_TIMEOUT = 6,     /* a bounded device wait gave up                  */
  SABLE_ERR_KERNEL = 7,      /* a kernel's own bounds check tripped            */
  SABLE_ERR_UNSUPPORTED = 8  /* valid request the library does not implement  */
} sable_status;

/* Extractor kinds (Section 3.2).  SABLE_X_CSR claims everything left and must
 * come last for the plan to be complete. */
typedef enum { SABLE_X_VDIA = 0, SABLE_X_VBR = 1, SABLE_X_CSR = 2 } sable_extractor;

/* Arithmetic of the VBR blocks in SpMM.  SABLE_BF16_BLOCKS stores each block
 * as bfloat16 (round to nearest even) of value / s_b with a per-block power of
 * two s_b = 2^ceil(log2 max|a|), rounds the B rows it multiplies to bfloat16,
 * runs the block products on the tensor cores (tcgen05, FP32 accumulation)
 * and multiplies by s_b; VDIA and CSR parts stay FP32.
 * SABLE_FP32_SPLIT keeps FP32 accuracy on the tensor cores: each block value
 * / s_b and each B value is the sum of three bfloat16 terms (the value
 * rounded, then its exact FP32 remainders rounded: 24 significant bits), and
 * the six term products down to 2^-24 of the product are accumulated in
 * FP32.  SABLE_FP32 runs the blocks on the FP32 FMA pipes. */
typedef enum { SABLE_FP32 = 0, SABLE_BF16_BLOCKS = 1, SABLE_FP32_SPLIT = 2 } sable_precision;

/* Extractor parameters.  Fields an extractor does not use are ignored.
 *   delta        density floor (Section 4.1: 0.5 for blocks; Section 5 uses
 *                0.75 for bands)
 *   a_min        minimum area of a block / of a band candidate (2500)
 *   l_seg        minimum rows of a VDIA segment (Algorithm 4)
 *   w_max        largest ribbon half-width FitRibbon may reach (<= 512)
 *   d_max        largest |diagonal offset| considered (0 = all)
 *   count_min    entries a diagonal needs to be a candidate (0 = ceil(delta*l_seg))
 *   coverage_min share of entries blocks must cover, else none are kept (0.08)
 *   max_span     cap on FindBlock's outer span (Algorithm 2)
 *   tile         candidate-region pre-pass cell size; 0 runs Algorithm 1 on
 *                the whole matrix
 *   passes       VDIA: runs of Algorithm 3, each over the residual the previous
 *                one left and with its own row mask, so a row may carry bands
 *                of several passes at different offsets (multi-ribbon VDIA; a
 *                segment's diagonal set is its own, Section 4.2.1); added as
 *                that many consecutive band stages; 1..8, default 1 */
typedef struct {
  double delta;
  int64_t a_min;
  int32_t l_seg;
  int32_t w_max;
  int64_t d_max;
  int64_t count_min;
  double coverage_min;
  int32_t max_span;
  int32_t tile;
  int32_t passes;
} sable_extract_params;

/* Summary of an extracted plan.  Byte counts are the algorithmic bytes one
 * call must move: every stored value, index and pointer once, x (or B) once
 * and y (or C) written once. */
typedef struct {
  int64_t m, n, nnz;                 /* canonical entries (duplicates summed)  */
  int64_t nnz_vdia, nnz_vbr, nnz_csr;/* entries claimed by each format         */
  int64_t n_segments, n_diagonals;   /* VDIA segments, sum of their diagonals  */
  int64_t vdia_cells;                /* stored VDIA cells (entries + padding)  */
  int64_t n_blocks, vbr_cells;       /* VBR blocks and their stored cells      */
  int64_t n_items;                   /* row tiles of the SpMV launch           */
  int64_t spmv_bytes;                /* algorithmic bytes of one sable_spmv    */
  int64_t csr_spmv_bytes;            /* same for plain CSR of the whole matrix */
} sable_plan_stats;

typedef struct sable_plan_s *sable_plan_t;
typedef struct sable_batch_s *sable_batch_t;

/* Fill `out` with the defaults for one extractor kind. */
void sable_default_params(sable_extractor kind, sable_extract_params *out);

/* Create a plan from host COO triples (copied).  nnz may be 0.  Duplicate
 * coordinates are summed (FP64 in input order, rounded once to FP32);
 * explicit zeros are structural entries.  Errors: SABLE_ERR_INVALID for a
 * negative size, m or n >= 2^31, nnz >= 2^31, a NULL array with nnz > 0 or
 * an index outside the matrix; SABLE_ERR_OOM. */
sable_status sable_plan_create(int64_t m, int64_t n, int64_t nnz, const int32_t *row,
                               const int32_t *col, const float *val, sable_plan_t *out);

/* Append an extractor (Section 3, "Extract").  params NULL = defaults.
 * Errors: SABLE_ERR_ORDER after sable_extract; SABLE_ERR_INVALID. */
sable_status sable_plan_add_extractor(sable_plan_t plan, sable_extractor kind,
                                      const sable_extract_params *params);

/* Append a stage of given regions instead of a search: the saved region
 * table of an earlier extraction, so that a plan can be rebuilt without
 * running the extractors again, e.g. for the same structure with new values
 * (the paper keeps its extracted regions on disk and reuses them when only
 * the values change, Section 3.4).  kind SABLE_X_VDIA: `count` rows of
 * (row_start, nrows, lowest offset j - i, ndiags), rows within [0, m),
 * offsets within [-(m-1), n-1]; kind SABLE_X_VBR: `count` rows of (row0,
 * nrows, col0, ncols) inside the matrix.  int64, row-major, copied.  At
 * sable_extract the stage runs in its place among the stages: its regions,
 * in the given order, claim the residual entries inside their areas that no
 * earlier region claimed; a region is kept even if it claims nothing.  With
 * sable_plan_get_region_stages this reproduces an extraction exactly.
 * Errors: SABLE_ERR_ORDER after sable_extract; SABLE_ERR_INVALID (kind CSR,
 * a region outside the matrix, count < 0); SABLE_ERR_OOM. */
sable_status sable_plan_add_regions(sable_plan_t plan, sable_extractor kind, const int64_t *regions,
                                    int64_t count);

/* Where sable_extract runs the extractors' counting steps (the inspector).
 * SABLE_INSPECT_HOST (default): everything on the host.  SABLE_INSPECT_DEVICE:
 * on the current CUDA device, integer arithmetic only, for each band stage the
 * diagonal histogram M[d] of Algorithm 3 and FitRibbon (Section 4.2) of every
 * residual entry on a candidate diagonal, and for each block stage with tile > 0 the
 * entry counts of the candidate-region pre-pass's cells; candidate order,
 * GrowSegments (Algorithm 4), acceptance, FindBlock (Algorithm 2) and Trim
 * stay on the host.  Both give the same regions, entry for entry (each FP64
 * density test of the host becomes an integer threshold the host computes
 * with the same FP64 expression). */
typedef enum { SABLE_INSPECT_HOST = 0, SABLE_INSPECT_DEVICE = 1 } sable_inspector;

/* Choose the inspector of a plan's sable_extract.  Errors: SABLE_ERR_ORDER
 * after sable_extract; SABLE_ERR_INVALID for another value. */
sable_status sable_plan_set_inspector(sable_plan_t plan, sable_inspector where);

/* Run the extractors in order over the residual, check that the residual is
 * empty and that the regions partition the entries exactly, and build the
 * host tables (Section 3, "Extract"/"Dispatch", Section 3.4).  With the host
 * inspector no CUDA call is made; with the device inspector each searching
 * band or block stage copies its residual CSR to the current device and works
 * on a stream of its own, synchronously, freeing what it allocated before it
 * returns.  Errors: SABLE_ERR_INCOMPLETE if entries are left unclaimed;
 * SABLE_ERR_ORDER if called twice; device inspector: SABLE_ERR_UNSUPPORTED
 * (nothing done, not sticky) for a block stage with tile > 64, SABLE_ERR_CUDA
 * (no device, or a CUDA call failed) and SABLE_ERR_OOM. */
sable_status sable_extract(sable_plan_t plan);

/* Copy the plan's tables to the current CUDA device (asynchronously on
 * `stream`; host copies are kept until destroy).  Errors: SABLE_ERR_ORDER
 * before sable_extract; SABLE_ERR_OOM / SABLE_ERR_CUDA. */
sable_status sable_plan_upload(sable_plan_t plan, void *stream);

/* y := A x.  x: device, n floats; y: device, m floats (overwritten).  One
 * launch over the plan's row tiles; when the upload cut a tile whose CSR range
 * is longer than two chunks (rows of tens of thousands of entries; a chunk is
 * the entries of one tile at the byte target, at least 4096), partial tiles
 * sum the rest of that range on other CTAs and a second, small launch adds
 * their row sums to y.  Those partial sums live in the plan's device memory:
 * two SpMVs of such a plan must not run at the same time (on two streams).
 * Errors: SABLE_ERR_ORDER before upload; SABLE_ERR_INVALID; SABLE_ERR_CUDA. */
sable_status sable_spmv(sable_plan_t plan, const float *x, float *y, void *stream);

/* C := A B.  B: device, n x N row-major with leading dimension ldb >= N;
 * C: device, m x N row-major, ldc >= N (overwritten).  1 <= N <= 65535 * 32;
 * ldb, ldc <= INT32_MAX.  SABLE_BF16_BLOCKS / SABLE_FP32_SPLIT as documented
 * at sable_precision: the tensor-core launch stores the blocks' rows of C,
 * then one row-split launch adds each row's VDIA diagonals, FP32 blocks and
 * CSR entries.  VBR blocks of different stages that share rows stay on the
 * FP32 path in every precision.  Errors: SABLE_ERR_ORDER before upload;
 * SABLE_ERR_INVALID; SABLE_ERR_CUDA. */
sable_status sable_spmm(sable_plan_t plan, const float *B, int64_t N, int64_t ldb, float *C,
                        int64_t ldc, sable_precision prec, void *stream);

/* Plain CSR SpMV of the whole canonical matrix (no extraction), with the
 * library's CSR kernel: the "plain GPU CSR" comparison point.  Requires
 * upload.  y := A x as for sable_spmv. */
sable_status sable_csr_spmv(sable_plan_t plan, const float *x, float *y, void *stream);

/* Plain CSR SpMM of the whole canonical matrix (comparison point). */
sable_status sable_csr_spmm(sable_plan_t plan, const float *B, int64_t N, int64_t ldb,
                            float *C, int64_t ldc, void *stream);

/* Statistics of an extracted plan.  Errors: SABLE_ERR_ORDER before extract. */
sable_status sable_plan_info(sable_plan_t plan, sable_plan_stats *out);

/* Host exports of an extracted plan (for checking; sizes from plan_info).
 * segments: n_segments x 4 int64 (row_start, nrows, lowest offset, ndiags),
 *           sorted by row_start; diagonals of a segment are consecutive
 *           offsets.
 * blocks:   n_blocks x 4 int64 (row0, nrows, col0, ncols), sorted by row0.
 * vdia values: vdia_cells floats, segment by segment, diagonal-major
 *           (Fig. 4 layout, no padding).
 * vbr values: vbr_cells floats, block by block, column-major (Fig. 9).
 * csr: row_ptr m+1 int64, col nnz_csr int32, val nnz_csr floats, rows sorted,
 *           columns ascending within a row. */
sable_status sable_plan_get_segments(sable_plan_t plan, int64_t *out);
sable_status sable_plan_get_blocks(sable_plan_t plan, int64_t *out);
sable_status sable_plan_get_vdia_values(sable_plan_t plan, float *out);
sable_status sable_plan_get_vbr_values(sable_plan_t plan, float *out);
sable_status sable_plan_get_csr(sable_plan_t plan, int64_t *row_ptr, int32_t *col, float *val);
/* The stage (0-based position among the extractors and region stages, in the
 * order they were added) that produced each segment and each block, in the
 * order of sable_plan_get_segments / sable_plan_get_blocks: n_segments and
 * n_blocks int32.  Together they are the plan's region table. */
sable_status sable_plan_get_region_stages(sable_plan_t plan, int32_t *seg_stage, int32_t *blk_stage);

/* New values for the same structure: the extracted regions and, after
 * upload, the device tables are kept and only the values are replaced (the
 * paper's inspector-executor reuse: the regions depend on the structure only,
 * so a program built for one matrix serves every matrix with the same
 * pattern, Sections 2 and 3.4).  val: host, the nnz floats of the COO given to
 * sable_plan_create, in that order (duplicates are summed again as there:
 * FP64 in input order, rounded once).  The BF16 copies of the blocks and
 * their scales are recomputed.  With an uploaded plan the device must be the
 * plan's; the values are copied on `stream`, which the call waits for.
 * Errors: SABLE_ERR_INVALID; SABLE_ERR_ORDER before sable_extract;
 * SABLE_ERR_OOM / SABLE_ERR_CUDA. */
sable_status sable_plan_update_values(sable_plan_t plan, const float *val, void *stream);

/* Start the plan over from its canonical matrix: drop the stages, the
 * extraction and the device tables (cudaFree, which waits for the device),
 * keep the matrix and the tiling, clear the recorded error.  New stages can
 * then be added and extracted: one matrix, many plans, without copying and
 * sorting the COO input again.  Errors: SABLE_ERR_INVALID; SABLE_ERR_CUDA. */
sable_status sable_plan_reset(sable_plan_t plan);

/* Tuning of the row tiles of the SpMV launch; takes effect at the next
 * upload.  spmv_rows: rows of an SpMV tile, a multiple of 4 in [4, 1024];
 * spmv_bytes: target algorithmic bytes per SpMV tile (>= 64).  SpMM is row
 * split (a lane group per row) and depends only on the column panel and depth
 * below.  Errors: SABLE_ERR_INVALID. */
sable_status sable_plan_set_tiling(sable_plan_t plan, int32_t spmv_rows, int64_t spmv_bytes);

/* The plan's current tiling. */
typedef struct {
  int32_t spmv_rows;
  int64_t spmv_bytes;
  int32_t spmm_cols;   /* 0 = widest panel the operands allow; else 32, 64 or 128 */
  int32_t spmm_depth;  /* B rows in flight per lane group in SpMM: 4 or 8 */
} sable_tiling;
sable_status sable_plan_get_tiling(sable_plan_t plan, sable_tiling *out);

/* Columns of C (and B) one SpMM CTA works on: 128, 64 or 32.  With N, ldb,
 * ldc multiples of 4 and 16-byte aligned B, C every lane holds four columns
 * and a group of 32, 16 or 8 lanes owns a row, so narrow panels put several
 * rows on a warp; otherwise 64 means two columns per lane (even N, ldb, ldc,
 * 8-byte alignment) and 32 one.  0 picks the widest the operands allow, or
 * for N <= 32 (<= 64) the 32- (64-) column panel.  The column panels of one
 * launch run one after another, so a narrower panel keeps a smaller slice of
 * B live in L2 while its rows are gathered.  Takes effect at the next SpMM
 * call.  Errors: SABLE_ERR_INVALID. */
sable_status sable_plan_set_spmm_cols(sable_plan_t plan, int32_t cols);

/* B rows each lane group has in flight in SpMM: 4 (default) or 8 (more loads
 * in flight, more registers: at most 4 CTAs per SM).  Takes effect at the
 * next SpMM call.  Errors: SABLE_ERR_INVALID. */
sable_status sable_plan_set_spmm_depth(sable_plan_t plan, int32_t depth);

/* Autotuner (no counterpart in the paper, which runs one generated kernel per
 * region): time the plan's op over candidate tilings with CUDA events on
 * `stream` and leave the plan uploaded with the fastest.  op 0 = SpMV (in =
 * x, out = y), 4 = plain CSR SpMV (sable_csr_spmv), 1 = SpMM FP32, 2 = SpMM
 * with BF16 blocks, 3 = SpMM with SABLE_FP32_SPLIT blocks (in = B, n x N, out =
 * C, m x N, row-major with leading dimension N); in / out are device buffers
 * the timed launches read and overwrite.  Candidates: SpMV rows {32, 64, 128,
 * 256, 512, 1024} x bytes {4K, 16K, 48K, 160K}, and 1024 rows with the bytes that cut
 * the plan into 1, 2 or 3 full waves of the CTAs the GPU holds at once; SpMM
 * (column panel, rows in flight) in {128, 64, 32} x {4, 8}; the other op's
 * tiling is kept.  Each candidate is
 * uploaded (sable_plan_upload, which reallocates the plan's device tables and
 * waits for the device), then timed as the best of two rounds of `reps`
 * launches: for the SpMV ops the `reps` launches are captured in one CUDA
 * graph on a stream of the library's own and the graph is replayed on
 * `stream` (a small plan's launch is shorter than the host's work per call);
 * for SpMM, after two warm-up runs, `reps` back-to-back launches.  The winner is remembered per shape class
 * (op, floor log2 of N, m and nnz, and the quarters of the entries in VDIA
 * and in VBR) for the life of the process; with use_cache != 0 a known class
 * is applied and timed without a search.  chosen / chosen_ms (host, may be
 * NULL) receive the tiling and its mean launch time.  Repeated launches of one
 * plan keep a matrix smaller than L2 resident there, so small plans are tuned
 * warm.  Errors: SABLE_ERR_INVALID; SABLE_ERR_ORDER before extract; errors of
 * upload and of the op. */
sable_status sable_autotune(sable_plan_t plan, int32_t op, int64_t N, const float *in, float *out, int32_t reps,
                            int32_t use_cache, sable_tiling *chosen, float *chosen_ms, void *stream);
/* Forget every remembered tiling; returns how many there were. */
int64_t sable_autotune_cache_clear(void);

/* ---- Batches: many matrices in one grouped launch per op ----------------
 * A batch is built from `count` uploaded plans (same device; the plans must
 * outlive the batch).  It concatenates their row-tile tables, each tile
 * tagged with its matrix, so that one launch computes every region of every
 * matrix.  Errors: SABLE_ERR_ORDER if a plan is not uploaded;
 * SABLE_ERR_INVALID (NULL, other device, plan in error); SABLE_ERR_OOM;
 * SABLE_ERR_UNSUPPORTED for a plan whose SpMV tiles were cut (a CSR range of
 * more than two chunks, see sable_spmv): run such a plan on its own. */
sable_status sable_batch_create(const sable_plan_t *plans, int32_t count, sable_batch_t *out);

/* y_i := A_i x_i for every matrix i of the batch, one launch.  x and y are
 * DEVICE arrays of `count` device pointers (x_i: n_i floats, y_i: m_i floats). */
sable_status sable_batch_spmv(sable_batch_t batch, const float *const *x, float *const *y, void *stream);

/* C_i := A_i B_i, one launch (two with tensor-core blocks).  B and C are
 * DEVICE arrays of device pointers; B_i is n_i x N and C_i is m_i x N,
 * row-major with leading dimension N; when N is a multiple of 4 every B_i and
 * C_i must be 16-byte aligned, when N is even 8-byte aligned.  The rows of all
 * matrices are split over the warps of one persistent launch (a warp per row,
 * as in sable_spmm), with the column panel and B rows in flight of the first
 * plan's tiling (sable_plan_set_spmm_cols / sable_plan_set_spmm_depth). */
sable_status sable_batch_spmm(sable_batch_t batch, const float *const *B, int64_t N, float *const *C,
                              sable_precision prec, void *stream);

/* Capture the batch's SpMV / SpMM launches (with these operand tables) into a
 * CUDA graph; sable_graph_launch replays it on a stream.  The operand tables
 * and the buffers they point to are read at every replay. */
typedef struct sable_graph_s *sable_graph_t;
sable_status sable_batch_graph_spmv(sable_batch_t batch, const float *const *x, float *const *y,
                                    sable_graph_t *out);
sable_status sable_batch_graph_spmm(sable_batch_t batch, const float *const *B, int64_t N, float *const *C,
                                    sable_precision prec, sable_graph_t *out);
sable_status sable_graph_launch(sable_graph_t graph, void *stream);
sable_status sable_graph_destroy(sable_graph_t graph);

/* Device error word of the batch (0, or a sable_status recorded by a kernel). */
sable_status sable_batch_status(sable_batch_t batch, int32_t *device_error);
sable_status sable_batch_destroy(sable_batch_t batch);

/* ---- Learned planner support (the planner itself is a layer on top of the
 * paper's pipeline; its knobs are the extractor order and thresholds of
 * Section 3.2 / 4.1 / 4.2 and Section 5's delta) ----------------------------
 *
 * Structural features of a COO matrix (device arrays row/col, nnz entries):
 * writes SABLE_NFEAT floats to `out` (device): sizes, row-length statistics
 * and histogram, the share of entries on sparse / dense diagonals (the
 * histogram M[d] of Algorithm 3), the share near the main diagonal, and the
 * share of entries in dense 8 x 8 tiles (the block extractor's candidate test,
 * counted in a hash table over at most 2^22 sampled entries).  The exact
 * definitions are in the implementation's header comment.  `work` is a device
 * workspace of at least sable_features_workspace_bytes(m, n, nnz) bytes.
 * Indices should lie in [0, m) x [0, n); the kernels check every entry,
 * skip one that does not (it is never used as an index) and then write every
 * feature as NaN, since the host cannot see the device arrays before the
 * asynchronous launch.  Errors: SABLE_ERR_INVALID; SABLE_ERR_CUDA. */
#define SABLE_NFEAT 24
int64_t sable_features_workspace_bytes(int64_t m, int64_t n, int64_t nnz);
sable_status sable_features(int64_t m, int64_t n, int64_t nnz, const int32_t *row, const int32_t *col,
                            void *work, int64_t work_bytes, float *out, void *stream);

/* sable_features without a caller workspace and without any allocation.  The
 * paper has no counterpart: this entry point serves callers that may not call
 * cudaMalloc, for instance a host framework that owns all of a GPU's memory
 * through its own pool and forbids outside allocations, a plugin interface
 * that hands over only input and output pointers, or latency-critical code
 * that cannot take the device-wide synchronisation cudaMalloc / cudaFree may
 * cause.  The scratch (row and diagonal counters, the tile hash table) is one
 * fixed array of SABLE_FEATURES_NOALLOC_MAX_BYTES (32 MiB) that every GPU
 * holds from loading the library's device code until the process exits.
 *  - Same inputs, output and results as sable_features (entries outside the
 *    matrix included: skipped, every feature NaN); no workspace argument.
 *  - Sizes whose workspace, sable_features_workspace_bytes(m, n, nnz), exceeds
 *    SABLE_FEATURES_NOALLOC_MAX_BYTES are rejected with SABLE_ERR_UNSUPPORTED
 *    before any device work (for example nnz <= 2^20 with 2m + n <= 2,000,000 fits).
 *  - The first call on a device looks up that device's address of the array
 *    (cudaGetSymbolAddress, with the device current); make that first call
 *    before any stream capture.  The address is kept for the life of the
 *    process: do not call this entry point after cudaDeviceReset or any other
 *    teardown of the device's primary context.
 *  - The call allocates nothing: no cudaMalloc, cudaFree or allocating library
 *    routine.  It clears the array's counters and table on `stream` before
 *    using them, since the array keeps the previous call's contents.
 *  - All calls on a device share the one array: calls that may overlap on the
 *    GPU (other streams, other host threads) race and give wrong features;
 *    order them (one stream, or events).
 * Errors: SABLE_ERR_INVALID (bad arguments); SABLE_ERR_UNSUPPORTED (too
 * large, or device ordinal >= 64); SABLE_ERR_CUDA. */
#define SABLE_FEATURES_NOALLOC_MAX_BYTES (32 << 20)
sable_status sable_features_noalloc(int64_t m, int64_t n, int64_t nnz, const int32_t *row, const int32_t *col,
                                    float *out, void *stream);

/* A multilayer perceptron n_in -> n_h1 (ReLU) -> n_h2 (ReLU) -> n_out (linear),
 * FP32.  Parameters live in one caller-owned device buffer of
 * sable_mlp_param_count() floats: W1 [n_in x n_h1], b1, W2 [n_h1 x n_h2], b2,
 * W3 [n_h2 x n_out], b3, matrices row-major.  `work` is a device workspace of
 * sable_mlp_work_floats(shape, batch) floats.  X is [batch x n_in], Y and T
 * are [batch x n_out], row-major, device. */
typedef struct {
  int32_t n_in, n_h1, n_h2, n_out;
} sable_mlp_shape;
int64_t sable_mlp_param_count(const sable_mlp_shape *shape);
int64_t sable_mlp_work_floats(const sable_mlp_shape *shape, int64_t batch);
/* Y = MLP(X). */
sable_status sable_mlp_forward(const sable_mlp_shape *shape, const float *params, const float *X, int64_t batch,
                               float *Y, float *work, void *stream);
/* Forward, masked mean squared error L = sum mask (Y - T)^2 / sum mask (mask
 * NULL = all ones; written to *loss, device, if loss is not NULL) and the
 * gradient dL/dparams into `grads` (same layout as params). */
sable_status sable_mlp_grad(const sable_mlp_shape *shape, const float *params, const float *X, const float *T,
                            const float *mask, int64_t batch, float *grads, float *loss, float *work, void *stream);
/* One Adam step (bias-corrected, step >= 1) on `count` parameters. */
sable_status sable_mlp_adam(int64_t count, float *params, const float *grads, float *m, float *v, int64_t step,
                            float lr, float beta1, float beta2, float eps, void *stream);

/* Calibration: `count` random 4-byte reads of x[0..n) (device), indices from a
 * fixed hash reduced modulo n, one kernel launch on `stream`; `out` (device,
 * one float) may be written.  Timing it gives the device's rate of random
 * single-word gathers, the ceiling of the CSR part of SpMV on matrices with
 * scattered entries.  No counterpart in the paper.  Errors: SABLE_ERR_INVALID. */
sable_status sable_probe_gather(const float *x, int64_t n, int64_t count, float *out, void *stream);

/* Calibration: `count` random row reads of B (device, row-major, n rows of
 * leading dimension ld floats; the caller's buffer holds (n - 1) * ld + N
 * floats), N columns each, row indices from a fixed hash reduced modulo n, one
 * warp per row, one kernel launch on `stream`; `out` (device, one float) may
 * be written.  Timing it gives the device's rate of random dense-row gathers,
 * the ceiling of the CSR part of SpMM (one row of B per entry).  No
 * counterpart in the paper.  Errors: SABLE_ERR_INVALID unless 4 <= N <= 128,
 * N and ld are multiples of 4, ld >= N and B is 16-byte aligned. */
sable_status sable_probe_row_gather(const float *B, int64_t n, int64_t ld, int32_t N, int64_t count, float *out,
                                    void *stream);

/* Calibration: `count` random 16-byte chunks of x (device, n >= 4 floats,
 * 16-byte aligned; chunk indices from a fixed hash reduced modulo n / 4)
 * copied into shared memory by the bulk-copy (TMA) unit, cp.async.bulk
 * completing on mbarriers, one launch on `stream`.  Timing it gives the rate
 * of random x reads that bypass the load path's per-line lookups, beside
 * sable_probe_gather's.  `out` (device, one float) may be written; `status`
 * (device, one int32) receives 0, or SABLE_ERR_TIMEOUT if a wait ran past
 * the wait limit (the kernel still waits, bounded, for its copies before it
 * exits).  No counterpart in the paper.  Errors: SABLE_ERR_INVALID. */
sable_status sable_probe_bulk_gather(const float *x, int64_t n, int64_t count, float *out, int32_t *status,
                                     void *stream);

/* The budget, in GPU clock cycles, of every bounded device wait of the
 * library (the tensor-core kernel's mbarrier waits, the bulk-copy probe),
 * read at each launch; default 4e9 (about 2 s).  A wait that runs past it
 * makes its kernel record SABLE_ERR_TIMEOUT, skip its remaining work, wait
 * (bounded) for its own copies in flight, free what it holds and return; the
 * CUDA context stays usable.  Process-wide.  No counterpart in the paper.
 * Errors: SABLE_ERR_INVALID unless 1000 <= cycles <= 2^40. */
sable_status sable_set_wait_limit(int64_t cycles);
int64_t sable_get_wait_limit(void);

/* A bounded wait that nothing satisfies (an mbarrier whose one expected
 * arrival never comes), with the current wait limit: `status` (device, one
 * int32) receives SABLE_ERR_TIMEOUT once the budget runs out.  For testing
 * that waits end with a status instead of a hang; nothing else is in flight.
 * No counterpart in the paper.  Errors: SABLE_ERR_INVALID; SABLE_ERR_CUDA. */
sable_status sable_probe_wait_limit(int32_t *status, void *stream);

/* Accuracy of a result, reduced on the device in FP64: the error of an FP32
 * result y against an FP64 reference (the oracle's), as the normwise
 * relative error max|y - ref| / max|ref| that the library's accuracy budget
 * is stated in (1e-5 FP32, 2e-2 BF16 blocks) and its 2-norm analogue.
 * y: device, count floats; ref: device, count doubles; out: device, 4
 * doubles = max_i |y_i - ref_i|, max_i |ref_i|, sum (y_i - ref_i)^2,
 * sum ref_i^2 (a NaN anywhere makes the maxima NaN).  work: device workspace
 * of sable_error_workspace_bytes() bytes.  Two launches of a fixed grid with
 * fixed-order reductions: the result is the same on every run.  No
 * counterpart in the paper.  Errors: SABLE_ERR_INVALID; SABLE_ERR_CUDA. */
int64_t sable_error_workspace_bytes(void);
sable_status sable_error_norms(const float *y, const double *ref, int64_t count, double *out, void *work,
                               int64_t work_bytes, void *stream);

/* The plan's device error word, 4 int32 copied to host `out` (synchronous):
 * a status recorded by a kernel (0 = none; SABLE_ERR_TIMEOUT from a bounded
 * wait of the tensor-core kernel; SABLE_ERR_KERNEL from an index check of the
 * debug build), then three words of detail: for an index check, its tag (1 =
 * SpMV CSR column, 2 = SpMV block column, 3 = SpMM CSR column, 4 = SpMM
 * block column), the index and its bound; 0 otherwise.  The debug build is
 * the library compiled with SABLE_CHECKS (`build.py --checks`): its SpMV and
 * row-split SpMM kernels test every column they gather with against the
 * matrix's width, record the first bad one here and skip it.  The word is
 * cleared at upload.  Errors: SABLE_ERR_ORDER before upload; SABLE_ERR_CUDA. */
sable_status sable_plan_device_error(sable_plan_t plan, int32_t *out);

/* Debug build only: overwrite entry `entry` (0 .. nnz_csr - 1, in row order)
 * of an uploaded plan's device CSR remainder columns with `value`, so that a
 * test can make the index checks record SABLE_ERR_KERNEL.  The release build
 * returns SABLE_ERR_UNSUPPORTED and changes nothing (its kernels do not check
 * columns).  No counterpart in the paper.  Errors: SABLE_ERR_UNSUPPORTED;
 * SABLE_ERR_INVALID; SABLE_ERR_ORDER before upload; SABLE_ERR_CUDA. */
sable_status sable_debug_set_csr_column(sable_plan_t plan, int64_t entry, int32_t value);

/* Testing hook, no counterpart in the paper: allocation-failure injection.
 * after >= 0 lets that many of the library's guarded allocations (plan
 * creation, extraction, the upload's host staging and its device
 * allocation, a batch's device allocation) pass and makes the next one fail
 * as if memory ran out, once; after < 0 turns injection off.  The failing
 * call returns SABLE_ERR_OOM, frees what it had allocated and leaves other
 * plans untouched (a plan that failed keeps SABLE_ERR_OOM as its sticky
 * status).  Process-wide; not for production use. */
void sable_debug_fail_allocations(int64_t after);

/* First error recorded on the plan (SABLE_OK if none). */
sable_status sable_plan_status(sable_plan_t plan);

/* Free host and device memory of the plan.  NULL is accepted. */
sable_status sable_plan_destroy(sable_plan_t plan);

/* Static description of a status code. */
const char *sable_status_string(sable_status s);

#ifdef __cplusplus
}
#endif
#endif /* SABLE_H */
