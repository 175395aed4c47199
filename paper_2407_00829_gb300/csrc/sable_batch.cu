// Batched SpMV / SpMM over many extracted plans in one grouped launch per op,
// and CUDA-graph capture of those launches.
//
// A batch concatenates the SpMV row-tile tables of its plans (each tile
// carries its matrix index), numbers the rows of all its matrices one after
// another for the row-split SpMM, and keeps a device table of the plans'
// device descriptors, so one persistent launch covers every region of every
// matrix (and, for SpMM with tensor-core blocks, one more launch covers every
// block tile on the tensor cores).  The plans must stay alive and uploaded
// while the batch is used.
#include <cuda_runtime.h>

#include <algorithm>
#include <new>
#include <vector>

#include "sable_internal.h"
#include "sable_trace.h"

using namespace sable;

struct sable_batch_s {
  std::vector<sable_plan_t> plans;
  int device = -1, sm_count = 1;
  char *blob = nullptr;
  const DevHybrid *mats = nullptr;
  const DevItem *items_v = nullptr;
  const int32_t *trip = nullptr;
  const int32_t *fg = nullptr;         // (matrix, block, row group) triples of the FP32 block kernel
  int n_fg = 0;
  const int64_t *row_base = nullptr;   // rows of the matrices before each one (count + 1)
  int64_t rows = 0;                    // all rows of the batch
  int *err = nullptr;
  int n_v = 0, n_trip = 0, rows_v = 0;
};

struct sable_graph_s {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {

sable_status batch_spmv_launch(sable_batch_t b, const float *const *x, float *const *y, cudaStream_t st) {
  return launch_spmv_grouped(b->mats, b->items_v, b->n_v, b->rows_v, x, y, b->sm_count, st);
}

sable_status batch_spmm_launch(sable_batch_t b, const float *const *B, int64_t N, float *const *C,
                               sable_precision prec, cudaStream_t st) {
  if (N < 1 || N > (int64_t)65535 * 32) return SABLE_ERR_INVALID;
  if (prec != SABLE_FP32 && prec != SABLE_BF16_BLOCKS && prec != SABLE_FP32_SPLIT) return SABLE_ERR_INVALID;
  // column panel and depth from the first plan's tiling
  const Tiling &T = b->plans.empty() ? Tiling{} : b->plans[0]->tiling;
  // blocks first (matrices whose blocks share no rows): they store their rows
  // of C on the tensor cores or, FP32, in groups of rows
  const bool first = b->n_trip > 0;
  if (first) {
    const sable_status s =
        prec == SABLE_FP32
            ? launch_vbr_rows(b->mats, b->fg, b->n_fg, nullptr, 0, nullptr, 0, B, C, (int)N, T.spmm_cols,
                              b->sm_count, st)
            : launch_vbr_tc(b->mats, b->trip, b->n_trip, nullptr, 0, nullptr, 0, B, C, (int)N, b->sm_count, b->err,
                            st, prec == SABLE_FP32_SPLIT ? 3 : 1);
    if (s) return s;
  }
  // the row-split grouped launch
  return launch_spmm_rows_grouped(b->mats, b->row_base, (int)b->plans.size(), b->rows, B, C, (int)N, first,
                                  T.spmm_cols, T.spmm_depth, b->sm_count, st);
}

sable_status capture(sable_batch_t b, sable_graph_t *out, bool spmm, const float *const *in, int64_t N,
                     float *const *o, sable_precision prec) {
  *out = nullptr;
  cudaStream_t st;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return SABLE_ERR_CUDA;
  sable_graph_s *g = new (std::nothrow) sable_graph_s();
  if (!g) {
    cudaStreamDestroy(st);
    return SABLE_ERR_OOM;
  }
  sable_status s = SABLE_OK;
  if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) s = SABLE_ERR_CUDA;
  if (!s) s = spmm ? batch_spmm_launch(b, in, N, o, prec, st) : batch_spmv_launch(b, in, o, st);
  cudaGraph_t graph = nullptr;
  const cudaError_t e = cudaStreamEndCapture(st, &graph);
  if (!s && e != cudaSuccess) s = SABLE_ERR_CUDA;
  if (!s && cudaGraphInstantiate(&g->exec, graph, 0) != cudaSuccess) s = SABLE_ERR_CUDA;
  g->graph = graph;
  cudaStreamDestroy(st);
  (void)cudaGetLastError();
  if (s) {
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    delete g;
    return s;
  }
  *out = g;
  return SABLE_OK;
}

}  // namespace

extern "C" {

sable_status sable_batch_create(const sable_plan_t *plans, int32_t count, sable_batch_t *out) {
  sable::TraceRange trace_("sable_batch_create");
  if (!out || count < 0 || (count > 0 && !plans)) return SABLE_ERR_INVALID;
  *out = nullptr;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return SABLE_ERR_CUDA;
  sable_batch_s *b = new (std::nothrow) sable_batch_s();
  if (!b) return SABLE_ERR_OOM;
  std::vector<DevHybrid> mats;
  std::vector<DevItem> iv;
  std::vector<int32_t> trip, fg;
  std::vector<int64_t> row_base(1, 0);
  try {
    for (int32_t i = 0; i < count; ++i) {
      sable_plan_t P = plans[i];
      if (!P || P->sticky || !P->uploaded || P->device != dev) {
        delete b;
        return P && !P->uploaded ? SABLE_ERR_ORDER : SABLE_ERR_INVALID;
      }
      if (P->dev.spmv.n_fix > 0) {   // cut tiles need their own second launch per plan
        delete b;
        return SABLE_ERR_UNSUPPORTED;
      }
      b->plans.push_back(P);
      mats.push_back(P->dev);
      for (DevItem it : P->h_items_v) {
        it.mat = i;
        iv.push_back(it);
      }
      for (size_t k = 0; k + 2 < P->h_trip.size(); k += 3) {
        trip.push_back(i);
        trip.push_back(P->h_trip[k + 1]);
        trip.push_back(P->h_trip[k + 2]);
      }
      for (size_t k = 0; k + 2 < P->h_fg.size(); k += 3) {
        fg.push_back(i);
        fg.push_back(P->h_fg[k + 1]);
        fg.push_back(P->h_fg[k + 2]);
      }
      row_base.push_back(row_base.back() + P->m);
      b->rows_v = std::max(b->rows_v, P->dev.spmv.rows_max);
    }
  } catch (const std::bad_alloc &) {
    delete b;
    return SABLE_ERR_OOM;
  }
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t s_err = 256, s_m = al(mats.size() * sizeof(DevHybrid)), s_v = al(iv.size() * sizeof(DevItem)),
               s_t = al(trip.size() * sizeof(int32_t)),
               s_r = al(row_base.size() * sizeof(int64_t)), s_f = al(fg.size() * sizeof(int32_t));
  const size_t total = s_err + s_m + s_v + s_t + s_r + s_f;
  if (alloc_fails() || cudaMalloc(&b->blob, total) != cudaSuccess) {
    (void)cudaGetLastError();
    delete b;
    return SABLE_ERR_OOM;
  }
  char *p = b->blob;
  b->err = reinterpret_cast<int *>(p);
  p += s_err;
  b->mats = reinterpret_cast<const DevHybrid *>(p);
  p += s_m;
  b->items_v = reinterpret_cast<const DevItem *>(p);
  p += s_v;
  b->trip = reinterpret_cast<const int32_t *>(p);
  p += s_t;
  b->row_base = reinterpret_cast<const int64_t *>(p);
  p += s_r;
  b->fg = reinterpret_cast<const int32_t *>(p);
  cudaError_t e = cudaMemset(b->err, 0, s_err);
  if (e == cudaSuccess && !mats.empty())
    e = cudaMemcpy((void *)b->mats, mats.data(), mats.size() * sizeof(DevHybrid), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !iv.empty())
    e = cudaMemcpy((void *)b->items_v, iv.data(), iv.size() * sizeof(DevItem), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !trip.empty())
    e = cudaMemcpy((void *)b->trip, trip.data(), trip.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy((void *)b->row_base, row_base.data(), row_base.size() * sizeof(int64_t), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !fg.empty())
    e = cudaMemcpy((void *)b->fg, fg.data(), fg.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    cudaFree(b->blob);
    delete b;
    return SABLE_ERR_CUDA;
  }
  b->n_v = (int)iv.size();
  b->n_trip = (int)(trip.size() / 3);
  b->n_fg = (int)(fg.size() / 3);
  b->rows = row_base.back();
  b->device = dev;
  cudaDeviceGetAttribute(&b->sm_count, cudaDevAttrMultiProcessorCount, dev);
  *out = b;
  return SABLE_OK;
}

sable_status sable_batch_spmv(sable_batch_t b, const float *const *x, float *const *y, void *stream) {
  sable::TraceRange trace_("sable_batch_spmv");
  if (!b || (b->n_v > 0 && (!x || !y))) return SABLE_ERR_INVALID;
  return batch_spmv_launch(b, x, y, (cudaStream_t)stream);
}

sable_status sable_batch_spmm(sable_batch_t b, const float *const *B, int64_t N, float *const *C,
                              sable_precision prec, void *stream) {
  sable::TraceRange trace_("sable_batch_spmm");
  if (!b || (b->rows > 0 && (!B || !C))) return SABLE_ERR_INVALID;
  return batch_spmm_launch(b, B, N, C, prec, (cudaStream_t)stream);
}

sable_status sable_batch_graph_spmv(sable_batch_t b, const float *const *x, float *const *y, sable_graph_t *out) {
  if (!b || !out || (b->n_v > 0 && (!x || !y))) return SABLE_ERR_INVALID;
  return capture(b, out, false, x, 0, y, SABLE_FP32);
}

sable_status sable_batch_graph_spmm(sable_batch_t b, const float *const *B, int64_t N, float *const *C,
                                    sable_precision prec, sable_graph_t *out) {
  if (!b || !out || (b->rows > 0 && (!B || !C))) return SABLE_ERR_INVALID;
  return capture(b, out, true, B, N, C, prec);
}

sable_status sable_graph_launch(sable_graph_t g, void *stream) {
  sable::TraceRange trace_("sable_graph_launch");
  if (!g || !g->exec) return SABLE_ERR_INVALID;
  return cudaGraphLaunch(g->exec, (cudaStream_t)stream) == cudaSuccess ? SABLE_OK : SABLE_ERR_CUDA;
}

sable_status sable_graph_destroy(sable_graph_t g) {
  if (!g) return SABLE_OK;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  delete g;
  return SABLE_OK;
}

sable_status sable_batch_status(sable_batch_t b, int32_t *device_error) {
  if (!b || !device_error) return SABLE_ERR_INVALID;
  int v = 0;
  if (cudaMemcpy(&v, b->err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return SABLE_ERR_CUDA;
  *device_error = v;
  return SABLE_OK;
}

sable_status sable_batch_destroy(sable_batch_t b) {
  if (!b) return SABLE_OK;
  if (b->blob) {
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != b->device) cudaSetDevice(b->device);
    cudaFree(b->blob);
    if (cur >= 0 && cur != b->device) cudaSetDevice(cur);
    (void)cudaGetLastError();
  }
  delete b;
  return SABLE_OK;
}

}  // extern "C"
