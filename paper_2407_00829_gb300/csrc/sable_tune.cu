// Autotuner: picks the row-tile shape of a plan's SpMV or SpMM launch by
// timing candidate tilings on the device with CUDA events, through the same
// entry points a user calls, and remembers the choice per shape class (op,
// N, and the plan's size and format mix, all bucketed) for the rest of the
// process.  The extraction thresholds (delta, A_min, extractor order) are the
// planner's choice; this picks what the launch does with the extracted plan.
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <utility>
#include <vector>

#include "sable_internal.h"
#include "sable_trace.h"

namespace sable {
namespace {

using Key = std::tuple<int, int, int, int, int, int>;   // op, log2 N, log2 m, log2 nnz, vdia 1/4s, vbr 1/4s

std::mutex g_mu;
std::map<Key, sable_tiling> g_cache;

int floor_log2(int64_t v) {
  int k = 0;
  while (v > 1) {
    v >>= 1;
    ++k;
  }
  return k;
}

Key shape_class(const sable_plan_stats &s, int op, int64_t N) {
  const int64_t z = std::max<int64_t>(1, s.nnz);
  return Key{op, (op == 0 || op == 4) ? -1 : floor_log2(N), floor_log2(std::max<int64_t>(1, s.m)), floor_log2(z),
             (int)(4 * s.nnz_vdia / z), (int)(4 * s.nnz_vbr / z)};
}

sable_status run_op(sable_plan_t P, int op, int64_t N, const float *in, float *out, cudaStream_t st) {
  if (op == 0) return sable_spmv(P, in, out, st);
  if (op == 4) return sable_csr_spmv(P, in, out, st);
  return sable_spmm(P, in, N, N, out, N, op == 2 ? SABLE_BF16_BLOCKS : op == 3 ? SABLE_FP32_SPLIT : SABLE_FP32, st);
}

// mean device time of one SpMV launch over `reps` launches captured in one
// CUDA graph (on a side stream) and replayed on `st`, best of two rounds: a
// small plan's launch is shorter than the host's work per call, so launches
// issued one by one would time the host
sable_status time_graph(sable_plan_t P, int op, const float *in, float *out, int reps, cudaStream_t st,
                        cudaEvent_t e0, cudaEvent_t e1, float *ms) {
  cudaStream_t cs = nullptr;
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ge = nullptr;
  sable_status s = SABLE_OK;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) s = SABLE_ERR_CUDA;
  if (!s && cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) s = SABLE_ERR_CUDA;
  if (!s) {
    for (int r = 0; r < reps && !s; ++r) s = run_op(P, op, 0, in, out, cs);
    if (cudaStreamEndCapture(cs, &g) != cudaSuccess && !s) s = SABLE_ERR_CUDA;   // ends the capture either way
  }
  if (!s && cudaGraphInstantiate(&ge, g, 0) != cudaSuccess) s = SABLE_ERR_CUDA;
  float best = -1.f;
  if (!s && cudaGraphLaunch(ge, st) != cudaSuccess) s = SABLE_ERR_CUDA;   // warm-up
  for (int round = 0; round < 2 && !s; ++round) {
    float t = 0.f;
    if (cudaEventRecord(e0, st) != cudaSuccess || cudaGraphLaunch(ge, st) != cudaSuccess ||
        cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) {
      s = SABLE_ERR_CUDA;
      break;
    }
    t /= (float)reps;
    if (best < 0.f || t < best) best = t;
  }
  if (ge) cudaGraphExecDestroy(ge);
  if (g) cudaGraphDestroy(g);
  if (cs) cudaStreamDestroy(cs);
  (void)cudaGetLastError();
  *ms = best;
  return s;
}

// mean device time of one launch over `reps` back-to-back launches, best of two rounds
sable_status time_op(sable_plan_t P, int op, int64_t N, const float *in, float *out, int reps, cudaStream_t st,
                     cudaEvent_t e0, cudaEvent_t e1, float *ms) {
  if (op == 0 || op == 4) return time_graph(P, op, in, out, reps, st, e0, e1, ms);
  sable_status s = SABLE_OK;
  for (int w = 0; w < 2 && !s; ++w) s = run_op(P, op, N, in, out, st);
  float best = -1.f;
  for (int round = 0; round < 2 && !s; ++round) {
    if (cudaEventRecord(e0, st) != cudaSuccess) return SABLE_ERR_CUDA;
    for (int r = 0; r < reps && !s; ++r) s = run_op(P, op, N, in, out, st);
    if (s) break;
    float t = 0.f;
    if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&t, e0, e1) != cudaSuccess)
      return SABLE_ERR_CUDA;
    t /= (float)reps;
    if (best < 0.f || t < best) best = t;
  }
  *ms = best;
  return s;
}

sable_status apply(sable_plan_t P, const sable_tiling &t, cudaStream_t st) {
  const Tiling &now = P->tiling;
  const bool same_tables = P->uploaded && now.rows_per_item == t.spmv_rows && now.item_bytes == t.spmv_bytes;
  sable_status s = sable_plan_set_tiling(P, t.spmv_rows, t.spmv_bytes);
  if (!s) s = sable_plan_set_spmm_cols(P, t.spmm_cols);
  if (!s) s = sable_plan_set_spmm_depth(P, t.spmm_depth);
  if (!s && !same_tables) s = sable_plan_upload(P, st);   // the column panel needs no new tables
  return s;
}

}  // namespace
}  // namespace sable

using namespace sable;

extern "C" {

sable_status sable_plan_get_tiling(sable_plan_t P, sable_tiling *out) {
  if (!P || !out) return SABLE_ERR_INVALID;
  out->spmv_rows = P->tiling.rows_per_item;
  out->spmv_bytes = P->tiling.item_bytes;
  out->spmm_cols = P->tiling.spmm_cols;
  out->spmm_depth = P->tiling.spmm_depth;
  return SABLE_OK;
}

sable_status sable_autotune(sable_plan_t P, int32_t op, int64_t N, const float *in, float *out, int32_t reps,
                            int32_t use_cache, sable_tiling *chosen, float *chosen_ms, void *stream) {
  sable::TraceRange trace_("sable_autotune");
  const bool spmv = op == 0 || op == 4;
  if (!P || op < 0 || op > 4 || (!spmv && N < 1) || !in || !out || reps < 1 || reps > 10000)
    return SABLE_ERR_INVALID;
  if (P->sticky) return P->sticky;
  if (!P->extracted) return SABLE_ERR_ORDER;
  cudaStream_t st = (cudaStream_t)stream;
  const Key key = shape_class(P->stats, op, N);
  sable_tiling cur{};
  sable_plan_get_tiling(P, &cur);
  std::vector<sable_tiling> cand;
  bool cached = false;
  if (use_cache) {
    std::lock_guard<std::mutex> lock(g_mu);
    auto it = g_cache.find(key);
    if (it != g_cache.end()) {
      sable_tiling t = cur;
      if (spmv) {
        t.spmv_rows = it->second.spmv_rows;
        t.spmv_bytes = it->second.spmv_bytes;
      } else {
        t.spmm_cols = it->second.spmm_cols;
        t.spmm_depth = it->second.spmm_depth;
      }
      cand.push_back(t);
      cached = true;
    }
  }
  if (!cached) {
    if (spmv) {
      // short tiles (32, 64 rows) give small matrices enough CTAs to fill the GPU
      for (int32_t rows : {32, 64, 128, 256, 512, 1024})
        for (int64_t bytes : {4 << 10, 16 << 10, 48 << 10, 160 << 10})
          cand.push_back({rows, bytes, cur.spmm_cols, cur.spmm_depth});
      // tiles sized for exactly 1, 2 or 3 full waves of resident CTAs
      int dev = 0, sms = 0;
      if (cudaGetDevice(&dev) == cudaSuccess &&
          cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && sms > 0) {
        const int64_t slots = (int64_t)spmv_resident_ctas(kRangeRows) * sms;
        const int64_t total = op == 4 ? P->stats.csr_spmv_bytes : P->stats.spmv_bytes;
        for (int64_t k = 1; k <= 3; ++k) {
          const int64_t bytes = total / (k * slots) + total / (50 * k * slots) + 64;
          cand.push_back({kRangeRows, bytes, cur.spmm_cols, cur.spmm_depth});
        }
      }
      (void)cudaGetLastError();
    } else {
      // one matrix's SpMM is row split: only the column panel and depth matter
      for (const auto &cd : {std::pair<int32_t, int32_t>{128, 4}, {128, 8}, {64, 4}, {64, 8}, {32, 4}, {32, 8}})
        cand.push_back({cur.spmv_rows, cur.spmv_bytes, cd.first, cd.second});
    }
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    (void)cudaGetLastError();
    return SABLE_ERR_CUDA;
  }
  sable_status s = SABLE_OK;
  int best = -1;
  float best_ms = 0.f;
  for (size_t c = 0; c < cand.size() && !s; ++c) {
    float ms = 0.f;
    s = apply(P, cand[c], st);
    if (!s) s = time_op(P, op, N, in, out, reps, st, e0, e1, &ms);
    if (!s && (best < 0 || ms < best_ms)) {
      best = (int)c;
      best_ms = ms;
    }
  }
  if (!s && cand.size() > 1) s = apply(P, cand[best], st);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s) return s;
  if (!cached) {
    std::lock_guard<std::mutex> lock(g_mu);
    g_cache[key] = cand[best];
  }
  if (chosen) *chosen = cand[best];
  if (chosen_ms) *chosen_ms = best_ms;
  return SABLE_OK;
}

int64_t sable_autotune_cache_clear(void) {
  std::lock_guard<std::mutex> lock(g_mu);
  const int64_t n = (int64_t)g_cache.size();
  g_cache.clear();
  return n;
}

}  // extern "C"
