// Plan life cycle on the host: COO ingest and canonical form, the ordered
// extractor list, extraction over the shrinking residual (Section 3,
// "Initialize" / "Extract"), the completeness check (Section 3, "Dispatch"),
// and host exports.  No CUDA call is made here.
#include <algorithm>
#include <thread>
#include <atomic>
#include <cmath>
#include <cstring>
#include <new>
#include <numeric>

#include <stdexcept>

#include "sable_internal.h"
#include "sable_trace.h"

using namespace sable;

namespace sable {
namespace {
std::atomic<int64_t> g_fail_after{-1};   // guarded allocations to let pass; -1 = injection off
}
bool alloc_fails() {
  int64_t v = g_fail_after.load(std::memory_order_relaxed);
  while (v >= 0) {
    if (g_fail_after.compare_exchange_weak(v, v - 1, std::memory_order_relaxed)) return v == 0;
  }
  return false;
}
void alloc_point() {
  if (alloc_fails()) throw std::bad_alloc();
}
}  // namespace sable

namespace sable {

sable_status fail(sable_plan_t p, sable_status s) {
  if (p && p->sticky == SABLE_OK) p->sticky = s;
  return s;
}

// Residual (owner < 0) of the canonical matrix as CSR, or its transpose.
// Rows (or columns) keep their inner indices ascending.  Threads over row
// ranges on large matrices: each range counts its entries per output line,
// the counts are turned into per-range offsets line by line, and each range
// fills its own slots (ranges in row order, so every line stays sorted).
static Csr residual(const sable_plan_s &P, bool transpose) {
  Csr R;
  const Csr &C = P.canon;
  R.m = transpose ? P.n : P.m;
  R.n = transpose ? P.m : P.n;
  R.rp.assign(R.m + 1, 0);
  const int T = std::max(1, std::min(C.nnz() >= (1 << 20) ? host_threads() : 1, (int)std::max<int64_t>(C.m, 1)));
  const int64_t chunk = (C.m + T - 1) / T;
  auto run = [&](auto &&f) {
    if (T == 1) {
      f(0);
      return;
    }
    std::vector<std::thread> th;
    for (int t = 0; t < T; ++t) th.emplace_back(f, t);
    for (auto &x : th) x.join();
  };
  // cnt[t][o]: entries of range t on output line o, then that range's first slot on line o
  // (int32: a plan holds fewer than 2^31 entries)
  std::vector<std::vector<int32_t>> cnt(T, std::vector<int32_t>(transpose ? R.m : 0, 0));
  std::vector<int64_t> rowcnt(transpose ? 0 : C.m, 0);
  run([&](int t) {
    const int64_t a = t * chunk, b = std::min(C.m, a + chunk);
    for (int64_t i = a; i < b; ++i)
      for (int64_t k = C.rp[i]; k < C.rp[i + 1]; ++k)
        if (P.owner[k] < 0) {
          if (transpose) ++cnt[t][C.ci[k]];
          else ++rowcnt[i];
        }
  });
  if (transpose) {
    for (int64_t o = 0; o < R.m; ++o) {
      int64_t at = R.rp[o];
      for (int t = 0; t < T; ++t) {
        const int64_t c = cnt[t][o];
        cnt[t][o] = (int32_t)at;
        at += c;
      }
      R.rp[o + 1] = at;
    }
  } else {
    for (int64_t i = 0; i < C.m; ++i) R.rp[i + 1] = R.rp[i] + rowcnt[i];
  }
  R.ci.resize(R.rp[R.m]);
  R.id.resize(R.rp[R.m]);
  run([&](int t) {
    const int64_t a = t * chunk, b = std::min(C.m, a + chunk);
    for (int64_t i = a; i < b; ++i) {
      int64_t q = transpose ? 0 : R.rp[i];
      for (int64_t k = C.rp[i]; k < C.rp[i + 1]; ++k) {
        if (P.owner[k] >= 0) continue;
        if (transpose) {
          const int64_t s = cnt[t][C.ci[k]]++;
          R.ci[s] = (int32_t)i;
          R.id[s] = k;
        } else {
          R.ci[q] = C.ci[k];
          R.id[q] = k;
          ++q;
        }
      }
    }
  });
  return R;
}

}  // namespace sable

extern "C" {

const char *sable_status_string(sable_status s) {
  switch (s) {
    case SABLE_OK: return "ok";
    case SABLE_ERR_INVALID: return "invalid argument";
    case SABLE_ERR_OOM: return "out of memory";
    case SABLE_ERR_CUDA: return "CUDA runtime error";
    case SABLE_ERR_INCOMPLETE: return "incomplete plan: entries left unclaimed";
    case SABLE_ERR_ORDER: return "call out of order for this plan";
    case SABLE_ERR_TIMEOUT: return "bounded device wait timed out";
    case SABLE_ERR_KERNEL: return "kernel bounds check failed";
    case SABLE_ERR_UNSUPPORTED: return "unsupported request";
  }
  return "unknown status";
}

void sable_default_params(sable_extractor kind, sable_extract_params *o) {
  if (!o) return;
  o->delta = kind == SABLE_X_VDIA ? 0.75 : 0.5;
  o->a_min = 2500;
  o->l_seg = 32;
  o->w_max = 64;
  o->d_max = 0;
  o->count_min = 0;
  o->coverage_min = 0.08;
  o->max_span = 512;
  o->tile = 8;
  o->passes = 1;
}

sable_status sable_plan_create(int64_t m, int64_t n, int64_t nnz, const int32_t *row,
                               const int32_t *col, const float *val, sable_plan_t *out) {
  if (!out) return SABLE_ERR_INVALID;
  *out = nullptr;
  if (m < 0 || n < 0 || nnz < 0 || m >= INT32_MAX || n >= INT32_MAX || nnz >= INT32_MAX)
    return SABLE_ERR_INVALID;
  if (nnz > 0 && (!row || !col || !val)) return SABLE_ERR_INVALID;
  for (int64_t k = 0; k < nnz; ++k)
    if (row[k] < 0 || row[k] >= m || col[k] < 0 || col[k] >= n) return SABLE_ERR_INVALID;
  sable_plan_s *P = new (std::nothrow) sable_plan_s();
  if (!P) return SABLE_ERR_OOM;
  try {
    alloc_point();
    P->m = m;
    P->n = n;
    // bucket by row, keeping input order, then order each row by column
    std::vector<int64_t> cnt(m + 1, 0);
    for (int64_t k = 0; k < nnz; ++k) ++cnt[row[k] + 1];
    for (int64_t i = 0; i < m; ++i) cnt[i + 1] += cnt[i];
    std::vector<int64_t> order(nnz);
    {
      std::vector<int64_t> pos(cnt.begin(), cnt.end() - 1);
      for (int64_t k = 0; k < nnz; ++k) order[pos[row[k]]++] = k;
    }
    Csr &C = P->canon;
    C.m = m;
    C.n = n;
    C.rp.assign(m + 1, 0);
    P->canon_of.assign(nnz, 0);
    // rows are independent: sort each row's bucket by column (stable: equal
    // columns keep input order) and count its distinct columns, then fill;
    // threads over row ranges on large matrices, the same result either way
    const int T = nnz >= (1 << 20) ? host_threads() : 1;
    auto over_rows = [&](auto &&f) {
      if (T <= 1) {
        f(0, m);
        return;
      }
      std::vector<std::thread> th;
      const int64_t chunk = (m + T - 1) / T;
      for (int t = 0; t < T; ++t) {
        const int64_t a = t * chunk, b = std::min(m, a + chunk);
        if (a >= b) break;
        th.emplace_back([&f, a, b] { f(a, b); });
      }
      for (auto &x : th) x.join();
    };
    over_rows([&](int64_t a, int64_t b) {
      for (int64_t i = a; i < b; ++i) {
        int64_t *q = order.data() + cnt[i], *e = order.data() + cnt[i + 1];
        std::stable_sort(q, e, [&](int64_t u, int64_t z) { return col[u] < col[z]; });
        int64_t distinct = 0;
        for (int64_t *r = q; r < e; ++r) distinct += (r == q || col[*r] != col[*(r - 1)]);
        C.rp[i + 1] = distinct;
      }
    });
    for (int64_t i = 0; i < m; ++i) C.rp[i + 1] += C.rp[i];
    C.ci.resize(C.rp[m]);
    P->cval.resize(C.rp[m]);
    over_rows([&](int64_t a, int64_t b) {
      for (int64_t i = a; i < b; ++i) {
        int64_t id = C.rp[i];
        const int64_t *e = order.data() + cnt[i + 1];
        for (const int64_t *q = order.data() + cnt[i]; q < e; ++id) {
          const int32_t c = col[*q];
          double sum = 0.0;
          for (; q < e && col[*q] == c; ++q) {   // input order
            sum += (double)val[*q];
            P->canon_of[*q] = (int32_t)id;
          }
          C.ci[id] = c;
          P->cval[id] = (float)sum;
        }
      }
    });
    C.id.clear();
    P->owner.assign(C.ci.size(), OWN_NONE);
  } catch (const std::bad_alloc &) {
    delete P;
    return SABLE_ERR_OOM;
  }
  *out = P;
  return SABLE_OK;
}

sable_status sable_plan_add_extractor(sable_plan_t P, sable_extractor kind,
                                      const sable_extract_params *params) {
  if (!P) return SABLE_ERR_INVALID;
  if (P->sticky) return P->sticky;
  if (P->extracted) return SABLE_ERR_ORDER;
  if (kind != SABLE_X_VDIA && kind != SABLE_X_VBR && kind != SABLE_X_CSR) return SABLE_ERR_INVALID;
  sable_extract_params p;
  sable_default_params(kind, &p);
  if (params) p = *params;
  if (!(p.delta > 0.0 && p.delta <= 1.0) || p.a_min < 1 || p.l_seg < 1 || p.w_max < 0 || p.w_max > 512 ||
      p.d_max < 0 || p.count_min < 0 || !(p.coverage_min >= 0.0) || p.max_span < 1 ||
      p.tile < 0 || p.passes < 1 || p.passes > 8 || (kind != SABLE_X_VDIA && p.passes != 1))
    return SABLE_ERR_INVALID;
  // multi-ribbon VDIA: one band stage per pass, each over the residual of the last
  const int passes = p.passes;
  p.passes = 1;
  try {
    for (int k = 0; k < passes; ++k) {
      P->extractors.push_back({kind, p});
      P->stage_regions.emplace_back();
      P->stage_fixed.push_back(0);
    }
  } catch (const std::bad_alloc &) {
    return fail(P, SABLE_ERR_OOM);
  }
  return SABLE_OK;
}

sable_status sable_plan_add_regions(sable_plan_t P, sable_extractor kind, const int64_t *regions,
                                    int64_t count) {
  if (!P) return SABLE_ERR_INVALID;
  if (P->sticky) return P->sticky;
  if (P->extracted) return SABLE_ERR_ORDER;
  if ((kind != SABLE_X_VDIA && kind != SABLE_X_VBR) || count < 0 || (count > 0 && !regions))
    return SABLE_ERR_INVALID;
  for (int64_t t = 0; t < count; ++t) {
    const int64_t *g = regions + 4 * t;
    if (kind == SABLE_X_VDIA) {
      // rows [row0, row0 + nrows), offsets off_lo .. off_lo + ndiag - 1 within [-(m-1), n-1]
      if (g[0] < 0 || g[1] < 1 || g[1] > P->m - g[0] || g[3] < 1 || g[2] < -(P->m - 1) ||
          g[3] > P->n - g[2] || g[3] > INT32_MAX / 4)
        return SABLE_ERR_INVALID;
    } else {
      if (g[0] < 0 || g[1] < 1 || g[1] > P->m - g[0] || g[2] < 0 || g[3] < 1 || g[3] > P->n - g[2])
        return SABLE_ERR_INVALID;
    }
  }
  try {
    sable_extract_params p;
    sable_default_params(kind, &p);
    P->extractors.push_back({kind, p});
    P->stage_regions.emplace_back(regions, regions + 4 * count);
    P->stage_fixed.push_back(1);
  } catch (const std::bad_alloc &) {
    return fail(P, SABLE_ERR_OOM);
  }
  return SABLE_OK;
}

sable_status sable_plan_set_inspector(sable_plan_t P, sable_inspector where) {
  if (!P) return SABLE_ERR_INVALID;
  if (P->sticky) return P->sticky;
  if (P->extracted) return SABLE_ERR_ORDER;
  if (where != SABLE_INSPECT_HOST && where != SABLE_INSPECT_DEVICE) return SABLE_ERR_INVALID;
  P->inspector = (int)where;
  return SABLE_OK;
}

namespace {
// the device copy of one stage's residual, released on every way out
struct DevStage {
  sable::DevResidual *d = nullptr;
  ~DevStage() { sable::dev_residual_close(d); }
};
}  // namespace

sable_status sable_extract(sable_plan_t P) {
  sable::TraceRange trace_("sable_extract");
  if (!P) return SABLE_ERR_INVALID;
  if (P->sticky) return P->sticky;
  if (P->extracted) return SABLE_ERR_ORDER;
  const bool on_device = P->inspector == SABLE_INSPECT_DEVICE;
  if (on_device)
    for (size_t st = 0; st < P->extractors.size(); ++st)
      if (!P->stage_fixed[st] && P->extractors[st].first == SABLE_X_VBR && P->extractors[st].second.tile > 64)
        return SABLE_ERR_UNSUPPORTED;
  try {
    alloc_point();
    const Csr &C = P->canon;
    const int64_t nnz = C.nnz();
    std::vector<int32_t> region(nnz, -1);
    std::vector<Segment> segs;   // acceptance order
    std::vector<Block> blks;
    std::vector<int32_t> sstage, bstage;
    for (size_t st = 0; st < P->extractors.size(); ++st) {
      const auto &ex = P->extractors[st];
      const sable_extract_params &p = ex.second;
      Csr R = residual(*P, false);
      if (P->stage_fixed[st]) {
        // given regions, in order: each claims the stage's residual entries in
        // its area that no earlier region of the stage claimed
        const std::vector<int64_t> &G = P->stage_regions[st];
        for (size_t t = 0; t + 3 < G.size(); t += 4) {
          const int64_t r0 = G[t], nr = G[t + 1];
          const int64_t lo = G[t + 2], hi = G[t + 2] + G[t + 3] - 1;   // offsets (VDIA) or columns (VBR)
          const bool vd = ex.first == SABLE_X_VDIA;
          const int32_t rid = (int32_t)(vd ? segs.size() : blks.size());
          if (vd) {
            segs.push_back({r0, nr, G[t + 2], G[t + 3]});
            sstage.push_back((int32_t)st);
          } else {
            blks.push_back({r0, nr, G[t + 2], G[t + 3]});
            bstage.push_back((int32_t)st);
          }
          for (int64_t r = r0; r < r0 + nr; ++r) {
            const int64_t clo = vd ? r + lo : lo, chi = vd ? r + hi : hi;
            const int32_t *b = R.ci.data() + R.rp[r], *e = R.ci.data() + R.rp[r + 1];
            for (const int32_t *q = std::lower_bound(b, e, (int32_t)std::max<int64_t>(clo, 0));
                 q < e && *q <= chi; ++q) {
              const int64_t k = R.id[q - R.ci.data()];
              if (P->owner[k] >= 0) continue;
              P->owner[k] = vd ? OWN_VDIA : OWN_VBR;
              region[k] = rid;
            }
          }
        }
      } else if (ex.first == SABLE_X_CSR) {
        for (int64_t q = 0; q < R.nnz(); ++q) P->owner[R.id[q]] = OWN_CSR;
      } else if (ex.first == SABLE_X_VDIA) {
        DevStage ds;
        if (on_device)
          if (sable_status e = dev_residual_open(R, &ds.d)) return fail(P, e);
        for (const BandSeg &s : extract_bands(R, p, ds.d)) {
          const int32_t sid = (int32_t)segs.size();
          segs.push_back({s.i0, s.i1 - s.i0, s.d - s.L, s.L + s.U + 1});
          sstage.push_back((int32_t)st);
          for (int64_t r = s.i0; r < s.i1; ++r)
            for (int64_t q = R.rp[r]; q < R.rp[r + 1]; ++q) {
              const int64_t o = (int64_t)R.ci[q] - r;
              if (o >= s.d - s.L && o <= s.d + s.U) {
                P->owner[R.id[q]] = OWN_VDIA;
                region[R.id[q]] = sid;
              }
            }
        }
      } else {
        Csr RT = residual(*P, true);
        DevStage ds;
        if (on_device && p.tile > 0)
          if (sable_status e = dev_residual_open(R, &ds.d)) return fail(P, e);
        for (const BlockFound &b : partition_blocks(R, RT, p, ds.d)) {
          const int32_t bid = (int32_t)blks.size();
          blks.push_back({b.r0, b.r1 - b.r0, b.c0, b.c1 - b.c0});
          bstage.push_back((int32_t)st);
          for (int64_t r = b.r0; r < b.r1; ++r)
            for (int64_t q = R.rp[r]; q < R.rp[r + 1]; ++q)
              if (R.ci[q] >= b.c0 && R.ci[q] < b.c1) {
                P->owner[R.id[q]] = OWN_VBR;
                region[R.id[q]] = bid;
              }
        }
      }
    }
    for (int64_t k = 0; k < nnz; ++k)
      if (P->owner[k] < 0) return fail(P, SABLE_ERR_INCOMPLETE);

    Hybrid &H = P->hyb;
    H.m = P->m;
    H.n = P->n;
    // order segments and blocks by first row; remember where each went
    std::vector<int32_t> so(segs.size()), bo(blks.size());
    std::iota(so.begin(), so.end(), 0);
    std::iota(bo.begin(), bo.end(), 0);
    std::stable_sort(so.begin(), so.end(), [&](int32_t a, int32_t b) {
      return segs[a].row0 != segs[b].row0 ? segs[a].row0 < segs[b].row0 : segs[a].off_lo < segs[b].off_lo;
    });
    std::stable_sort(bo.begin(), bo.end(), [&](int32_t a, int32_t b) {
      return blks[a].r0 != blks[b].r0 ? blks[a].r0 < blks[b].r0 : blks[a].c0 < blks[b].c0;
    });
    std::vector<int32_t> sidx(segs.size()), bidx(blks.size());
    std::vector<int64_t> sptr(segs.size() + 1, 0), bptr(blks.size() + 1, 0);
    H.segs.clear();
    P->seg_stage.assign(so.size(), 0);
    P->blk_stage.assign(bo.size(), 0);
    for (size_t t = 0; t < so.size(); ++t) {
      sidx[so[t]] = (int32_t)t;
      P->seg_stage[t] = sstage[so[t]];
      H.segs.push_back(segs[so[t]]);
      sptr[t + 1] = sptr[t] + segs[so[t]].nrows * segs[so[t]].ndiag;
    }
    H.blks.clear();
    for (size_t t = 0; t < bo.size(); ++t) {
      bidx[bo[t]] = (int32_t)t;
      P->blk_stage[t] = bstage[bo[t]];
      H.blks.push_back(blks[bo[t]]);
      bptr[t + 1] = bptr[t] + blks[bo[t]].nr * blks[bo[t]].nc;
    }
    H.vdia_canon.assign(sptr.back(), 0.0f);
    H.vbr_canon.assign(bptr.back(), 0.0f);
    H.crp.assign(P->m + 1, 0);
    H.cci.clear();
    H.ccv.clear();
    int64_t nv = 0, nb = 0, nc = 0;
    P->dest.assign(nnz, 0);
    for (int64_t i = 0; i < C.m; ++i) {
      for (int64_t k = C.rp[i]; k < C.rp[i + 1]; ++k) {
        const int64_t j = C.ci[k];
        if (P->owner[k] == OWN_VDIA) {
          const int32_t s = sidx[region[k]];
          const Segment &g = H.segs[s];
          P->dest[k] = sptr[s] + (j - i - g.off_lo) * g.nrows + (i - g.row0);
          H.vdia_canon[P->dest[k]] = P->cval[k];
          ++nv;
        } else if (P->owner[k] == OWN_VBR) {
          const int32_t b = bidx[region[k]];
          const Block &g = H.blks[b];
          P->dest[k] = bptr[b] + (j - g.c0) * g.nr + (i - g.r0);
          H.vbr_canon[P->dest[k]] = P->cval[k];
          ++nb;
        } else {
          P->dest[k] = (int64_t)H.ccv.size();
          H.cci.push_back((int32_t)j);
          H.ccv.push_back(P->cval[k]);
          ++nc;
        }
      }
      H.crp[i + 1] = (int64_t)H.cci.size();
    }
    if (nv + nb + nc != nnz) return fail(P, SABLE_ERR_INCOMPLETE);

    sable_plan_stats &S = P->stats;
    S = sable_plan_stats{};
    S.m = P->m;
    S.n = P->n;
    S.nnz = nnz;
    S.nnz_vdia = nv;
    S.nnz_vbr = nb;
    S.nnz_csr = nc;
    S.n_segments = (int64_t)H.segs.size();
    for (auto &g : H.segs) S.n_diagonals += g.ndiag;
    S.vdia_cells = sptr.back();
    S.n_blocks = (int64_t)H.blks.size();
    S.vbr_cells = bptr.back();
    S.csr_spmv_bytes = 8 * nnz + 4 * (P->m + 1) + 4 * P->n + 4 * P->m;
    S.spmv_bytes = 4 * (S.vdia_cells + S.vbr_cells + nc) + 4 * nc + 4 * (P->m + 1) +
                   32 * (S.n_segments + S.n_blocks) + 4 * P->n + 4 * P->m;
  } catch (const std::bad_alloc &) {
    return fail(P, SABLE_ERR_OOM);
  } catch (const InspectError &e) {
    return fail(P, e.status);
  }
  P->extracted = true;
  return SABLE_OK;
}

sable_status sable_plan_info(sable_plan_t P, sable_plan_stats *out) {
  if (!P || !out) return SABLE_ERR_INVALID;
  if (!P->extracted) return SABLE_ERR_ORDER;
  *out = P->stats;
  return SABLE_OK;
}

sable_status sable_plan_get_segments(sable_plan_t P, int64_t *out) {
  if (!P || !out) return SABLE_ERR_INVALID;
  if (!P->extracted) return SABLE_ERR_ORDER;
  for (size_t s = 0; s < P->hyb.segs.size(); ++s) {
    const Segment &g = P->hyb.segs[s];
    out[4 * s] = g.row0;
    out[4 * s + 1] = g.nrows;
    out[4 * s + 2] = g.off_lo;
    out[4 * s + 3] = g.ndiag;
  }
  return SABLE_OK;
}

sable_status sable_plan_get_blocks(sable_plan_t P, int64_t *out) {
  if (!P || !out) return SABLE_ERR_INVALID;
  if (!P->extracted) return SABLE_ERR_ORDER;
  for (size_t b = 0; b < P->hyb.blks.size(); ++b) {
    const Block &g = P->hyb.blks[b];
    out[4 * b] = g.r0;
    out[4 * b + 1] = g.nr;
    out[4 * b + 2] = g.c0;
    out[4 * b + 3] = g.nc;
  }
  return SABLE_OK;
}

sable_status sable_plan_get_region_stages(sable_plan_t P, int32_t *seg_stage, int32_t *blk_stage) {
  if (!P) return SABLE_ERR_INVALID;
  if (!P->extracted) return SABLE_ERR_ORDER;
  if ((!seg_stage && !P->seg_stage.empty()) || (!blk_stage && !P->blk_stage.empty())) return SABLE_ERR_INVALID;
  if (!P->seg_stage.empty()) std::memcpy(seg_stage, P->seg_stage.data(), P->seg_stage.size() * 4);
  if (!P->blk_stage.empty()) std::memcpy(blk_stage, P->blk_stage.data(), P->blk_stage.size() * 4);
  return SABLE_OK;
}

sable_status sable_plan_get_vdia_values(sable_plan_t P, float *out) {
  if (!P || (!out && !P->hyb.vdia_canon.empty())) return SABLE_ERR_INVALID;
  if (!P->extracted) return SABLE_ERR_ORDER;
  if (!P->hyb.vdia_canon.empty())
    std::memcpy(out, P->hyb.vdia_canon.data(), P->hyb.vdia_canon.size() * sizeof(float));
  return SABLE_OK;
}

sable_status sable_plan_get_vbr_values(sable_plan_t P, float *out) {
  if (!P || (!out && !P->hyb.vbr_canon.empty())) return SABLE_ERR_INVALID;
  if (!P->extracted) return SABLE_ERR_ORDER;
  if (!P->hyb.vbr_canon.empty())
    std::memcpy(out, P->hyb.vbr_canon.data(), P->hyb.vbr_canon.size() * sizeof(float));
  return SABLE_OK;
}

sable_status sable_plan_get_csr(sable_plan_t P, int64_t *row_ptr, int32_t *col, float *val) {
  if (!P || !row_ptr) return SABLE_ERR_INVALID;
  if (!P->extracted) return SABLE_ERR_ORDER;
  const Hybrid &H = P->hyb;
  std::memcpy(row_ptr, H.crp.data(), H.crp.size() * sizeof(int64_t));
  if (!H.cci.empty()) {
    if (!col || !val) return SABLE_ERR_INVALID;
    std::memcpy(col, H.cci.data(), H.cci.size() * sizeof(int32_t));
    std::memcpy(val, H.ccv.data(), H.ccv.size() * sizeof(float));
  }
  return SABLE_OK;
}

sable_status sable_plan_set_tiling(sable_plan_t P, int32_t spmv_rows, int64_t spmv_bytes) {
  if (!P) return SABLE_ERR_INVALID;
  if (spmv_rows < 4 || spmv_rows > kRangeRows || spmv_rows % 4 || spmv_bytes < 64) return SABLE_ERR_INVALID;
  P->tiling.rows_per_item = spmv_rows;
  P->tiling.item_bytes = spmv_bytes;
  return SABLE_OK;
}

sable_status sable_plan_set_spmm_cols(sable_plan_t P, int32_t cols) {
  if (!P || (cols != 0 && cols != 32 && cols != 64 && cols != 128)) return SABLE_ERR_INVALID;
  P->tiling.spmm_cols = cols;
  return SABLE_OK;
}

sable_status sable_plan_set_spmm_depth(sable_plan_t P, int32_t depth) {
  if (!P || (depth != 4 && depth != 8)) return SABLE_ERR_INVALID;
  P->tiling.spmm_depth = depth;
  return SABLE_OK;
}

sable_status sable_plan_status(sable_plan_t P) { return P ? P->sticky : SABLE_ERR_INVALID; }

void sable_debug_fail_allocations(int64_t after) {
  sable::g_fail_after.store(after < 0 ? -1 : after, std::memory_order_relaxed);
}

}  // extern "C"
