// Block partitioner: Section 4.1, Algorithm 1 (Partition / Decompose) and
// Algorithm 2 (FindBlock), host C++ with FindBlock's outer loop spread over
// threads (thread-local histograms and bests, merged deterministically).
//
// Readings (identical to the library's documented behaviour):
//  * Density floor and score base are delta (printed as 0.5 = default delta):
//    score = area * (density - delta)^1.5, compared through its square.
//  * FindBlock's outer span is capped at max_span lines.
//  * Ties keep the first window in scan order (o0, o1, i1 ascending; strict
//    '>'); across threads the merge keeps the highest score, then the lowest
//    o0, which is the sequential scan's choice.  The CSR search wins a tie
//    against the CSC search.
//  * Trim: per round, remove the one edge (top, bottom, left, right) with the
//    largest strict density gain (first on a tie), until none helps.
//  * width(B) = number of columns.
//  * With tile > 0, Decompose runs on candidate regions rather than the whole
//    matrix: cells of tile x tile with entries >= delta * cell area are hot,
//    8-connected hot cells form components, their bounding boxes (grown by one
//    cell, clipped) are merged until disjoint and visited in (row, column)
//    order.  A component taller than max_span rows whose hot cells fill less
//    than a quarter of its bounding box (a diagonal band) gives instead one
//    box per slab of ceil(max_span / tile) cell rows, counted from its first
//    row: the bounding box of its cells in that slab, grown by one cell in
//    columns and, at the component's two ends, in rows.  Slabs touch but do
//    not overlap, so the merge keeps them apart.
//  With the device inspector the cell counts come from the GPU
//  (sable_inspect.cu), with the same hot cells.
//  The two scan shortcuts below (starting a window scan at the first
//  non-empty histogram slot, stopping once the window is past the last one)
//  reproduce the printed loop's results exactly, given delta > 0.
#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <thread>

#include "sable_internal.h"

namespace sable {

int host_threads() {
  static int t = [] {
    const char *e = std::getenv("SABLE_THREADS");
    int v = e ? std::atoi(e) : (int)std::thread::hardware_concurrency();
    if (v < 1) v = 1;
    if (v > 64) v = 64;
    return v;
  }();
  return t;
}

namespace {

// Algorithm 2's score a (d - delta)^1.5 is compared through its square,
// (nnz - delta a)^3 / a (same order for d >= delta), which needs only IEEE
// multiply, subtract and divide and so rounds the same on every processor.
inline double score2(int64_t nnz, int64_t a, double delta) {
  double t = (double)nnz - delta * (double)a;
  if (t < 0.0) t = 0.0;   // d >= delta by division, but the product may round below it
  return t * t * t / (double)a;
}

// Best window of a region: score (squared, above), outer [o0, o1), inner
// [i0, i1) (half-open); sc < 0 = none.
struct Best {
  double sc = -1.0;
  int64_t o0 = 0, o1 = 0, i0 = 0, i1 = 0;
};

struct Region { int64_t r0, r1, c0, c1; };

int64_t isqrt_ceil(int64_t a) {
  int64_t s = (int64_t)std::sqrt((double)a);
  while (s * s > a) --s;
  while ((s + 1) * (s + 1) <= a) ++s;
  return s * s >= a ? s : s + 1;
}

// One outer start o0 of Algorithm 2.
void scan_start(const Csr &M, int64_t o0, int64_t O1, int64_t I0, int64_t I1,
                const sable_extract_params &p, int64_t s_min, std::vector<int32_t> &H,
                std::vector<int32_t> &touched, Best &best) {
  const int64_t L_in = I1 - I0;
  int64_t tmin = INT64_MAX, tmax = -1, hmax = 0, total = 0;
  const double omd = 1.0 - p.delta, ub_unit = omd * omd * omd;   // (1 - delta)^3
  const int64_t o_end = std::min<int64_t>(O1, o0 + (int64_t)p.max_span);
  for (int64_t o1 = o0; o1 < o_end; ++o1) {
    const int32_t *b = M.ci.data() + M.rp[o1], *e = M.ci.data() + M.rp[o1 + 1];
    for (const int32_t *q = std::lower_bound(b, e, (int32_t)I0); q < e && *q < I1; ++q) {
      const int64_t rel = *q - I0;
      const int32_t h = ++H[rel];
      if (h == 1) touched.push_back((int32_t)rel);
      if (h > hmax) hmax = h;
      ++total;
      if (rel < tmin) tmin = rel;
      if (rel > tmax) tmax = rel;
    }
    const int64_t s = o1 - o0 + 1;
    if (s < s_min || tmax < 0) continue;
    // Exact shortcuts (the printed scan would record nothing for this span):
    //  - every window's density is at most hmax / s;
    //  - every window's score is at most ub(total) (see below), so it cannot
    //    exceed the best score found so far, which only a strictly larger
    //    score replaces.
    if ((double)hmax < p.delta * (double)s) continue;
    {
      double ub;
      if (total >= p.a_min) ub = (double)total * (double)total * ub_unit;
      else if ((double)total >= p.delta * (double)p.a_min)
        ub = score2(total, p.a_min, p.delta);
      else continue;
      if (best.sc >= 0 && ub * (1.0 + 1e-9) <= best.sc) continue;
    }
    // state of the printed scan after the leading empty slots [0, tmin)
    const int64_t w_small = (p.a_min + s - 1) / s - 1;   // widest window with area < a_min
    int64_t i0 = tmin - std::min<int64_t>(tmin, w_small);
    int64_t nnz = 0;
    for (int64_t i1 = tmin; i1 < L_in; ++i1) {
      nnz += H[i1];
      while (i0 <= i1) {
        const int64_t a = s * (i1 - i0 + 1);
        if (a < p.a_min) break;
        const double d = (double)nnz / (double)a;
        if (d >= p.delta) {
          const double sc = score2(nnz, a, p.delta);
          if (sc > best.sc) best = {sc, o0, o1 + 1, I0 + i0, I0 + i1 + 1};
          break;
        }
        nnz -= H[i0];
        ++i0;
      }
      if (i1 >= tmax && nnz == 0) break;   // only empty slots remain
    }
  }
  for (int32_t t : touched) H[t] = 0;
  touched.clear();
}

Best find_block(const Csr &M, int64_t O0, int64_t O1, int64_t I0, int64_t I1,
                const sable_extract_params &p) {
  const int64_t s_min = isqrt_ceil(p.a_min);
  const int64_t count = O1 - O0, L_in = I1 - I0;
  if (count <= 0 || L_in <= 0) return Best{};
  int T = host_threads();
  if (count < 32) T = 1;
  if (T > count) T = (int)count;
  std::vector<Best> bests(T);
  std::atomic<int64_t> next{O0};
  auto worker = [&](int t) {
    std::vector<int32_t> H(L_in, 0), touched;
    Best b;
    for (;;) {
      const int64_t o0 = next.fetch_add(1);
      if (o0 >= O1) break;
      scan_start(M, o0, O1, I0, I1, p, s_min, H, touched, b);
    }
    bests[t] = b;
  };
  if (T == 1) {
    worker(0);
  } else {
    std::vector<std::thread> th;
    for (int t = 0; t < T; ++t) th.emplace_back(worker, t);
    for (auto &x : th) x.join();
  }
  Best out;
  for (const Best &b : bests) {
    if (b.sc < 0) continue;
    if (b.sc > out.sc || (b.sc == out.sc && b.o0 < out.o0)) out = b;
  }
  return out;
}

int64_t block_nnz(const Csr &R, int64_t r0, int64_t r1, int64_t c0, int64_t c1) {
  int64_t z = 0;
  for (int64_t r = r0; r < r1; ++r) z += R.count(r, c0, c1 - 1);
  return z;
}

void trim(const Csr &R, const Csr &RT, int64_t &r0, int64_t &r1, int64_t &c0, int64_t &c1,
          int64_t &nnz) {
  nnz = block_nnz(R, r0, r1, c0, c1);
  for (;;) {
    const int64_t area = (r1 - r0) * (c1 - c0);
    int best = -1;
    int64_t bn = 0, ba = 1;
    int64_t en[4], el[4];
    bool ok[4] = {false, false, false, false};
    if (r1 - r0 >= 2) {
      en[0] = R.count(r0, c0, c1 - 1);
      en[1] = R.count(r1 - 1, c0, c1 - 1);
      el[0] = el[1] = c1 - c0;
      ok[0] = ok[1] = true;
    }
    if (c1 - c0 >= 2) {
      en[2] = RT.count(c0, r0, r1 - 1);
      en[3] = RT.count(c1 - 1, r0, r1 - 1);
      el[2] = el[3] = r1 - r0;
      ok[2] = ok[3] = true;
    }
    for (int k = 0; k < 4; ++k) {
      if (!ok[k]) continue;
      const int64_t nn = nnz - en[k], na = area - el[k];
      if (nn * area <= nnz * na) continue;
      if (best < 0 || nn * ba > bn * na) {
        best = k;
        bn = nn;
        ba = na;
      }
    }
    if (best < 0) return;
    nnz = bn;
    if (best == 0) ++r0;
    else if (best == 1) --r1;
    else if (best == 2) ++c0;
    else --c1;
  }
}

std::vector<Region> candidate_regions(const Csr &R, const sable_extract_params &p, DevResidual *dev) {
  const int64_t m = R.m, n = R.n, g = p.tile;
  const int64_t TI = (m + g - 1) / g, TJ = (n + g - 1) / g;
  std::vector<int64_t> hot;
  if (dev) {
    // cell counts on the device; thr[a] = least count c with c >= delta * a (FP64)
    std::vector<int32_t> thr(g * g + 1, 0);
    for (int64_t a = 1; a <= g * g; ++a) {
      int64_t c = 0;
      while (c <= a && !((double)c >= p.delta * (double)a)) ++c;
      thr[a] = (int32_t)c;
    }
    if (sable_status st = dev_hot_cells(dev, (int)g, thr, hot)) throw InspectError{st};
  } else {
    // per tile row: the cells of its entries, sorted, counted in runs; tile
    // rows in parallel, concatenated in order (keys ascending)
    const int T = R.nnz() >= (1 << 20) ? host_threads() : 1;
    std::vector<std::vector<int64_t>> part(T);
    const int64_t per = (TI + T - 1) / T;
    auto work = [&](int t) {
      std::vector<int32_t> cells;
      const int64_t I1 = std::min(TI, (t + 1) * per);
      for (int64_t I = t * per; I < I1; ++I) {
        const int64_t r0 = I * g, r1 = std::min(m, r0 + g);
        cells.clear();
        for (int64_t k = R.rp[r0]; k < R.rp[r1]; ++k) cells.push_back((int32_t)(R.ci[k] / g));
        std::sort(cells.begin(), cells.end());
        for (size_t a = 0; a < cells.size();) {
          size_t b = a;
          while (b < cells.size() && cells[b] == cells[a]) ++b;
          const int64_t J = cells[a];
          const int64_t area = (r1 - r0) * std::min(g, n - J * g);
          if ((double)(b - a) >= p.delta * (double)area) part[t].push_back(I * TJ + J);
          a = b;
        }
      }
    };
    if (T == 1) {
      work(0);
    } else {
      std::vector<std::thread> th;
      for (int t = 0; t < T; ++t) th.emplace_back(work, t);
      for (auto &x : th) x.join();
    }
    for (auto &v : part) hot.insert(hot.end(), v.begin(), v.end());
  }
  std::vector<uint8_t> seen(hot.size(), 0);
  std::vector<std::array<int64_t, 4>> boxes;
  std::vector<size_t> stack, comp;
  const int64_t S = std::max<int64_t>(1, ((int64_t)p.max_span + g - 1) / g);   // slab height, tiles
  for (size_t t = 0; t < hot.size(); ++t) {
    if (seen[t]) continue;
    seen[t] = 1;
    stack.assign(1, t);
    comp.clear();
    int64_t I0 = hot[t] / TJ, I1 = I0 + 1, J0 = hot[t] % TJ, J1 = J0 + 1;
    while (!stack.empty()) {
      const size_t q = stack.back();
      stack.pop_back();
      comp.push_back(q);
      const int64_t a = hot[q] / TJ, b = hot[q] % TJ;
      I0 = std::min(I0, a);
      I1 = std::max(I1, a + 1);
      J0 = std::min(J0, b);
      J1 = std::max(J1, b + 1);
      for (int da = -1; da <= 1; ++da)
        for (int db = -1; db <= 1; ++db) {
          const int64_t aa = a + da, bb = b + db;
          if (aa < 0 || bb < 0 || aa >= TI || bb >= TJ) continue;
          auto it = std::lower_bound(hot.begin(), hot.end(), aa * TJ + bb);
          if (it != hot.end() && *it == aa * TJ + bb) {
            const size_t z = it - hot.begin();
            if (!seen[z]) {
              seen[z] = 1;
              stack.push_back(z);
            }
          }
        }
    }
    if (I1 - I0 > S && (int64_t)comp.size() * 4 < (I1 - I0) * (J1 - J0)) {
      // tall, sparsely filled component (a band): one box per slab of S tile rows
      for (int64_t a = I0; a < I1; a += S) {
        const int64_t b = std::min(I1, a + S);
        int64_t s0 = INT64_MAX, s1 = -1;
        for (size_t q : comp) {
          const int64_t r = hot[q] / TJ, c = hot[q] % TJ;
          if (r >= a && r < b) {
            s0 = std::min(s0, c);
            s1 = std::max(s1, c + 1);
          }
        }
        boxes.push_back({a == I0 ? std::max<int64_t>(0, a - 1) : a, b == I1 ? std::min(TI, b + 1) : b,
                         std::max<int64_t>(0, s0 - 1), std::min(TJ, s1 + 1)});
      }
    } else {
      boxes.push_back({std::max<int64_t>(0, I0 - 1), std::min(TI, I1 + 1), std::max<int64_t>(0, J0 - 1),
                       std::min(TJ, J1 + 1)});
    }
  }
  bool merged = true;
  while (merged) {
    merged = false;
    std::sort(boxes.begin(), boxes.end());
    for (size_t x = 0; x < boxes.size() && !merged; ++x)
      for (size_t y = x + 1; y < boxes.size(); ++y) {
        auto &A = boxes[x], &B = boxes[y];
        if (A[0] < B[1] && B[0] < A[1] && A[2] < B[3] && B[2] < A[3]) {
          A = {std::min(A[0], B[0]), std::max(A[1], B[1]), std::min(A[2], B[2]),
               std::max(A[3], B[3])};
          boxes.erase(boxes.begin() + y);
          merged = true;
          break;
        }
      }
  }
  std::sort(boxes.begin(), boxes.end());
  std::vector<Region> out;
  for (auto &b : boxes) out.push_back({b[0] * g, std::min(m, b[1] * g), b[2] * g, std::min(n, b[3] * g)});
  return out;
}

struct Partitioner {
  const Csr &R, &RT;
  const sable_extract_params &p;
  std::vector<uint8_t> used_r, used_c;
  std::vector<BlockFound> blocks;

  Partitioner(const Csr &R_, const Csr &RT_, const sable_extract_params &p_)
      : R(R_), RT(RT_), p(p_), used_r(R_.m, 0), used_c(R_.n, 0) {}

  void decompose(int64_t r0, int64_t r1, int64_t c0, int64_t c1) {
    if ((r1 - r0) * (c1 - c0) < p.a_min) return;
    Best b = find_block(R, r0, r1, c0, c1, p);
    const Best bt = find_block(RT, c0, c1, r0, r1, p);
    if (bt.sc > b.sc) b = Best{bt.sc, bt.i0, bt.i1, bt.o0, bt.o1};
    if (b.sc < 0) return;
    int64_t br0 = b.o0, br1 = b.o1, bc0 = b.i0, bc1 = b.i1;
    if ((br1 - br0) * (bc1 - bc0) < p.a_min) return;
    for (int64_t r = br0; r < br1; ++r)
      if (used_r[r]) return;
    for (int64_t c = bc0; c < bc1; ++c)
      if (used_c[c]) return;
    int64_t z;
    trim(R, RT, br0, br1, bc0, bc1, z);
    const int64_t area = (br1 - br0) * (bc1 - bc0);
    if ((double)z / (double)area < p.delta || area < p.a_min) return;
    blocks.push_back({br0, br1, bc0, bc1, z});
    for (int64_t r = br0; r < br1; ++r) used_r[r] = 1;
    for (int64_t c = bc0; c < bc1; ++c) used_c[c] = 1;
    decompose(r0, br0, c0, c1);
    decompose(br1, r1, c0, c1);
    decompose(br0, br1, c0, bc0);
    decompose(br0, br1, bc1, c1);
  }
};

}  // namespace

std::vector<BlockFound> partition_blocks(const Csr &R, const Csr &RT, const sable_extract_params &p,
                                         DevResidual *dev) {
  Partitioner P(R, RT, p);
  std::vector<Region> regions;
  if (p.tile <= 0) regions.push_back({0, R.m, 0, R.n});
  else regions = candidate_regions(R, p, dev);
  for (const Region &g : regions) P.decompose(g.r0, g.r1, g.c0, g.c1);
  std::vector<BlockFound> out;
  int64_t covered = 0;
  for (auto &b : P.blocks)
    if (b.c1 - b.c0 != 1) {
      out.push_back(b);
      covered += b.nnz;
    }
  if ((double)covered < p.coverage_min * (double)R.nnz()) out.clear();
  return out;
}

}  // namespace sable
