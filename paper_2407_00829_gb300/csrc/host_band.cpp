// Band extractor: Appendix D, Algorithm 3 (ExtractBands) and Algorithm 4
// (GrowSegments), with the FitRibbon step that Section 4.2 names but does not
// define.  Host C++, threaded over rows where rows are independent; with the
// device inspector, M[d] and FitRibbon of every entry on a candidate diagonal
// run on the GPU (sable_inspect.cu), with the same results.
//
// Readings (identical to the library's documented behaviour):
//  * M[d] counts residual entries on diagonal d = j - i, |d| <= d_max.
//    Candidates: M[d] >= count_min, by decreasing M[d], ties by increasing d.
//  * FitRibbon(i, d): (0,0,0) unless row i holds an entry at column i + d.
//    Otherwise the ribbon grows from that cell; each step reaches the nearest
//    entry below or above the ribbon (adding one entry and the zeros between),
//    takes the narrower result (below on a tie) if its density stays >= delta
//    and the side's extent stays <= w_max, and stops otherwise.  k_i = entries
//    in the final ribbon.
//  * GrowSegments as printed: rolling maximum (L, U); a widened extent recounts
//    the whole segment, an unchanged one adds row j's entries inside the
//    ribbon; the segment ends when its density drops below delta; segments
//    shorter than l_seg rows are dropped.
//  * A candidate is accepted when the summed area of its segments is >= a_min
//    and their density is >= delta; accepted rows are masked for later
//    candidates.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <thread>
#include <unordered_map>

#include "sable_internal.h"

namespace sable {

int64_t Csr::count(int64_t i, int64_t lo, int64_t hi) const {
  if (hi < lo) return 0;
  const int32_t *b = ci.data() + rp[i], *e = ci.data() + rp[i + 1];
  const int32_t *a = std::lower_bound(b, e, (int32_t)std::max<int64_t>(lo, INT32_MIN));
  const int32_t *z = std::upper_bound(a, e, (int32_t)std::min<int64_t>(hi, INT32_MAX));
  return z - a;
}

template <class F>
static void parallel_rows(int64_t n, F &&f) {
  const int T = host_threads();
  if (T <= 1 || n < 4096) {
    f(0, n);
    return;
  }
  std::vector<std::thread> th;
  const int64_t chunk = (n + T - 1) / T;
  for (int t = 0; t < T; ++t) {
    int64_t a = t * chunk, b = std::min(n, a + chunk);
    if (a >= b) break;
    th.emplace_back([&, a, b] { f(a, b); });
  }
  for (auto &x : th) x.join();
}

struct Ext { int32_t l, u, k; };

static Ext fit_ribbon(const Csr &R, int64_t i, int64_t d, double delta, int64_t w_max) {
  const int64_t c = i + d;
  if (c < 0 || c >= R.n) return {0, 0, 0};
  const int32_t *b = R.ci.data() + R.rp[i], *e = R.ci.data() + R.rp[i + 1];
  const int32_t *p = std::lower_bound(b, e, (int32_t)c);
  if (p == e || *p != c) return {0, 0, 0};
  const int64_t len = e - b;
  int64_t lo = p - b, hi = lo, l = 0, u = 0, z = 1;
  for (;;) {
    int64_t wb = -1, wa = -1, nl = 0, nu = 0;
    if (lo > 0 && c - b[lo - 1] <= w_max) {
      nl = c - b[lo - 1];
      wb = nl + u + 1;
    }
    if (hi + 1 < len && b[hi + 1] - c <= w_max) {
      nu = b[hi + 1] - c;
      wa = l + nu + 1;
    }
    if (wb < 0 && wa < 0) break;
    const bool below = wb >= 0 && (wa < 0 || wb <= wa);
    const int64_t w = below ? wb : wa;
    if ((double)(z + 1) / (double)w < delta) break;
    ++z;
    if (below) {
      l = nl;
      --lo;
    } else {
      u = nu;
      ++hi;
    }
  }
  return {(int32_t)l, (int32_t)u, (int32_t)z};
}

// Entries of row r whose offset (col - r) lies in [olo, ohi].
static inline int64_t ribbon_count(const Csr &R, int64_t r, int64_t olo, int64_t ohi) {
  return R.count(r, r + olo, r + ohi);
}

// GrowSegments (Algorithm 4) for offset d over the rows holding an entry on d:
// list positions t in [0, len), rows[t] ascending; k_of(t) = 0 where FitRibbon
// gave no ribbon (or the row is masked), ext_of(t) its (l, u, k).  Shared by
// the host FitRibbon and the device inspector's.
template <class K, class E>
static void grow_segments(const Csr &R, int64_t d, const sable_extract_params &p, int64_t len, const int32_t *rows,
                          K &&k_of, E &&ext_of, std::vector<BandSeg> &S) {
  int64_t t = 0;
  while (t < len) {
    if (k_of(t) == 0) {
      ++t;
      continue;
    }
    const int64_t i0 = rows[t];
    int64_t L = ext_of(t).l, U = ext_of(t).u;
    int64_t z = ribbon_count(R, i0, d - L, d + U);
    int64_t j = i0 + 1, u = t + 1;
    while (u < len && rows[u] == j && k_of(u) > 0) {
      const Ext eu = ext_of(u);
      const int64_t L2 = std::max<int64_t>(L, eu.l), U2 = std::max<int64_t>(U, eu.u);
      int64_t z2;
      if (L2 != L || U2 != U) {
        z2 = 0;
        for (int64_t r = i0; r <= j; ++r) z2 += ribbon_count(R, r, d - L2, d + U2);
      } else {
        z2 = z + ribbon_count(R, j, d - L, d + U);
      }
      if ((double)z2 / (double)((L2 + U2 + 1) * (j - i0 + 1)) < p.delta) break;
      L = L2;
      U = U2;
      z = z2;
      ++j;
      ++u;
    }
    if (j - i0 >= p.l_seg) S.push_back({i0, j, d, L, U, z});
    t = u;   // the next segment may start at row j (listed) or at the next listed row
  }
}

std::vector<BandSeg> extract_bands(const Csr &R, const sable_extract_params &p, DevResidual *dev) {
  const int64_t m = R.m, n = R.n;
  const int64_t d_max = p.d_max > 0 ? p.d_max : std::max(m, n);
  const int64_t count_min =
      p.count_min > 0 ? p.count_min : (int64_t)std::ceil(p.delta * (double)p.l_seg);
  // M[d] over the offset range [-(m-1), n-1]
  const int64_t span = m + n;
  std::vector<int64_t> M;
  if (dev) {
    if (sable_status st = dev_diag_counts(dev, d_max, M)) throw InspectError{st};
  } else {
    M.assign(span > 0 ? span + 1 : 1, 0);
    for (int64_t i = 0; i < m; ++i)
      for (int64_t k = R.rp[i]; k < R.rp[i + 1]; ++k) {
        const int64_t d = (int64_t)R.ci[k] - i;
        if (d <= d_max && -d <= d_max) ++M[d + m];
      }
  }
  std::vector<int64_t> D;
  for (int64_t t = 0; t < span; ++t)
    if (M[t] > 0 && M[t] >= count_min) D.push_back(t - m);
  std::stable_sort(D.begin(), D.end(), [&](int64_t a, int64_t b) {
    if (M[a + m] != M[b + m]) return M[a + m] > M[b + m];
    return a < b;
  });

  std::vector<uint8_t> used(m, 0);
  std::vector<BandSeg> out;
  auto accept = [&](std::vector<BandSeg> &S) {
    if (S.empty()) return;
    int64_t area = 0, zz = 0;
    for (auto &sg : S) {
      area += (sg.L + sg.U + 1) * (sg.i1 - sg.i0);
      zz += sg.z;
    }
    if (area < p.a_min || (double)zz / (double)area < p.delta) return;
    for (auto &sg : S) {
      for (int64_t r = sg.i0; r < sg.i1; ++r) used[r] = 1;
      out.push_back(sg);
    }
  };

  // for every offset the rows holding a residual entry on it (ascending), and
  // where that entry sits in the residual: FitRibbon(i, d) is (0, 0, 0) for
  // every other row, so only these are visited
  std::vector<int64_t> start(span + 1, 0);
  for (int64_t t = 0; t < span; ++t) start[t + 1] = start[t] + M[t];
  std::vector<int32_t> drow(start[span]);
  std::vector<int64_t> dpos(dev ? start[span] : 0);
  {
    std::vector<int64_t> pos(start.begin(), start.end() - 1);
    for (int64_t i = 0; i < m; ++i)
      for (int64_t k = R.rp[i]; k < R.rp[i + 1]; ++k) {
        const int64_t d = (int64_t)R.ci[k] - i;
        if (d <= d_max && -d <= d_max) {
          const int64_t q = pos[d + m]++;
          drow[q] = (int32_t)i;
          if (dev) dpos[q] = k;
        }
      }
  }
  // device inspector: FitRibbon of every entry on a candidate diagonal in one
  // launch (the results do not depend on the row mask, applied below)
  std::vector<uint32_t> ext_e;
  if (dev) {
    const int w_max = (int)p.w_max;
    std::vector<int32_t> zt(2 * (size_t)w_max + 2, 0);
    for (int64_t w = 1; w < (int64_t)zt.size(); ++w) {
      int64_t q = 0;
      while (q <= w && (double)q / (double)w < p.delta) ++q;
      zt[w] = (int32_t)q;
    }
    std::vector<unsigned char> cand(span + 1, 0);
    for (const int64_t d : D) cand[d + m] = 1;
    if (sable_status st = dev_fit_ribbons(dev, d_max, cand, w_max, zt, ext_e)) throw InspectError{st};
  }
  std::vector<Ext> ext;
  for (const int64_t d : D) {
    const int32_t *rows = drow.data() + start[d + m];
    const int64_t len = M[d + m];
    std::vector<BandSeg> S;
    if (dev) {
      const int64_t *at = dpos.data() + start[d + m];
      grow_segments(
          R, d, p, len, rows, [&](int64_t t) -> int64_t { return used[rows[t]] ? 0 : (int64_t)(ext_e[at[t]] >> 20); },
          [&](int64_t t) {
            const uint32_t e = ext_e[at[t]];
            return Ext{(int32_t)(e & 1023u), (int32_t)((e >> 10) & 1023u), (int32_t)(e >> 20)};
          },
          S);
    } else {
      ext.resize(len);
      auto fit = [&](int64_t a, int64_t b) {
        for (int64_t t = a; t < b; ++t)
          ext[t] = used[rows[t]] ? Ext{0, 0, 0} : fit_ribbon(R, rows[t], d, p.delta, p.w_max);
      };
      if (len < 65536) fit(0, len);
      else parallel_rows(len, fit);
      grow_segments(
          R, d, p, len, rows, [&](int64_t t) -> int64_t { return ext[t].k; }, [&](int64_t t) { return ext[t]; }, S);
    }
    accept(S);
  }
  return out;
}

}  // namespace sable
