// Learned planner support on the device: structural features of a COO
// matrix and a small multilayer perceptron (forward, backward, Adam), all
// FP32, deterministic (no atomics in the MLP).
//
// Features (kFeat values, each scaled to about [0, 1]):
//   0 log2(m+1)/24   1 log2(n+1)/24   2 log2(nnz+1)/32
//   3 log2(mean entries per row + 1)/8   4 coefficient of variation of row lengths / 8
//   5 log2(max row length + 1)/16
//   6..13  share of rows with length 0, 1, 2-3, 4-7, 8-15, 16-31, 32-63, >= 64
//   14..17 share of entries on diagonals d = j - i whose count M[d] (Algorithm 3's
//          histogram) is < min(m,n)/64, < /16, < /4, >= min(m,n)/4
//   18     share of entries with |j - i| <= 64
//   19..22 share of (sampled) entries lying in 8 x 8 tiles holding >= 48, >= 32,
//          >= 16, >= 8 (sampled) entries  (block density, the block extractor's
//          candidate test); tiles are counted in a hash table
//   23     log2(N + 1)/8, N = dense columns of the product (0 for SpMV), set by
//          the caller after the call (written 0 here)
// Entries whose row is outside [0, m) or column outside [0, n) are skipped
// (never used as an index) and counted; if there is any, every feature is
// written as NaN.  The final step is FP32, with the row-length variance's
// numerator m sum L^2 - (sum L)^2 formed exactly in 128-bit integers.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>

#include "sable_internal.h"

namespace sable {
namespace {

constexpr int kFeat = 24;
constexpr int kThreads = 256;
constexpr unsigned long long kEmpty = 0xffffffffffffffffull;

constexpr int kAccOutside = 21;   // acc slot: entries outside the matrix

__global__ void feat_count(int64_t nnz, const int32_t *__restrict__ row, const int32_t *__restrict__ col,
                           int64_t m, int64_t n, int32_t *__restrict__ rowlen, int32_t *__restrict__ dcount,
                           unsigned long long *__restrict__ keys, int32_t *__restrict__ cnt, int64_t slots,
                           int64_t stride, int64_t ntile_cols, unsigned long long *__restrict__ acc) {
  unsigned long long near = 0, outside = 0;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nnz; k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = row[k], j = col[k];
    if ((uint64_t)i >= (uint64_t)m || (uint64_t)j >= (uint64_t)n) {
      ++outside;
      continue;
    }
    atomicAdd(&rowlen[i], 1);
    atomicAdd(&dcount[j - i + m - 1], 1);
    near += (j - i <= 64 && i - j <= 64);
    if (k % stride == 0) {
      const unsigned long long key = (unsigned long long)((i >> 3) * ntile_cols + (j >> 3));
      unsigned long long h = (key * 0x9E3779B97F4A7C15ull) >> 20;
      for (int64_t probe = 0; probe < slots; ++probe) {
        const int64_t s = (int64_t)((h + probe) & (unsigned long long)(slots - 1));
        const unsigned long long old = atomicCAS(&keys[s], kEmpty, key);
        if (old == kEmpty || old == key) {
          atomicAdd(&cnt[s], 1);
          break;
        }
      }
    }
  }
  atomicAdd(&acc[0], near);
  if (outside) atomicAdd(&acc[kAccOutside], outside);
}

__global__ void feat_tiles(int64_t nnz, const int32_t *__restrict__ row, const int32_t *__restrict__ col,
                           int64_t m, int64_t n, const unsigned long long *__restrict__ keys,
                           const int32_t *__restrict__ cnt, int64_t slots, int64_t stride, int64_t ntile_cols,
                           unsigned long long *__restrict__ acc) {
  unsigned long long b[4] = {0, 0, 0, 0}, sampled = 0;
  for (int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * stride; k < nnz;
       k += (int64_t)gridDim.x * blockDim.x * stride) {
    const int64_t i = row[k], j = col[k];
    if ((uint64_t)i >= (uint64_t)m || (uint64_t)j >= (uint64_t)n) continue;   // counted by feat_count
    const unsigned long long key = (unsigned long long)((i >> 3) * ntile_cols + (j >> 3));
    unsigned long long h = (key * 0x9E3779B97F4A7C15ull) >> 20;
    int c = 0;
    for (int64_t probe = 0; probe < slots; ++probe) {
      const int64_t s = (int64_t)((h + probe) & (unsigned long long)(slots - 1));
      if (keys[s] == key) {
        c = cnt[s];
        break;
      }
      if (keys[s] == kEmpty) break;
    }
    ++sampled;
    b[0] += c >= 48;
    b[1] += c >= 32;
    b[2] += c >= 16;
    b[3] += c >= 8;
  }
  for (int q = 0; q < 4; ++q) atomicAdd(&acc[1 + q], b[q]);
  atomicAdd(&acc[5], sampled);
}

// rows: histogram, sum, sum of squares, max; diagonals: entry-weighted bins
__global__ void feat_reduce(int64_t m, int64_t nd, const int32_t *__restrict__ rowlen,
                            const int32_t *__restrict__ dcount, int64_t mn, unsigned long long *__restrict__ acc) {
  unsigned long long h[8] = {0, 0, 0, 0, 0, 0, 0, 0}, s = 0, s2 = 0, mx = 0, dg[4] = {0, 0, 0, 0};
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = tid; i < m; i += step) {
    const unsigned long long L = (unsigned)rowlen[i];
    s += L;
    s2 += L * L;
    mx = L > mx ? L : mx;
    const int bin = L == 0 ? 0 : min(7, 1 + (63 - __clzll((long long)L)));
    ++h[bin];
  }
  for (int64_t d = tid; d < nd; d += step) {
    const unsigned long long c = (unsigned)dcount[d];
    if (!c) continue;
    const int bin = c * 64 < (unsigned long long)mn ? 0 : c * 16 < (unsigned long long)mn ? 1 : c * 4 < (unsigned long long)mn ? 2 : 3;
    dg[bin] += c;
  }
  for (int q = 0; q < 8; ++q) atomicAdd(&acc[6 + q], h[q]);
  atomicAdd(&acc[14], s);
  atomicAdd(&acc[15], s2);
  atomicMax(&acc[16], mx);
  for (int q = 0; q < 4; ++q) atomicAdd(&acc[17 + q], dg[q]);
}

__global__ void feat_final(int64_t m, int64_t n, int64_t nnz, const unsigned long long *__restrict__ acc,
                           float *__restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (acc[kAccOutside] != 0) {   // an entry outside the matrix: no feature is meaningful
    for (int q = 0; q < kFeat; ++q) out[q] = __int_as_float(0x7fc00000);
    return;
  }
  const float M = (float)m, NZ = (float)nnz;
  const unsigned long long s = acc[14], s2 = acc[15];
  const float mean = m > 0 ? (float)s / M : 0.f;
  // coefficient of variation sqrt(var) / mean = sqrt(m s2 - s^2) / s, the
  // numerator exact: m s2 < 2^94 as a 128-bit product, s^2 < 2^62
  float cv = 0.f;
  if (m > 0 && s > 0) {
    const unsigned long long mu = (unsigned long long)m;
    const unsigned long long lo1 = mu * s2, hi1 = __umul64hi(mu, s2), sq = s * s;
    const unsigned long long lo = lo1 - sq, hi = hi1 - (lo1 < sq ? 1ull : 0ull);
    const float num = (float)hi * 18446744073709551616.0f + (float)lo;
    cv = sqrtf(num) / (float)s;
  }
  out[0] = log2f(M + 1.f) / 24.f;
  out[1] = log2f((float)n + 1.f) / 24.f;
  out[2] = log2f(NZ + 1.f) / 32.f;
  out[3] = log2f(mean + 1.f) / 8.f;
  out[4] = cv / 8.f;
  out[5] = log2f((float)acc[16] + 1.f) / 16.f;
  for (int q = 0; q < 8; ++q) out[6 + q] = m > 0 ? (float)acc[6 + q] / M : 0.f;
  for (int q = 0; q < 4; ++q) out[14 + q] = nnz > 0 ? (float)acc[17 + q] / NZ : 0.f;
  out[18] = nnz > 0 ? (float)acc[0] / NZ : 0.f;
  const float smp = (float)acc[5];
  for (int q = 0; q < 4; ++q) out[19 + q] = smp > 0.f ? (float)acc[1 + q] / smp : 0.f;
  out[23] = 0.f;
}

struct FeatWork {
  int64_t slots, stride;
  size_t o_rowlen, o_dcount, o_keys, o_cnt, o_acc, total;
};

FeatWork feat_layout(int64_t m, int64_t n, int64_t nnz) {
  FeatWork w{};
  const int64_t cap = 1 << 22;   // sampled entries put in the tile table
  w.stride = std::max<int64_t>(1, (nnz + cap - 1) / cap);
  const int64_t samples = (nnz + w.stride - 1) / w.stride;
  int64_t slots = 1024;
  while (slots < 2 * samples) slots <<= 1;
  w.slots = slots;
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  size_t off = 0;
  w.o_rowlen = off;
  off += al((size_t)std::max<int64_t>(m, 1) * 4);
  w.o_dcount = off;
  off += al((size_t)std::max<int64_t>(m + n, 1) * 4);
  w.o_keys = off;
  off += al((size_t)slots * 8);
  w.o_cnt = off;
  off += al((size_t)slots * 4);
  w.o_acc = off;
  off += al(32 * 8);
  w.total = off;
  return w;
}

// ------------------------------------------------------------------ MLP
// Layout of the parameters: W1 [in x h1], b1 [h1], W2 [h1 x h2], b2 [h2],
// W3 [h2 x out], b3 [out]; matrices row-major.  Activations ReLU, ReLU, linear.
struct Offs {
  int64_t w1, b1, w2, b2, w3, b3, total;
};

Offs mlp_offs(const sable_mlp_shape &s) {
  Offs o{};
  o.w1 = 0;
  o.b1 = o.w1 + (int64_t)s.n_in * s.n_h1;
  o.w2 = o.b1 + s.n_h1;
  o.b2 = o.w2 + (int64_t)s.n_h1 * s.n_h2;
  o.w3 = o.b2 + s.n_h2;
  o.b3 = o.w3 + (int64_t)s.n_h2 * s.n_out;
  o.total = o.b3 + s.n_out;
  return o;
}

// Z[b, j] = sum_i X[b, i] W[i, j] + bias[j]; A = relu(Z) if relu
__global__ void dense_fwd(const float *__restrict__ X, const float *__restrict__ W, const float *__restrict__ bias,
                          int64_t B, int in, int out, float *__restrict__ Z, float *__restrict__ A, bool relu) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= B * out) return;
  const int64_t b = t / out;
  const int j = (int)(t - b * out);
  float z = bias[j];
  for (int i = 0; i < in; ++i) z = fmaf(X[b * in + i], W[(int64_t)i * out + j], z);
  Z[t] = z;
  A[t] = relu ? fmaxf(z, 0.f) : z;
}

// masked mean squared error and its gradient with respect to Y
__global__ void mse_loss(const float *__restrict__ Y, const float *__restrict__ T, const float *__restrict__ mask,
                         int64_t count, float *__restrict__ dY, float *__restrict__ loss) {
  __shared__ float s_num[kThreads], s_den[kThreads];
  float num = 0.f, den = 0.f;
  for (int64_t t = threadIdx.x; t < count; t += blockDim.x) {
    const float mk = mask ? mask[t] : 1.f;
    const float d = Y[t] - T[t];
    num += mk * d * d;
    den += mk;
  }
  s_num[threadIdx.x] = num;
  s_den[threadIdx.x] = den;
  __syncthreads();
  for (int k = blockDim.x / 2; k > 0; k >>= 1) {
    if ((int)threadIdx.x < k) {
      s_num[threadIdx.x] += s_num[threadIdx.x + k];
      s_den[threadIdx.x] += s_den[threadIdx.x + k];
    }
    __syncthreads();
  }
  const float D = fmaxf(s_den[0], 1.f);
  for (int64_t t = threadIdx.x; t < count; t += blockDim.x) {
    const float mk = mask ? mask[t] : 1.f;
    dY[t] = 2.f * mk * (Y[t] - T[t]) / D;
  }
  if (threadIdx.x == 0 && loss) *loss = s_num[0] / D;
}

// dZ = dA * relu'(Z) (or dA when linear)
__global__ void relu_bwd(const float *__restrict__ dA, const float *__restrict__ Z, int64_t count, bool relu,
                         float *__restrict__ dZ) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < count) dZ[t] = relu ? (Z[t] > 0.f ? dA[t] : 0.f) : dA[t];
}

// dW[i, j] = sum_b X[b, i] dZ[b, j]; db[j] = sum_b dZ[b, j] (row i = in for the bias)
__global__ void dense_wgrad(const float *__restrict__ X, const float *__restrict__ dZ, int64_t B, int in, int out,
                            float *__restrict__ dW, float *__restrict__ db) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)(in + 1) * out) return;
  const int i = (int)(t / out), j = (int)(t - (int64_t)i * out);
  float g = 0.f;
  if (i < in)
    for (int64_t b = 0; b < B; ++b) g = fmaf(X[b * in + i], dZ[b * out + j], g);
  else
    for (int64_t b = 0; b < B; ++b) g += dZ[b * out + j];
  if (i < in) dW[(int64_t)i * out + j] = g;
  else db[j] = g;
}

// dX[b, i] = sum_j dZ[b, j] W[i, j]
__global__ void dense_xgrad(const float *__restrict__ dZ, const float *__restrict__ W, int64_t B, int in, int out,
                            float *__restrict__ dX) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= B * in) return;
  const int64_t b = t / in;
  const int i = (int)(t - b * in);
  float g = 0.f;
  for (int j = 0; j < out; ++j) g = fmaf(dZ[b * out + j], W[(int64_t)i * out + j], g);
  dX[t] = g;
}

__global__ void adam_step(int64_t count, float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                          float *__restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= count) return;
  const float gt = g[t];
  const float mt = b1 * m[t] + (1.f - b1) * gt;
  const float vt = b2 * v[t] + (1.f - b2) * gt * gt;
  m[t] = mt;
  v[t] = vt;
  p[t] -= lr * (mt / c1) / (sqrtf(vt / c2) + eps);
}

inline int blocks_for(int64_t n) { return (int)std::max<int64_t>(1, (n + kThreads - 1) / kThreads); }

bool shape_ok(const sable_mlp_shape *s) {
  return s && s->n_in > 0 && s->n_h1 > 0 && s->n_h2 > 0 && s->n_out > 0 && s->n_in <= 4096 && s->n_h1 <= 4096 &&
         s->n_h2 <= 4096 && s->n_out <= 4096;
}

// work: Z1 A1 Z2 A2 Y dY dA2 dZ2 dA1 dZ1 (B x width each; sized by sable_mlp_work_floats)
struct Work {
  float *z1, *a1, *z2, *a2, *y, *dy, *da2, *dz2, *da1, *dz1;
};

Work work_of(const sable_mlp_shape &s, int64_t B, float *w) {
  Work k;
  k.z1 = w;
  k.a1 = k.z1 + B * s.n_h1;
  k.z2 = k.a1 + B * s.n_h1;
  k.a2 = k.z2 + B * s.n_h2;
  k.y = k.a2 + B * s.n_h2;
  k.dy = k.y + B * s.n_out;
  k.da2 = k.dy + B * s.n_out;
  k.dz2 = k.da2 + B * s.n_h2;
  k.da1 = k.dz2 + B * s.n_h2;
  k.dz1 = k.da1 + B * s.n_h1;
  return k;
}

void forward(const sable_mlp_shape &s, const float *P, const float *X, int64_t B, const Work &k, cudaStream_t st) {
  const Offs o = mlp_offs(s);
  dense_fwd<<<blocks_for(B * s.n_h1), kThreads, 0, st>>>(X, P + o.w1, P + o.b1, B, s.n_in, s.n_h1, k.z1, k.a1, true);
  dense_fwd<<<blocks_for(B * s.n_h2), kThreads, 0, st>>>(k.a1, P + o.w2, P + o.b2, B, s.n_h1, s.n_h2, k.z2, k.a2, true);
  dense_fwd<<<blocks_for(B * s.n_out), kThreads, 0, st>>>(k.a2, P + o.w3, P + o.b3, B, s.n_h2, s.n_out, k.y, k.y, false);
}

}  // namespace
}  // namespace sable

using namespace sable;

// Scratch of sable_features_noalloc: one fixed device array, created when the
// library's device code is loaded on a GPU and held there until the process
// exits.  Host code may not use the symbol's host-side address; each device's
// own address is looked up once (with that device current) and then passed to
// the kernels.
static __device__ __align__(256) unsigned char g_feat_scratch[SABLE_FEATURES_NOALLOC_MAX_BYTES];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void *g_scratch_addr[kMaxDevices] = {};

sable_status feat_scratch_address(void **out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return SABLE_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return SABLE_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_feat_scratch) != cudaSuccess || !p) return SABLE_ERR_CUDA;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return SABLE_OK;
}
}  // namespace

extern "C" {

int64_t sable_features_workspace_bytes(int64_t m, int64_t n, int64_t nnz) {
  if (m < 0 || n < 0 || nnz < 0) return -1;
  return (int64_t)feat_layout(m, n, nnz).total;
}

sable_status sable_features(int64_t m, int64_t n, int64_t nnz, const int32_t *row, const int32_t *col,
                            void *work, int64_t work_bytes, float *out, void *stream) {
  if (m < 0 || n < 0 || nnz < 0 || !out || !work || (nnz > 0 && (!row || !col))) return SABLE_ERR_INVALID;
  const FeatWork w = feat_layout(m, n, nnz);
  if (work_bytes < (int64_t)w.total) return SABLE_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  char *base = static_cast<char *>(work);
  int32_t *rowlen = reinterpret_cast<int32_t *>(base + w.o_rowlen);
  int32_t *dcount = reinterpret_cast<int32_t *>(base + w.o_dcount);
  unsigned long long *keys = reinterpret_cast<unsigned long long *>(base + w.o_keys);
  int32_t *cnt = reinterpret_cast<int32_t *>(base + w.o_cnt);
  unsigned long long *acc = reinterpret_cast<unsigned long long *>(base + w.o_acc);
  cudaError_t e = cudaMemsetAsync(base, 0, w.o_keys, st);                       // rowlen, dcount
  if (e == cudaSuccess) e = cudaMemsetAsync(keys, 0xff, (size_t)w.slots * 8, st);  // empty keys
  if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, (size_t)w.slots * 4, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(acc, 0, 32 * 8, st);
  if (e != cudaSuccess) return SABLE_ERR_CUDA;
  const int64_t ntc = (n + 7) / 8;
  const int grid = (int)std::min<int64_t>(4096, std::max<int64_t>(1, (nnz + kThreads - 1) / kThreads));
  if (nnz > 0) {
    feat_count<<<grid, kThreads, 0, st>>>(nnz, row, col, m, n, rowlen, dcount, keys, cnt, w.slots, w.stride, ntc,
                                          acc);
    feat_tiles<<<grid, kThreads, 0, st>>>(nnz, row, col, m, n, keys, cnt, w.slots, w.stride, ntc, acc);
  }
  const int64_t nd = m + n > 0 ? m + n - 1 : 0;
  const int gridr = (int)std::min<int64_t>(4096, std::max<int64_t>(1, (std::max(m, nd) + kThreads - 1) / kThreads));
  feat_reduce<<<gridr, kThreads, 0, st>>>(m, nd, rowlen, dcount, std::max<int64_t>(1, std::min(m, n)), acc);
  feat_final<<<1, 32, 0, st>>>(m, n, nnz, acc, out);
  return cudaGetLastError() == cudaSuccess ? SABLE_OK : SABLE_ERR_CUDA;
}

sable_status sable_features_noalloc(int64_t m, int64_t n, int64_t nnz, const int32_t *row, const int32_t *col,
                                    float *out, void *stream) {
  if (m < 0 || n < 0 || nnz < 0 || !out || (nnz > 0 && (!row || !col))) return SABLE_ERR_INVALID;
  const FeatWork w = feat_layout(m, n, nnz);
  if (w.total > (size_t)SABLE_FEATURES_NOALLOC_MAX_BYTES) return SABLE_ERR_UNSUPPORTED;
  void *scratch = nullptr;
  const sable_status got = feat_scratch_address(&scratch);
  if (got != SABLE_OK) return got;
  cudaStream_t st = (cudaStream_t)stream;
  char *base = static_cast<char *>(scratch);
  int32_t *rowlen = reinterpret_cast<int32_t *>(base + w.o_rowlen);
  int32_t *dcount = reinterpret_cast<int32_t *>(base + w.o_dcount);
  unsigned long long *keys = reinterpret_cast<unsigned long long *>(base + w.o_keys);
  int32_t *cnt = reinterpret_cast<int32_t *>(base + w.o_cnt);
  unsigned long long *acc = reinterpret_cast<unsigned long long *>(base + w.o_acc);
  // the array keeps the previous call's contents: reset counters and the table
  cudaError_t e = cudaMemsetAsync(base, 0, w.o_keys, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(keys, 0xff, (size_t)w.slots * 8, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, (size_t)w.slots * 4, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(acc, 0, 32 * 8, st);
  if (e != cudaSuccess) return SABLE_ERR_CUDA;
  const int64_t ntc = (n + 7) / 8;
  const int grid = (int)std::min<int64_t>(4096, std::max<int64_t>(1, (nnz + kThreads - 1) / kThreads));
  if (nnz > 0) {
    feat_count<<<grid, kThreads, 0, st>>>(nnz, row, col, m, n, rowlen, dcount, keys, cnt, w.slots, w.stride, ntc,
                                          acc);
    feat_tiles<<<grid, kThreads, 0, st>>>(nnz, row, col, m, n, keys, cnt, w.slots, w.stride, ntc, acc);
  }
  const int64_t nd = m + n > 0 ? m + n - 1 : 0;
  const int gridr = (int)std::min<int64_t>(4096, std::max<int64_t>(1, (std::max(m, nd) + kThreads - 1) / kThreads));
  feat_reduce<<<gridr, kThreads, 0, st>>>(m, nd, rowlen, dcount, std::max<int64_t>(1, std::min(m, n)), acc);
  feat_final<<<1, 32, 0, st>>>(m, n, nnz, acc, out);
  return cudaGetLastError() == cudaSuccess ? SABLE_OK : SABLE_ERR_CUDA;
}

int64_t sable_mlp_param_count(const sable_mlp_shape *s) { return shape_ok(s) ? mlp_offs(*s).total : -1; }

int64_t sable_mlp_work_floats(const sable_mlp_shape *s, int64_t batch) {
  if (!shape_ok(s) || batch < 1) return -1;
  // Work: Z1 A1 dA1 dZ1 (h1 each), Z2 A2 dA2 dZ2 (h2 each), Y dY (out each), per row
  return batch * (4 * (int64_t)s->n_h1 + 4 * (int64_t)s->n_h2 + 2 * (int64_t)s->n_out);
}

sable_status sable_mlp_forward(const sable_mlp_shape *s, const float *params, const float *X, int64_t batch, float *Y,
                               float *work, void *stream) {
  if (!shape_ok(s) || !params || !X || !Y || !work || batch < 1) return SABLE_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  const Work k = work_of(*s, batch, work);
  forward(*s, params, X, batch, k, st);
  if (cudaMemcpyAsync(Y, k.y, (size_t)batch * s->n_out * 4, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return SABLE_ERR_CUDA;
  return cudaGetLastError() == cudaSuccess ? SABLE_OK : SABLE_ERR_CUDA;
}

sable_status sable_mlp_grad(const sable_mlp_shape *s, const float *params, const float *X, const float *T,
                            const float *mask, int64_t batch, float *grads, float *loss, float *work, void *stream) {
  if (!shape_ok(s) || !params || !X || !T || !grads || !work || batch < 1) return SABLE_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  const Offs o = mlp_offs(*s);
  const Work k = work_of(*s, batch, work);
  forward(*s, params, X, batch, k, st);
  mse_loss<<<1, kThreads, 0, st>>>(k.y, T, mask, batch * s->n_out, k.dy, loss);
  // layer 3 (linear): dZ3 = dY
  dense_wgrad<<<blocks_for((int64_t)(s->n_h2 + 1) * s->n_out), kThreads, 0, st>>>(
      k.a2, k.dy, batch, s->n_h2, s->n_out, grads + o.w3, grads + o.b3);
  dense_xgrad<<<blocks_for(batch * s->n_h2), kThreads, 0, st>>>(k.dy, params + o.w3, batch, s->n_h2, s->n_out, k.da2);
  relu_bwd<<<blocks_for(batch * s->n_h2), kThreads, 0, st>>>(k.da2, k.z2, batch * s->n_h2, true, k.dz2);
  dense_wgrad<<<blocks_for((int64_t)(s->n_h1 + 1) * s->n_h2), kThreads, 0, st>>>(
      k.a1, k.dz2, batch, s->n_h1, s->n_h2, grads + o.w2, grads + o.b2);
  dense_xgrad<<<blocks_for(batch * s->n_h1), kThreads, 0, st>>>(k.dz2, params + o.w2, batch, s->n_h1, s->n_h2, k.da1);
  relu_bwd<<<blocks_for(batch * s->n_h1), kThreads, 0, st>>>(k.da1, k.z1, batch * s->n_h1, true, k.dz1);
  dense_wgrad<<<blocks_for((int64_t)(s->n_in + 1) * s->n_h1), kThreads, 0, st>>>(
      X, k.dz1, batch, s->n_in, s->n_h1, grads + o.w1, grads + o.b1);
  return cudaGetLastError() == cudaSuccess ? SABLE_OK : SABLE_ERR_CUDA;
}

sable_status sable_mlp_adam(int64_t count, float *params, const float *grads, float *m, float *v, int64_t step,
                            float lr, float beta1, float beta2, float eps, void *stream) {
  if (count < 0 || step < 1 || (count > 0 && (!params || !grads || !m || !v))) return SABLE_ERR_INVALID;
  if (count == 0) return SABLE_OK;
  const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
  adam_step<<<blocks_for(count), kThreads, 0, (cudaStream_t)stream>>>(count, params, grads, m, v, lr, beta1, beta2,
                                                                    eps, c1, c2);
  return cudaGetLastError() == cudaSuccess ? SABLE_OK : SABLE_ERR_CUDA;
}

}  // extern "C"
