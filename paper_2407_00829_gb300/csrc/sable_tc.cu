// VBR blocks of SpMM on the 5th-generation tensor cores (tcgen05), BF16
// operands with FP32 accumulation in tensor memory (TMEM).
//
// Each VBR block (Appendix B) is a dense nr x nc matrix; its SpMM part is the
// dense product C[r0:r0+nr, :] = Blk * B[c0:c0+nc, :].  Blocks are stored at
// upload as bf16(a / s_b), rounded to nearest even, with the per-block
// power-of-two scale s_b = 2^ceil(log2 max|a|), cut into tiles of 128 rows x
// 64 columns laid out exactly as the tensor core reads shared memory (the
// canonical K-major layout without swizzle: 8 x 8 "core matrices" of 128
// contiguous bytes, adjacent along K 128 bytes apart, adjacent along M 1024
// bytes apart).
//
// One CTA (4 warps) computes one job = (block, 128-row tile, 128-column tile
// of B/C).  Per 64-wide K step: a TMA bulk copy brings the A tile (16 KB),
// the 128 threads convert the matching 64 x 128 slice of B from FP32 to BF16
// (round to nearest even) into the same layout (B as an N x K K-major
// operand), and one thread issues four tcgen05.mma (M=128, N=128, K=16) into
// a 128-column FP32 accumulator in TMEM; tcgen05.commit signals an mbarrier
// when they finish.  The epilogue reads the accumulator with tcgen05.ld
// (warp w owns TMEM lanes / rows 32w..32w+31), multiplies by s_b and writes
// the block's rows of C.  Every wait is bounded; on time-out the kernel
// records SABLE_ERR_TIMEOUT, skips the rest of its job, frees its TMEM and
// returns.
//
// FP32-accurate variant (NS = 3): every operand value v is written as the sum
// of three bf16 terms, v1 = bf16(v), v2 = bf16(v - v1), v3 = bf16(v - v1 - v2)
// (each difference exact in FP32), 24 significant bits in all; the six
// products whose order is at most that of v1 * w3 (v3 w1, v2 w2, v1 w3, v2 w1,
// v1 w2, v1 w1, smallest first) are accumulated in FP32 in TMEM.  The dropped
// terms are below 2^-24 of the product, FP32's own rounding.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "sable_internal.h"
#include "sable_wait.cuh"

namespace sable {

namespace {

constexpr int kTcThreads = 128;
constexpr int kTileM = 128, kTileN = 128, kTileK = 64;
constexpr int kTileBytes = kTileM * kTileK * 2;        // 16 KB, A and B tiles alike
constexpr unsigned kTmemCols = 128;
constexpr int kStageFloats = 4 * 32 * 33;               // epilogue transpose: 4 warps x 32 rows x 33

template <int NS>
union TileOrStage {
  unsigned char a[NS][kTileBytes];   // A tile, one per bf16 term (K steps)
  float stage[kStageFloats];         // epilogue: accumulator rows transposed for whole-row stores
};

template <int NS>
struct TcShared {
  alignas(1024) TileOrStage<NS> u;                 // the A tiles are free in the epilogue
  alignas(1024) unsigned char b[NS][kTileBytes];   // B tile, one per bf16 term
  uint64_t bar_a;     // A tiles landed
  uint64_t bar_mma;   // MMAs of the K step finished
  uint32_t tmem_base;
  int dead;
};

__device__ __forceinline__ unsigned su32(const void *p) { return smem_u32(p); }

// Shared-memory matrix descriptor: canonical K-major layout, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(const void *p, unsigned lbo, unsigned sbo) {
  const uint64_t addr = su32(p);
  return ((addr & 0x3FFFFull) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

// Instruction descriptor: D = FP32, A = B = BF16, both K-major, M = N = 128.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTileN >> 3) << 17) |
                            ((uint32_t)(kTileM >> 4) << 24);

template <int NS>
__global__ void __launch_bounds__(kTcThreads, 1)
vbr_tc_kernel(const DevHybrid *__restrict__ mats, const int32_t *__restrict__ trip, int n_jobs, int ntn,
              const float *B0, int64_t ldb0, float *C0, int64_t ldc0, const float *const *Bs, float *const *Cs,
              int N, int *err, long long limit) {
  extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
  // align the working area to 1024 bytes
  TcShared<NS> &S =
      *reinterpret_cast<TcShared<NS> *>((reinterpret_cast<uintptr_t>(tc_smem_raw) + 1023) & ~(uintptr_t)1023);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&S.bar_a)) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&S.bar_mma)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    S.dead = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&S.tmem_base)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = S.tmem_base;
  unsigned ph_a = 0, ph_m = 0;

  for (int job = blockIdx.x; job < n_jobs; job += gridDim.x) {
    const int pair = job / ntn, n0 = (job - pair * ntn) * kTileN;
    const int mat = trip[3 * pair], bi = trip[3 * pair + 1], t = trip[3 * pair + 2];
    const DevHybrid &A = mats[mat];
    const float *__restrict__ B = Bs ? Bs[mat] : B0;
    float *__restrict__ C = Cs ? Cs[mat] : C0;
    const int64_t ldb = Bs ? N : ldb0, ldc = Cs ? N : ldc0;
    const DevBlk blk = A.blks[bi];
    const float scale = A.vbr_scale[bi];
    const int nkt = (blk.nc + kTileK - 1) / kTileK;
    const size_t toff = blk.bf_off + (size_t)t * nkt * (kTileM * kTileK);
    const uint16_t *atiles[3] = {A.vbr_bf16 + toff, NS > 1 ? A.vbr_bf16_mid + toff : nullptr,
                                 NS > 1 ? A.vbr_bf16_lo + toff : nullptr};
    bool ok = true;
    for (int kt = 0; kt < nkt && ok; ++kt) {
      // A tiles by TMA bulk copy
      if (tid == 0) {
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(&S.bar_a)),
                     "r"((unsigned)(NS * kTileBytes))
                     : "memory");
#pragma unroll
        for (int sp = 0; sp < NS; ++sp)
          asm volatile(
              "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                  su32(S.u.a[sp])),
              "l"(atiles[sp] + (size_t)kt * (kTileM * kTileK)), "r"((unsigned)kTileBytes), "r"(su32(&S.bar_a))
              : "memory");
      }
      // B slice: rows k of B (K dim), columns n (N dim) -> bf16, K-major core matrices
      const int kb = blk.c0 + kt * kTileK;
      const int kvalid = min(kTileK, blk.c0 + blk.nc - kb);
      {
        const int n = tid;                       // one column of the tile per thread
        const bool ncol = n0 + n < N;
        const float *bp = B + (size_t)kb * ldb + n0 + n;
        // all 64 rows of the thread's column in flight at once: one load latency per K step
#pragma unroll
        for (int k8 = 0; k8 < kTileK / 8; ++k8) {
          uint32_t w[NS][4];
#pragma unroll
          for (int h = 0; h < 4; ++h) {
            const int ka = 8 * k8 + 2 * h, kb2 = ka + 1;
            float f0 = (ncol && ka < kvalid) ? __ldg(bp + (size_t)ka * ldb) : 0.f;
            float f1 = (ncol && kb2 < kvalid) ? __ldg(bp + (size_t)kb2 * ldb) : 0.f;
#pragma unroll
            for (int sp = 0; sp < NS; ++sp) {   // term sp, then the exact remainder
              const __nv_bfloat16 b0 = __float2bfloat16_rn(f0), b1 = __float2bfloat16_rn(f1);
              w[sp][h] = (uint32_t)__bfloat16_as_ushort(b0) | ((uint32_t)__bfloat16_as_ushort(b1) << 16);
              f0 -= __bfloat162float(b0);
              f1 -= __bfloat162float(b1);
            }
          }
#pragma unroll
          for (int sp = 0; sp < NS; ++sp)
            *reinterpret_cast<uint4 *>(S.b[sp] + (n >> 3) * 1024 + k8 * 128 + (n & 7) * 16) =
                make_uint4(w[sp][0], w[sp][1], w[sp][2], w[sp][3]);
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncthreads();
      if (tid == 0) {
        if (!mbar_wait(&S.bar_a, ph_a, limit)) {
          // the A copies are still in flight: wait for them (bounded, longer)
          // before this CTA can leave, then give up
          (void)mbar_wait(&S.bar_a, ph_a, drain_limit(limit));
          atomicExch(err, (int)SABLE_ERR_TIMEOUT);
          S.dead = 1;
        } else {
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          // products (A term, B term), smallest first: one for NS = 1, six for NS = 3
          constexpr int kPairs = NS == 1 ? 1 : 6;
          constexpr int kPa[6] = {2, 1, 0, 1, 0, 0}, kPb[6] = {0, 1, 2, 0, 1, 0};
#pragma unroll
          for (int ks = 0; ks < kTileK / 16; ++ks) {
#pragma unroll
            for (int pr = 0; pr < kPairs; ++pr) {
              const int ta = NS == 1 ? 0 : kPa[pr], tb = NS == 1 ? 0 : kPb[pr];
              const uint64_t ad = smem_desc(S.u.a[ta] + ks * 256, 128, 1024);
              const uint64_t bd = smem_desc(S.b[tb] + ks * 256, 128, 1024);
              const uint32_t acc = (kt > 0 || ks > 0 || pr > 0) ? 1u : 0u;
              asm volatile(
                  "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                  "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                  "l"(ad), "l"(bd), "r"(kIdesc), "r"(acc)
                  : "memory");
            }
          }
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                           su32(&S.bar_mma))
                       : "memory");
        }
      }
      ph_a ^= 1u;
      __syncthreads();
      if (S.dead) {
        ok = false;
        break;
      }
      // the tiles are overwritten next step: wait for the MMAs to finish reading them
      bool done = __all_sync(0xffffffffu, mbar_wait(&S.bar_mma, ph_m, limit));
      if (!done) {   // the MMAs still read shared memory and write TMEM: wait (bounded, longer)
        (void)__all_sync(0xffffffffu, mbar_wait(&S.bar_mma, ph_m, drain_limit(limit)));
        if (lane == 0) atomicExch(err, (int)SABLE_ERR_TIMEOUT);
        S.dead = 1;
      }
      ph_m ^= 1u;
      __syncthreads();
      if (S.dead) ok = false;
    }
    if (!ok) break;
    // epilogue: TMEM -> registers -> scale -> shared (transpose) -> C, whole
    // rows per store instruction.  The A/B tiles are free: the MMAs are done.
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    float *stage = S.u.stage + warp * (32 * 33);                             // 32 rows x 33 (padded)
    const int rbase = t * kTileM + 32 * warp;                             // first row of my warp in the block
#pragma unroll 1
    for (int ch = 0; ch < kTileN / 32; ++ch) {
      uint32_t r[32];
      const uint32_t taddr = tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(32 * ch);
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
          "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
            "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
            "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
            "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int j = 0; j < 32; ++j) stage[lane * 33 + j] = __uint_as_float(r[j]) * scale;
      __syncwarp();
      const int col = n0 + 32 * ch + lane;
#pragma unroll 4
      for (int rr = 0; rr < 32; ++rr) {
        const int row = rbase + rr;
        if (row < blk.nr && col < N) C[(size_t)(blk.r0 + row) * ldc + col] = stage[rr * 33 + lane];
      }
      __syncwarp();
    }
    // all warps have read the accumulator before the next job overwrites it;
    // the staging writes (generic proxy) are ordered before the next job's
    // bulk copies (async proxy) into the same bytes
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

}  // namespace

template <int NS>
size_t tc_smem_bytes() { return sizeof(TcShared<NS>) + 1024; }
static_assert(sizeof(TileOrStage<1>) >= (size_t)kStageFloats * 4 && sizeof(TileOrStage<3>) >= (size_t)kStageFloats * 4,
              "epilogue staging area inside the A-tile region");

// Host: bf16 of a float, round to nearest even (NaN kept quiet).
static uint16_t to_bf16(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  if ((u & 0x7F800000u) == 0x7F800000u && (u & 0x007FFFFFu)) return (uint16_t)((u >> 16) | 0x40);
  const uint32_t r = u + 0x7FFFu + ((u >> 16) & 1u);
  return (uint16_t)(r >> 16);
}

// Host: power-of-two scale 2^ceil(log2 amax) (1 for an all-zero block).
static float pow2_scale(float amax) {
  if (!(amax > 0.f) || !std::isfinite(amax)) return 1.f;
  int e;
  const float m = std::frexp(amax, &e);   // amax = m 2^e, m in [0.5, 1)
  return std::ldexp(1.f, m == 0.5f ? e - 1 : e);
}

// bf16 value of a host bf16 bit pattern
static float from_bf16(uint16_t h) {
  const uint32_t u = (uint32_t)h << 16;
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}

void pack_vbr_bf16(const std::vector<Block> &blks, const std::vector<float> &canon,
                   std::vector<uint16_t> &packed, std::vector<float> &scales, std::vector<int64_t> &offs,
                   std::vector<uint16_t> *mid, std::vector<uint16_t> *lo) {
  packed.clear();
  scales.clear();
  offs.clear();
  if (mid) mid->clear();
  if (lo) lo->clear();
  int64_t voff = 0;
  for (const Block &b : blks) {
    float amax = 0.f;
    for (int64_t k = 0; k < b.nr * b.nc; ++k) amax = std::max(amax, std::fabs(canon[voff + k]));
    const float s = pow2_scale(amax);
    scales.push_back(s);
    offs.push_back((int64_t)packed.size());
    const int64_t nt = (b.nr + kTileM - 1) / kTileM, nkt = (b.nc + kTileK - 1) / kTileK;
    const size_t base = packed.size();
    packed.resize(base + (size_t)(nt * nkt * kTileM * kTileK), 0);
    if (mid) mid->resize(packed.size(), 0);
    if (lo) lo->resize(packed.size(), 0);
    for (int64_t t = 0; t < nt; ++t)
      for (int64_t kt = 0; kt < nkt; ++kt) {
        uint16_t *tile = packed.data() + base + (size_t)((t * nkt + kt) * kTileM * kTileK);
        for (int m = 0; m < kTileM; ++m) {
          const int64_t r = t * kTileM + m;
          if (r >= b.nr) break;
          for (int k = 0; k < kTileK; ++k) {
            const int64_t c = kt * kTileK + k;
            if (c >= b.nc) break;
            const float v = canon[voff + c * b.nr + r] / s;     // exact: s is a power of two
            const size_t at = (size_t)(tile - packed.data()) + (m >> 3) * 512 + (k >> 3) * 64 + (m & 7) * 8 + (k & 7);
            const uint16_t h1 = to_bf16(v);
            packed[at] = h1;
            if (mid && lo) {   // the next two terms of v, each from an exact FP32 remainder
              const float r1 = v - from_bf16(h1);
              const uint16_t h2 = to_bf16(r1);
              (*mid)[at] = h2;
              (*lo)[at] = to_bf16(r1 - from_bf16(h2));
            }
          }
        }
      }
    voff += b.nr * b.nc;
  }
}

void vbr_tc_pairs(const std::vector<Block> &blks, int32_t mat, std::vector<int32_t> &trip) {
  for (size_t bi = 0; bi < blks.size(); ++bi) {
    const int64_t nt = (blks[bi].nr + kTileM - 1) / kTileM;
    for (int64_t t = 0; t < nt; ++t) {
      trip.push_back(mat);
      trip.push_back((int32_t)bi);
      trip.push_back((int32_t)t);
    }
  }
}

sable_status launch_vbr_tc(const DevHybrid *mats, const int32_t *trip, int n_trip, const float *B, int64_t ldb,
                           float *C, int64_t ldc, const float *const *Bs, float *const *Cs, int N, int sm_count,
                           int *err, cudaStream_t_ st, int terms) {
  const int ntn = (N + kTileN - 1) / kTileN;
  const long long nj = (long long)n_trip * ntn;
  if (nj == 0) return SABLE_OK;
  if (nj > INT32_MAX || (terms != 1 && terms != 3)) return SABLE_ERR_INVALID;
  // at most 4 CTAs per SM so that their TMEM allocations (128 columns each) fit;
  // the three-term variant's tiles allow 2
  const size_t smem_req = terms == 1 ? std::max(tc_smem_bytes<1>(), (size_t)56 * 1024) : tc_smem_bytes<3>();
  const int per_sm = terms == 1 ? 4 : 2;
  auto k = terms == 1 ? vbr_tc_kernel<1> : vbr_tc_kernel<3>;
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_req);
  const int grid = std::max(1, std::min((int)nj, per_sm * std::max(sm_count, 1)));
  k<<<grid, kTcThreads, smem_req, st>>>(mats, trip, (int)nj, ntn, B, ldb, C, ldc, Bs, Cs, N, err,
                                        wait_limit_cycles());
  if (cudaGetLastError() != cudaSuccess) {
    (void)cudaGetLastError();
    return SABLE_ERR_CUDA;
  }
  return SABLE_OK;
}

}  // namespace sable
