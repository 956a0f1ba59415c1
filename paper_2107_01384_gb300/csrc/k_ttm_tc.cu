// Split-precision mode-k product on the 5th-generation tensor cores.
//
// Projection (Algorithm 1): Y[l][j][c] = sum_i U[i][j] X[l][i][c], i.e. for
// every "column" gamma = (l, c) of the (L, n, R) view, y_gamma = U^T x_gamma.
// As a GEMM: D[gamma][j] = sum_i A[gamma][i] B[j][i] with M = gamma (128 per
// tile, any L and R), N = a chunk of <= 32 output indices j (padded to 16),
// K = n.  The same kernel runs the expansion Y = U ._k X with B[a][b] = U[a][b].
// Both operands are cut into three integer slices (tc::slice3i): X on the
// tensor's power-of-two scale (projections) or on one power of two per column
// gamma (expansions: a row of the MMA sums inside one column, so the column's
// scale factors out exactly), the factor on the scale 2^8 (|U| <= 1).  The
// nine slice products go, by order s + t, into five TMEM accumulators.  By
// Cauchy-Schwarz every partial sum of an order is below 2^16 sqrt(n) (a factor
// column or row has norm <= 1), so for the sizes here the FP32 tensor-core
// accumulation is exact without flushing, and the epilogue rounds the
// combined orders once: the output carries an unbiased round-to-nearest
// error instead of the one-signed drift of truncating FP32 accumulation.
//
// Warp roles (480 threads):
//   warps 0-3  epilogue: tcgen05.ld of a finished accumulator set -> Y (FP32),
//              overlapped with the next tile's MMAs (two TMEM buffers);
//   warps 4-11 converters: slicing into K-major 128-byte-swizzled stages.
//              FP32 data whose unfolding tiles are boxes of a tensor map
//              (R = 1, R a multiple of 128, or R a power of two below 128)
//              arrive as raw tiles in a ring of shared-memory buffers filled
//              by warp 14 with TMA tensor copies -- the mode-k unfolding is
//              the box geometry, no transpose is written anywhere -- and the
//              converters slice from shared memory; other data is loaded
//              with coalesced global loads (the unfolding is index
//              arithmetic).  With several output chunks the operand is sliced
//              once beforehand (ttm_preslice_a) and one thread of warp 4
//              bulk-copies each stage's image instead, the chunks of one M
//              tile running side by side so that the image is read from L2;
//   warp 12    MMA issuer (one elected thread), 9 MMAs per K step;
//   warp 13    B producer: bulk-async copies (cp.async.bulk, TMA engine) of the
//              pre-sliced, pre-swizzled factor tiles, completing on the
//              stage's mbarrier;
//   warp 14    raw-tile producer (TMA tensor copies, see above).
// TMEM: buffer b at column 256 b, order o at +32 o.
// All waits are bounded (2 s); on time-out the CTA raises an error flag,
// waits for its own MMAs, frees TMEM and returns.
#include <stdint.h>
#include <stdlib.h>

#include <algorithm>

#include "atc_internal.cuh"
#include "tc_common.cuh"

namespace atc {
namespace {
using namespace tc;

constexpr int kEpiWarps = 4;
constexpr int kConvWarps = 8;
constexpr int kConvThreads = kConvWarps * 32;
constexpr int kMmaWarp = kEpiWarps + kConvWarps;  // 12
constexpr int kProdWarp = kMmaWarp + 1;           // 13
constexpr int kRawWarp = kProdWarp + 1;           // 14
constexpr int kThreads = (kRawWarp + 1) * 32;     // 480
constexpr int kMaxRaw = 3;                        // raw-tile ring depth
constexpr uint32_t kRawBytes = 128 * 64 * 4;      // one raw FP32 tile: 128 columns x 64 K
constexpr int KT = 64;
constexpr int UNITS = 128 * 8 / kConvThreads;     // 4
constexpr int kMaxN = 32;                         // output indices per launch
constexpr uint32_t kOrdStride = 32;               // TMEM columns per order (allocation granule)

enum { TM_ROW = 0, TM_ROWVEC = 1, TM_GEN = 2 };

struct TtmArgs {
  const void* x;
  int64_t L, Bdim, R;    // input view (L, Bdim, R); K = Bdim
  int apad;              // output indices per chunk padded to 16 (N of the MMA, <= kMaxN)
  int64_t Atot;          // output mode size
  int nkt;               // K tiles
  int64_t mtiles;        // ceil(L*R / 128)
  const uint8_t* bw;     // [3 slices][nkt][apad][128 B] pre-swizzled
  void* y;               // (L, Atot, R)
  const SliceScale* xs;  // slice scale of x
  const signed char* cshift;  // per-column (gamma) scale exponents, or nullptr: xs for every column
  int* err;
  int nstage;            // pipeline depth (<= 4)
  int rowmode;           // TM_ROW / TM_ROWVEC when R == 1
  int64_t csz;           // output indices per chunk
  size_t wb;             // bytes of one chunk's factor slices
  unsigned nchunk_launch;
  // products with several output chunks: the data operand already sliced into
  // the converters' shared-memory image, one 3 x 16 KB block per (M tile,
  // K tile) (ttm_preslice_a); nullptr: the converter warps slice it
  const uint8_t* aimg;
  // raw FP32 tiles by TMA (the kernel's tensor map): box {rb, 64, 128 / rb}
  // over (R, K, L) when R > 1 (rb = min(R, 128), a power of two), {64, 128}
  // over (K, L) when R == 1
  int tma;
  int rb_log2;
  int nraw;
  // one output chunk whose factor slices fit: they are copied into shared
  // memory once per CTA (after the stages and the raw ring) instead of once
  // per K step, so no MMA waits on an L2 round trip for its B tile
  int bres;
  // work items: chunk_fast -> item w = (M tile w / nchunk, chunk w % nchunk),
  // so that the chunks of one M tile run side by side, CTA blockIdx.x taking
  // items blockIdx.x + t gridDim.x; else item = M tile, chunk = blockIdx.y
  int chunk_fast;
};

template <typename T>
__device__ __forceinline__ void ld8(const T* p, float (&v)[8]);
template <>
__device__ __forceinline__ void ld8<float>(const float* p, float (&v)[8]) {
  const float4 a = __ldg(reinterpret_cast<const float4*>(p));
  const float4 b = __ldg(reinterpret_cast<const float4*>(p) + 1);
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
  v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}
template <>
__device__ __forceinline__ void ld8<double>(const double* p, float (&v)[8]) {
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const double2 a = __ldg(reinterpret_cast<const double2*>(p) + i);
    v[2 * i] = (float)a.x;
    v[2 * i + 1] = (float)a.y;
  }
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"((uint64_t)src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

template <typename TX, bool BF16, bool GEN>
__global__ void __launch_bounds__(kThreads, 1)
    ttm_tc_kernel(TtmArgs a, const __grid_constant__ CUtensorMap xmap) {
  typedef float TY;
  constexpr int MAXST = 4;
  const int NSTAGE = a.nstage;
  const int NRAW = a.nraw;
  const int MODE = GEN ? TM_GEN : a.rowmode;
  constexpr uint32_t A_BYTES = 128 * 128;  // 128 rows x 64 16-bit
  extern __shared__ uint8_t smem_raw[];
  __shared__ uint64_t full_bar[MAXST], bfull_bar[MAXST], empty_bar[MAXST], accf_bar[2], acce_bar[2], done_bar;
  __shared__ uint64_t raw_full[kMaxRaw], raw_empty[kMaxRaw], bres_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  volatile int* abort = &abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // this CTA's work items t = 0 .. nmine-1: (M tile, output chunk) -- all
  // chunks share the padded width apad
  const bool cf = a.chunk_fast != 0;
  const int64_t nch = cf ? (int64_t)a.nchunk_launch : 1;
  const int64_t nwork = a.mtiles * nch;
  const int64_t wb0 = blockIdx.x, wst = gridDim.x;
  auto tile_mt = [&](int64_t t) -> int64_t {
    const int64_t w = wb0 + t * wst;
    return cf ? w / nch : w;
  };
  auto tile_ch = [&](int64_t t) -> int64_t {
    const int64_t w = wb0 + t * wst;
    return cf ? w - (w / nch) * nch : (int64_t)blockIdx.y;
  };
  const uint32_t B_BYTES = (uint32_t)a.apad * 128u;
  const uint32_t STAGE = 3 * A_BYTES + (a.bres ? 0u : ((3 * B_BYTES + 1023u) & ~1023u));
  uint8_t* rawbuf = smem + (size_t)NSTAGE * STAGE;  // raw-tile ring (TMA path)
  uint8_t* bresbuf = rawbuf + (size_t)NRAW * kRawBytes;  // resident factor slices [slice][kt][apad][128 B]
  const int64_t nmine = (nwork > wb0) ? (nwork - 1 - wb0) / wst + 1 : 0;
  const int64_t iters = nmine * a.nkt;
  const int64_t LR = a.L * a.R;
  const int shift = a.xs->shift;

  if (tid == 0) {
    for (int s = 0; s < NSTAGE; ++s) {
      mbar_init(&full_bar[s], a.aimg ? 1 : kConvThreads);
      mbar_init(&bfull_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    for (int s = 0; s < NRAW; ++s) {
      mbar_init(&raw_full[s], 1);
      mbar_init(&raw_empty[s], kConvThreads);
    }
    mbar_init(&bres_bar, 1);
    mbar_init(&done_bar, 1);
    for (int b = 0; b < 2; ++b) {
      mbar_init(&accf_bar[b], 1);
      mbar_init(&acce_bar[b], kEpiWarps * 32);
    }
    abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == kMmaWarp) tmem_alloc(&tmem_slot, 512);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;

  if (warp >= kEpiWarps && warp < kMmaWarp && a.aimg) {
    // --------------------------------------- pre-sliced data operand (bulk copies)
    if (tid == kEpiWarps * 32) {
      int64_t issued = 0;
      for (int64_t it = 0; it < iters; ++it) {
        const int s = (int)(it % NSTAGE);
        const int64_t mt = tile_mt(it / a.nkt);
        const int kt = (int)(it % a.nkt);
        if (!mbar_wait(&empty_bar[s], ((uint32_t)(it / NSTAGE) & 1u) ^ 1u, abort)) break;
        mbar_arrive_expect_tx(&full_bar[s], 3 * A_BYTES);
        bulk_g2s(smem + (size_t)s * STAGE, a.aimg + ((size_t)mt * a.nkt + kt) * 3 * A_BYTES, 3 * A_BYTES, &full_bar[s]);
        issued = it + 1;
      }
      // drain: every issued copy must land before the CTA may exit
      const int64_t first = issued > NSTAGE ? issued - NSTAGE : 0;
      for (int64_t it = first; it < issued; ++it)
        mbar_wait_drain(&full_bar[it % NSTAGE], (uint32_t)(it / NSTAGE) & 1u);
    }
  } else if (warp >= kEpiWarps && warp < kMmaWarp && a.tma) {
    // ------------------------------ converters on raw tiles from the TMA ring
    const int ct = tid - kEpiWarps * 32;
    const float sc = ldexpf(1.0f, shift);
    const int rbl = a.rb_log2;
    const uint32_t rbm = (1u << rbl) - 1u;
    for (int64_t it = 0; it < iters; ++it) {
      const int rs = (int)(it % NRAW);
      if (!mbar_wait(&raw_full[rs], (uint32_t)(it / NRAW) & 1u, abort)) break;
      const int s = (int)(it % NSTAGE);
      if (!mbar_wait(&empty_bar[s], ((uint32_t)(it / NSTAGE) & 1u) ^ 1u, abort)) break;
      const float* raw = reinterpret_cast<const float*>(rawbuf + (size_t)rs * kRawBytes);
      uint8_t* a0s = smem + (size_t)s * STAGE;
      const int64_t g0 = tile_mt(it / a.nkt) * 128;
#pragma unroll
      for (int u = 0; u < UNITS; ++u) {
        const int g = ct + kConvThreads * u;
        int m, q;
        float v[8];
        if (MODE == TM_GEN) {
          // raw tile [l][k][c] (c fastest), row m = l * rb + c
          m = g & 127;
          q = g >> 7;
          const uint32_t base = ((((uint32_t)m >> rbl) * 64u + 8u * (uint32_t)q) << rbl) + ((uint32_t)m & rbm);
#pragma unroll
          for (int e = 0; e < 8; ++e) v[e] = raw[base + ((uint32_t)e << rbl)];
        } else {
          // raw tile [m][k]
          m = g >> 3;
          q = g & 7;
          const float4* r4 = reinterpret_cast<const float4*>(raw + m * 64 + 8 * q);
          const float4 x0 = r4[0], x1 = r4[1];
          v[0] = x0.x; v[1] = x0.y; v[2] = x0.z; v[3] = x0.w;
          v[4] = x1.x; v[5] = x1.y; v[6] = x1.z; v[7] = x1.w;
        }
        float scu = sc;
        if (a.cshift) {
          const int64_t gam = g0 + m;
          scu = (gam < LR) ? ldexpf(1.0f, (int)__ldg(a.cshift + gam)) : 0.f;
        }
        uint32_t p0[4], p1[4], p2[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          float a0x, a1x, a2x, a0y, a1y, a2y;
          slice3i(v[2 * e] * scu, a0x, a1x, a2x);
          slice3i(v[2 * e + 1] * scu, a0y, a1y, a2y);
          p0[e] = Pack<BF16>::two(a0x, a0y);
          p1[e] = Pack<BF16>::two(a1x, a1y);
          p2[e] = Pack<BF16>::two(a2x, a2y);
        }
        const uint32_t off = sw128_off((uint32_t)m, (uint32_t)(8 * q));
        *reinterpret_cast<uint4*>(a0s + off) = make_uint4(p0[0], p0[1], p0[2], p0[3]);
        *reinterpret_cast<uint4*>(a0s + A_BYTES + off) = make_uint4(p1[0], p1[1], p1[2], p1[3]);
        *reinterpret_cast<uint4*>(a0s + 2 * A_BYTES + off) = make_uint4(p2[0], p2[1], p2[2], p2[3]);
      }
      mbar_arrive(&raw_empty[rs]);  // the raw tile is consumed
      fence_proxy_async_smem();
      mbar_arrive(&full_bar[s]);
    }
  } else if (warp >= kEpiWarps && warp < kMmaWarp) {
    // ------------------------------------------------------------ converters
    const int ct = tid - kEpiWarps * 32;
    const float sc = ldexpf(1.0f, shift);
    const TX* __restrict__ x = reinterpret_cast<const TX*>(a.x);
    float bufA[UNITS][8], bufB[UNITS][8];
    auto load = [&](float (&buf)[UNITS][8], int64_t it) {
      const int64_t mt = tile_mt(it / a.nkt);
      const int kt = (int)(it % a.nkt);
      const int64_t g0 = mt * 128;
#pragma unroll
      for (int u = 0; u < UNITS; ++u) {
        const int g = ct + kConvThreads * u;
        if (MODE == TM_GEN) {
          const int m = g & 127, q = g >> 7;
          const int64_t gam = g0 + m;
          const int64_t l = gam / a.R, c = gam - l * a.R;
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const int64_t i = (int64_t)kt * KT + 8 * q + e;
            buf[u][e] = (gam < LR && i < a.Bdim) ? (float)__ldg(x + (l * a.Bdim + i) * a.R + c) : 0.f;
          }
        } else {
          const int m = g >> 3, q = g & 7;
          const int64_t gam = g0 + m;
          const int64_t i0 = (int64_t)kt * KT + 8 * q;
          if (MODE == TM_ROWVEC) {
            if (gam < LR && i0 < a.Bdim) {
              ld8<TX>(x + gam * a.Bdim + i0, buf[u]);
            } else {
#pragma unroll
              for (int e = 0; e < 8; ++e) buf[u][e] = 0.f;
            }
          } else {
#pragma unroll
            for (int e = 0; e < 8; ++e)
              buf[u][e] = (gam < LR && i0 + e < a.Bdim) ? (float)__ldg(x + gam * a.Bdim + i0 + e) : 0.f;
          }
        }
      }
    };
    auto store = [&](float (&buf)[UNITS][8], int64_t it) -> bool {
      const int s = (int)(it % NSTAGE);
      const uint32_t ph = ((uint32_t)(it / NSTAGE) & 1u) ^ 1u;
      if (!mbar_wait(&empty_bar[s], ph, abort)) return false;
      uint8_t* a0s = smem + (size_t)s * STAGE;
#pragma unroll
      for (int u = 0; u < UNITS; ++u) {
        const int g = ct + kConvThreads * u;
        int m, q;
        if (MODE == TM_GEN) { m = g & 127; q = g >> 7; } else { m = g >> 3; q = g & 7; }
        float scu = sc;
        if (a.cshift) {
          const int64_t gam = tile_mt(it / a.nkt) * 128 + m;
          scu = (gam < LR) ? ldexpf(1.0f, (int)__ldg(a.cshift + gam)) : 0.f;
        }
        uint32_t p0[4], p1[4], p2[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          float a0x, a1x, a2x, a0y, a1y, a2y;
          slice3i(buf[u][2 * e] * scu, a0x, a1x, a2x);
          slice3i(buf[u][2 * e + 1] * scu, a0y, a1y, a2y);
          p0[e] = Pack<BF16>::two(a0x, a0y);
          p1[e] = Pack<BF16>::two(a1x, a1y);
          p2[e] = Pack<BF16>::two(a2x, a2y);
        }
        const uint32_t off = sw128_off((uint32_t)m, (uint32_t)(8 * q));
        *reinterpret_cast<uint4*>(a0s + off) = make_uint4(p0[0], p0[1], p0[2], p0[3]);
        *reinterpret_cast<uint4*>(a0s + A_BYTES + off) = make_uint4(p1[0], p1[1], p1[2], p1[3]);
        *reinterpret_cast<uint4*>(a0s + 2 * A_BYTES + off) = make_uint4(p2[0], p2[1], p2[2], p2[3]);
      }
      fence_proxy_async_smem();
      mbar_arrive(&full_bar[s]);
      return true;
    };
    if (iters > 0) load(bufA, 0);
    for (int64_t it = 0; it < iters; it += 2) {
      if (it + 1 < iters) load(bufB, it + 1);
      if (!store(bufA, it)) break;
      if (it + 1 < iters) {
        if (it + 2 < iters) load(bufA, it + 2);
        if (!store(bufB, it + 1)) break;
      }
    }
  } else if (warp == kProdWarp) {
    // ---------------------------------------------------------- B producer
    if (lane == 0 && a.bres) {
      // every K tile of the three slices at once (each slice is contiguous)
      const uint32_t slice_bytes = (uint32_t)a.nkt * B_BYTES;
      mbar_arrive_expect_tx(&bres_bar, 3 * slice_bytes);
#pragma unroll
      for (int q = 0; q < 3; ++q) bulk_g2s(bresbuf + q * slice_bytes, a.bw + (size_t)q * slice_bytes, slice_bytes, &bres_bar);
      mbar_wait_drain(&bres_bar, 0);
    } else if (lane == 0) {
      const size_t slice_bytes = (size_t)a.nkt * B_BYTES;
      int64_t issued = 0;
      for (int64_t it = 0; it < iters; ++it) {
        const int s = (int)(it % NSTAGE);
        const int kt = (int)(it % a.nkt);
        if (!mbar_wait(&empty_bar[s], ((uint32_t)(it / NSTAGE) & 1u) ^ 1u, abort)) break;
        uint8_t* bb = smem + (size_t)s * STAGE + 3 * A_BYTES;
        const uint8_t* bwc = a.bw + (size_t)tile_ch(it / a.nkt) * a.wb;
        mbar_arrive_expect_tx(&bfull_bar[s], 3 * B_BYTES);
#pragma unroll
        for (int q = 0; q < 3; ++q)
          bulk_g2s(bb + q * B_BYTES, bwc + q * slice_bytes + (size_t)kt * B_BYTES, B_BYTES, &bfull_bar[s]);
        issued = it + 1;
      }
      // drain: every issued copy must land before the CTA may exit
      const int64_t first = issued > NSTAGE ? issued - NSTAGE : 0;
      for (int64_t it = first; it < issued; ++it)
        mbar_wait_drain(&bfull_bar[it % NSTAGE], (uint32_t)(it / NSTAGE) & 1u);
    }
  } else if (warp == kRawWarp) {
    // ---------------------------------------------- raw-tile producer (TMA)
    if (lane == 0 && a.tma && !a.aimg) {
      int64_t issued = 0;
      for (int64_t it = 0; it < iters; ++it) {
        const int rs = (int)(it % NRAW);
        if (!mbar_wait(&raw_empty[rs], ((uint32_t)(it / NRAW) & 1u) ^ 1u, abort)) break;
        const int64_t g0 = tile_mt(it / a.nkt) * 128;
        const int kt = (int)(it % a.nkt);
        mbar_arrive_expect_tx(&raw_full[rs], kRawBytes);
        void* dst = rawbuf + (size_t)rs * kRawBytes;
        if (GEN) {
          const int64_t l = g0 / a.R, c0 = g0 - l * a.R;
          tma_load_3d(dst, &xmap, &raw_full[rs], (int)c0, kt * KT, (int)l);
        } else {
          tma_load_2d(dst, &xmap, &raw_full[rs], kt * KT, (int)g0);
        }
        issued = it + 1;
      }
      // drain: every issued copy must land before the CTA may exit
      const int64_t first = issued > NRAW ? issued - NRAW : 0;
      for (int64_t it = first; it < issued; ++it)
        mbar_wait_drain(&raw_full[it % NRAW], (uint32_t)(it / NRAW) & 1u);
    }
  } else if (warp == kMmaWarp) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      const uint32_t idesc = idesc_f16(BF16 ? 1 : 0, 128, a.apad);
      int64_t it = 0;
      bool ok = true;
      if (a.bres && nmine > 0) ok = mbar_wait(&bres_bar, 0u, abort);
      const uint32_t bslice = a.bres ? (uint32_t)a.nkt * B_BYTES : B_BYTES;  // distance between slices
      for (int64_t t = 0; t < nmine && ok; ++t) {
        const int ab = (int)(t & 1);
        if (!mbar_wait(&acce_bar[ab], ((uint32_t)(t >> 1) & 1u) ^ 1u, abort)) break;
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)ab * 256u;
        for (int kt = 0; kt < a.nkt; ++kt, ++it) {
          const int s = (int)(it % NSTAGE);
          if (!mbar_wait(&full_bar[s], (uint32_t)(it / NSTAGE) & 1u, abort) ||
              (!a.bres && !mbar_wait(&bfull_bar[s], (uint32_t)(it / NSTAGE) & 1u, abort))) { ok = false; break; }
          tc_fence_after();
          const uint32_t xa = smem_u32(smem + (size_t)s * STAGE);
          const uint32_t wa = a.bres ? smem_u32(bresbuf) + (uint32_t)kt * B_BYTES : xa + 3 * A_BYTES;
#pragma unroll
          for (int j = 0; j < KT / 16; ++j) {
            const uint32_t o = 32u * j;
            const uint64_t X0 = desc_k128(xa + o), X1 = desc_k128(xa + A_BYTES + o), X2 = desc_k128(xa + 2 * A_BYTES + o);
            const uint64_t W0 = desc_k128(wa + o), W1 = desc_k128(wa + bslice + o), W2 = desc_k128(wa + 2 * bslice + o);
            const uint32_t acc = (kt | j) ? 1u : 0u;
            umma_f16(d, X0, W0, idesc, acc);
            umma_f16(d + kOrdStride, X0, W1, idesc, acc);
            umma_f16(d + kOrdStride, X1, W0, idesc, 1u);
            umma_f16(d + 2 * kOrdStride, X0, W2, idesc, acc);
            umma_f16(d + 2 * kOrdStride, X1, W1, idesc, 1u);
            umma_f16(d + 2 * kOrdStride, X2, W0, idesc, 1u);
            umma_f16(d + 3 * kOrdStride, X1, W2, idesc, acc);
            umma_f16(d + 3 * kOrdStride, X2, W1, idesc, 1u);
            umma_f16(d + 4 * kOrdStride, X2, W2, idesc, acc);
          }
          umma_commit(&empty_bar[s]);
        }
        if (ok) umma_commit(&accf_bar[ab]);
      }
      umma_commit(&done_bar);
      mbar_wait_drain(&done_bar, 0);  // every issued MMA has completed
    }
  } else {
    // ------------------------------------------------------------- epilogue
    // y = (sum_o 2^-8o acc_o) 2^-(shift + 8): one rounding, then exact power-of-two scaling
    const int e_glob = -(shift + 8);
    TY* __restrict__ y = reinterpret_cast<TY*>(a.y);
    for (int64_t t = 0; t < nmine; ++t) {
      const int ab = (int)(t & 1);
      // warp-uniform wait: the tcgen05.ld below is .sync.aligned
      int okw = 1;
      if (lane == 0) okw = mbar_wait(&accf_bar[ab], (uint32_t)(t >> 1) & 1u, abort) ? 1 : 0;
      okw = __shfl_sync(0xffffffffu, okw, 0);
      __syncwarp();
      if (!okw) break;
      tc_fence_after();
      const int64_t mt = tile_mt(t);
      const int64_t j0 = tile_ch(t) * a.csz;
      const int Ach = (int)min(a.csz, a.Atot - j0);
      const int64_t gam = mt * 128 + 32 * warp + lane;
      const bool valid = gam < LR;
      const int64_t l = valid ? gam / a.R : 0, c = valid ? gam - l * a.R : 0;
      const int e_out = (a.cshift && valid) ? -((int)__ldg(a.cshift + gam) + 8) : e_glob;
      const float f1 = ldexpf(1.0f, e_out / 2), f2 = ldexpf(1.0f, e_out - e_out / 2);
      TY* yo = y + (l * a.Atot + j0) * a.R + c;
      const uint32_t tb = tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)ab * 256u;
#pragma unroll 1
      for (int c0 = 0; c0 < a.apad; c0 += 8) {
        uint32_t r0[8], r1[8], r2[8], r3[8], r4[8];
        tmem_ld8(tb + (uint32_t)c0, r0);
        tmem_ld8(tb + kOrdStride + (uint32_t)c0, r1);
        tmem_ld8(tb + 2 * kOrdStride + (uint32_t)c0, r2);
        tmem_ld8(tb + 3 * kOrdStride + (uint32_t)c0, r3);
        tmem_ld8(tb + 4 * kOrdStride + (uint32_t)c0, r4);
        tmem_ld_wait();
        if (valid) {
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const int j = c0 + e;
            if (j < Ach) {
              float sv, tv;
              combine_orders(__uint_as_float(r0[e]), __uint_as_float(r1[e]), __uint_as_float(r2[e]),
                             __uint_as_float(r3[e]), __uint_as_float(r4[e]), sv, tv);
              yo[(int64_t)j * a.R] = (TY)(((sv + tv) * f1) * f2);
            }
          }
        }
      }
      tc_fence_before();
      mbar_arrive(&acce_bar[ab]);
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == kMmaWarp) tmem_dealloc(tmem, 512);
  if (tid == 0 && abort_flag) atomicExch(a.err, 1);
}

}  // namespace
}  // namespace atc

namespace atc {
namespace {

// Per-column scale exponents of the (L, K, R) input: column gamma = (l, c)
// gets shift_gamma = 8 - E with max_i |x[l][i][c]| < 2^E, so that its values
// times 2^shift_gamma stay below 2^8 (the slice range).  The sum of every MMA
// row runs over i inside one column, so the column's power of two factors out
// exactly; the epilogue removes it.  A zero column gets 0.
__device__ __forceinline__ signed char col_shift_of(float m) {
  if (!(m > 0.f)) return 0;
  int E = 0;
  frexpf(m, &E);  // m = f 2^E, f in [0.5, 1)
  int sh = 8 - E;
  sh = sh < -120 ? -120 : (sh > 120 ? 120 : sh);
  return (signed char)sh;
}
template <typename TX>
__global__ void col_shift_rows_kernel(const TX* __restrict__ x, int64_t L, int64_t K, signed char* __restrict__ cs) {
  // R == 1: a warp per row l (contiguous)
  const int lane = threadIdx.x & 31;
  for (int64_t l = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; l < L;
       l += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    float m = 0.f;
    for (int64_t i = lane; i < K; i += 32) m = fmaxf(m, fabsf((float)__ldg(x + l * K + i)));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) cs[l] = col_shift_of(m);
  }
}
template <typename TX>
__global__ void col_shift_cols_kernel(const TX* __restrict__ x, int64_t L, int64_t K, int64_t R,
                                      signed char* __restrict__ cs) {
  // R > 1: a thread per column, consecutive threads on consecutive c (coalesced)
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < L * R; g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t l = g / R, c = g - l * R;
    const TX* p = x + l * K * R + c;
    float m = 0.f;
    for (int64_t i = 0; i < K; ++i) m = fmaxf(m, fabsf((float)__ldg(p + i * R)));
    cs[g] = col_shift_of(m);
  }
}

// W tiles for the MMA B operand: W[a][b] = U[b][j0 + a] (projection) or
// U[j0 + a][b] (expansion), cut into the three fixed-point slices on the
// scale 2^8 (|U| <= 1) and laid out per K tile exactly as the
// 128-byte-swizzled K-major shared-memory image: [slice][kt][apad][64].
template <bool BF16>
__global__ void ttm_prep_b(const double* __restrict__ u, int64_t csz, int64_t Atot, int nchunk, int Bdim, int expand,
                           int apad, int nkt, uint8_t* __restrict__ bw, size_t wb) {
  // W tiles of every chunk: W_ch[a][b] = U[b][j0 + a] (projection) or U[j0 + a][b]
  // (expansion), j0 = ch * csz, cut into three integer slices on the scale
  // 2^8 (|U| <= 1), laid out per K tile exactly as the 128-byte-swizzled
  // K-major shared-memory image: [chunk][slice][kt][apad][64].
  const int64_t per = (int64_t)nkt * apad * 64;
  const int64_t total = per * nchunk;
  const size_t slice_bytes = (size_t)nkt * apad * 128;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
    const int ch = (int)(idx / per);
    const int64_t e = idx - (int64_t)ch * per;
    const int il = (int)(e & 63);
    const int64_t rest = e >> 6;
    const int j = (int)(rest % apad);
    const int kt = (int)(rest / apad);
    const int b = kt * 64 + il;
    const int64_t j0 = (int64_t)ch * csz;
    const int64_t A = min(csz, Atot - j0);
    double w = 0.0;
    if (j < A && b < Bdim) w = expand ? u[(j0 + j) * (int64_t)Bdim + b] : u[(int64_t)b * Atot + j0 + j];
    // integer slices of v = 256 w in FP64 (exact steps, one final rounding)
    const double v = w * 256.0;
    const double a0 = rint(v);
    const double t = (v - a0) * 256.0;
    const double a1 = rint(t);
    const double a2 = rint((t - a1) * 256.0);
    uint8_t* base = bw + (size_t)ch * wb;
    const size_t off = (size_t)kt * apad * 128 + tc::sw128_off((uint32_t)j, (uint32_t)il);
    *reinterpret_cast<uint16_t*>(base + off) = tc::Pack<BF16>::one((float)a0);
    *reinterpret_cast<uint16_t*>(base + slice_bytes + off) = tc::Pack<BF16>::one((float)a1);
    *reinterpret_cast<uint16_t*>(base + 2 * slice_bytes + off) = tc::Pack<BF16>::one((float)a2);
  }
}

// The data operand of a product with several output chunks sliced once into
// the converter warps' shared-memory image: per (M tile, K tile), three
// 128 x 64 16-bit slices in the 128-byte-swizzled K-major layout,
// [m tile][k tile][slice][16 KB].  The output chunks then copy it with the
// bulk engine instead of each re-slicing it.  Same loads, scales and slicing
// as the converter warps, one thread per (m tile, k tile, row, group of 8 K
// values).
template <typename TX, bool GEN, bool BF16>
__global__ void ttm_preslice_a(TtmArgs a, uint8_t* __restrict__ img) {
  constexpr uint32_t A_BYTES = 128 * 128;
  const int MODE = GEN ? TM_GEN : a.rowmode;
  const float sc = ldexpf(1.0f, a.xs->shift);
  const TX* __restrict__ x = reinterpret_cast<const TX*>(a.x);
  const int64_t LR = a.L * a.R;
  const int64_t total = a.mtiles * a.nkt * 1024;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t tile = idx >> 10;  // mt * nkt + kt
    const int64_t mt = tile / a.nkt;
    const int64_t k0 = (tile - mt * a.nkt) * KT;
    const int g = (int)(idx & 1023);
    int m, q;
    if (MODE == TM_GEN) { m = g & 127; q = g >> 7; } else { m = g >> 3; q = g & 7; }
    const int64_t gam = mt * 128 + m;
    float buf[8];
    if (MODE == TM_GEN) {
      const int64_t l = gam / a.R, c = gam - l * a.R;
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int64_t i = k0 + 8 * q + e;
        buf[e] = (gam < LR && i < a.Bdim) ? (float)__ldg(x + (l * a.Bdim + i) * a.R + c) : 0.f;
      }
    } else if (MODE == TM_ROWVEC && gam < LR && k0 + 8 * q < a.Bdim) {
      ld8<TX>(x + gam * a.Bdim + k0 + 8 * q, buf);
    } else {
#pragma unroll
      for (int e = 0; e < 8; ++e)
        buf[e] = (gam < LR && k0 + 8 * q + e < a.Bdim) ? (float)__ldg(x + gam * a.Bdim + k0 + 8 * q + e) : 0.f;
    }
    float scu = sc;
    if (a.cshift) scu = (gam < LR) ? ldexpf(1.0f, (int)__ldg(a.cshift + gam)) : 0.f;
    uint32_t p0[4], p1[4], p2[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      float a0x, a1x, a2x, a0y, a1y, a2y;
      slice3i(buf[2 * e] * scu, a0x, a1x, a2x);
      slice3i(buf[2 * e + 1] * scu, a0y, a1y, a2y);
      p0[e] = Pack<BF16>::two(a0x, a0y);
      p1[e] = Pack<BF16>::two(a1x, a1y);
      p2[e] = Pack<BF16>::two(a2x, a2y);
    }
    uint8_t* base = img + (size_t)tile * 3 * A_BYTES + sw128_off((uint32_t)m, (uint32_t)(8 * q));
    *reinterpret_cast<uint4*>(base) = make_uint4(p0[0], p0[1], p0[2], p0[3]);
    *reinterpret_cast<uint4*>(base + A_BYTES) = make_uint4(p1[0], p1[1], p1[2], p1[3]);
    *reinterpret_cast<uint4*>(base + 2 * A_BYTES) = make_uint4(p2[0], p2[1], p2[2], p2[3]);
  }
}

template <typename TX, bool BF16, bool GEN>
int ttm_launch_t(const TtmArgs& a, const CUtensorMap& map, dim3 grid, int smem, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    ATC_CUDA_TRY(cudaFuncSetAttribute(ttm_tc_kernel<TX, BF16, GEN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      225 * 1024));
    attr = true;
  }
  // algorithmic work: the data tensor read once, the output written once, the
  // factor read once; 2 Atot Bdim per output column; issued: nine slice
  // products over the padded tiles
  const double cols = (double)a.L * (double)a.R;
  const double bytes = cols * (double)a.Bdim * sizeof(TX) + cols * (double)a.Atot * 4.0 +
                       (double)a.Atot * (double)a.Bdim * 8.0;
  const double flops = 2.0 * cols * (double)a.Atot * (double)a.Bdim;
  const double issued = 9.0 * 2.0 * (double)a.mtiles * 128.0 * (double)a.apad * (double)a.nchunk_launch *
                        (double)a.nkt * KT;
  KTimed kt_(s, "ttm_tc_kernel", bytes, flops, issued);
  ttm_tc_kernel<TX, BF16, GEN><<<grid, kThreads, smem, s>>>(a, map);
  ATC_LAUNCHED(1);
  return ATC_OK;
}

template <typename TX, bool BF16>
int ttm_launch_g(const TtmArgs& a, const CUtensorMap& map, bool gen, dim3 grid, int smem, cudaStream_t s) {
  return gen ? ttm_launch_t<TX, BF16, true>(a, map, grid, smem, s) : ttm_launch_t<TX, BF16, false>(a, map, grid, smem, s);
}

int g_nsm_ttm = 0;
// per-column scales replace the tensor's slice scale: a zero scale stands in
__device__ SliceScale g_unit_scale;
// largest pre-sliced data image (6 bytes per element of the data operand)
constexpr size_t kMaxImageBytes = (size_t)16 << 30;
// largest factor slice image kept resident in shared memory
constexpr size_t kMaxResidentB = (size_t)48 << 10;

}  // namespace

int tc_error_flag(int** flag);

namespace {

// Driver of the projection / expansion.  percol: per-column scale exponents for the data operand (expansions, whose
// inputs -- cores and partly expanded cores -- span many orders of magnitude
// across columns); otherwise one power of two for the whole tensor.
int ttm_run(const void* x, int xdtype, int64_t L, int64_t n, int64_t R, const double* u, int64_t r, int expand,
            int precision, void* y, cudaStream_t s, const SliceScale* xs, bool percol) {
  const int64_t Atot = expand ? n : r;
  const int64_t Bdim = expand ? r : n;
  if (Bdim > 1024) return fail(ATC_EUNSUP, "split-precision TTM supports contraction length <= 1024 (got %lld)",
                               (long long)Bdim);
  if (g_nsm_ttm == 0) {
    int dev = 0;
    ATC_CUDA_TRY(cudaGetDevice(&dev));
    ATC_CUDA_TRY(cudaDeviceGetAttribute(&g_nsm_ttm, cudaDevAttrMultiProcessorCount, dev));
  }
  const bool bf16 = (precision == ATC_PREC_SPLIT_BF16);
  if (!xs && percol) {
    // every column carries its own power of two (cshift): the tensor-wide
    // scale is never read, so no pass over the data computes it
    void* p = nullptr;
    ATC_CUDA_TRY(cudaGetSymbolAddress(&p, g_unit_scale));
    xs = reinterpret_cast<const SliceScale*>(p);
  }
  if (!xs) ATC_TRY(slice_scale(x, xdtype, L * Bdim * R, s, &xs));
  int* err = nullptr;
  ATC_TRY(tc_error_flag(&err));
  const int nkt = (int)((Bdim + KT - 1) / KT);
  const int64_t mtiles = (L * R + 127) / 128;
  // the output indices in chunks of at most kMaxN (two TMEM buffers of five orders)
  const int nchunk = (int)((Atot + kMaxN - 1) / kMaxN);
  const int64_t csz = (Atot + nchunk - 1) / nchunk;
  const int apad_max = (int)((csz + 15) / 16 * 16);
  const size_t wb = (size_t)3 * nkt * apad_max * 128;
  // work items (M tile, chunk), chunks of one M tile side by side; one
  // persistent CTA per SM at most
  const int64_t nwork = mtiles * nchunk;
  const int grid = (int)(nwork < g_nsm_ttm ? nwork : g_nsm_ttm);
  uint8_t* bw = nullptr;
  ATC_TRY(Scratch::get(SLOT_TTM_U, wb * nchunk + 256, (void**)&bw));
  signed char* cshift = nullptr;
  if (percol && L * R > 0) {
    ATC_TRY(Scratch::get(SLOT_COLSHIFT, (size_t)(L * R) + 256, (void**)&cshift));
    const int blocks = 4 * g_nsm_ttm;
    if (R == 1) {
      if (xdtype == ATC_F32) col_shift_rows_kernel<float><<<blocks, 256, 0, s>>>((const float*)x, L, Bdim, cshift);
      else col_shift_rows_kernel<double><<<blocks, 256, 0, s>>>((const double*)x, L, Bdim, cshift);
    } else {
      if (xdtype == ATC_F32) col_shift_cols_kernel<float><<<blocks, 256, 0, s>>>((const float*)x, L, Bdim, R, cshift);
      else col_shift_cols_kernel<double><<<blocks, 256, 0, s>>>((const double*)x, L, Bdim, R, cshift);
    }
    ATC_LAUNCHED(1);
  }
  {
    TtmArgs a;
    a.x = x;
    a.L = L;
    a.Bdim = Bdim;
    a.R = R;
    a.apad = apad_max;
    a.Atot = Atot;
    a.nkt = nkt;
    a.mtiles = mtiles;
    a.y = y;
    a.xs = xs;
    a.cshift = cshift;
    a.err = err;
    a.rowmode = (Bdim % 8 == 0) ? TM_ROWVEC : TM_ROW;
    a.csz = csz;
    a.wb = wb;
    a.nchunk_launch = (unsigned)nchunk;
    a.bw = bw;
    a.aimg = nullptr;
    a.tma = 0;
    a.rb_log2 = 0;
    a.nraw = 0;
    a.chunk_fast = nchunk > 1 ? 1 : 0;
    const uint32_t bbytes = (uint32_t)a.apad * 128u;
    const size_t bres_bytes = (size_t)3 * nkt * bbytes;
    a.bres = (nchunk == 1 && bres_bytes <= kMaxResidentB) ? 1 : 0;
    const uint32_t stage = 3u * 128u * 128u + (a.bres ? 0u : ((3u * bbytes + 1023u) & ~1023u));
    const size_t bres_smem = a.bres ? ((bres_bytes + 1023) & ~(size_t)1023) : 0;
    // the data operand: pre-sliced image (several chunks), raw FP32 tiles by
    // TMA (tensor-map geometry), or the converters' global loads
    const size_t img_bytes = (size_t)mtiles * nkt * 3 * 128 * 128;
    const bool use_img = mtiles > 0 && nchunk > 1 && img_bytes <= kMaxImageBytes;
    CUtensorMap map;
    memset(&map, 0, sizeof(map));
    if (!use_img && mtiles > 0 && xdtype == ATC_F32 && ((uintptr_t)x & 15u) == 0) {
      bool ok = false;
      int rbl = 0;
      if (R == 1) {
        if (Bdim % 4 == 0) {
          const int64_t dims[2] = {Bdim, L}, strides[1] = {Bdim * 4};
          const uint32_t box[2] = {(uint32_t)KT, 128u};
          ok = make_raw_map_f32(&map, x, 2, dims, strides, box) == ATC_OK;
        }
      } else if (R % 128 == 0 || (R < 128 && R >= 4 && (128 % R) == 0)) {
        const int64_t rb = R < 128 ? R : 128;
        while ((1 << rbl) < rb) ++rbl;
        const int64_t dims[3] = {R, Bdim, L}, strides[2] = {R * 4, R * Bdim * 4};
        const uint32_t box[3] = {(uint32_t)rb, (uint32_t)KT, (uint32_t)(128 / rb)};
        ok = make_raw_map_f32(&map, x, 3, dims, strides, box) == ATC_OK;
      }
      if (!ok) cudaGetLastError();
      for (int nraw = kMaxRaw; ok && nraw >= 2 && !a.tma; --nraw) {
        if ((size_t)224 * 1024 >= (size_t)nraw * kRawBytes + 2 * (size_t)stage + bres_smem) {
          a.tma = 1;
          a.nraw = nraw;
          a.rb_log2 = rbl;
        }
      }
    }
    const size_t raw_bytes = (size_t)a.nraw * kRawBytes;
    a.nstage = (int)(((size_t)224 * 1024 - raw_bytes - bres_smem) / stage);
    if (a.nstage > 4) a.nstage = 4;
    if (a.nstage < 2) return fail(ATC_EUNSUP, "TTM stage does not fit in shared memory");
    const int smem = (int)(a.nstage * stage + raw_bytes + bres_smem + 1024);
    {
      const int64_t tot = (int64_t)nkt * a.apad * 64 * nchunk;
      const int blocks = (int)((tot + 255) / 256 < 4096 ? (tot + 255) / 256 : 4096);
      if (bf16) ttm_prep_b<true><<<blocks, 256, 0, s>>>(u, csz, Atot, nchunk, (int)Bdim, expand, a.apad, nkt, bw, wb);
      else ttm_prep_b<false><<<blocks, 256, 0, s>>>(u, csz, Atot, nchunk, (int)Bdim, expand, a.apad, nkt, bw, wb);
      ATC_LAUNCHED(1);
    }
    // several output chunks: slice the data operand once instead of once per
    // chunk; the chunks of an M tile read its image while it sits in L2
    if (use_img) {
      uint8_t* img = nullptr;
      ATC_TRY(Scratch::get(SLOT_TTM_AIMG, img_bytes, (void**)&img));
      const int64_t tot = mtiles * nkt * 1024;
      const int blocks = (int)((tot + 255) / 256 < 8 * g_nsm_ttm ? (tot + 255) / 256 : 8 * g_nsm_ttm);
      const bool gen = (R != 1), pb = bf16;
      if (xdtype == ATC_F32) {
        if (gen) {
          if (pb) ttm_preslice_a<float, true, true><<<blocks, 256, 0, s>>>(a, img);
          else ttm_preslice_a<float, true, false><<<blocks, 256, 0, s>>>(a, img);
        } else {
          if (pb) ttm_preslice_a<float, false, true><<<blocks, 256, 0, s>>>(a, img);
          else ttm_preslice_a<float, false, false><<<blocks, 256, 0, s>>>(a, img);
        }
      } else {
        if (gen) {
          if (pb) ttm_preslice_a<double, true, true><<<blocks, 256, 0, s>>>(a, img);
          else ttm_preslice_a<double, true, false><<<blocks, 256, 0, s>>>(a, img);
        } else {
          if (pb) ttm_preslice_a<double, false, true><<<blocks, 256, 0, s>>>(a, img);
          else ttm_preslice_a<double, false, false><<<blocks, 256, 0, s>>>(a, img);
        }
      }
      ATC_LAUNCHED(1);
      a.aimg = img;
    }
    if (mtiles > 0) {
      const bool gen = (R != 1);
      const dim3 g3((unsigned)grid, 1u);
      if (xdtype == ATC_F32) {
        if (bf16) ATC_TRY((ttm_launch_g<float, true>(a, map, gen, g3, smem, s)));
        else ATC_TRY((ttm_launch_g<float, false>(a, map, gen, g3, smem, s)));
      } else {
        if (bf16) ATC_TRY((ttm_launch_g<double, true>(a, map, gen, g3, smem, s)));
        else ATC_TRY((ttm_launch_g<double, false>(a, map, gen, g3, smem, s)));
      }
    }
  }
  return ATC_OK;
}

}  // namespace

int launch_ttm_split(const void* x, int xdtype, int64_t L, int64_t n, int64_t R, const double* u, int64_t r,
                     int expand, int precision, void* y, int ydtype, cudaStream_t s, const SliceScale* xs) {
  if (ydtype != ATC_F32) return fail(ATC_EUNSUP, "split-precision TTM writes FP32 output");
  return ttm_run(x, xdtype, L, n, R, u, r, expand, precision, y, s, xs, expand != 0);
}

}  // namespace atc
