// Split-precision mode-k product on the 5th-generation tensor cores.
//
// Projection (Algorithm 1): Y[l][j][c] = sum_i U[i][j] X[l][i][c], i.e. for
// every "column" gamma = (l, c) of the (L, n, R) view, y_gamma = U^T x_gamma.
// As a GEMM: D[gamma][j] = sum_i A[gamma][i] B[j][i] with M = gamma (128 per
// tile, any L and R), N = a chunk of <= 32 output indices j (padded to 16),
// K = n.  The same kernel runs the expansion Y = U ._k X with B[a][b] = U[a][b],
// and, in residual mode, sums (X' - U ._k Y)^2 instead of writing the product.
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
// Warp roles (448 threads):
//   warps 0-3  epilogue: tcgen05.ld of a finished accumulator set -> Y (FP32),
//              overlapped with the next tile's MMAs (two TMEM buffers);
//   warps 4-11 converters: coalesced loads of X (the unfolding is index
//              arithmetic), slicing, K-major 128-byte-swizzled stores to smem;
//              for single-K-tile products with several output chunks the
//              operand is sliced once beforehand (ttm_preslice_a) and one
//              thread of warp 4 bulk-copies each stage's image instead;
//   warp 12    MMA issuer (one elected thread), 9 MMAs per K step;
//   warp 13    B producer: bulk-async copies (cp.async.bulk, TMA engine) of the
//              pre-sliced, pre-swizzled factor tiles, completing on the
//              stage's mbarrier.
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
constexpr int kThreads = (kProdWarp + 1) * 32;    // 448
constexpr int KT = 64;
constexpr int UNITS = 128 * 8 / kConvThreads;     // 4
constexpr int kMaxN = 32;                         // output indices per launch
constexpr uint32_t kOrdStride = 32;               // TMEM columns per order (allocation granule)

enum { TM_ROW = 0, TM_ROWVEC = 1, TM_GEN = 2 };

struct TtmArgs {
  const void* x;
  int64_t L, Bdim, R;    // input view (L, Bdim, R); K = Bdim
  int A;                 // output indices in this chunk (N of the MMA, <= kMaxN)
  int apad;              // A padded to 16
  int64_t Atot, j0;      // output mode size and this chunk's first index
  int nkt;               // K tiles
  int64_t mtiles;        // ceil(L*R / 128)
  const uint8_t* bw;     // [3 slices][nkt][apad][128 B] pre-swizzled
  void* y;               // (L, Atot, R)
  const SliceScale* xs;  // slice scale of x
  const signed char* cshift;  // per-column (gamma) scale exponents, or nullptr: xs for every column
  int* err;
  int nstage;            // pipeline depth (<= 4)
  int rowmode;           // TM_ROW / TM_ROWVEC when R == 1
  // residual mode: instead of writing Y, accumulate sum (xres - Y)^2 over this
  // chunk's outputs, one FP64 partial per CTA in res_part[blockIdx.x]
  const void* xres;      // (L, Atot, R) tensor compared with the product
  double* res_part;
  int64_t csz;           // output indices per chunk (blockIdx.y = chunk)
  size_t wb;             // bytes of one chunk's factor slices
  unsigned nchunk_launch;
  // single-K-tile products with several output chunks: the data operand
  // already sliced into the converters' shared-memory image, one 3 x 16 KB
  // block per M tile (ttm_preslice_a); nullptr: the converter warps slice it
  const uint8_t* aimg;
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

template <typename TX, bool BF16, bool GEN, bool RES, typename TR>
__global__ void __launch_bounds__(kThreads, 1) ttm_tc_kernel(TtmArgs a) {  // a is modified per chunk (by value)
  typedef float TY;
  constexpr int MAXST = 4;
  const int NSTAGE = a.nstage;
  const int MODE = GEN ? TM_GEN : a.rowmode;
  constexpr uint32_t A_BYTES = 128 * 128;  // 128 rows x 64 16-bit
  extern __shared__ uint8_t smem_raw[];
  __shared__ uint64_t full_bar[MAXST], bfull_bar[MAXST], empty_bar[MAXST], accf_bar[2], acce_bar[2], done_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  __shared__ double res_smem[kEpiWarps];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  volatile int* abort = &abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // chunk of output indices of this CTA row (all chunks share the padded width apad)
  {
    const int64_t j0c = (int64_t)blockIdx.y * a.csz;
    a.j0 = j0c;
    a.A = (int)min((int64_t)a.csz, a.Atot - j0c);
    a.bw += (size_t)blockIdx.y * a.wb;
    if (a.res_part) a.res_part += (size_t)blockIdx.y * gridDim.x;
  }
  const uint32_t B_BYTES = (uint32_t)a.apad * 128u;
  const uint32_t STAGE = 3 * A_BYTES + ((3 * B_BYTES + 1023u) & ~1023u);
  const int64_t nmine = (a.mtiles > blockIdx.x) ? (a.mtiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int64_t iters = nmine * a.nkt;
  const int64_t LR = a.L * a.R;
  const int shift = a.xs->shift;

  if (tid == 0) {
    for (int s = 0; s < NSTAGE; ++s) {
      mbar_init(&full_bar[s], a.aimg ? 1 : kConvThreads);
      mbar_init(&bfull_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
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
        const int64_t mt = blockIdx.x + (it / a.nkt) * gridDim.x;
        if (!mbar_wait(&empty_bar[s], ((uint32_t)(it / NSTAGE) & 1u) ^ 1u, abort)) break;
        mbar_arrive_expect_tx(&full_bar[s], 3 * A_BYTES);
        bulk_g2s(smem + (size_t)s * STAGE, a.aimg + (size_t)mt * 3 * A_BYTES, 3 * A_BYTES, &full_bar[s]);
        issued = it + 1;
      }
      // drain: every issued copy must land before the CTA may exit
      const int64_t first = issued > NSTAGE ? issued - NSTAGE : 0;
      for (int64_t it = first; it < issued; ++it)
        mbar_wait_drain(&full_bar[it % NSTAGE], (uint32_t)(it / NSTAGE) & 1u);
    }
  } else if (warp >= kEpiWarps && warp < kMmaWarp) {
    // ------------------------------------------------------------ converters
    const int ct = tid - kEpiWarps * 32;
    const float sc = ldexpf(1.0f, shift);
    const TX* __restrict__ x = reinterpret_cast<const TX*>(a.x);
    float bufA[UNITS][8], bufB[UNITS][8];
    auto load = [&](float (&buf)[UNITS][8], int64_t it) {
      const int64_t mt = blockIdx.x + (it / a.nkt) * gridDim.x;
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
          const int64_t gam = ((int64_t)blockIdx.x + (it / a.nkt) * gridDim.x) * 128 + m;
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
    if (lane == 0) {
      const size_t slice_bytes = (size_t)a.nkt * B_BYTES;
      int64_t issued = 0;
      for (int64_t it = 0; it < iters; ++it) {
        const int s = (int)(it % NSTAGE);
        const int kt = (int)(it % a.nkt);
        if (!mbar_wait(&empty_bar[s], ((uint32_t)(it / NSTAGE) & 1u) ^ 1u, abort)) break;
        uint8_t* bb = smem + (size_t)s * STAGE + 3 * A_BYTES;
        mbar_arrive_expect_tx(&bfull_bar[s], 3 * B_BYTES);
#pragma unroll
        for (int q = 0; q < 3; ++q)
          bulk_g2s(bb + q * B_BYTES, a.bw + q * slice_bytes + (size_t)kt * B_BYTES, B_BYTES, &bfull_bar[s]);
        issued = it + 1;
      }
      // drain: every issued copy must land before the CTA may exit
      const int64_t first = issued > NSTAGE ? issued - NSTAGE : 0;
      for (int64_t it = first; it < issued; ++it)
        mbar_wait_drain(&bfull_bar[it % NSTAGE], (uint32_t)(it / NSTAGE) & 1u);
    }
  } else if (warp == kMmaWarp) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      const uint32_t idesc = idesc_f16(BF16 ? 1 : 0, 128, a.apad);
      int64_t it = 0;
      bool ok = true;
      for (int64_t t = 0; t < nmine && ok; ++t) {
        const int ab = (int)(t & 1);
        if (!mbar_wait(&acce_bar[ab], ((uint32_t)(t >> 1) & 1u) ^ 1u, abort)) break;
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)ab * 256u;
        for (int kt = 0; kt < a.nkt; ++kt, ++it) {
          const int s = (int)(it % NSTAGE);
          if (!mbar_wait(&full_bar[s], (uint32_t)(it / NSTAGE) & 1u, abort) ||
              !mbar_wait(&bfull_bar[s], (uint32_t)(it / NSTAGE) & 1u, abort)) { ok = false; break; }
          tc_fence_after();
          const uint32_t xa = smem_u32(smem + (size_t)s * STAGE);
          const uint32_t wa = xa + 3 * A_BYTES;
#pragma unroll
          for (int j = 0; j < KT / 16; ++j) {
            const uint32_t o = 32u * j;
            const uint64_t X0 = desc_k128(xa + o), X1 = desc_k128(xa + A_BYTES + o), X2 = desc_k128(xa + 2 * A_BYTES + o);
            const uint64_t W0 = desc_k128(wa + o), W1 = desc_k128(wa + B_BYTES + o), W2 = desc_k128(wa + 2 * B_BYTES + o);
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
    const TR* __restrict__ xr = reinterpret_cast<const TR*>(a.xres);
    float racc = 0.f;  // residual mode: this thread's sum of squares
    for (int64_t t = 0; t < nmine; ++t) {
      const int ab = (int)(t & 1);
      // warp-uniform wait: the tcgen05.ld below is .sync.aligned
      int okw = 1;
      if (lane == 0) okw = mbar_wait(&accf_bar[ab], (uint32_t)(t >> 1) & 1u, abort) ? 1 : 0;
      okw = __shfl_sync(0xffffffffu, okw, 0);
      __syncwarp();
      if (!okw) break;
      tc_fence_after();
      const int64_t mt = blockIdx.x + t * gridDim.x;
      const int64_t gam = mt * 128 + 32 * warp + lane;
      const bool valid = gam < LR;
      const int64_t l = valid ? gam / a.R : 0, c = valid ? gam - l * a.R : 0;
      const int e_out = (a.cshift && valid) ? -((int)__ldg(a.cshift + gam) + 8) : e_glob;
      const float f1 = ldexpf(1.0f, e_out / 2), f2 = ldexpf(1.0f, e_out - e_out / 2);
      TY* yo = y + (l * a.Atot + a.j0) * a.R + c;
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
          const TR* xo = RES ? xr + (l * a.Atot + a.j0) * a.R + c : nullptr;
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const int j = c0 + e;
            if (j < a.A) {
              float sv, tv;
              combine_orders(__uint_as_float(r0[e]), __uint_as_float(r1[e]), __uint_as_float(r2[e]),
                             __uint_as_float(r3[e]), __uint_as_float(r4[e]), sv, tv);
              const float z = ((sv + tv) * f1) * f2;
              if (RES) {
                const float dd = (float)(__ldg(xo + (int64_t)j * a.R) - (TR)z);
                racc = fmaf(dd, dd, racc);
              } else {
                yo[(int64_t)j * a.R] = (TY)z;
              }
            }
          }
        }
      }
      tc_fence_before();
      mbar_arrive(&acce_bar[ab]);
    }
    if (RES) {
      // fixed-order FP64 reduction over the 128 epilogue threads
      double v = (double)racc;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) res_smem[warp] = v;
      asm volatile("bar.sync 1, 128;" ::: "memory");
      if (tid == 0) a.res_part[blockIdx.x] = ((res_smem[0] + res_smem[1]) + (res_smem[2] + res_smem[3]));
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

// The data operand of a single-K-tile product (contraction <= 64) sliced once
// into the converter warps' shared-memory image: per M tile, three 128 x 64
// 16-bit slices in the 128-byte-swizzled K-major layout, [m tile][slice][16 KB].
// The output chunks (blockIdx.y of the product) then copy it with the bulk
// engine instead of each re-slicing it.  Same loads, scales and slicing as the
// converter warps, one thread per (m tile, row, group of 8 K values).
template <typename TX, bool GEN, bool BF16>
__global__ void ttm_preslice_a(TtmArgs a, uint8_t* __restrict__ img) {
  constexpr uint32_t A_BYTES = 128 * 128;
  const int MODE = GEN ? TM_GEN : a.rowmode;
  const float sc = ldexpf(1.0f, a.xs->shift);
  const TX* __restrict__ x = reinterpret_cast<const TX*>(a.x);
  const int64_t LR = a.L * a.R;
  const int64_t total = a.mtiles * 1024;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t mt = idx >> 10;
    const int g = (int)(idx & 1023);
    int m, q;
    if (MODE == TM_GEN) { m = g & 127; q = g >> 7; } else { m = g >> 3; q = g & 7; }
    const int64_t gam = mt * 128 + m;
    float buf[8];
    if (MODE == TM_GEN) {
      const int64_t l = gam / a.R, c = gam - l * a.R;
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int64_t i = 8 * q + e;
        buf[e] = (gam < LR && i < a.Bdim) ? (float)__ldg(x + (l * a.Bdim + i) * a.R + c) : 0.f;
      }
    } else if (MODE == TM_ROWVEC && gam < LR && 8 * q < a.Bdim) {
      ld8<TX>(x + gam * a.Bdim + 8 * q, buf);
    } else {
#pragma unroll
      for (int e = 0; e < 8; ++e)
        buf[e] = (gam < LR && 8 * q + e < a.Bdim) ? (float)__ldg(x + gam * a.Bdim + 8 * q + e) : 0.f;
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
    uint8_t* base = img + (size_t)mt * 3 * A_BYTES + sw128_off((uint32_t)m, (uint32_t)(8 * q));
    *reinterpret_cast<uint4*>(base) = make_uint4(p0[0], p0[1], p0[2], p0[3]);
    *reinterpret_cast<uint4*>(base + A_BYTES) = make_uint4(p1[0], p1[1], p1[2], p1[3]);
    *reinterpret_cast<uint4*>(base + 2 * A_BYTES) = make_uint4(p2[0], p2[1], p2[2], p2[3]);
  }
}

template <typename TX, bool BF16, bool GEN, bool RES, typename TR>
int ttm_launch_t(const TtmArgs& a, int grid, int smem, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    ATC_CUDA_TRY(cudaFuncSetAttribute(ttm_tc_kernel<TX, BF16, GEN, RES, TR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      225 * 1024));
    attr = true;
  }
  // algorithmic work: the data tensor read once, the output (or, with the
  // fused residual, the compared tensor) once, the factor once; 2 Atot Bdim per
  // output column; issued: nine slice products over the padded tiles
  const double cols = (double)a.L * (double)a.R;
  const double bytes = cols * (double)a.Bdim * sizeof(TX) + cols * (double)a.Atot * (RES ? sizeof(TR) : 4.0) +
                       (double)a.Atot * (double)a.Bdim * 8.0;
  const double flops = 2.0 * cols * (double)a.Atot * (double)a.Bdim;
  const double issued = 9.0 * 2.0 * (double)a.mtiles * 128.0 * (double)a.apad * (double)a.nchunk_launch *
                        (double)a.nkt * KT;
  KTimed kt_(s, RES ? "ttm_tc_kernel(fused residual)" : "ttm_tc_kernel", bytes, flops, issued);
  ttm_tc_kernel<TX, BF16, GEN, RES, TR><<<dim3(grid, a.nchunk_launch), kThreads, smem, s>>>(a);
  ATC_LAUNCHED(1);
  return ATC_OK;
}

template <typename TX, bool BF16>
int ttm_launch_g(const TtmArgs& a, bool gen, int grid, int smem, cudaStream_t s) {
  return gen ? ttm_launch_t<TX, BF16, true, false, float>(a, grid, smem, s)
             : ttm_launch_t<TX, BF16, false, false, float>(a, grid, smem, s);
}

template <typename TR>
int ttm_launch_res(const TtmArgs& a, bool gen, int grid, int smem, cudaStream_t s) {
  return gen ? ttm_launch_t<float, true, true, true, TR>(a, grid, smem, s)
             : ttm_launch_t<float, true, false, true, TR>(a, grid, smem, s);
}

// fixed-order sum of the residual partials
__global__ void sum_res_partials(const double* __restrict__ p, int np, double* __restrict__ out) {
  __shared__ double sh[256];
  double v = 0.0;
  for (int i = threadIdx.x; i < np; i += 256) v += p[i];
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}

int g_nsm_ttm = 0;

}  // namespace

int tc_error_flag(int** flag);

namespace {

// Shared driver of the projection / expansion (res == nullptr) and of the
// residual energy sum ||xres - U ._k X||^2 (res != nullptr, expansion only).
// percol: per-column scale exponents for the data operand (expansions, whose
// inputs -- cores and partly expanded cores -- span many orders of magnitude
// across columns); otherwise one power of two for the whole tensor.
int ttm_run(const void* x, int xdtype, int64_t L, int64_t n, int64_t R, const double* u, int64_t r, int expand,
            int precision, void* y, cudaStream_t s, const SliceScale* xs, const void* xres, int xres_dtype,
            double* res, bool percol) {
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
  const int grid = (int)(mtiles < g_nsm_ttm ? mtiles : g_nsm_ttm);
  uint8_t* bw = nullptr;
  ATC_TRY(Scratch::get(SLOT_TTM_U, wb * nchunk + (size_t)8 * nchunk * (grid + 1) + 256, (void**)&bw));
  double* part = reinterpret_cast<double*>(bw + wb * nchunk);
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
    a.A = (int)std::min<int64_t>(csz, Atot);
    a.apad = apad_max;
    a.Atot = Atot;
    a.j0 = 0;
    a.nkt = nkt;
    a.mtiles = mtiles;
    a.y = y;
    a.xs = xs;
    a.cshift = cshift;
    a.err = err;
    a.rowmode = (Bdim % 8 == 0) ? TM_ROWVEC : TM_ROW;
    a.xres = xres;
    a.res_part = res ? part : nullptr;
    a.csz = csz;
    a.wb = wb;
    a.nchunk_launch = (unsigned)nchunk;
    a.bw = bw;
    a.aimg = nullptr;
    const uint32_t bbytes = (uint32_t)a.apad * 128u;
    const uint32_t stage = 3u * 128u * 128u + ((3u * bbytes + 1023u) & ~1023u);
    a.nstage = (int)((224u * 1024u) / stage);
    if (a.nstage > 4) a.nstage = 4;
    if (a.nstage < 2) return fail(ATC_EUNSUP, "TTM stage does not fit in shared memory");
    const int smem = (int)(a.nstage * stage + 1024);
    {
      const int64_t tot = (int64_t)nkt * a.apad * 64 * nchunk;
      const int blocks = (int)((tot + 255) / 256 < 4096 ? (tot + 255) / 256 : 4096);
      if (bf16 || res) ttm_prep_b<true><<<blocks, 256, 0, s>>>(u, csz, Atot, nchunk, (int)Bdim, expand, a.apad, nkt, bw, wb);
      else ttm_prep_b<false><<<blocks, 256, 0, s>>>(u, csz, Atot, nchunk, (int)Bdim, expand, a.apad, nkt, bw, wb);
      ATC_LAUNCHED(1);
    }
    // one K tile and several output chunks: slice the data operand once (the
    // image stays in L2 when it is at most 64 MB) instead of once per chunk
    if (mtiles > 0 && nkt == 1 && nchunk > 1 && (size_t)mtiles * 3 * 128 * 128 <= ((size_t)64 << 20)) {
      uint8_t* img = nullptr;
      ATC_TRY(Scratch::get(SLOT_TTM_AIMG, (size_t)mtiles * 3 * 128 * 128, (void**)&img));
      const int64_t tot = mtiles * 1024;
      const int blocks = (int)((tot + 255) / 256 < 8 * g_nsm_ttm ? (tot + 255) / 256 : 8 * g_nsm_ttm);
      const bool gen = (R != 1), pb = bf16 || res;
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
      if (res) {
        if (xdtype != ATC_F32) return fail(ATC_EUNSUP, "residual mode expects an FP32 projected tensor");
        if (xres_dtype == ATC_F32) ATC_TRY(ttm_launch_res<float>(a, gen, grid, smem, s));
        else ATC_TRY(ttm_launch_res<double>(a, gen, grid, smem, s));
      } else if (xdtype == ATC_F32) {
        if (bf16) ATC_TRY((ttm_launch_g<float, true>(a, gen, grid, smem, s)));
        else ATC_TRY((ttm_launch_g<float, false>(a, gen, grid, smem, s)));
      } else {
        if (bf16) ATC_TRY((ttm_launch_g<double, true>(a, gen, grid, smem, s)));
        else ATC_TRY((ttm_launch_g<double, false>(a, gen, grid, smem, s)));
      }
    }
  }
  if (res) {
    if (mtiles == 0) {
      ATC_CUDA_TRY(cudaMemsetAsync(res, 0, sizeof(double), s));
    } else {
      sum_res_partials<<<1, 256, 0, s>>>(part, nchunk * grid, res);
      ATC_LAUNCHED(1);
    }
  }
  return ATC_OK;
}

}  // namespace

int launch_ttm_split(const void* x, int xdtype, int64_t L, int64_t n, int64_t R, const double* u, int64_t r,
                     int expand, int precision, void* y, int ydtype, cudaStream_t s, const SliceScale* xs) {
  if (ydtype != ATC_F32) return fail(ATC_EUNSUP, "split-precision TTM writes FP32 output");
  return ttm_run(x, xdtype, L, n, R, u, r, expand, precision, y, s, xs, nullptr, 0, nullptr, expand != 0);
}

// The residual ||x - U ._k y||^2 as the tensor-core expansion into a scratch
// tensor (the epilogue's stores do not stall it) followed by one streaming pass
// over x and the expansion; the differences and their rounding are those of the
// fused residual epilogue of ttm_tc_kernel (res != nullptr), whose dependent
// loads of x left HBM mostly idle.  ATC_RESIDUAL_FUSED=1 (read on every call)
// selects the fused epilogue instead; it needs no scratch tensor.
int launch_ttm_residual(const float* y, int64_t L, int64_t r, int64_t R, const double* u, int64_t n, const void* x,
                        int xdtype, double* rho, cudaStream_t s) {
  const char* fused = getenv("ATC_RESIDUAL_FUSED");
  if (fused && fused[0] == '1')
    return ttm_run(y, ATC_F32, L, n, R, u, r, 1, ATC_PREC_SPLIT_BF16, nullptr, s, nullptr, x, xdtype, rho, true);
  float* z = nullptr;
  ATC_TRY(Scratch::get(SLOT_RES_TMP, sizeof(float) * (size_t)(L * n * R) + 256, (void**)&z));
  ATC_TRY(ttm_run(y, ATC_F32, L, n, R, u, r, 1, ATC_PREC_SPLIT_BF16, z, s, nullptr, nullptr, 0, nullptr, true));
  return launch_diff_norm2(x, xdtype, z, L * n * R, rho, s);
}

}  // namespace atc
