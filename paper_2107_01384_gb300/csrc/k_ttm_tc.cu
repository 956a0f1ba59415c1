// Split-precision mode-k product on the 5th-generation tensor cores.
//
// Projection (Algorithm 1): Y[l][j][c] = sum_i U[i][j] X[l][i][c], i.e. for
// every "column" gamma = (l, c) of the (L, n, R) view, y_gamma = U^T x_gamma.
// As a GEMM: D[gamma][j] = sum_i A[gamma][i] B[j][i] with M = gamma (128 per
// tile, any L and R), N = r (padded to 16, <= 256), K = n.  The same kernel
// runs the expansion Y = U ._k X with B[a][b] = U[a][b].
// Three split products (x ~ xh + xl, u ~ uh + ul in bf16 or pre-scaled fp16):
//   D = Xh Uh^T + Xl Uh^T + Xh Ul^T,  FP32 accumulation in TMEM.
//
// Warp roles (448 threads):
//   warps 0-3  epilogue: tcgen05.ld of a finished accumulator -> Y (FP32/FP64),
//              overlapped with the next tile's MMAs (two TMEM accumulators);
//   warps 4-11 converters: coalesced loads of X (the unfolding is index
//              arithmetic), split, K-major 128-byte-swizzled stores to smem;
//   warp 12    MMA issuer (one elected thread);
//   warp 13    B producer: bulk-async copies (cp.async.bulk, TMA engine) of the
//              pre-split, pre-swizzled factor tiles, completing on the
//              stage's mbarrier.
// All waits are bounded (2 s); on time-out the CTA raises an error flag,
// waits for its own MMAs, frees TMEM and returns.
#include <stdint.h>

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

enum { TM_ROW = 0, TM_ROWVEC = 1, TM_GEN = 2 };

struct TtmArgs {
  const void* x;
  int64_t L, Bdim, R;    // input view (L, Bdim, R); K = Bdim
  int A;                 // output mode size (N of the MMA, <= 256)
  int apad;              // A padded to 16
  int nkt;               // K tiles
  int64_t mtiles;        // ceil(L*R / 128)
  const uint8_t* bh;     // [nkt][apad][128 B] pre-swizzled
  const uint8_t* bl;
  void* y;               // (L, A, R)
  const float* xscale;   // device pre-scale of x or nullptr
  float uscale;          // pre-scale of the factor
  int* err;
  int nstage;            // pipeline depth (<= 4)
  int rowmode;           // TM_ROW / TM_ROWVEC when R == 1
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

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"((uint64_t)src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

template <typename TX, bool BF16, bool GEN>
__global__ void __launch_bounds__(kThreads, 1) ttm_tc_kernel(TtmArgs a) {
  typedef float TY;
  constexpr int MAXST = 4;
  const int NSTAGE = a.nstage;
  const int MODE = GEN ? TM_GEN : a.rowmode;
  constexpr uint32_t A_BYTES = 128 * 128;  // 128 rows x 64 16-bit
  extern __shared__ uint8_t smem_raw[];
  __shared__ uint64_t full_bar[MAXST], bfull_bar[MAXST], empty_bar[MAXST], accf_bar[2], acce_bar[2], done_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  volatile int* abort = &abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t B_BYTES = (uint32_t)a.apad * 128u;
  const uint32_t STAGE = 2 * A_BYTES + ((2 * B_BYTES + 1023u) & ~1023u);
  const int64_t nmine = (a.mtiles > blockIdx.x) ? (a.mtiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int64_t iters = nmine * a.nkt;
  const int64_t LR = a.L * a.R;

  if (tid == 0) {
    for (int s = 0; s < NSTAGE; ++s) {
      mbar_init(&full_bar[s], kConvThreads);
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

  if (warp >= kEpiWarps && warp < kMmaWarp) {
    // ------------------------------------------------------------ converters
    const int ct = tid - kEpiWarps * 32;
    const float sc = a.xscale ? *a.xscale : 1.0f;
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
      uint8_t* ah = smem + (size_t)s * STAGE;
      uint8_t* al = ah + A_BYTES;
#pragma unroll
      for (int u = 0; u < UNITS; ++u) {
        const int g = ct + kConvThreads * u;
        int m, q;
        if (MODE == TM_GEN) { m = g & 127; q = g >> 7; } else { m = g >> 3; q = g & 7; }
        uint32_t h[4], l[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) Split<BF16>::run(buf[u][2 * e] * sc, buf[u][2 * e + 1] * sc, h[e], l[e], 1.0f);
        const uint32_t off = sw128_off((uint32_t)m, (uint32_t)(8 * q));
        *reinterpret_cast<uint4*>(ah + off) = make_uint4(h[0], h[1], h[2], h[3]);
        *reinterpret_cast<uint4*>(al + off) = make_uint4(l[0], l[1], l[2], l[3]);
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
      int64_t issued = 0;
      for (int64_t it = 0; it < iters; ++it) {
        const int s = (int)(it % NSTAGE);
        const int kt = (int)(it % a.nkt);
        if (!mbar_wait(&empty_bar[s], ((uint32_t)(it / NSTAGE) & 1u) ^ 1u, abort)) break;
        uint8_t* bb = smem + (size_t)s * STAGE + 2 * A_BYTES;
        mbar_arrive_expect_tx(&bfull_bar[s], 2 * B_BYTES);
        bulk_g2s(bb, a.bh + (size_t)kt * B_BYTES, B_BYTES, &bfull_bar[s]);
        bulk_g2s(bb + B_BYTES, a.bl + (size_t)kt * B_BYTES, B_BYTES, &bfull_bar[s]);
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
          const uint32_t ah = smem_u32(smem + (size_t)s * STAGE);
          const uint32_t al = ah + A_BYTES;
          const uint32_t bh = ah + 2 * A_BYTES;
          const uint32_t bl = bh + B_BYTES;
#pragma unroll
          for (int j = 0; j < KT / 16; ++j) {
            const uint64_t dah = desc_k128(ah + 32 * j), dal = desc_k128(al + 32 * j);
            const uint64_t dbh = desc_k128(bh + 32 * j), dbl = desc_k128(bl + 32 * j);
            umma_f16(d, dah, dbh, idesc, (kt | j) ? 1u : 0u);
            umma_f16(d, dal, dbh, idesc, 1u);
            umma_f16(d, dah, dbl, idesc, 1u);
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
    const float inv = 1.0f / ((a.xscale ? *a.xscale : 1.0f) * a.uscale);
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
      const int64_t mt = blockIdx.x + t * gridDim.x;
      const int64_t gam = mt * 128 + 32 * warp + lane;
      const bool valid = gam < LR;
      const int64_t l = valid ? gam / a.R : 0, c = valid ? gam - l * a.R : 0;
      TY* yo = y + (l * a.A) * a.R + c;
#pragma unroll 1
      for (int c0 = 0; c0 < a.apad; c0 += 16) {
        uint32_t r[16];
        tmem_ld16(tmem + (uint32_t)ab * 256u + (uint32_t)c0 + ((uint32_t)(32 * warp) << 16), r);
        tmem_ld_wait();
        if (valid) {
#pragma unroll
          for (int e = 0; e < 16; ++e) {
            const int j = c0 + e;
            if (j < a.A) yo[(int64_t)j * a.R] = (TY)(__uint_as_float(r[e]) * inv);
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

// W tiles for the MMA B operand: W[a][b] = U[b][a] (projection) or U[a][b]
// (expansion), split into two 16-bit halves, laid out per K tile exactly as
// the 128-byte-swizzled K-major shared-memory image.
template <bool BF16>
__global__ void ttm_prep_b(const double* __restrict__ u, int A, int Bdim, int expand, int apad, int nkt, float uscale,
                           uint8_t* __restrict__ bh, uint8_t* __restrict__ bl) {
  const int64_t total = (int64_t)nkt * apad * 64;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
    const int il = (int)(idx & 63);
    const int64_t rest = idx >> 6;
    const int j = (int)(rest % apad);
    const int kt = (int)(rest / apad);
    const int b = kt * 64 + il;
    double w = 0.0;
    if (j < A && b < Bdim) w = expand ? u[(int64_t)j * Bdim + b] : u[(int64_t)b * A + j];
    const float wf = (float)(w * (double)uscale);
    uint16_t h, l;
    if (BF16) {
      const __nv_bfloat16 hh = __float2bfloat16_rn(wf);
      const float rem = (float)(w * (double)uscale - (double)__bfloat162float(hh));
      h = __bfloat16_as_ushort(hh);
      l = __bfloat16_as_ushort(__float2bfloat16_rn(rem));
    } else {
      const __half hh = __float2half_rn(wf);
      const float rem = (float)(w * (double)uscale - (double)__half2float(hh));
      h = __half_as_ushort(hh);
      l = __half_as_ushort(__float2half_rn(rem));
    }
    const size_t off = (size_t)kt * apad * 128 + tc::sw128_off((uint32_t)j, (uint32_t)il);
    *reinterpret_cast<uint16_t*>(bh + off) = h;
    *reinterpret_cast<uint16_t*>(bl + off) = l;
  }
}

template <typename T>
__global__ void ttm_xscale_kernel(const T* __restrict__ x, int64_t N, unsigned* __restrict__ mx_bits) {
  float m = 0.f;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    m = fmaxf(m, fabsf((float)x[i]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(mx_bits, __float_as_uint(m));
}
__global__ void ttm_xscale_finish(const unsigned* __restrict__ mx_bits, float* __restrict__ scale) {
  const float m = __uint_as_float(*mx_bits);
  int e = 0;
  if (m > 0.f) frexpf(m, &e);
  *scale = (m > 0.f) ? ldexpf(1.0f, 14 - e) : 1.0f;
}

template <typename TX, bool BF16, bool GEN>
int ttm_launch_t(const TtmArgs& a, int grid, int smem, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    ATC_CUDA_TRY(cudaFuncSetAttribute(ttm_tc_kernel<TX, BF16, GEN>, cudaFuncAttributeMaxDynamicSharedMemorySize, 197 * 1024));
    attr = true;
  }
  ttm_tc_kernel<TX, BF16, GEN><<<grid, kThreads, smem, s>>>(a);
  ATC_LAUNCHED(1);
  return ATC_OK;
}

template <typename TX, bool BF16>
int ttm_launch_g(const TtmArgs& a, bool gen, int grid, int smem, cudaStream_t s) {
  return gen ? ttm_launch_t<TX, BF16, true>(a, grid, smem, s) : ttm_launch_t<TX, BF16, false>(a, grid, smem, s);
}

int g_nsm_ttm = 0;

}  // namespace

int tc_error_flag(int** flag);

int launch_ttm_split(const void* x, int xdtype, int64_t L, int64_t n, int64_t R, const double* u, int64_t r,
                     int expand, int precision, void* y, int ydtype, cudaStream_t s) {
  const int64_t A = expand ? n : r;
  const int64_t Bdim = expand ? r : n;
  if (A > 256) return fail(ATC_EUNSUP, "split-precision TTM supports output mode <= 256 (got %lld)", (long long)A);
  if (ydtype != ATC_F32) return fail(ATC_EUNSUP, "split-precision TTM writes FP32 output");
  if (g_nsm_ttm == 0) {
    int dev = 0;
    ATC_CUDA_TRY(cudaGetDevice(&dev));
    ATC_CUDA_TRY(cudaDeviceGetAttribute(&g_nsm_ttm, cudaDevAttrMultiProcessorCount, dev));
  }
  const bool bf16 = (precision == ATC_PREC_SPLIT_BF16);
  TtmArgs a;
  a.x = x;
  a.L = L;
  a.Bdim = Bdim;
  a.R = R;
  a.A = (int)A;
  a.apad = (int)((A + 15) / 16 * 16);
  a.nkt = (int)((Bdim + KT - 1) / KT);
  a.mtiles = (L * R + 127) / 128;
  a.y = y;
  a.uscale = bf16 ? 1.0f : 8192.0f;
  a.rowmode = (Bdim % 8 == 0) ? TM_ROWVEC : TM_ROW;
  const uint32_t bbytes = (uint32_t)a.apad * 128u;
  const uint32_t stage = 2u * 128u * 128u + ((2u * bbytes + 1023u) & ~1023u);
  a.nstage = (int)((192u * 1024u) / stage);
  if (a.nstage > 4) a.nstage = 4;
  if (a.nstage < 2) return fail(ATC_EUNSUP, "TTM stage does not fit in shared memory");
  const int smem = (int)(a.nstage * stage + 1024);
  uint8_t* bw = nullptr;
  const size_t wb = (size_t)a.nkt * bbytes;
  ATC_TRY(Scratch::get(SLOT_TTM_U, 2 * wb + 256, (void**)&bw));
  a.bh = bw;
  a.bl = bw + wb;
  int* err = nullptr;
  ATC_TRY(tc_error_flag(&err));
  a.err = err;
  a.xscale = nullptr;
  if (!bf16) {
    unsigned* mx = reinterpret_cast<unsigned*>(err + 8);
    float* scale = reinterpret_cast<float*>(err + 9);
    ATC_CUDA_TRY(cudaMemsetAsync(mx, 0, sizeof(unsigned), s));
    const int64_t N = L * Bdim * R;
    const int blocks = (int)((N + 255) / 256 < 1216 ? (N + 255) / 256 : 1216);
    if (xdtype == ATC_F32) ttm_xscale_kernel<float><<<blocks, 256, 0, s>>>((const float*)x, N, mx);
    else ttm_xscale_kernel<double><<<blocks, 256, 0, s>>>((const double*)x, N, mx);
    ttm_xscale_finish<<<1, 1, 0, s>>>(mx, scale);
    ATC_LAUNCHED(2);
    a.xscale = scale;
  }
  {
    const int64_t tot = (int64_t)a.nkt * a.apad * 64;
    const int blocks = (int)((tot + 255) / 256 < 1024 ? (tot + 255) / 256 : 1024);
    if (bf16) ttm_prep_b<true><<<blocks, 256, 0, s>>>(u, a.A, (int)Bdim, expand, a.apad, a.nkt, a.uscale, bw, bw + wb);
    else ttm_prep_b<false><<<blocks, 256, 0, s>>>(u, a.A, (int)Bdim, expand, a.apad, a.nkt, a.uscale, bw, bw + wb);
    ATC_LAUNCHED(1);
  }
  if (a.mtiles == 0) return ATC_OK;
  const int grid = (int)(a.mtiles < g_nsm_ttm ? a.mtiles : g_nsm_ttm);
  const bool gen = (R != 1);
  if (xdtype == ATC_F32) {
    if (bf16) ATC_TRY((ttm_launch_g<float, true>(a, gen, grid, smem, s)));
    else ATC_TRY((ttm_launch_g<float, false>(a, gen, grid, smem, s)));
  } else {
    if (bf16) ATC_TRY((ttm_launch_g<double, true>(a, gen, grid, smem, s)));
    else ATC_TRY((ttm_launch_g<double, false>(a, gen, grid, smem, s)));
  }
  return ATC_OK;
}

}  // namespace atc
