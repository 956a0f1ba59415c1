// Split-precision mode Gram matrix on the 5th-generation tensor cores.
//
// G = X_(k) X_(k)^T over the (L, n, R) view (Section 3.1 unfolding, Gram form
// of the Algorithm 1 SVD step).  Every element x is split into two 16-bit
// halves, x ~ h + l (bf16, or fp16 after a power-of-two pre-scale), and
//   acc = H H^T + H (2L)^T + L L^T  (three tcgen05 MMAs per K step)
//   G   = (acc + acc^T) / 2 = (H + L)(H + L)^T,
// i.e. the full product of the split values: only the residual x - h - l
// and the FP32 accumulation perturb G.  Keeping L L^T matters: it is positive
// semi-definite and, if dropped, inflates every tail eigenvalue (the energy
// that decides the rank).  The symmetrisation is done in FP64 after the
// split-K partial sums.
//
// Kernel structure (one CTA per K chunk, n <= 256):
//   * 8 converter warps stream FP32/FP64 elements from HBM with coalesced
//     loads (the mode-k unfolding is pure index arithmetic: kappa = (l, c)),
//     split them and write H and 2L as K-major 128-byte-swizzled bf16/fp16
//     tiles into a multi-stage shared-memory ring (producer -> mbarrier);
//   * one elected thread issues tcgen05.mma (M = 128 rows per i-block, N = n
//     padded to 16, K = 16) into FP32 TMEM accumulators and releases ring
//     slots with tcgen05.commit;
//   * after the K loop, four warps read the accumulators with tcgen05.ld and
//     write FP32 partials; a second kernel sums the partials in FP64 in a
//     fixed order and symmetrises.
// Every wait is bounded (2 s); on time-out the CTA raises an error flag, waits
// for its issued MMAs, frees its TMEM and returns.
#include <stdint.h>

#include "atc_internal.cuh"
#include "tc_common.cuh"

namespace atc {
namespace {
using namespace tc;

constexpr int kConvWarps = 8;
constexpr int kConvThreads = kConvWarps * 32;
constexpr int kThreads = kConvThreads + 32;  // + MMA warp
constexpr int KT = 64;                       // K elements per pipeline stage

enum { LM_KC8 = 0, LM_IC1 = 1, LM_GEN = 2 };

struct GramArgs {
  const void* x;
  int64_t n, R, K;
  int64_t kchunk;      // K elements per CTA (multiple of KT)
  float* part;         // [split][blk][npad][128] FP32
  const float* scale;  // device power-of-two pre-scale, or nullptr
  int* err;
  int npad;
  int mode;            // LM_*
};

template <typename T>
__device__ __forceinline__ void load8(const T* p, float (&v)[8]);
template <>
__device__ __forceinline__ void load8<float>(const float* p, float (&v)[8]) {
  const float4 a = __ldg(reinterpret_cast<const float4*>(p));
  const float4 b = __ldg(reinterpret_cast<const float4*>(p) + 1);
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
  v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}
template <>
__device__ __forceinline__ void load8<double>(const double* p, float (&v)[8]) {
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const double2 a = __ldg(reinterpret_cast<const double2*>(p) + i);
    v[2 * i] = (float)a.x;
    v[2 * i + 1] = (float)a.y;
  }
}

template <typename T, bool BF16, int NBLK>
__global__ void __launch_bounds__(kThreads, 1) gram_tc_kernel(GramArgs a) {
  const int MODE = a.mode;
  constexpr int ROWS = NBLK * 128;
  constexpr int TILE_BYTES = ROWS * 128;          // one operand: ROWS x 64 16-bit
  constexpr int STAGE_BYTES = 3 * TILE_BYTES;     // H, 2L and L
  constexpr int NSTAGE = (NBLK == 2) ? 2 : 4;
  constexpr int UNITS = ROWS * 8 / kConvThreads;  // 8-element units per converter thread
  constexpr uint32_t TMEM_COLS = NBLK * 256;
  extern __shared__ uint8_t smem_raw[];
  __shared__ uint64_t full_bar[NSTAGE], empty_bar[NSTAGE], done_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  volatile int* abort = &abort_flag;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t n = a.n, R = a.R;
  const int64_t kb = (int64_t)blockIdx.x * a.kchunk;
  const int64_t ke = min(a.K, kb + a.kchunk);
  const int ntiles = (int)((ke - kb + KT - 1) / KT);
  const T* __restrict__ x = reinterpret_cast<const T*>(a.x);

  if (tid == 0) {
    for (int s = 0; s < NSTAGE; ++s) {
      mbar_init(&full_bar[s], kConvThreads);
      mbar_init(&empty_bar[s], 1);
    }
    mbar_init(&done_bar, 1);
    abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == kConvWarps) tmem_alloc(&tmem_slot, TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;

  if (warp < kConvWarps) {
    // ------------------------------------------------------------ converters
    const float sc = a.scale ? *a.scale : 1.0f;
    float bufA[UNITS][8], bufB[UNITS][8];
    auto load_tile = [&](float (&buf)[UNITS][8], int t) {
      const int64_t k0 = kb + (int64_t)t * KT;
#pragma unroll
      for (int u = 0; u < UNITS; ++u) {
        const int g = tid + kConvThreads * u;
        if (MODE == LM_KC8) {
          const int row = g >> 3, q = g & 7;
          const int64_t kap = k0 + 8 * q;
          if (row < n && kap < ke) {
            const int64_t l = kap / R, c = kap - l * R;
            load8<T>(x + (l * n + row) * R + c, buf[u]);
          } else {
#pragma unroll
            for (int e = 0; e < 8; ++e) buf[u][e] = 0.f;
          }
        } else if (MODE == LM_IC1) {
          const int row = g % ROWS, q = g / ROWS;
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const int64_t kap = k0 + 8 * q + e;
            buf[u][e] = (row < n && kap < ke) ? (float)__ldg(x + kap * n + row) : 0.f;
          }
        } else {
          const int row = g >> 3, q = g & 7;
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const int64_t kap = k0 + 8 * q + e;
            float v = 0.f;
            if (row < n && kap < ke) {
              const int64_t l = kap / R, c = kap - l * R;
              v = (float)__ldg(x + (l * n + row) * R + c);
            }
            buf[u][e] = v;
          }
        }
      }
    };
    auto store_tile = [&](float (&buf)[UNITS][8], int t) -> bool {
      const int s = t % NSTAGE;
      const uint32_t ph = ((uint32_t)(t / NSTAGE) & 1u) ^ 1u;
      if (!mbar_wait(&empty_bar[s], ph, abort)) return false;
      uint8_t* hbase = smem + s * STAGE_BYTES;
      uint8_t* lbase = hbase + TILE_BYTES;      // 2L
      uint8_t* l1base = lbase + TILE_BYTES;     // L
#pragma unroll
      for (int u = 0; u < UNITS; ++u) {
        const int g = tid + kConvThreads * u;
        int row, q;
        if (MODE == LM_IC1) { row = g % ROWS; q = g / ROWS; } else { row = g >> 3; q = g & 7; }
        uint32_t h[4], l1[4], l2[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) Split<BF16>::run(buf[u][2 * e] * sc, buf[u][2 * e + 1] * sc, h[e], l1[e], 1.0f);
#pragma unroll
        for (int e = 0; e < 4; ++e) l2[e] = Split<BF16>::twice(l1[e]);
        const uint32_t off = sw128_off((uint32_t)row, (uint32_t)(8 * q));
        *reinterpret_cast<uint4*>(hbase + off) = make_uint4(h[0], h[1], h[2], h[3]);
        *reinterpret_cast<uint4*>(lbase + off) = make_uint4(l2[0], l2[1], l2[2], l2[3]);
        *reinterpret_cast<uint4*>(l1base + off) = make_uint4(l1[0], l1[1], l1[2], l1[3]);
      }
      fence_proxy_async_smem();
      mbar_arrive(&full_bar[s]);
      return true;
    };
    if (ntiles > 0) load_tile(bufA, 0);
    for (int t = 0; t < ntiles; t += 2) {
      if (t + 1 < ntiles) load_tile(bufB, t + 1);
      if (!store_tile(bufA, t)) break;
      if (t + 1 < ntiles) {
        if (t + 2 < ntiles) load_tile(bufA, t + 2);
        if (!store_tile(bufB, t + 1)) break;
      }
    }
  } else if (lane == 0) {
    // ------------------------------------------------------------ MMA issuer
    constexpr uint32_t IDESC = idesc_f16(BF16 ? 1 : 0, 128, 0);
    const uint32_t idesc = IDESC | ((uint32_t)(a.npad >> 3) << 17);
    for (int t = 0; t < ntiles; ++t) {
      const int s = t % NSTAGE;
      if (!mbar_wait(&full_bar[s], (uint32_t)(t / NSTAGE) & 1u, abort)) break;
      tc_fence_after();
      const uint32_t hb = smem_u32(smem + s * STAGE_BYTES);
      const uint32_t lb = hb + TILE_BYTES;      // 2L
      const uint32_t l1b = lb + TILE_BYTES;     // L
#pragma unroll
      for (int j = 0; j < KT / 16; ++j) {
#pragma unroll
        for (int b = 0; b < NBLK; ++b) {
          const uint32_t d = tmem + b * 256;
          const uint64_t ad = desc_k128(hb + b * 16384 + 32 * j);
          umma_f16(d, ad, desc_k128(hb + 32 * j), idesc, (t | j) ? 1u : 0u);
          umma_f16(d, ad, desc_k128(lb + 32 * j), idesc, 1u);
          umma_f16(d, desc_k128(l1b + b * 16384 + 32 * j), desc_k128(l1b + 32 * j), idesc, 1u);
        }
      }
      umma_commit(&empty_bar[s]);
    }
    umma_commit(&done_bar);
  }

  // ---------------------------------------------------------------- epilogue
  if (warp < 4) {
    const bool ok = mbar_wait_drain(&done_bar, 0) && !abort_flag;
    tc_fence_after();
    float* out = a.part + (int64_t)blockIdx.x * (NBLK * 128) * a.npad;
#pragma unroll 1
    for (int b = 0; b < NBLK; ++b) {
#pragma unroll 1
      for (int c0 = 0; c0 < a.npad; c0 += 16) {
        uint32_t r[16];
        tmem_ld16(tmem + b * 256 + c0 + ((uint32_t)(32 * warp) << 16), r);
        tmem_ld_wait();
        float* o = out + ((int64_t)b * a.npad + c0) * 128 + 32 * warp + lane;
#pragma unroll
        for (int e = 0; e < 16; ++e) o[e * 128] = (ok && ntiles > 0) ? __uint_as_float(r[e]) : 0.f;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == kConvWarps) tmem_dealloc(tmem, TMEM_COLS);
  if (tid == 0 && abort_flag) atomicExch(a.err, 1);
}

// S[i][j] = inv_scale2 * sum_s part[s][(blk(i) * npad + j) * 128 + i % 128] in FP64 (fixed order)
__global__ void gram_tc_reduce(const float* __restrict__ part, int nsplit, int64_t n, int npad, int nblk,
                               const float* __restrict__ scale, double* __restrict__ s_out) {
  const int64_t total = n * n;
  const int64_t per = (int64_t)nblk * 128 * npad;
  double inv = 1.0;
  if (scale) {
    const double sc = (double)*scale;
    inv = 1.0 / (sc * sc);
  }
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = idx / n, i = idx - j * n;  // i fastest: coalesced partial reads
    const int64_t off = ((i >> 7) * npad + j) * 128 + (i & 127);
    double acc = 0.0;
    for (int s = 0; s < nsplit; ++s) acc += (double)part[(int64_t)s * per + off];
    s_out[i * n + j] = acc * inv;
  }
}

__global__ void symmetrize(const double* __restrict__ s_in, int64_t n, double* __restrict__ g) {
  const int64_t total = n * n;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx / n, j = idx - i * n;
    g[idx] = 0.5 * (s_in[i * n + j] + s_in[j * n + i]);
  }
}

// power-of-two scale so that max|x| * scale lies in [2^13, 2^14): fp16 halves stay finite
template <typename T>
__global__ void fp16_scale_kernel(const T* __restrict__ x, int64_t N, unsigned* __restrict__ mx_bits) {
  float m = 0.f;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    m = fmaxf(m, fabsf((float)x[i]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(mx_bits, __float_as_uint(m));
}
__global__ void fp16_scale_finish(const unsigned* __restrict__ mx_bits, float* __restrict__ scale) {
  const float m = __uint_as_float(*mx_bits);
  int e = 0;
  if (m > 0.f) frexpf(m, &e);  // m in [2^(e-1), 2^e)
  *scale = (m > 0.f) ? ldexpf(1.0f, 14 - e) : 1.0f;
}

template <typename T, bool BF16, int NBLK>
int launch_t(const GramArgs& a, int nsplit, cudaStream_t s) {
  constexpr int ROWS = NBLK * 128;
  constexpr int NSTAGE = (NBLK == 2) ? 2 : 4;
  const int smem = NSTAGE * 3 * ROWS * 128 + 1024;
  static bool attr = false;
  if (!attr) {
    ATC_CUDA_TRY(cudaFuncSetAttribute(gram_tc_kernel<T, BF16, NBLK>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    attr = true;
  }
  gram_tc_kernel<T, BF16, NBLK><<<nsplit, kThreads, smem, s>>>(a);
  ATC_LAUNCHED(1);
  return ATC_OK;
}

template <typename T, bool BF16>
int launch_mode(const GramArgs& a, int nblk, int nsplit, cudaStream_t s) {
  if (nblk == 1) return launch_t<T, BF16, 1>(a, nsplit, s);
  return launch_t<T, BF16, 2>(a, nsplit, s);
}

int g_nsm = 0;

}  // namespace

int tc_error_flag(int** flag) { return Scratch::get(SLOT_TC_ERR, 64, (void**)flag); }

int launch_gram_split(const void* x, int dtype, int64_t L, int64_t n, int64_t R, int precision, double* g,
                      cudaStream_t s) {
  if (n > 256) return fail(ATC_EUNSUP, "split-precision Gram supports n <= 256 (n = %lld)", (long long)n);
  if (g_nsm == 0) {
    int dev = 0;
    ATC_CUDA_TRY(cudaGetDevice(&dev));
    ATC_CUDA_TRY(cudaDeviceGetAttribute(&g_nsm, cudaDevAttrMultiProcessorCount, dev));
  }
  const int64_t K = L * R;
  const int nblk = (n <= 128) ? 1 : 2;
  const int npad = (int)((n + 15) / 16 * 16);
  const int mode = (R == 1) ? LM_IC1 : ((R % 8 == 0) ? LM_KC8 : LM_GEN);
  const int64_t ktiles = (K + KT - 1) / KT;
  int64_t tpc = (ktiles + g_nsm - 1) / g_nsm;
  if (tpc < 4) tpc = 4;
  const int nsplit = (int)((ktiles + tpc - 1) / tpc);
  GramArgs a;
  a.x = x;
  a.n = n;
  a.R = R;
  a.K = K;
  a.kchunk = tpc * KT;
  a.npad = npad;
  a.mode = mode;
  const size_t part_elems = (size_t)nsplit * nblk * 128 * npad;
  uint8_t* ws = nullptr;
  ATC_TRY(Scratch::get(SLOT_GRAM_PART, part_elems * 4 + (size_t)n * n * 8 + 1024, (void**)&ws));
  a.part = reinterpret_cast<float*>(ws);
  double* S = reinterpret_cast<double*>(ws + ((part_elems * 4 + 255) & ~(size_t)255));
  int* err = nullptr;
  ATC_TRY(tc_error_flag(&err));
  a.err = err;
  float* scale = nullptr;
  a.scale = nullptr;
  const bool bf16 = (precision == ATC_PREC_SPLIT_BF16);
  if (!bf16) {
    unsigned* mx = reinterpret_cast<unsigned*>(err + 4);
    scale = reinterpret_cast<float*>(err + 5);
    ATC_CUDA_TRY(cudaMemsetAsync(mx, 0, sizeof(unsigned), s));
    const int64_t N = K * n;
    const int blocks = (int)((N + 255) / 256 < 1216 ? (N + 255) / 256 : 1216);
    if (dtype == ATC_F32)
      fp16_scale_kernel<float><<<blocks, 256, 0, s>>>((const float*)x, N, mx);
    else
      fp16_scale_kernel<double><<<blocks, 256, 0, s>>>((const double*)x, N, mx);
    fp16_scale_finish<<<1, 1, 0, s>>>(mx, scale);
    ATC_LAUNCHED(2);
    a.scale = scale;
  }
  if (dtype == ATC_F32) {
    if (bf16) ATC_TRY((launch_mode<float, true>(a, nblk, nsplit, s)));
    else ATC_TRY((launch_mode<float, false>(a, nblk, nsplit, s)));
  } else {
    if (bf16) ATC_TRY((launch_mode<double, true>(a, nblk, nsplit, s)));
    else ATC_TRY((launch_mode<double, false>(a, nblk, nsplit, s)));
  }
  const int64_t tot = n * n;
  const int rb = (int)((tot + 255) / 256 < 2048 ? (tot + 255) / 256 : 2048);
  gram_tc_reduce<<<rb, 256, 0, s>>>(a.part, nsplit, n, npad, nblk, a.scale, S);
  symmetrize<<<rb, 256, 0, s>>>(S, n, g);
  ATC_LAUNCHED(2);
  return ATC_OK;
}

}  // namespace atc
