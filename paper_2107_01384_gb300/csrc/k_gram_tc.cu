// Split-precision mode Gram matrix on the 5th-generation tensor cores.
//
// G = X_(k) X_(k)^T over the (L, n, R) view (Section 3.1 unfolding, Gram form
// of the Algorithm 1 SVD step).  Every element x is split into two 16-bit
// halves x ~ h + l (fp16 after a power-of-two pre-scale, or bf16) and the
// tensor cores form the full product of the split values,
//   diagonal tile     acc = H H^T + H (2L)^T + L L^T,   G = (acc + acc^T) / 2
//   off-diagonal tile acc = H_i H_j^T + H_i L_j^T + L_i H_j^T + L_i L_j^T,
// i.e. (H + L)(H + L)^T: only the split residual x - h - l perturbs G.
//
// Accuracy of the small eigenvalues is what decides the rank: the energy left
// in the tail is ~rel_eps^2 of the total, far below FP32 resolution of a long
// sum.  So the FP32 TMEM accumulator only ever holds FLUSH K-tiles (256
// products per entry); it is then added, with an error-free two-sum, into a
// double-float (hi, lo) accumulator that also lives in TMEM, and the CTA's
// partial is written in FP64.  The partials of the K splits are summed in FP64.
//
// Kernel structure (one CTA per (128x128 tile, K chunk)):
//   warps 0-7   converters: coalesced loads of the unfolding (index arithmetic,
//               no transpose), split, K-major 128-byte-swizzled smem tiles;
//   warps 8-11  flush / epilogue: tcgen05.ld of a finished FP32 accumulator,
//               two-sum into the TMEM (hi, lo) pair (tcgen05.st), final FP64 write;
//   warp 12     MMA issuer (one elected thread), two FP32 accumulators in
//               ping-pong so the MMAs never wait for a flush.
// TMEM columns: [0,128) acc0, [128,256) acc1, [256,384) hi, [384,512) lo.
// Every wait is bounded (2 s); on time-out the CTA raises an error flag, waits
// for its own MMAs, frees its TMEM and returns.
#include <stdint.h>

#include "atc_internal.cuh"
#include "tc_common.cuh"

namespace atc {
namespace {
using namespace tc;

constexpr int kConvWarps = 8;
constexpr int kConvThreads = kConvWarps * 32;
constexpr int kFlushWarp0 = kConvWarps;        // 8..11
constexpr int kMmaWarp = kConvWarps + 4;       // 12
constexpr int kThreads = (kMmaWarp + 1) * 32;  // 416
constexpr int KT = 64;                         // K elements per pipeline stage
constexpr int FLUSH = 4;                       // K tiles per FP32 accumulation
constexpr int NSTAGE = 3;
constexpr int SLOT = 128 * 128;                // bytes of one 128 x 64 16-bit tile
constexpr int STAGE_BYTES = 4 * SLOT;

enum { LM_KC8 = 0, LM_IC1 = 1, LM_GEN = 2 };

struct GramArgs {
  const void* x;
  int64_t n, R, K;
  int64_t kchunk;      // K elements per CTA (multiple of KT)
  int nsplit;
  int ntile;           // 128-row blocks
  double* part;        // [split][pair][128 cols][128 rows]
  const float* scale;  // device power-of-two pre-scale, or nullptr
  int* err;
  int mode;            // LM_*
};

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
          taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
      "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
      : "memory");
}
__device__ __forceinline__ void tmem_st_wait() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

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

// tile pair index -> (ti <= tj), row-major over the upper triangle
__device__ __forceinline__ void pair_of(int p, int ntile, int& ti, int& tj) {
  int t = p;
  ti = 0;
  while (t >= ntile - ti) { t -= ntile - ti; ++ti; }
  tj = ti + t;
}

template <typename T, bool BF16>
__global__ void __launch_bounds__(kThreads, 1) gram_tc_kernel(GramArgs a) {
  constexpr int UNITS = 8;  // 8-element units per converter thread (256 rows x 8 chunks / 256)
  extern __shared__ uint8_t smem_raw[];
  __shared__ uint64_t full_bar[NSTAGE], empty_bar[NSTAGE], accf_bar[2], acce_bar[2], done_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  volatile int* abort = &abort_flag;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int pair = blockIdx.x / a.nsplit, split = blockIdx.x % a.nsplit;
  int ti, tj;
  pair_of(pair, a.ntile, ti, tj);
  const bool diag = (ti == tj);
  const int nrows = diag ? 128 : 256;
  const int64_t n = a.n, R = a.R;
  const int64_t kb = (int64_t)split * a.kchunk;
  const int64_t ke = min(a.K, kb + a.kchunk);
  const int ntiles = (ke > kb) ? (int)((ke - kb + KT - 1) / KT) : 0;
  const int ngroups = (ntiles + FLUSH - 1) / FLUSH;
  const T* __restrict__ x = reinterpret_cast<const T*>(a.x);
  const int MODE = a.mode;

  if (tid == 0) {
    for (int s = 0; s < NSTAGE; ++s) {
      mbar_init(&full_bar[s], kConvThreads);
      mbar_init(&empty_bar[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&accf_bar[b], 1);
      mbar_init(&acce_bar[b], 128);
    }
    mbar_init(&done_bar, 1);
    abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == kMmaWarp) tmem_alloc(&tmem_slot, 512);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;

  if (warp < kConvWarps) {
    // ------------------------------------------------------------ converters
    const float sc = a.scale ? *a.scale : 1.0f;
    float bufA[UNITS][8], bufB[UNITS][8];
    // global row of local row r (0..nrows-1)
    auto grow = [&](int r) -> int64_t { return (r < 128) ? (int64_t)ti * 128 + r : (int64_t)tj * 128 + (r - 128); };
    auto unit_rq = [&](int g, int& r, int& q) {
      if (MODE == LM_IC1) { r = g % nrows; q = g / nrows; } else { r = g >> 3; q = g & 7; }
    };
    auto load_tile = [&](float (&buf)[UNITS][8], int t) {
      const int64_t k0 = kb + (int64_t)t * KT;
#pragma unroll
      for (int u = 0; u < UNITS; ++u) {
        const int g = tid + kConvThreads * u;
        int r, q;
        unit_rq(g, r, q);
        const int64_t row = grow(r);
        const bool live = (g < nrows * 8) && row < n;
        if (MODE == LM_KC8) {
          const int64_t kap = k0 + 8 * q;
          if (live && kap < ke) {
            const int64_t l = kap / R, c = kap - l * R;
            load8<T>(x + (l * n + row) * R + c, buf[u]);
          } else {
#pragma unroll
            for (int e = 0; e < 8; ++e) buf[u][e] = 0.f;
          }
        } else if (MODE == LM_IC1) {
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const int64_t kap = k0 + 8 * q + e;
            buf[u][e] = (live && kap < ke) ? (float)__ldg(x + kap * n + row) : 0.f;
          }
        } else {
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const int64_t kap = k0 + 8 * q + e;
            float v = 0.f;
            if (live && kap < ke) {
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
      uint8_t* st = smem + s * STAGE_BYTES;
#pragma unroll
      for (int u = 0; u < UNITS; ++u) {
        const int g = tid + kConvThreads * u;
        if (g >= nrows * 8) continue;
        int r, q;
        unit_rq(g, r, q);
        uint32_t h[4], l1[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) Split<BF16>::run(buf[u][2 * e] * sc, buf[u][2 * e + 1] * sc, h[e], l1[e], 1.0f);
        const int rr = r & 127;
        const uint32_t off = sw128_off((uint32_t)rr, (uint32_t)(8 * q));
        if (diag) {
          // slots: 0 = H, 1 = L, 2 = 2L
          uint32_t l2[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) l2[e] = Split<BF16>::twice(l1[e]);
          *reinterpret_cast<uint4*>(st + off) = make_uint4(h[0], h[1], h[2], h[3]);
          *reinterpret_cast<uint4*>(st + SLOT + off) = make_uint4(l1[0], l1[1], l1[2], l1[3]);
          *reinterpret_cast<uint4*>(st + 2 * SLOT + off) = make_uint4(l2[0], l2[1], l2[2], l2[3]);
        } else {
          // slots: 0 = H_i, 1 = L_i, 2 = H_j, 3 = L_j
          uint8_t* base = st + ((r < 128) ? 0 : 2 * SLOT);
          *reinterpret_cast<uint4*>(base + off) = make_uint4(h[0], h[1], h[2], h[3]);
          *reinterpret_cast<uint4*>(base + SLOT + off) = make_uint4(l1[0], l1[1], l1[2], l1[3]);
        }
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
  } else if (warp == kMmaWarp) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      const uint32_t idesc = idesc_f16(BF16 ? 1 : 0, 128, 128);
      bool ok = true;
      for (int g = 0; g < ngroups && ok; ++g) {
        const int ab = g & 1;
        if (!mbar_wait(&acce_bar[ab], ((uint32_t)(g >> 1) & 1u) ^ 1u, abort)) break;
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)ab * 128u;
        const int t1 = min(ntiles, (g + 1) * FLUSH);
        for (int t = g * FLUSH; t < t1; ++t) {
          const int s = t % NSTAGE;
          if (!mbar_wait(&full_bar[s], (uint32_t)(t / NSTAGE) & 1u, abort)) { ok = false; break; }
          tc_fence_after();
          const uint32_t s0 = smem_u32(smem + s * STAGE_BYTES);
#pragma unroll
          for (int j = 0; j < KT / 16; ++j) {
            const uint32_t acc0 = (t == g * FLUSH && j == 0) ? 0u : 1u;
            if (diag) {
              const uint64_t dh = desc_k128(s0 + 32 * j);
              umma_f16(d, dh, dh, idesc, acc0);
              umma_f16(d, dh, desc_k128(s0 + 2 * SLOT + 32 * j), idesc, 1u);
              const uint64_t dl = desc_k128(s0 + SLOT + 32 * j);
              umma_f16(d, dl, dl, idesc, 1u);
            } else {
              const uint64_t hi_ = desc_k128(s0 + 32 * j), li_ = desc_k128(s0 + SLOT + 32 * j);
              const uint64_t hj_ = desc_k128(s0 + 2 * SLOT + 32 * j), lj_ = desc_k128(s0 + 3 * SLOT + 32 * j);
              umma_f16(d, hi_, hj_, idesc, acc0);
              umma_f16(d, hi_, lj_, idesc, 1u);
              umma_f16(d, li_, hj_, idesc, 1u);
              umma_f16(d, li_, lj_, idesc, 1u);
            }
          }
          umma_commit(&empty_bar[s]);
        }
        if (ok) umma_commit(&accf_bar[ab]);
      }
      umma_commit(&done_bar);
      mbar_wait_drain(&done_bar, 0);
    }
  } else {
    // ------------------------------------------- flush (two-sum) and epilogue
    const int w = warp - kFlushWarp0;  // 0..3 == warp % 4: TMEM lanes 32w..32w+31
    const uint32_t lane_off = (uint32_t)(32 * w) << 16;
    const uint32_t thi = tmem + 256u + lane_off, tlo = tmem + 384u + lane_off;
    {
      uint32_t z[16];
#pragma unroll
      for (int e = 0; e < 16; ++e) z[e] = 0u;
#pragma unroll 1
      for (int c0 = 0; c0 < 128; c0 += 16) {
        tmem_st16(thi + c0, z);
        tmem_st16(tlo + c0, z);
      }
      tmem_st_wait();
    }
    bool ok = true;
    for (int g = 0; g < ngroups; ++g) {
      const int ab = g & 1;
      int okw = 1;
      if (lane == 0) okw = mbar_wait(&accf_bar[ab], (uint32_t)(g >> 1) & 1u, abort) ? 1 : 0;
      okw = __shfl_sync(0xffffffffu, okw, 0);
      __syncwarp();
      if (!okw) { ok = false; break; }
      tc_fence_after();
      const uint32_t tacc = tmem + (uint32_t)ab * 128u + lane_off;
#pragma unroll 1
      for (int c0 = 0; c0 < 128; c0 += 16) {
        uint32_t ra[16], rh[16], rl[16];
        tmem_ld16(tacc + c0, ra);
        tmem_ld16(thi + c0, rh);
        tmem_ld16(tlo + c0, rl);
        tmem_ld_wait();
#pragma unroll
        for (int e = 0; e < 16; ++e) {
          const float av = __uint_as_float(ra[e]), hv = __uint_as_float(rh[e]);
          const float s = hv + av;
          const float bp = s - hv;
          const float err = (hv - (s - bp)) + (av - bp);
          rh[e] = __float_as_uint(s);
          rl[e] = __float_as_uint(__uint_as_float(rl[e]) + err);
        }
        tmem_st16(thi + c0, rh);
        tmem_st16(tlo + c0, rl);
      }
      tmem_st_wait();
      tc_fence_before();
      mbar_arrive(&acce_bar[ab]);
    }
    // final: (hi + lo) in FP64, lane-major per column (coalesced across lanes)
    ok = ok && !abort_flag;
    double* out = a.part + ((int64_t)split * (a.ntile * (a.ntile + 1) / 2) + pair) * (128 * 128);
#pragma unroll 1
    for (int c0 = 0; c0 < 128; c0 += 16) {
      uint32_t rh[16], rl[16];
      tmem_ld16(thi + c0, rh);
      tmem_ld16(tlo + c0, rl);
      tmem_ld_wait();
#pragma unroll
      for (int e = 0; e < 16; ++e) {
        const double v = (double)__uint_as_float(rh[e]) + (double)__uint_as_float(rl[e]);
        out[(int64_t)(c0 + e) * 128 + 32 * w + lane] = ok ? v : 0.0;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == kMmaWarp) tmem_dealloc(tmem, 512);
  if (tid == 0 && abort_flag) atomicExch(a.err, 1);
}

// G[i][j] from the split partials, summed in FP64 in split order, scaled by
// 1/scale^2 and symmetrised inside diagonal tiles.
__global__ void gram_tc_assemble(const double* __restrict__ part, int nsplit, int ntile, int64_t n,
                                 const float* __restrict__ scale, double* __restrict__ g) {
  const int npair = ntile * (ntile + 1) / 2;
  double inv = 1.0;
  if (scale) {
    const double sc = (double)*scale;
    inv = 1.0 / (sc * sc);
  }
  const int64_t total = n * n;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t ocol = idx / n, orow = idx - (idx / n) * n;  // row fastest: coalesced partial reads
    int64_t i = orow, j = ocol;
    if (i / 128 > j / 128) { const int64_t t = i; i = j; j = t; }
    const int ti = (int)(i / 128), tj = (int)(j / 128);
    // pair index of (ti, tj), ti <= tj, row-major upper triangle
    const int p = ti * ntile - ti * (ti - 1) / 2 + (tj - ti);
    const int64_t ar = i & 127, bc = j & 127;
    double s1 = 0.0, s2 = 0.0;
    for (int s = 0; s < nsplit; ++s) {
      const double* t = part + ((int64_t)s * npair + p) * (128 * 128);
      s1 += t[bc * 128 + ar];          // acc[ar][bc] (lane-major: column bc, row ar)
      if (ti == tj) s2 += t[ar * 128 + bc];
    }
    const double v = (ti == tj) ? 0.5 * (s1 + s2) : s1;
    g[orow * n + ocol] = v * inv;
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

template <typename T, bool BF16>
int launch_t(const GramArgs& a, int grid, cudaStream_t s) {
  const int smem = NSTAGE * STAGE_BYTES + 1024;
  static bool attr = false;
  if (!attr) {
    ATC_CUDA_TRY(cudaFuncSetAttribute(gram_tc_kernel<T, BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    attr = true;
  }
  gram_tc_kernel<T, BF16><<<grid, kThreads, smem, s>>>(a);
  ATC_LAUNCHED(1);
  return ATC_OK;
}

int g_nsm = 0;

}  // namespace

int tc_error_flag(int** flag) { return Scratch::get(SLOT_TC_ERR, 64, (void**)flag); }

int launch_gram_split(const void* x, int dtype, int64_t L, int64_t n, int64_t R, int precision, double* g,
                      cudaStream_t s) {
  if (n > 1024) return fail(ATC_EUNSUP, "split-precision Gram supports n <= 1024 (n = %lld)", (long long)n);
  if (g_nsm == 0) {
    int dev = 0;
    ATC_CUDA_TRY(cudaGetDevice(&dev));
    ATC_CUDA_TRY(cudaDeviceGetAttribute(&g_nsm, cudaDevAttrMultiProcessorCount, dev));
  }
  const int64_t K = L * R;
  const int ntile = (int)((n + 127) / 128);
  const int npair = ntile * (ntile + 1) / 2;
  const int mode = (R == 1) ? LM_IC1 : ((R % 8 == 0) ? LM_KC8 : LM_GEN);
  const int64_t ktiles = (K + KT - 1) / KT;
  // about one CTA per SM over all tile pairs, at least two flush groups per CTA
  int64_t want = (g_nsm + npair - 1) / npair;
  int64_t tpc = (ktiles + want - 1) / want;
  if (tpc < 2 * FLUSH) tpc = 2 * FLUSH;
  int nsplit = (int)((ktiles + tpc - 1) / tpc);
  if (nsplit < 1) nsplit = 1;
  GramArgs a;
  a.x = x;
  a.n = n;
  a.R = R;
  a.K = K;
  a.kchunk = tpc * KT;
  a.nsplit = nsplit;
  a.ntile = ntile;
  a.mode = mode;
  const size_t part_elems = (size_t)nsplit * npair * 128 * 128;
  ATC_TRY(Scratch::get(SLOT_GRAM_PART, part_elems * 8 + 1024, (void**)&a.part));
  int* err = nullptr;
  ATC_TRY(tc_error_flag(&err));
  a.err = err;
  a.scale = nullptr;
  const bool bf16 = (precision == ATC_PREC_SPLIT_BF16);
  if (!bf16) {
    unsigned* mx = reinterpret_cast<unsigned*>(err + 4);
    float* scale = reinterpret_cast<float*>(err + 5);
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
  const int grid = npair * nsplit;
  if (dtype == ATC_F32) {
    if (bf16) ATC_TRY((launch_t<float, true>(a, grid, s)));
    else ATC_TRY((launch_t<float, false>(a, grid, s)));
  } else {
    if (bf16) ATC_TRY((launch_t<double, true>(a, grid, s)));
    else ATC_TRY((launch_t<double, false>(a, grid, s)));
  }
  const int64_t tot = n * n;
  const int rb = (int)((tot + 255) / 256 < 2048 ? (tot + 255) / 256 : 2048);
  gram_tc_assemble<<<rb, 256, 0, s>>>(a.part, nsplit, ntile, n, a.scale, g);
  ATC_LAUNCHED(1);
  return ATC_OK;
}

}  // namespace atc
