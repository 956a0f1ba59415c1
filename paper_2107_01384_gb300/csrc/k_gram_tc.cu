// Split-precision mode Gram matrix on the 5th-generation tensor cores.
//
// G = X_(k) X_(k)^T over the (L, n, R) view (Section 3.1 unfolding, Gram form
// of the Algorithm 1 SVD step).  The rank rule compares the energy left in
// the eigenvalue tail, ~rel_eps^2 of the total, with a budget, so G must be
// accurate far below FP32 resolution and, above all, free of bias: the FP32
// accumulation of the tensor cores truncates, and a floating hi/lo split fed
// to it shifts every entry of G by ~1e-6 relative in one direction - more
// than the whole tail at rel_eps = 1e-3.  Dropping the low-order products of
// a fixed-point split is not safe either: for smooth data the low slices are
// correlated and their products add up.
//
// So every element is cut into three integer slices on one power-of-two
// scale for the whole tensor (tc::slice3i: v = x 2^shift ~ a0 + a1 2^-8 +
// a2 2^-16), and the tensor cores form all nine slice products, grouped by
// order o = s + t into five accumulators acc_o = sum_{s+t=o} A_s B_t^T.  A
// window of FLUSH K tiles (128 products per entry) keeps every acc_o an
// integer below 2^24, so the FP32 accumulation is exact; after each window the
// orders are combined (tc::combine_orders) into a double-float (hi, lo)
// accumulator in TMEM, and the CTA's partial is written in FP64.  The
// partials of the K splits are summed in FP64 and scaled by 2^(-2 shift).
// What remains is the rounding of x to 24 bits below 2^E >= max|x|: unbiased,
// |x - x~| <= 2^(E-25).
//
// Tiles are 128 rows (block ti) x 64 columns (block cj), cj >= 2 ti, which
// covers the upper triangle; one CTA per (tile, K chunk):
//   warps 0-15  converters: coalesced loads of the unfolding (index arithmetic,
//               no transpose), slicing, K-major 128-byte-swizzled smem tiles;
//   warps 16-19 flush / epilogue: tcgen05.ld of the finished window, combine
//               into the TMEM (hi, lo) pair (tcgen05.st), final FP64 write;
//   warp 20     MMA issuer (one elected thread): 9 MMAs (M 128, N 64, K 16)
//               per K step.
// TMEM columns: acc_o at [64 o, 64 o + 64), hi at [320, 384), lo at [384, 448).
// Every wait is bounded (2 s); on time-out the CTA raises an error flag, waits
// for its own MMAs, frees its TMEM and returns.
#include <stdint.h>
#include <stdlib.h>

#include "atc_internal.cuh"
#include "tc_common.cuh"

namespace atc {
namespace {
using namespace tc;

constexpr int kConvWarps = 16;
constexpr int kConvThreads = kConvWarps * 32;
constexpr int kFlushWarp0 = kConvWarps;        // 16..19 (warp % 4 == TMEM lane quarter)
constexpr int kMmaWarp = kConvWarps + 4;       // 20
constexpr int kThreads = (kMmaWarp + 1) * 32;  // 672
constexpr int KT = 64;                         // K elements per pipeline stage
constexpr int FLUSH = 2;                       // K tiles per exact window (128 products)
constexpr int NSTAGE = 3;
constexpr int TM = 128, TN = 64;               // tile rows (A block) and columns (B block)
constexpr int ROWS = TM + TN;                  // rows loaded per K tile
constexpr int SLOT_A = TM * 128;               // bytes of one 128 x 64 16-bit slice tile
constexpr int SLOT_B = TN * 128;
constexpr int STAGE_BYTES = 3 * SLOT_A + 3 * SLOT_B;
constexpr int UNITS = ROWS * 8 / kConvThreads;  // 8-element units per converter thread (3)
static_assert(ROWS * 8 == UNITS * kConvThreads, "unit split");

enum { LM_KC8 = 0, LM_IC1 = 1, LM_GEN = 2 };

struct GramArgs {
  const void* x;
  int64_t n, R, K;
  int64_t kchunk;  // K elements per CTA (multiple of KT)
  int nsplit;
  int nt128, nc64;  // row blocks of 128, column blocks of 64
  int npair;
  double* part;     // [split][pair][64 cols][128 rows]
  const SliceScale* xs;
  int* err;
  int mode;         // LM_*
};

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
          taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
      "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
      : "memory");
}
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t (&r)[8]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr), "r"(r[0]),
               "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
               : "memory");
}
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
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

// tile index -> (ti, cj) with cj >= 2 ti, row-major
__device__ __forceinline__ void tile_of(int p, int nc64, int& ti, int& cj) {
  int t = p;
  ti = 0;
  while (t >= nc64 - 2 * ti) { t -= nc64 - 2 * ti; ++ti; }
  cj = 2 * ti + t;
}

template <typename T, bool BF16>
__global__ void __launch_bounds__(kThreads, 1) gram_tc_kernel(GramArgs a) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ uint64_t full_bar[NSTAGE], empty_bar[NSTAGE], accf_bar, acce_bar, done_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  volatile int* abort = &abort_flag;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int pair = blockIdx.x / a.nsplit, split = blockIdx.x % a.nsplit;
  int ti, cj;
  tile_of(pair, a.nc64, ti, cj);
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
    mbar_init(&accf_bar, 1);
    mbar_init(&acce_bar, 128);
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
    const float sc = ldexpf(1.0f, a.xs->shift);
    float bufA[UNITS][8], bufB[UNITS][8];
    // global row of local row r (0..ROWS-1): A block rows, then B block rows
    auto grow = [&](int r) -> int64_t { return (r < TM) ? (int64_t)ti * TM + r : (int64_t)cj * TN + (r - TM); };
    auto unit_rq = [&](int g, int& r, int& q) {
      if (MODE == LM_IC1) { r = g % ROWS; q = g / ROWS; } else { r = g >> 3; q = g & 7; }
    };
    auto load_tile = [&](float (&buf)[UNITS][8], int t) {
      const int64_t k0 = kb + (int64_t)t * KT;
#pragma unroll
      for (int u = 0; u < UNITS; ++u) {
        const int g = tid + kConvThreads * u;
        int r, q;
        unit_rq(g, r, q);
        const int64_t row = grow(r);
        const bool live = row < n;
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
        int r, q;
        unit_rq(g, r, q);
        uint32_t p0[4], p1[4], p2[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          float a0x, a1x, a2x, a0y, a1y, a2y;
          slice3i(buf[u][2 * e] * sc, a0x, a1x, a2x);
          slice3i(buf[u][2 * e + 1] * sc, a0y, a1y, a2y);
          p0[e] = Pack<BF16>::two(a0x, a0y);
          p1[e] = Pack<BF16>::two(a1x, a1y);
          p2[e] = Pack<BF16>::two(a2x, a2y);
        }
        uint8_t* base;
        uint32_t sl, rr;
        if (r < TM) { base = st; sl = SLOT_A; rr = (uint32_t)r; }
        else { base = st + 3 * SLOT_A; sl = SLOT_B; rr = (uint32_t)(r - TM); }
        const uint32_t off = sw128_off(rr, (uint32_t)(8 * q));
        *reinterpret_cast<uint4*>(base + off) = make_uint4(p0[0], p0[1], p0[2], p0[3]);
        *reinterpret_cast<uint4*>(base + sl + off) = make_uint4(p1[0], p1[1], p1[2], p1[3]);
        *reinterpret_cast<uint4*>(base + 2 * sl + off) = make_uint4(p2[0], p2[1], p2[2], p2[3]);
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
      const uint32_t idesc = idesc_f16(BF16 ? 1 : 0, TM, TN);
      bool ok = true;
      for (int g = 0; g < ngroups && ok; ++g) {
        // the flush warps must have drained the previous window
        if (!mbar_wait(&acce_bar, ((uint32_t)g & 1u) ^ 1u, abort)) break;
        tc_fence_after();
        const int t1 = min(ntiles, (g + 1) * FLUSH);
        for (int t = g * FLUSH; t < t1; ++t) {
          const int s = t % NSTAGE;
          if (!mbar_wait(&full_bar[s], (uint32_t)(t / NSTAGE) & 1u, abort)) { ok = false; break; }
          tc_fence_after();
          const uint32_t sa = smem_u32(smem + s * STAGE_BYTES), sb = sa + 3 * SLOT_A;
#pragma unroll
          for (int j = 0; j < KT / 16; ++j) {
            const uint32_t acc = (t == g * FLUSH && j == 0) ? 0u : 1u;
            const uint32_t o = 32u * j;
            const uint64_t A0 = desc_k128(sa + o), A1 = desc_k128(sa + SLOT_A + o), A2 = desc_k128(sa + 2 * SLOT_A + o);
            const uint64_t B0 = desc_k128(sb + o), B1 = desc_k128(sb + SLOT_B + o), B2 = desc_k128(sb + 2 * SLOT_B + o);
            umma_f16(tmem + 0u, A0, B0, idesc, acc);
            umma_f16(tmem + 64u, A0, B1, idesc, acc);
            umma_f16(tmem + 64u, A1, B0, idesc, 1u);
            umma_f16(tmem + 128u, A0, B2, idesc, acc);
            umma_f16(tmem + 128u, A1, B1, idesc, 1u);
            umma_f16(tmem + 128u, A2, B0, idesc, 1u);
            umma_f16(tmem + 192u, A1, B2, idesc, acc);
            umma_f16(tmem + 192u, A2, B1, idesc, 1u);
            umma_f16(tmem + 256u, A2, B2, idesc, acc);
          }
          umma_commit(&empty_bar[s]);
        }
        if (ok) umma_commit(&accf_bar);
      }
      umma_commit(&done_bar);
      mbar_wait_drain(&done_bar, 0);
    }
  } else {
    // ---------------------------------------- flush (combine) and epilogue
    const int w = warp - kFlushWarp0;  // == warp % 4: TMEM lanes 32w..32w+31
    const uint32_t tl = tmem + ((uint32_t)(32 * w) << 16);
    const uint32_t thi = tl + 320u, tlo = tl + 384u;
    {
      uint32_t z[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) z[e] = 0u;
#pragma unroll 1
      for (int c0 = 0; c0 < TN; c0 += 8) {
        tmem_st8(thi + c0, z);
        tmem_st8(tlo + c0, z);
      }
      tmem_st_wait();
    }
    bool ok = true;
    for (int g = 0; g < ngroups; ++g) {
      int okw = 1;
      if (lane == 0) okw = mbar_wait(&accf_bar, (uint32_t)g & 1u, abort) ? 1 : 0;
      okw = __shfl_sync(0xffffffffu, okw, 0);
      __syncwarp();
      if (!okw) { ok = false; break; }
      tc_fence_after();
#pragma unroll 1
      for (int c0 = 0; c0 < TN; c0 += 8) {
        uint32_t r0[8], r1[8], r2[8], r3[8], r4[8], rh[8], rl[8];
        tmem_ld8(tl + c0, r0);
        tmem_ld8(tl + 64u + c0, r1);
        tmem_ld8(tl + 128u + c0, r2);
        tmem_ld8(tl + 192u + c0, r3);
        tmem_ld8(tl + 256u + c0, r4);
        tmem_ld8(thi + c0, rh);
        tmem_ld8(tlo + c0, rl);
        tmem_ld_wait();
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          float sv, tv, s1, e1;
          combine_orders(__uint_as_float(r0[e]), __uint_as_float(r1[e]), __uint_as_float(r2[e]),
                         __uint_as_float(r3[e]), __uint_as_float(r4[e]), sv, tv);
          // double-float (hi, lo) += s + t, renormalised so that |lo| <= ulp(hi) / 2
          two_sum(__uint_as_float(rh[e]), sv, s1, e1);
          e1 += __uint_as_float(rl[e]) + tv;
          const float h2 = s1 + e1;
          rh[e] = __float_as_uint(h2);
          rl[e] = __float_as_uint(e1 - (h2 - s1));
        }
        tmem_st8(thi + c0, rh);
        tmem_st8(tlo + c0, rl);
      }
      tmem_st_wait();
      tc_fence_before();
      mbar_arrive(&acce_bar);
    }
    // final: (hi + lo) in FP64, lane-major per column (coalesced across lanes)
    ok = ok && !abort_flag;
    double* out = a.part + ((int64_t)split * a.npair + pair) * (TM * TN);
#pragma unroll 1
    for (int c0 = 0; c0 < TN; c0 += 8) {
      uint32_t rh[8], rl[8];
      tmem_ld8(thi + c0, rh);
      tmem_ld8(tlo + c0, rl);
      tmem_ld_wait();
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const double v = (double)__uint_as_float(rh[e]) + (double)__uint_as_float(rl[e]);
        out[(int64_t)(c0 + e) * TM + 32 * w + lane] = ok ? v : 0.0;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == kMmaWarp) tmem_dealloc(tmem, 512);
  if (tid == 0 && abort_flag) atomicExch(a.err, 1);
}

// ------------------------------------------------ pre-sliced, TMA-fed variant
// The slices are formed once per mode by slice_planes_kernel (an HBM-bound
// pass) into NS = 3 (24-bit fixed point) or NS = 4 (32-bit) 16-bit planes in
// the unfolded (n, Kp) layout, Kp = K rounded up to 64 with zero padding; the
// Gram CTAs then pull 128 x 64 (A rows) and 64 x 64 (B rows) tiles of every
// plane with TMA (128-byte swizzle, the smem image the MMA descriptors
// expect), so no warp re-slices a row block per tile.  Warp 0 issues the
// copies, warp 1 the MMAs (all slice products of order s + t <= 4 -- nine for
// three slices, thirteen for four -- into five order accumulators), warps 2-5
// flush each exact window into a double-float running sum kept in their
// registers.  With four slices every partial sum of an order stays below
// 3 * 2^22 < 2^24 in a window of 128 products (|a0| <= 256, other slices
// <= 128), so the FP32 accumulation is still exact.
constexpr int kTmaThreads = 192;
template <int NS>
struct TmaCfg {
  static constexpr int STAGES = (NS == 3) ? 3 : 2;  // 216 KB / 192 KB of stages
  static constexpr int STAGE = NS * (SLOT_A + SLOT_B);
};

struct GramTmaArgs {
  int64_t kchunk;  // multiple of KT
  int64_t Kp;
  int nsplit, nc64, npair;
  double* part;
  int* err;
};

struct GramMaps {
  CUtensorMap a[4], b[4];  // per slice plane: 128-row and 64-row boxes
};

template <bool BF16, int NS>
__global__ void __launch_bounds__(kTmaThreads, 1)
    gram_tma_kernel(const __grid_constant__ GramMaps maps, GramTmaArgs a) {
  constexpr int TNS = TmaCfg<NS>::STAGES;
  constexpr int T_STAGE = TmaCfg<NS>::STAGE;
  extern __shared__ uint8_t smem_raw[];
  __shared__ uint64_t full_bar[TNS], empty_bar[TNS], accf_bar, acce_bar, done_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  volatile int* abort = &abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int pair = blockIdx.x / a.nsplit, split = blockIdx.x % a.nsplit;
  int ti, cj;
  tile_of(pair, a.nc64, ti, cj);
  const int64_t kb = (int64_t)split * a.kchunk;
  const int64_t ke = min(a.Kp, kb + a.kchunk);
  const int ntiles = (ke > kb) ? (int)((ke - kb) / KT) : 0;
  const int ngroups = (ntiles + FLUSH - 1) / FLUSH;
  if (tid == 0) {
    for (int s = 0; s < TNS; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    mbar_init(&accf_bar, 1);
    mbar_init(&acce_bar, 128);
    mbar_init(&done_bar, 1);
    abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 1) tmem_alloc(&tmem_slot, 512);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;

  if (warp == 0) {
    // ---------------------------------------------------------- TMA producer
    if (lane == 0) {
      int issued = 0;
      for (int t = 0; t < ntiles; ++t) {
        const int s = t % TNS;
        if (!mbar_wait(&empty_bar[s], ((uint32_t)(t / TNS) & 1u) ^ 1u, abort)) break;
        uint8_t* st = smem + s * T_STAGE;
        mbar_arrive_expect_tx(&full_bar[s], (uint32_t)T_STAGE);
        const int k0 = (int)(kb + (int64_t)t * KT);
#pragma unroll
        for (int q = 0; q < NS; ++q) {
          tma_load_2d(st + q * SLOT_A, &maps.a[q], &full_bar[s], k0, ti * TM);
          tma_load_2d(st + NS * SLOT_A + q * SLOT_B, &maps.b[q], &full_bar[s], k0, cj * TN);
        }
        issued = t + 1;
      }
      // every issued copy must land before the CTA may exit
      for (int t = (issued > TNS ? issued - TNS : 0); t < issued; ++t)
        mbar_wait_drain(&full_bar[t % TNS], (uint32_t)(t / TNS) & 1u);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      const uint32_t idesc = idesc_f16(BF16 ? 1 : 0, TM, TN);
      bool ok = true;
      for (int g = 0; g < ngroups && ok; ++g) {
        if (!mbar_wait(&acce_bar, ((uint32_t)g & 1u) ^ 1u, abort)) break;
        tc_fence_after();
        const int t1 = min(ntiles, (g + 1) * FLUSH);
        for (int t = g * FLUSH; t < t1; ++t) {
          const int s = t % TNS;
          if (!mbar_wait(&full_bar[s], (uint32_t)(t / TNS) & 1u, abort)) { ok = false; break; }
          tc_fence_after();
          const uint32_t sa = smem_u32(smem + s * T_STAGE), sb = sa + NS * SLOT_A;
#pragma unroll
          for (int j = 0; j < KT / 16; ++j) {
            const uint32_t acc = (t == g * FLUSH && j == 0) ? 0u : 1u;
            const uint32_t o = 32u * j;
            // order o = s + t <= 4 into TMEM columns [64 o, 64 o + 64); the first
            // product of an order in a window starts it (acc), the others add
#pragma unroll
            for (int od = 0; od <= 4; ++od) {
              bool first = true;
#pragma unroll
              for (int sa_i = 0; sa_i < NS; ++sa_i) {
                const int tb_i = od - sa_i;
                if (tb_i < 0 || tb_i >= NS) continue;
                umma_f16(tmem + 64u * od, desc_k128(sa + sa_i * SLOT_A + o), desc_k128(sb + tb_i * SLOT_B + o), idesc,
                         first ? acc : 1u);
                first = false;
              }
            }
          }
          umma_commit(&empty_bar[s]);
        }
        if (ok) umma_commit(&accf_bar);
      }
      umma_commit(&done_bar);
      mbar_wait_drain(&done_bar, 0);
    }
  } else {
    // --------------------------------- flush into registers and epilogue
    const int w = warp & 3;  // TMEM lane quarter of this warp
    const uint32_t tl = tmem + ((uint32_t)(32 * w) << 16);
    float hi[TN], lo[TN];
#pragma unroll
    for (int c = 0; c < TN; ++c) { hi[c] = 0.f; lo[c] = 0.f; }
    bool ok = true;
    for (int g = 0; g < ngroups; ++g) {
      int okw = 1;
      if (lane == 0) okw = mbar_wait(&accf_bar, (uint32_t)g & 1u, abort) ? 1 : 0;
      okw = __shfl_sync(0xffffffffu, okw, 0);
      __syncwarp();
      if (!okw) { ok = false; break; }
      tc_fence_after();
#pragma unroll
      for (int c0 = 0; c0 < TN; c0 += 16) {
        uint32_t r0[16], r1[16], r2[16], r3[16], r4[16];
        tmem_ld16(tl + c0, r0);
        tmem_ld16(tl + 64u + c0, r1);
        tmem_ld16(tl + 128u + c0, r2);
        tmem_ld16(tl + 192u + c0, r3);
        tmem_ld16(tl + 256u + c0, r4);
        tmem_ld_wait();
#pragma unroll
        for (int e = 0; e < 16; ++e) {
          float sv, tv, s1, e1;
          combine_orders(__uint_as_float(r0[e]), __uint_as_float(r1[e]), __uint_as_float(r2[e]),
                         __uint_as_float(r3[e]), __uint_as_float(r4[e]), sv, tv);
          two_sum(hi[c0 + e], sv, s1, e1);
          e1 += lo[c0 + e] + tv;
          const float h2 = s1 + e1;
          lo[c0 + e] = e1 - (h2 - s1);
          hi[c0 + e] = h2;
        }
      }
      tc_fence_before();
      mbar_arrive(&acce_bar);
    }
    ok = ok && !abort_flag;
    double* out = a.part + ((int64_t)split * a.npair + pair) * (TM * TN);
#pragma unroll
    for (int c = 0; c < TN; ++c) {
      const double v = (double)hi[c] + (double)lo[c];
      out[(int64_t)c * TM + 32 * w + lane] = ok ? v : 0.0;
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tmem, 512);
  if (tid == 0 && abort_flag) atomicExch(a.err, 1);
}

// --------------------------- in-kernel unfolding: raw tiles by TMA, sliced here
// FP32 input whose mode-k unfolding tiles are boxes of a tensor map: R = 1
// (X is (L, n), a K tile is 32 consecutive rows l, the box {128 i, 32 l}) or
// R a multiple of 64 (a K tile of 32 lies inside one l: the box {32 r, 128 i,
// 1 l} over (R, n, L)).  Warp 0 streams raw A (128 rows) and B (64 rows)
// tiles of 32 K values into a ring of shared-memory buffers with TMA tensor
// copies -- the unfolding is the box geometry, nothing is transposed or
// written back to HBM; warps 6-21 cut two raw halves at a time into the three
// 16-bit slice planes of a K-major 128-byte-swizzled stage (tc::slice3i, the
// tensor's power-of-two scale; sixteen warps, so that the dependent
// add/multiply chains of the slicing overlap); warp 1 issues the nine slice
// products per K step into the five order accumulators; warps 2-5 and 22-25
// (two per TMEM lane quarter, 32 columns each) flush each exact window into a
// double-float sum kept in TMEM columns [320, 448).
constexpr int kRawConvWarps = 16;
constexpr int kRawConvThreads = kRawConvWarps * 32;
constexpr int kRawFlushThreads = 256;
constexpr int kRawThreads = (6 + kRawConvWarps + 4) * 32;  // 832
constexpr int kRawHalf = 32;                            // K values per raw tile
constexpr int kRawStages = 3;
constexpr uint32_t kRawA = TM * kRawHalf * 4, kRawB = TN * kRawHalf * 4;  // 16 KB, 8 KB
constexpr int kRawConvStages = 2;
constexpr int kRawStage = 3 * (SLOT_A + SLOT_B);  // 72 KB of slices
constexpr int kRawSmem = kRawConvStages * kRawStage + kRawStages * (int)(kRawA + kRawB) + 1024;
constexpr int kRawUnits = ROWS * 8 / kRawConvThreads;  // 3
static_assert(ROWS * 8 == kRawUnits * kRawConvThreads, "unit split");

struct GramRawArgs {
  int64_t R;        // 1, or a multiple of 64
  int64_t kchunk;   // K elements per CTA (multiple of KT)
  int64_t Kp;       // K rounded up to KT
  int nsplit, nc64, npair;
  double* part;
  const SliceScale* xs;
  int* err;
};

template <bool BF16>
__global__ void __launch_bounds__(kRawThreads, 1)
    gram_raw_kernel(const __grid_constant__ CUtensorMap mapa, const __grid_constant__ CUtensorMap mapb, GramRawArgs a) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ uint64_t full_bar[kRawConvStages], empty_bar[kRawConvStages], raw_full[kRawStages], raw_empty[kRawStages];
  __shared__ uint64_t accf_bar, acce_bar, done_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint8_t* rawbuf = smem + kRawConvStages * kRawStage;
  volatile int* abort = &abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int pair = blockIdx.x / a.nsplit, split = blockIdx.x % a.nsplit;
  int ti, cj;
  tile_of(pair, a.nc64, ti, cj);
  const int64_t kb = (int64_t)split * a.kchunk;
  const int64_t ke = min(a.Kp, kb + a.kchunk);
  const int ntiles = (ke > kb) ? (int)((ke - kb) / KT) : 0;
  const int nhalves = 2 * ntiles;
  const int ngroups = (ntiles + FLUSH - 1) / FLUSH;
  if (tid == 0) {
    for (int s = 0; s < kRawConvStages; ++s) {
      mbar_init(&full_bar[s], kRawConvThreads);
      mbar_init(&empty_bar[s], 1);
    }
    for (int s = 0; s < kRawStages; ++s) {
      mbar_init(&raw_full[s], 1);
      mbar_init(&raw_empty[s], kRawConvThreads);
    }
    mbar_init(&accf_bar, 1);
    mbar_init(&acce_bar, kRawFlushThreads);
    mbar_init(&done_bar, 1);
    abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 1) tmem_alloc(&tmem_slot, 512);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;

  if (warp == 0) {
    // ------------------------------------------------- raw-tile producer (TMA)
    if (lane == 0) {
      int issued = 0;
      for (int h = 0; h < nhalves; ++h) {
        const int rs = h % kRawStages;
        if (!mbar_wait(&raw_empty[rs], ((uint32_t)(h / kRawStages) & 1u) ^ 1u, abort)) break;
        uint8_t* dst = rawbuf + (size_t)rs * (kRawA + kRawB);
        mbar_arrive_expect_tx(&raw_full[rs], kRawA + kRawB);
        const int64_t k0 = kb + (int64_t)h * kRawHalf;
        if (a.R == 1) {
          tma_load_2d(dst, &mapa, &raw_full[rs], ti * TM, (int)k0);
          tma_load_2d(dst + kRawA, &mapb, &raw_full[rs], cj * TN, (int)k0);
        } else {
          const int64_t l = k0 / a.R, r0 = k0 - l * a.R;
          tma_load_3d(dst, &mapa, &raw_full[rs], (int)r0, ti * TM, (int)l);
          tma_load_3d(dst + kRawA, &mapb, &raw_full[rs], (int)r0, cj * TN, (int)l);
        }
        issued = h + 1;
      }
      for (int h = (issued > kRawStages ? issued - kRawStages : 0); h < issued; ++h)
        mbar_wait_drain(&raw_full[h % kRawStages], (uint32_t)(h / kRawStages) & 1u);
    }
  } else if (warp >= 6 && warp < 6 + kRawConvWarps) {
    // ---------------------------------------------------------- converters
    const int ct = tid - 6 * 32;
    const float sc = ldexpf(1.0f, a.xs->shift);
    const bool rows_k = a.R != 1;  // raw tiles [row][k] (else [k][row])
    for (int t = 0; t < ntiles; ++t) {
      const int h0 = 2 * t, h1 = 2 * t + 1;
      const int r0s = h0 % kRawStages, r1s = h1 % kRawStages;
      if (!mbar_wait(&raw_full[r0s], (uint32_t)(h0 / kRawStages) & 1u, abort)) break;
      if (!mbar_wait(&raw_full[r1s], (uint32_t)(h1 / kRawStages) & 1u, abort)) break;
      const int s = t % kRawConvStages;
      if (!mbar_wait(&empty_bar[s], ((uint32_t)(t / kRawConvStages) & 1u) ^ 1u, abort)) break;
      const float* raw0 = reinterpret_cast<const float*>(rawbuf + (size_t)r0s * (kRawA + kRawB));
      const float* raw1 = reinterpret_cast<const float*>(rawbuf + (size_t)r1s * (kRawA + kRawB));
      uint8_t* st = smem + (size_t)s * kRawStage;
#pragma unroll
      for (int u = 0; u < kRawUnits; ++u) {
        const int g = ct + kRawConvThreads * u;
        // unit = (row of the A and B blocks stacked, group q of 8 K values);
        // q < 4 from the first raw half, q >= 4 from the second
        int row, q;
        if (rows_k) { row = g >> 3; q = g & 7; } else { row = g % ROWS; q = g / ROWS; }
        const bool isb = row >= TM;
        const int rr = isb ? row - TM : row;
        const float* hb = (q < 4) ? raw0 : raw1;
        const float* tile = isb ? hb + kRawA / 4 : hb;
        const int kk = 8 * (q & 3);
        float v[8];
        if (rows_k) {
          const float4* p4 = reinterpret_cast<const float4*>(tile + rr * kRawHalf + kk);
          const float4 x0 = p4[0], x1 = p4[1];
          v[0] = x0.x; v[1] = x0.y; v[2] = x0.z; v[3] = x0.w;
          v[4] = x1.x; v[5] = x1.y; v[6] = x1.z; v[7] = x1.w;
        } else {
          const int ld = isb ? TN : TM;  // raw [k][row], rows contiguous
#pragma unroll
          for (int e = 0; e < 8; ++e) v[e] = tile[(kk + e) * ld + rr];
        }
        uint32_t p0[4], p1[4], p2[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          float a0x, a1x, a2x, a0y, a1y, a2y;
          slice3i(v[2 * e] * sc, a0x, a1x, a2x);
          slice3i(v[2 * e + 1] * sc, a0y, a1y, a2y);
          p0[e] = Pack<BF16>::two(a0x, a0y);
          p1[e] = Pack<BF16>::two(a1x, a1y);
          p2[e] = Pack<BF16>::two(a2x, a2y);
        }
        uint8_t* base = isb ? st + 3 * SLOT_A : st;
        const uint32_t slot = isb ? SLOT_B : SLOT_A;
        const uint32_t off = sw128_off((uint32_t)rr, (uint32_t)(8 * q));
        *reinterpret_cast<uint4*>(base + off) = make_uint4(p0[0], p0[1], p0[2], p0[3]);
        *reinterpret_cast<uint4*>(base + slot + off) = make_uint4(p1[0], p1[1], p1[2], p1[3]);
        *reinterpret_cast<uint4*>(base + 2 * slot + off) = make_uint4(p2[0], p2[1], p2[2], p2[3]);
      }
      mbar_arrive(&raw_empty[r0s]);
      mbar_arrive(&raw_empty[r1s]);
      fence_proxy_async_smem();
      mbar_arrive(&full_bar[s]);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      const uint32_t idesc = idesc_f16(BF16 ? 1 : 0, TM, TN);
      bool ok = true;
      for (int g = 0; g < ngroups && ok; ++g) {
        if (!mbar_wait(&acce_bar, ((uint32_t)g & 1u) ^ 1u, abort)) break;
        tc_fence_after();
        const int t1 = min(ntiles, (g + 1) * FLUSH);
        for (int t = g * FLUSH; t < t1; ++t) {
          const int s = t % kRawConvStages;
          if (!mbar_wait(&full_bar[s], (uint32_t)(t / kRawConvStages) & 1u, abort)) { ok = false; break; }
          tc_fence_after();
          const uint32_t sa = smem_u32(smem + (size_t)s * kRawStage), sb = sa + 3 * SLOT_A;
#pragma unroll
          for (int j = 0; j < KT / 16; ++j) {
            const uint32_t acc = (t == g * FLUSH && j == 0) ? 0u : 1u;
            const uint32_t o = 32u * j;
#pragma unroll
            for (int od = 0; od <= 4; ++od) {
              bool first = true;
#pragma unroll
              for (int sa_i = 0; sa_i < 3; ++sa_i) {
                const int tb_i = od - sa_i;
                if (tb_i < 0 || tb_i >= 3) continue;
                umma_f16(tmem + 64u * od, desc_k128(sa + sa_i * SLOT_A + o), desc_k128(sb + tb_i * SLOT_B + o), idesc,
                         first ? acc : 1u);
                first = false;
              }
            }
          }
          umma_commit(&empty_bar[s]);
        }
        if (ok) umma_commit(&accf_bar);
      }
      umma_commit(&done_bar);
      mbar_wait_drain(&done_bar, 0);
    }
  } else {
    // ------------------------- flush into the TMEM (hi, lo) pair and epilogue
    // (the running double-float sum lives in TMEM columns [320, 448): the
    // converter warps leave too few registers to hold it)
    const int w = warp & 3;                             // TMEM lane quarter of this warp
    const uint32_t cb = (warp >= 6 + kRawConvWarps) ? 32u : 0u;  // this warp's 32 columns
    const uint32_t tl = tmem + ((uint32_t)(32 * w) << 16) + cb;
    const uint32_t thi = tl + 320u, tlo = tl + 384u;
    bool ok = true;
    for (int g = 0; g < ngroups; ++g) {
      int okw = 1;
      if (lane == 0) okw = mbar_wait(&accf_bar, (uint32_t)g & 1u, abort) ? 1 : 0;
      okw = __shfl_sync(0xffffffffu, okw, 0);
      __syncwarp();
      if (!okw) { ok = false; break; }
      tc_fence_after();
#pragma unroll 1
      for (int c0 = 0; c0 < 32; c0 += 8) {
        uint32_t r0[8], r1[8], r2[8], r3[8], r4[8], rh[8], rl[8];
        tmem_ld8(tl + c0, r0);
        tmem_ld8(tl + 64u + c0, r1);
        tmem_ld8(tl + 128u + c0, r2);
        tmem_ld8(tl + 192u + c0, r3);
        tmem_ld8(tl + 256u + c0, r4);
        if (g > 0) {
          tmem_ld8(thi + c0, rh);
          tmem_ld8(tlo + c0, rl);
        }
        tmem_ld_wait();
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          float sv, tv, s1, e1;
          combine_orders(__uint_as_float(r0[e]), __uint_as_float(r1[e]), __uint_as_float(r2[e]),
                         __uint_as_float(r3[e]), __uint_as_float(r4[e]), sv, tv);
          const float h0 = (g > 0) ? __uint_as_float(rh[e]) : 0.f, l0 = (g > 0) ? __uint_as_float(rl[e]) : 0.f;
          two_sum(h0, sv, s1, e1);
          e1 += l0 + tv;
          const float h2 = s1 + e1;
          rh[e] = __float_as_uint(h2);
          rl[e] = __float_as_uint(e1 - (h2 - s1));
        }
        tmem_st8(thi + c0, rh);
        tmem_st8(tlo + c0, rl);
      }
      tmem_st_wait();
      tc_fence_before();
      mbar_arrive(&acce_bar);
    }
    ok = ok && !abort_flag && ngroups > 0;
    double* out = a.part + ((int64_t)split * a.npair + pair) * (TM * TN) + (int64_t)cb * TM;
#pragma unroll 1
    for (int c0 = 0; c0 < 32; c0 += 8) {
      uint32_t rh[8], rl[8];
      if (ok) {
        tmem_ld8(thi + c0, rh);
        tmem_ld8(tlo + c0, rl);
        tmem_ld_wait();
      }
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const double v = ok ? (double)__uint_as_float(rh[e]) + (double)__uint_as_float(rl[e]) : 0.0;
        out[(int64_t)(c0 + e) * TM + 32 * w + lane] = v;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tmem, 512);
  if (tid == 0 && abort_flag) atomicExch(a.err, 1);
}

// Slices of the (L, n, R) tensor into three 16-bit planes laid out (n, Kp):
// plane[i][k] for k = l R + r (zero for k >= K).  For R = 1 the reads along k
// are strided by n, so that case goes through a 32 x 32 shared-memory transpose.
struct Planes {
  uint16_t* p[4];
};
template <bool BF16, int NS>
__device__ __forceinline__ void put_slices(const Planes& pl, int64_t idx, float v) {
  float a0, a1, a2, a3 = 0.f;
  if (NS == 4) slice4i(v, a0, a1, a2, a3);
  else slice3i(v, a0, a1, a2);
  pl.p[0][idx] = Pack<BF16>::one(a0);
  pl.p[1][idx] = Pack<BF16>::one(a1);
  pl.p[2][idx] = Pack<BF16>::one(a2);
  if (NS == 4) pl.p[3][idx] = Pack<BF16>::one(a3);
}
// FP64 input: the slices are cut from the double value v = x 2^shift (every
// step exact in binary64 for |v| < 256); rounding x to float first would keep
// only 24 significant bits, less than four slices resolve near max |x|
template <bool BF16, int NS>
__device__ __forceinline__ void put_slices_d(const Planes& pl, int64_t idx, double v) {
  if (NS == 3) {
    put_slices<BF16, NS>(pl, idx, (float)v);  // 24 bits below max |x|: float holds them
    return;
  }
  const double a0 = rint(v), t = (v - a0) * 256.0, a1 = rint(t), t2 = (t - a1) * 256.0, a2 = rint(t2);
  const double a3 = rint((t2 - a2) * 256.0);
  pl.p[0][idx] = Pack<BF16>::one((float)a0);
  pl.p[1][idx] = Pack<BF16>::one((float)a1);
  pl.p[2][idx] = Pack<BF16>::one((float)a2);
  pl.p[3][idx] = Pack<BF16>::one((float)a3);
}

template <typename T, bool BF16, int NS>
__global__ void slice_planes_kernel(const T* __restrict__ x, int64_t n, int64_t R, int64_t K, int64_t Kp,
                                    const SliceScale* __restrict__ xs, Planes pl) {
  const int64_t total = n * Kp;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx / Kp, k = idx - i * Kp;
    T v = 0;
    if (k < K) {
      const int64_t l = k / R, r = k - l * R;
      v = __ldg(x + (l * n + i) * R + r);
    }
    if (sizeof(T) == 8) put_slices_d<BF16, NS>(pl, idx, ldexp((double)v, xs->shift));
    else put_slices<BF16, NS>(pl, idx, ldexpf((float)v, xs->shift));
  }
}
template <typename T, bool BF16, int NS>
__global__ void slice_planes_t_kernel(const T* __restrict__ x, int64_t n, int64_t K, int64_t Kp,
                                      const SliceScale* __restrict__ xs, Planes pl) {
  // R == 1: x[k][i] (k = l), tile of 32 k x 32 i through shared memory
  __shared__ T tile[32][33];
  const int64_t i0 = (int64_t)blockIdx.y * 32, k0 = (int64_t)blockIdx.x * 32;
  for (int yy = threadIdx.y; yy < 32; yy += blockDim.y) {
    const int64_t k = k0 + yy, i = i0 + threadIdx.x;
    tile[yy][threadIdx.x] = (k < K && i < n) ? __ldg(x + k * n + i) : (T)0;
  }
  __syncthreads();
  for (int yy = threadIdx.y; yy < 32; yy += blockDim.y) {
    const int64_t i = i0 + yy, k = k0 + threadIdx.x;
    if (i < n && k < Kp) {
      const T v = tile[threadIdx.x][yy];
      if (sizeof(T) == 8) put_slices_d<BF16, NS>(pl, i * Kp + k, ldexp((double)v, xs->shift));
      else put_slices<BF16, NS>(pl, i * Kp + k, ldexpf((float)v, xs->shift));
    }
  }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
    cudaGetLastError();
  }
  return fn;
}

// 2D map over a (rows, Kp) plane of 16-bit values, box (64 k, box_rows rows), 128-byte swizzle
int make_map(CUtensorMap* m, void* base, int64_t rows, int64_t Kp, int box_rows, bool bf16) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return fail(ATC_EUNSUP, "cuTensorMapEncodeTiled unavailable");
  const cuuint64_t dims[2] = {(cuuint64_t)Kp, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)Kp * 2};
  const cuuint32_t box[2] = {64u, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1u, 1u};
  const CUresult r = fn(m, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, base, dims,
                        strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(ATC_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return ATC_OK;
}

// G[i][j] from the split partials, summed in FP64 in split order and scaled
// by 2^(-2 shift); (i, j) is read from the tile of (min, max), which covers it.
__global__ void gram_tc_assemble(const double* __restrict__ part, int nsplit, int npair, int nc64, int64_t n,
                                 const SliceScale* __restrict__ xs, double* __restrict__ g) {
  const double f = ldexp(1.0, -2 * xs->shift);
  const int64_t total = n * n;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t ocol = idx / n, orow = idx - (idx / n) * n;  // row fastest: coalesced partial reads
    const int64_t i = min(orow, ocol), j = max(orow, ocol);
    const int ti = (int)(i / TM), cj = (int)(j / TN);
    // tile index of (ti, cj): rows ti' < ti contribute nc64 - 2 ti' tiles each
    const int p = ti * nc64 - ti * (ti - 1) + (cj - 2 * ti);
    const int64_t ar = i - (int64_t)ti * TM, bc = j - (int64_t)cj * TN;
    // the split partials added in split order; eight loads in flight at a time
    const double* src = part + (int64_t)p * (TM * TN) + bc * TM + ar;
    const int64_t sstride = (int64_t)npair * (TM * TN);
    double v = 0.0;
    for (int s0 = 0; s0 < nsplit; s0 += 8) {
      double t[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) t[u] = (s0 + u < nsplit) ? __ldg(src + (s0 + u) * sstride) : 0.0;
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (s0 + u < nsplit) v += t[u];
    }
    g[orow * n + ocol] = v * f;
  }
}

// max |x| as float bits (non-negative floats order like their bit patterns)
template <typename T>
__global__ void absmax_kernel(const T* __restrict__ x, int64_t N, unsigned* __restrict__ mx_bits) {
  float m = 0.f;
  const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, stride = (int64_t)gridDim.x * blockDim.x;
  int64_t done = 0;
  if (sizeof(T) == 4 && ((uintptr_t)x & 15) == 0) {
    // 16-byte loads: four times the bytes in flight per thread
    const float4* x4 = reinterpret_cast<const float4*>(x);
    const int64_t n4 = N / 4;
    for (int64_t i = t0; i < n4; i += stride) {
      const float4 v = __ldg(x4 + i);
      m = fmaxf(m, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
    }
    done = n4 * 4;
  }
  for (int64_t i = done + t0; i < N; i += stride) m = fmaxf(m, fabsf((float)x[i]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(mx_bits, __float_as_uint(m));
}
// shift = 8 - E with max < 2^E, so that |x| 2^shift < 256; clamped so that
// 2^shift and 2^(-2 shift) stay finite (tensors that small or large read as
// if their maximum were at the clamp)
__global__ void slice_scale_finish(SliceScale* s) {
  const float m = __uint_as_float(s->maxbits);
  int e = 0;
  if (m > 0.f) frexpf(m, &e);  // m in [2^(e-1), 2^e)
  int sh = 8 - e;
  if (sh > 120) sh = 120;
  if (sh < -120) sh = -120;
  s->shift = (m > 0.f) ? sh : 0;
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
int g_scale_rot = 0;

// ATC_GRAM_CONVERT=1 (read on every call) selects the converter-warp kernel
// (the TMA-fed one is the default)
bool gram_tma_off() {
  const char* e = getenv("ATC_GRAM_CONVERT");
  return e && e[0] == '1';
}

}  // namespace

// layout of the SLOT_TC_ERR scratch: error word at byte 0, slice scales from byte 64
int tc_error_flag(int** flag) { return Scratch::get(SLOT_TC_ERR, 1024, (void**)flag); }

// Map over FP32 data of `rank` dimensions (innermost first: dims[0] elements
// contiguous, strides[d - 1] bytes between consecutive indices of dimension
// d), no swizzle, out-of-range elements read as zero.
int make_raw_map_f32(CUtensorMap* m, const void* base, int rank, const int64_t* dims, const int64_t* strides,
                     const uint32_t* box) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return fail(ATC_EUNSUP, "cuTensorMapEncodeTiled unavailable");
  if (rank < 1 || rank > 5) return fail(ATC_EINVAL, "bad tensor map rank %d", rank);
  cuuint64_t d[5], st[4];
  cuuint32_t bx[5], es[5];
  for (int i = 0; i < rank; ++i) {
    d[i] = (cuuint64_t)dims[i];
    bx[i] = box[i];
    es[i] = 1u;
    if (i > 0) st[i - 1] = (cuuint64_t)strides[i - 1];
  }
  const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, (cuuint32_t)rank, const_cast<void*>(base), d, st, bx, es,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(ATC_ECUDA, "cuTensorMapEncodeTiled (raw FP32) failed (%d)", (int)r);
  return ATC_OK;
}

int slice_scale(const void* x, int dtype, int64_t N, cudaStream_t s, const SliceScale** out) {
  int* base = nullptr;
  ATC_TRY(tc_error_flag(&base));
  // rotate over 8 records so that a caller can hold the scales of a few tensors
  SliceScale* sc = reinterpret_cast<SliceScale*>(reinterpret_cast<uint8_t*>(base) + 64) + (g_scale_rot++ & 7);
  ATC_CUDA_TRY(cudaMemsetAsync(sc, 0, sizeof(SliceScale), s));
  if (N > 0) {
    const int blocks = (int)((N + 255) / 256 < 1216 ? (N + 255) / 256 : 1216);
    KTimed kt_(s, "absmax_kernel", (double)N * (dtype == ATC_F32 ? 4.0 : 8.0));
    if (dtype == ATC_F32)
      absmax_kernel<float><<<blocks, 256, 0, s>>>((const float*)x, N, &sc->maxbits);
    else
      absmax_kernel<double><<<blocks, 256, 0, s>>>((const double*)x, N, &sc->maxbits);
    ATC_LAUNCHED(1);
  }
  slice_scale_finish<<<1, 1, 0, s>>>(sc);
  ATC_LAUNCHED(1);
  *out = sc;
  return ATC_OK;
}

int slice_scale_begin(cudaStream_t s, SliceScale** out) {
  int* base = nullptr;
  ATC_TRY(tc_error_flag(&base));
  SliceScale* sc = reinterpret_cast<SliceScale*>(reinterpret_cast<uint8_t*>(base) + 64) + (g_scale_rot++ & 7);
  ATC_CUDA_TRY(cudaMemsetAsync(sc, 0, sizeof(SliceScale), s));
  *out = sc;
  return ATC_OK;
}

int slice_scale_end(SliceScale* sc, cudaStream_t s) {
  slice_scale_finish<<<1, 1, 0, s>>>(sc);
  ATC_LAUNCHED(1);
  return ATC_OK;
}

namespace {
template <typename T, bool BF16, int NS>
void launch_slices(const T* x, int64_t n, int64_t R, int64_t K, int64_t Kp, const SliceScale* xs, const Planes& pl,
                   cudaStream_t s) {
  KTimed kt_(s, NS == 3 ? "slice_planes_kernel" : "slice_planes_kernel(4 slices)",
             (double)n * (double)K * sizeof(T) + (double)NS * 2.0 * (double)n * (double)Kp);
  if (R == 1) {
    const dim3 grid((unsigned)((Kp + 31) / 32), (unsigned)((n + 31) / 32));
    slice_planes_t_kernel<T, BF16, NS><<<grid, dim3(32, 8), 0, s>>>(x, n, K, Kp, xs, pl);
  } else {
    const int64_t tot = n * Kp;
    const int blocks = (int)((tot + 255) / 256 < 4 * 1216 ? (tot + 255) / 256 : 4 * 1216);
    slice_planes_kernel<T, BF16, NS><<<blocks, 256, 0, s>>>(x, n, R, K, Kp, xs, pl);
  }
}
template <bool BF16, int NS>
int launch_gram_tma(const GramMaps& maps, const GramTmaArgs& ta, int grid, cudaStream_t s, double bytes, double flops,
                    double issued) {
  const int smem = TmaCfg<NS>::STAGES * TmaCfg<NS>::STAGE + 1024;
  static bool attr = false;
  if (!attr) {
    ATC_CUDA_TRY(cudaFuncSetAttribute(gram_tma_kernel<BF16, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    attr = true;
  }
  KTimed kt_(s, NS == 3 ? "gram_tma_kernel" : "gram_tma_kernel(4 slices)", bytes, flops, issued);
  gram_tma_kernel<BF16, NS><<<grid, kTmaThreads, smem, s>>>(maps, ta);
  return ATC_OK;
}
}  // namespace

int launch_gram_split(const void* x, int dtype, int64_t L, int64_t n, int64_t R, int precision, double* g,
                      cudaStream_t s, const SliceScale* xs, int nslice) {
  if (n > 1024) return fail(ATC_EUNSUP, "split-precision Gram supports n <= 1024 (n = %lld)", (long long)n);
  if (nslice != 3 && nslice != 4) return fail(ATC_EINVAL, "split-precision Gram: %d slices", nslice);
  if (g_nsm == 0) {
    int dev = 0;
    ATC_CUDA_TRY(cudaGetDevice(&dev));
    ATC_CUDA_TRY(cudaDeviceGetAttribute(&g_nsm, cudaDevAttrMultiProcessorCount, dev));
  }
  const int64_t K = L * R;
  const int nt128 = (int)((n + TM - 1) / TM), nc64 = (int)((n + TN - 1) / TN);
  int npair = 0;
  for (int ti = 0; ti < nt128; ++ti) npair += nc64 - 2 * ti;
  const int mode = (R == 1) ? LM_IC1 : ((R % 8 == 0) ? LM_KC8 : LM_GEN);
  const int64_t ktiles = (K + KT - 1) / KT;
  // at most one CTA per SM over all tiles (one wave), at least two windows per CTA
  int64_t want = g_nsm / npair;
  if (want < 1) want = 1;
  int64_t tpc = (ktiles + want - 1) / want;
  if (tpc < 2 * FLUSH) tpc = 2 * FLUSH;
  int nsplit = (int)((ktiles + tpc - 1) / tpc);
  if (nsplit < 1) nsplit = 1;
  if (!xs) ATC_TRY(slice_scale(x, dtype, K * n, s, &xs));
  const bool bf16 = (precision == ATC_PREC_SPLIT_BF16);
  if (!encode_fn() && nslice == 4) return fail(ATC_EUNSUP, "four-slice Gram needs cuTensorMapEncodeTiled");
  // FP32, three slices, tensor-map geometry: the unfolding tiles come straight
  // from the tensor by TMA and are sliced in the kernel
  if (encode_fn() && !gram_tma_off() && nslice == 3 && dtype == ATC_F32 && ((uintptr_t)x & 15u) == 0 &&
      ((R == 1 && n % 4 == 0) || (R > 1 && R % kRawHalf == 0))) {
    CUtensorMap ma, mb;
    int rc = ATC_OK;
    if (R == 1) {
      const int64_t dims[2] = {n, L}, strides[1] = {n * 4};
      const uint32_t boxa[2] = {(uint32_t)TM, (uint32_t)kRawHalf}, boxb[2] = {(uint32_t)TN, (uint32_t)kRawHalf};
      rc = make_raw_map_f32(&ma, x, 2, dims, strides, boxa);
      if (!rc) rc = make_raw_map_f32(&mb, x, 2, dims, strides, boxb);
    } else {
      const int64_t dims[3] = {R, n, L}, strides[2] = {R * 4, R * n * 4};
      const uint32_t boxa[3] = {(uint32_t)kRawHalf, (uint32_t)TM, 1u}, boxb[3] = {(uint32_t)kRawHalf, (uint32_t)TN, 1u};
      rc = make_raw_map_f32(&ma, x, 3, dims, strides, boxa);
      if (!rc) rc = make_raw_map_f32(&mb, x, 3, dims, strides, boxb);
    }
    if (rc == ATC_OK) {
      GramRawArgs ra;
      ra.R = R;
      ra.kchunk = tpc * KT;
      ra.Kp = ktiles * KT;
      ra.nsplit = nsplit;
      ra.nc64 = nc64;
      ra.npair = npair;
      ra.xs = xs;
      const size_t part_elems = (size_t)nsplit * npair * TM * TN;
      ATC_TRY(Scratch::get(SLOT_GRAM_PART, part_elems * 8 + 1024, (void**)&ra.part));
      int* err = nullptr;
      ATC_TRY(tc_error_flag(&err));
      ra.err = err;
      const int grid = npair * nsplit;
      static bool attr_b = false, attr_h = false;
      bool& attr = bf16 ? attr_b : attr_h;
      if (!attr) {
        ATC_CUDA_TRY(cudaFuncSetAttribute(bf16 ? gram_raw_kernel<true> : gram_raw_kernel<false>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, kRawSmem));
        attr = true;
      }
      // algorithmic work: the tensor read once, the split partials written
      // once, n^2 K multiply-adds; issued: nine slice products per 128 x 64 tile
      const double gb = 4.0 * (double)n * (double)K + (double)part_elems * 8.0;
      const double gf = (double)n * (double)n * (double)K;
      const double gi = 9.0 * 2.0 * TM * TN * (double)ra.Kp * (double)npair;
      {
        KTimed kt_(s, "gram_raw_kernel", gb, gf, gi);
        if (bf16) gram_raw_kernel<true><<<grid, kRawThreads, kRawSmem, s>>>(ma, mb, ra);
        else gram_raw_kernel<false><<<grid, kRawThreads, kRawSmem, s>>>(ma, mb, ra);
      }
      ATC_LAUNCHED(1);
      const int64_t tot = n * n;
      const int rb = (int)((tot + 255) / 256 < 2048 ? (tot + 255) / 256 : 2048);
      {
        KTimed kt_(s, "gram_tc_assemble", (double)part_elems * 8.0 + (double)n * (double)n * 8.0);
        gram_tc_assemble<<<rb, 256, 0, s>>>(ra.part, nsplit, npair, nc64, n, xs, g);
      }
      ATC_LAUNCHED(1);
      return ATC_OK;
    }
    cudaGetLastError();  // no map: the pre-sliced path below
  }
  if (encode_fn() && (!gram_tma_off() || nslice == 4)) {
    // pre-sliced planes + TMA-fed tensor-core Gram
    const int64_t Kp = ktiles * KT;
    uint16_t* planes = nullptr;
    ATC_TRY(Scratch::get(SLOT_SLICES, (size_t)nslice * n * Kp * 2 + 1024, (void**)&planes));
    Planes pl;
    for (int q = 0; q < 4; ++q) pl.p[q] = planes + (q < nslice ? q : 0) * n * Kp;
    if (dtype == ATC_F32) {
      const float* xf = (const float*)x;
      if (nslice == 3) bf16 ? launch_slices<float, true, 3>(xf, n, R, K, Kp, xs, pl, s)
                            : launch_slices<float, false, 3>(xf, n, R, K, Kp, xs, pl, s);
      else bf16 ? launch_slices<float, true, 4>(xf, n, R, K, Kp, xs, pl, s)
                : launch_slices<float, false, 4>(xf, n, R, K, Kp, xs, pl, s);
    } else {
      const double* xd = (const double*)x;
      if (nslice == 3) bf16 ? launch_slices<double, true, 3>(xd, n, R, K, Kp, xs, pl, s)
                            : launch_slices<double, false, 3>(xd, n, R, K, Kp, xs, pl, s);
      else bf16 ? launch_slices<double, true, 4>(xd, n, R, K, Kp, xs, pl, s)
                : launch_slices<double, false, 4>(xd, n, R, K, Kp, xs, pl, s);
    }
    ATC_LAUNCHED(1);
    GramMaps maps;
    for (int q = 0; q < 4; ++q) {
      ATC_TRY(make_map(&maps.a[q], pl.p[q], n, Kp, TM, bf16));
      ATC_TRY(make_map(&maps.b[q], pl.p[q], n, Kp, TN, bf16));
    }
    GramTmaArgs ta;
    ta.kchunk = tpc * KT;
    ta.Kp = Kp;
    ta.nsplit = nsplit;
    ta.nc64 = nc64;
    ta.npair = npair;
    const size_t part_elems = (size_t)nsplit * npair * TM * TN;
    ATC_TRY(Scratch::get(SLOT_GRAM_PART, part_elems * 8 + 1024, (void**)&ta.part));
    int* err = nullptr;
    ATC_TRY(tc_error_flag(&err));
    ta.err = err;
    const int grid = npair * nsplit;
    // algorithmic work of this kernel: every plane element read once, the
    // split partials written once; the SYRK's n^2 K FLOPs (unique half, as
    // multiply-adds); issued: all slice products over the 128 x 64 tiles
    const double gb = (double)nslice * 2.0 * (double)n * (double)Kp + (double)part_elems * 8.0;
    const double gf = (double)n * (double)n * (double)K;
    const double gi = (nslice == 3 ? 9.0 : 13.0) * 2.0 * TM * TN * (double)Kp * (double)npair;
    if (nslice == 3)
      ATC_TRY((bf16 ? launch_gram_tma<true, 3>(maps, ta, grid, s, gb, gf, gi) : launch_gram_tma<false, 3>(maps, ta, grid, s, gb, gf, gi)));
    else
      ATC_TRY((bf16 ? launch_gram_tma<true, 4>(maps, ta, grid, s, gb, gf, gi) : launch_gram_tma<false, 4>(maps, ta, grid, s, gb, gf, gi)));
    ATC_LAUNCHED(1);
    const int64_t tot = n * n;
    const int rb = (int)((tot + 255) / 256 < 2048 ? (tot + 255) / 256 : 2048);
    {
      KTimed kt_(s, "gram_tc_assemble", (double)part_elems * 8.0 + (double)n * (double)n * 8.0);
      gram_tc_assemble<<<rb, 256, 0, s>>>(ta.part, nsplit, npair, nc64, n, xs, g);
    }
    ATC_LAUNCHED(1);
    return ATC_OK;
  }
  GramArgs a;
  a.x = x;
  a.n = n;
  a.R = R;
  a.K = K;
  a.kchunk = tpc * KT;
  a.nsplit = nsplit;
  a.nt128 = nt128;
  a.nc64 = nc64;
  a.npair = npair;
  a.mode = mode;
  a.xs = xs;
  const size_t part_elems = (size_t)nsplit * npair * TM * TN;
  ATC_TRY(Scratch::get(SLOT_GRAM_PART, part_elems * 8 + 1024, (void**)&a.part));
  int* err = nullptr;
  ATC_TRY(tc_error_flag(&err));
  a.err = err;
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
  gram_tc_assemble<<<rb, 256, 0, s>>>(a.part, nsplit, npair, nc64, n, xs, g);
  ATC_LAUNCHED(1);
  return ATC_OK;
}

}  // namespace atc
