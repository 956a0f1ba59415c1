// Core quantization, exact bit-plane tracking, breakpoint and block encoding.
//
// Section 3.3: scale by 2^k with 2^63 <= 2^k max|b| < 2^64, round to the nearest
//   integer (ties to even); bit planes from 63 downward, bit by bit in
//   vectorised order, tracking the error of encoding every bit so far; the
//   breakpoint is the first bit whose tracked error is <= the target.
//   Leading bits (up to a coefficient's first 1) are run-length coded per
//   plane, signs of newly significant coefficients and trailing bits are raw.
// Section 4.2: contiguous blocks encoded independently + a size table.
// Section 4.3: a coefficient known down to plane p is rebuilt as a~ + 2^(p-1);
//   the tracker uses the same reconstruction.
// Supplement S.6: run lengths are range-ANS coded (static per-plane tables).
//
// Tracking is exact: per-coefficient errors are integers < 2^128 (units of
// 2^-2k), per-plane sums are 192-bit two's-complement integers, so the
// breakpoint is independent of the reduction order.  Per plane p the tracker
// needs S_p = sum_i D_i(p) and the largest prefix sum M_p of
// D_i(p) = e_i(p+1) - e_i(p); segments combine as
// (S1, M1) + (S2, M2) = (S1 + S2, max(M1, S1 + M2)), an associative
// (order-preserving) reduction.  The first plane with E(p+1) - M_p <= T holds
// the breakpoint.
//
// Supplement S.3 (split bit-plane truncation): on the last plane p_star the
//   leading bits (coefficients not yet significant) and the trailing bits
//   (significant ones) get breakpoints of their own, i_lead and i_trail.  The
//   category with the higher efficiency (exact SSE reduction / encoded bits)
//   on plane p_star + 1 goes first: the walk takes its bits in coefficient
//   order, then those of the other category, and stops at the first bit whose
//   tracked error is <= the target.  p_star itself comes from the walk in
//   coefficient order; when the split walk does not reach the target on that
//   plane, i_lead = i_trail = i_star.
//
// Stream section "ATCQ" (little-endian):
//   char[4] "ATCQ" | u32 2 | u64 n | i32 k | u32 block_size | i32 p_star |
//   u32 priority (0 leading first, 1 trailing first) | u64 i_lead | u64 i_trail |
//   u32 nplanes | u32 17 | u16 freq[nplanes][17] |
//   u32 sizes[nblocks][nplanes][2] (rANS bytes, raw bytes) | payload
//   (per block, per plane 63 .. p_star: rANS bytes then raw bytes).
// Run r >= 0 -> symbol s = floor(log2(r+1)) coded with the plane's table, then
// s extra bits (r + 1 - 2^s) coded as a uniform symbol; 32-bit rANS state,
// L = 2^23, byte-wise renormalisation, 12-bit frequencies.
#include <limits.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <string>
#include <mutex>
#include <vector>

#include "atc_internal.cuh"

namespace atc {
namespace {

typedef unsigned __int128 u128;
constexpr int kNsym = 17;
constexpr int kScaleBits = 12;
constexpr uint32_t kM = 1u << kScaleBits;
constexpr uint32_t kRansL = 1u << 23;
constexpr int kPlaneChunk = 16;       // planes per tracker pass
constexpr int kPlaneGroup = 8;        // planes per load of each magnitude
constexpr int kSegBlocks = 304;       // 2 x 152 SMs
constexpr int kSegThreads = 256;
constexpr int kQHdr = 56;             // fixed part of the ATCQ header

// ------------------------------------------------------------ 192-bit signed
struct I192 {
  uint64_t w0, w1, w2;
};
__host__ __device__ __forceinline__ I192 i192_zero() { return {0, 0, 0}; }
__host__ __device__ __forceinline__ I192 i192_from_u128(u128 v) { return {(uint64_t)v, (uint64_t)(v >> 64), 0}; }
__host__ __device__ __forceinline__ I192 i192_add(I192 a, I192 b) {
  I192 r;
  u128 s = (u128)a.w0 + b.w0;
  r.w0 = (uint64_t)s;
  s = (u128)a.w1 + b.w1 + (uint64_t)(s >> 64);
  r.w1 = (uint64_t)s;
  r.w2 = a.w2 + b.w2 + (uint64_t)(s >> 64);
  return r;
}
__host__ __device__ __forceinline__ I192 i192_neg(I192 a) {
  I192 r = {~a.w0, ~a.w1, ~a.w2};
  return i192_add(r, {1, 0, 0});
}
__host__ __device__ __forceinline__ I192 i192_sub(I192 a, I192 b) { return i192_add(a, i192_neg(b)); }
__host__ __device__ __forceinline__ bool i192_lt(I192 a, I192 b) {  // signed
  if (a.w2 != b.w2) return (int64_t)a.w2 < (int64_t)b.w2;
  if (a.w1 != b.w1) return a.w1 < b.w1;
  return a.w0 < b.w0;
}
__host__ __device__ __forceinline__ bool i192_le(I192 a, I192 b) { return !i192_lt(b, a); }
// (u128 a) - (u128 b) as a signed 192-bit value
__host__ __device__ __forceinline__ I192 i192_diff(u128 a, u128 b) { return i192_sub(i192_from_u128(a), i192_from_u128(b)); }

// Ordered segment summary of one plane: sum and largest prefix sum.
struct Seg {
  I192 s, m;
  int empty;
};
__device__ __forceinline__ Seg seg_combine(const Seg& a, const Seg& b) {
  if (a.empty) return b;
  if (b.empty) return a;
  Seg r;
  r.s = i192_add(a.s, b.s);
  I192 t = i192_add(a.s, b.m);
  r.m = i192_lt(a.m, t) ? t : a.m;
  r.empty = 0;
  return r;
}

// Error of one coefficient once every plane >= p is known (p in [0, 64]).
__device__ __forceinline__ u128 coef_err(uint64_t q, int p) {
  if (p >= 64 || (q >> p) == 0) return (u128)q * q;
  if (p == 0) return 0;
  const uint64_t rem = q & ((1ull << p) - 1ull);
  const uint64_t c = 1ull << (p - 1);
  const uint64_t d = (rem >= c) ? rem - c : c - rem;
  return (u128)d * d;
}

// D(p) = e(p+1) - e(p): the error reduction of coefficient v's bit on plane p
// (signed; zero while v is zero through plane p), without forming either
// square.  With c = 2^(p-1) and r = v mod 2^p:
//   leading bit (v < 2^(p+1)):  q^2 - (r - c)^2 = 3c (c + 2r)
//   trailing bit 1:  r^2 - (r - c)^2      = c (2r - c)
//   trailing bit 0:  (2c - r)^2 - (r - c)^2 = c (3c - 2r)
// (the reconstruction of Section 4.3; plane 0, where c is not an integer,
// takes the two squares).  |D| < 2^128 (leading), < 2^126 (trailing).
__device__ __forceinline__ I192 plane_reduction(uint64_t v, int p) {
  if ((v >> p) == 0) return i192_zero();
  if (p == 0) return i192_diff(coef_err(v, 1), coef_err(v, 0));
  const uint64_t c = 1ull << (p - 1);
  const uint64_t r = v & ((c << 1) - 1ull);
  const bool above = (p < 63) && ((v >> (p + 1)) != 0);
  if (!above) return i192_from_u128(((u128)3 * ((u128)c + 2 * (u128)r)) << (p - 1));
  const bool bit = (v >> p) & 1ull;
  const __int128 base = bit ? (__int128)2 * r - (__int128)c : (__int128)3 * c - (__int128)2 * r;
  const I192 m = i192_from_u128((u128)(base < 0 ? -base : base) << (p - 1));
  return base < 0 ? i192_neg(m) : m;
}
// The same reduction with the power of two taken out: D_i(p) = x * 2^(p-1) for
// p >= 1 (x * 2^0 at plane 0), x an integer with |x| < 15 * 2^(p-1):
//   leading 3 (c + 2r), trailing 1: 2r - c, trailing 0: 3c - 2r.
// X = int64_t holds x for p <= 60, __int128 for every plane.  Sums of x over a
// thread's range are shifted back once, by plane_shift(p), when they leave it.
template <typename X>
__device__ __forceinline__ X plane_factor(uint64_t v, int p) {
  if ((v >> p) == 0) return (X)0;
  if (p == 0) return (v == 1 || (v & 1ull) == 0) ? (X)1 : (X)0;
  const uint64_t c = 1ull << (p - 1);
  const uint64_t r = v & ((c << 1) - 1ull);
  if (p == 63 || (v >> (p + 1)) == 0) return (X)3 * ((X)c + (X)2 * (X)r);
  return ((v >> p) & 1ull) ? (X)2 * (X)r - (X)c : (X)3 * (X)c - (X)2 * (X)r;
}
__device__ __forceinline__ int plane_shift(int p) { return p > 0 ? p - 1 : 0; }
// v * 2^sh as a signed 192-bit value (|v| < 2^127, sh <= 63)
__device__ __forceinline__ I192 i192_from_i128_shl(__int128 v, int sh) {
  const bool neg = v < 0;
  const u128 u = neg ? (u128)0 - (u128)v : (u128)v;
  const uint64_t lo = (uint64_t)u, hi = (uint64_t)(u >> 64);
  I192 r;
  if (sh == 0) r = {lo, hi, 0ull};
  else r = {lo << sh, (hi << sh) | (lo >> (64 - sh)), hi >> (64 - sh)};
  return neg ? i192_neg(r) : r;
}
// ceil(v / 2^sh) of a signed 192-bit v as a 128-bit integer, saturated to
// [-(2^126), 2^126] (a first-passage threshold: a saturated one is out of reach
// of every sum it is compared with)
__device__ __forceinline__ __int128 i192_ceil_shr(I192 v, int sh) {
  const bool neg = (int64_t)v.w2 < 0;
  if (neg) v = i192_neg(v);
  // |v| >> sh, and whether bits were dropped
  uint64_t w0 = v.w0, w1 = v.w1, w2 = v.w2;
  bool frac = false;
  if (sh > 0) {
    frac = (w0 << (64 - sh)) != 0;
    w0 = (w0 >> sh) | (w1 << (64 - sh));
    w1 = (w1 >> sh) | (w2 << (64 - sh));
    w2 >>= sh;
  }
  const __int128 cap = (__int128)1 << 126;
  if (w2 != 0 || (w1 >> 62) != 0) return neg ? -cap : cap;
  __int128 r = (__int128)(((u128)w1 << 64) | w0);
  // ceil of v / 2^sh: up for a positive v with dropped bits, truncation for a negative one
  if (!neg) return frac ? r + 1 : r;
  return -r;
}
template <typename A>
__device__ __forceinline__ A acc_lowest();
template <>
__device__ __forceinline__ int64_t acc_lowest<int64_t>() { return INT64_MIN; }
template <>
__device__ __forceinline__ __int128 acc_lowest<__int128>() { return (__int128)((u128)1 << 127); }

__device__ __forceinline__ uint64_t shfl_down_u64(uint64_t v, int d) { return __shfl_down_sync(0xffffffffu, v, d); }

__device__ Seg warp_seg_reduce(Seg x) {
  // ordered tree: lane i combines with lane i + off (i is the left operand)
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    Seg o;
    o.s.w0 = shfl_down_u64(x.s.w0, off);
    o.s.w1 = shfl_down_u64(x.s.w1, off);
    o.s.w2 = shfl_down_u64(x.s.w2, off);
    o.m.w0 = shfl_down_u64(x.m.w0, off);
    o.m.w1 = shfl_down_u64(x.m.w1, off);
    o.m.w2 = shfl_down_u64(x.m.w2, off);
    o.empty = __shfl_down_sync(0xffffffffu, x.empty, off);
    const int lane = threadIdx.x & 31;
    if ((lane & (2 * off - 1)) == 0 && lane + off < 32) x = seg_combine(x, o);
  }
  return x;
}

// --------------------------------------------------------------- quantizer
__global__ void maxabs_kernel(const double* __restrict__ b, int64_t n, unsigned long long* __restrict__ out) {
  double m = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double a = fabs(b[i]);
    if (!(a <= m)) m = a;  // NaN propagates
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    double t = __shfl_xor_sync(0xffffffffu, m, o);
    if (!(t <= m)) m = t;
  }
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));  // |x| bit patterns order like values
}

// 2^k * a for a >= 0 with k in [-1074, 1138]; exact whenever the result is normal
__device__ __forceinline__ double mul_pow2(double a, int k) {
  if (k > 1023) return (a * __longlong_as_double((int64_t)(k - 1023 + 1023) << 52)) * 0x1p1023;
  if (k < -1022) return (a * 0x1p-1022) * __longlong_as_double((int64_t)(k + 1022 + 1023) << 52);
  return a * __longlong_as_double((int64_t)(k + 1023) << 52);
}

__global__ void quantize_kernel(const double* __restrict__ b, int64_t n, const int* __restrict__ kp,
                                uint64_t* __restrict__ q, uint8_t* __restrict__ sg) {
  const int k = *kp;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = b[i];
    q[i] = __double2ull_rn(mul_pow2(fabs(v), k));
    sg[i] = signbit(v) ? 1 : 0;
  }
}

struct TrackState {
  // device scalars
  int k;
  int nan;
  int p_star;
  int found;
  int64_t i_star;
  I192 t_int;     // floor(target * 2^(2k)), valid if reachable
  int reachable;
  int pad;
  I192 e_next;    // E(p+1) for the next unexamined plane
  I192 e64;
  I192 e_star;    // tracked error at the breakpoint
  I192 e_plane;   // E(p_star + 1)
  int prio;       // split truncation of plane p_star: 0 leading first, 1 trailing first
  int split_hit;  // the split walk reached the target on plane p_star
  int64_t i_lead, i_trail;
};

__global__ void scale_exp_kernel(const unsigned long long* __restrict__ mx, double target, TrackState* st) {
  if (threadIdx.x != 0) return;
  const double m = __longlong_as_double((long long)*mx);
  int k = 0;
  st->nan = !(m == m) || isinf(m);
  if (m > 0.0 && !st->nan) {
    int e;
    frexp(m, &e);
    k = 64 - e;
  }
  st->k = k;
  // T_int = floor(target * 2^(2k)) as 192-bit (target < 0: unreachable)
  I192 t = i192_zero();
  int reach = 0;
  if (target >= 0.0) {
    reach = 1;
    if (isinf(target)) {
      t = {~0ull, ~0ull, 0x7fffffffffffffffull};
    } else if (target > 0.0) {
      int e;
      double f = frexp(target, &e);
      uint64_t mant = (uint64_t)(f * 9007199254740992.0);  // f * 2^53, exact
      int sh = e - 53 + 2 * k;
      if (sh >= 0) {
        if (sh + 53 > 190) {
          t = {~0ull, ~0ull, 0x7fffffffffffffffull};
        } else {
          int limb = sh / 64, bit = sh % 64;
          uint64_t w[3] = {0, 0, 0};
          w[limb] = mant << bit;
          if (bit && limb + 1 < 3) w[limb + 1] = mant >> (64 - bit);
          t = {w[0], w[1], w[2]};
        }
      } else {
        int r = -sh;
        t = {r >= 64 ? 0ull : (mant >> r), 0, 0};
      }
    }
  }
  st->t_int = t;
  st->reachable = reach;
  st->found = 0;
  st->p_star = -1;
}

__device__ __forceinline__ __int128 shfl_down_i128(__int128 v, int d) {
  const uint64_t lo = shfl_down_u64((uint64_t)(u128)v, d), hi = shfl_down_u64((uint64_t)((u128)v >> 64), d);
  return (__int128)(((u128)hi << 64) | lo);
}

// One group of up to kPlaneGroup planes (pg down to max(plo, pg - 7)) over
// the thread range [t_lo, t_hi): per plane the running sum of the factors x
// (plane_factor) and its largest prefix, in X / A integers; then per plane an
// ordered warp tree in 128 bits (an empty range: sum 0, largest prefix kNone,
// far below any real prefix, so that combining with it changes nothing), and
// one thread per plane combining the warps in order, shifted back to
// D = x * 2^(p-1).  wsum: kPlaneGroup x (kSegThreads / 32) summaries.
template <typename X, typename A>
__device__ __forceinline__ void plane_group(const uint64_t* __restrict__ q, int64_t t_lo, int64_t t_hi, int pg, int plo,
                                            int phi, Seg* wsum, Seg* __restrict__ out) {
  constexpr int kW = kSegThreads / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  A s[kPlaneGroup], m[kPlaneGroup];
#pragma unroll
  for (int k = 0; k < kPlaneGroup; ++k) {
    s[k] = (A)0;
    m[k] = acc_lowest<A>();
  }
  const int pgl = max(plo, pg - kPlaneGroup + 1);  // lowest plane of this group
  for (int64_t i = t_lo; i < t_hi; ++i) {
    const uint64_t v = q[i];
    // zero through every plane of the group: x = 0 there, which leaves the sum
    // and (once the first element has set it) the largest prefix unchanged
    if ((v >> pgl) == 0 && i != t_lo) continue;
#pragma unroll
    for (int k = 0; k < kPlaneGroup; ++k) {
      const int p = pg - k;
      if (p >= pgl) {
        s[k] += (A)plane_factor<X>(v, p);
        if (m[k] < s[k]) m[k] = s[k];
      }
    }
  }
  const bool empty = t_lo >= t_hi;
  const __int128 kNone = -((__int128)1 << 126);
#pragma unroll
  for (int k = 0; k < kPlaneGroup; ++k) {
    const int p = pg - k;
    if (p < pgl) break;
    __int128 ws = empty ? (__int128)0 : (__int128)s[k];
    __int128 wm = empty ? kNone : (__int128)m[k];
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const __int128 os = shfl_down_i128(ws, off), om = shfl_down_i128(wm, off);
      if ((lane & (2 * off - 1)) == 0 && lane + off < 32) {
        const __int128 t = ws + om;
        if (wm < t) wm = t;
        ws += os;
      }
    }
    if (lane == 0) {
      Seg r;
      r.empty = wm <= kNone / 2;
      r.s = r.empty ? i192_zero() : i192_from_i128_shl(ws, plane_shift(p));
      r.m = r.empty ? i192_zero() : i192_from_i128_shl(wm, plane_shift(p));
      wsum[k * kW + warp] = r;
    }
  }
  __syncthreads();
  if (threadIdx.x < kPlaneGroup && pg - (int)threadIdx.x >= pgl) {
    const int k = threadIdx.x, p = pg - k;
    Seg t = wsum[k * kW];
    for (int w = 1; w < kW; ++w) t = seg_combine(t, wsum[k * kW + w]);
    out[(int64_t)(phi - p) * gridDim.x + blockIdx.x] = t;
  }
  __syncthreads();
}

// Per segment (one CTA, contiguous coefficients) and plane p in [plo, phi]
// (at most kPlaneChunk planes): the ordered summary of D_i(p); plus sum q_i^2
// when first_pass.  Planes above 60 take 128-bit factors; below, 64-bit
// factors, summed in 64 bits where a thread range cannot overflow them.
__global__ void __launch_bounds__(kSegThreads, 2) plane_stats_kernel(const uint64_t* __restrict__ q, int64_t n,
                                                                   int64_t seg_len, int plo, int phi, int first_pass,
                                                                   Seg* __restrict__ out, I192* __restrict__ e64_out) {
  __shared__ Seg wsum[kPlaneGroup * (kSegThreads / 32)];
  const int64_t s_lo = blockIdx.x * seg_len;
  const int64_t s_hi = min(n, s_lo + seg_len);
  const int64_t per = (seg_len + blockDim.x - 1) / blockDim.x;
  const int64_t t_lo = min(s_hi, s_lo + threadIdx.x * per);
  const int64_t t_hi = min(s_hi, t_lo + per);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (first_pass) {
    Seg a;
    a.s = i192_zero();
    a.m = i192_zero();
    a.empty = (t_lo >= t_hi);
    for (int64_t i = t_lo; i < t_hi; ++i) a.s = i192_add(a.s, i192_from_u128((u128)q[i] * q[i]));
    a.m = a.s;
    Seg r = warp_seg_reduce(a);
    if (lane == 0) wsum[warp] = r;
    __syncthreads();
    if (threadIdx.x == 0) {
      Seg t = wsum[0];
      for (int w = 1; w < (int)(blockDim.x >> 5); ++w) t = seg_combine(t, wsum[w]);
      e64_out[blockIdx.x] = t.empty ? i192_zero() : t.s;
    }
    __syncthreads();
  }
  // bits of the longest thread range: |sum x| < per * 15 * 2^(pg-1) < 2^(lb + pg + 3)
  const int lb = per > 0 ? 64 - __clzll((unsigned long long)per) : 0;
  for (int pg = phi; pg >= plo; pg -= kPlaneGroup) {
    if (pg > 60) plane_group<__int128, __int128>(q, t_lo, t_hi, pg, plo, phi, wsum, out);
    else if (lb + pg + 3 <= 63) plane_group<int64_t, int64_t>(q, t_lo, t_hi, pg, plo, phi, wsum, out);
    else plane_group<int64_t, __int128>(q, t_lo, t_hi, pg, plo, phi, wsum, out);
  }
}

// Combine the segment summaries in order and look for the first plane whose
// lowest running error reaches the target.  One warp per plane: each lane
// folds a contiguous run of segments, then an ordered warp tree combines the
// lanes; thread 0 then walks the planes from the top.
__global__ void __launch_bounds__(32 * kPlaneChunk) plane_scan_kernel(const Seg* __restrict__ segs,
                                                                      const I192* __restrict__ e64_seg, int nseg,
                                                                      int plo, int phi, int first_pass, TrackState* st) {
  __shared__ Seg plane_sum[kPlaneChunk];
  __shared__ I192 e64_sh;
  if (st->found) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int per = (nseg + 31) / 32;
  const int b0 = min(nseg, lane * per), b1 = min(nseg, b0 + per);
  const int p = phi - warp;
  if (p >= plo) {
    Seg t;
    t.empty = 1;
    t.s = t.m = i192_zero();
    for (int b = b0; b < b1; ++b) t = seg_combine(t, segs[(int64_t)(phi - p) * nseg + b]);
    t = warp_seg_reduce(t);
    if (lane == 0) plane_sum[warp] = t;
  }
  if (first_pass && warp == 0) {
    I192 e = i192_zero();
    for (int b = b0; b < b1; ++b) e = i192_add(e, e64_seg[b]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      I192 o;
      o.w0 = __shfl_down_sync(0xffffffffu, e.w0, off);
      o.w1 = __shfl_down_sync(0xffffffffu, e.w1, off);
      o.w2 = __shfl_down_sync(0xffffffffu, e.w2, off);
      if (lane < off) e = i192_add(e, o);
    }
    if (lane == 0) e64_sh = e;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  if (first_pass) {
    const I192 e = e64_sh;
    st->e64 = e;
    st->e_next = e;
    if (st->reachable && i192_le(e, st->t_int)) {
      st->found = 1;
      st->p_star = 64;
      st->i_star = -1;  // fixed up by the host to n-1
      st->e_star = e;
      st->e_plane = e;
      return;
    }
  }
  I192 e_next = st->e_next, e_prev = e_next;
  for (int q = phi; q >= plo; --q) {
    Seg t = plane_sum[phi - q];
    if (t.empty) { t.s = t.m = i192_zero(); }
    const I192 lowest = i192_sub(e_next, t.m);
    if (st->reachable && i192_le(lowest, st->t_int)) {
      st->found = 1;
      st->p_star = q;
      st->e_plane = e_next;
      return;
    }
    e_prev = e_next;
    e_next = i192_sub(e_next, t.s);
  }
  st->e_next = e_next;
  if (plo == 0) {  // target not reached in coefficient order: everything encoded
    st->found = 1;
    st->p_star = 0;
    st->i_star = -1;
    st->e_star = e_next;
    st->e_plane = e_prev;  // E(1): the split walk of plane 0 starts there
  }
}

// Exact position of the breakpoint inside plane p_star: one CTA walks the
// segment summaries, then re-scans the segment that holds it.
// Block-wide exclusive prefix sum of one I192 per thread (two's-complement
// sums mod 2^192, so any grouping gives the sequential result); *total gets the
// sum over the block.  Three barriers.
constexpr int kIstarThreads = 512;  // >= kSegBlocks: one segment per thread
__device__ I192 i192_block_exscan(I192 v, I192* sh, I192* total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  I192 inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    I192 u;
    u.w0 = __shfl_up_sync(0xffffffffu, inc.w0, o);
    u.w1 = __shfl_up_sync(0xffffffffu, inc.w1, o);
    u.w2 = __shfl_up_sync(0xffffffffu, inc.w2, o);
    if (lane >= o) inc = i192_add(inc, u);
  }
  __syncthreads();
  if (lane == 31) sh[w] = inc;
  __syncthreads();
  if (w == 0) {
    I192 x = (lane < nw) ? sh[lane] : i192_zero();
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      I192 u;
      u.w0 = __shfl_up_sync(0xffffffffu, x.w0, o);
      u.w1 = __shfl_up_sync(0xffffffffu, x.w1, o);
      u.w2 = __shfl_up_sync(0xffffffffu, x.w2, o);
      if (lane >= o) x = i192_add(x, u);
    }
    if (lane < nw) sh[lane] = x;  // inclusive prefix over the warps
  }
  __syncthreads();
  const I192 warp_pre = (w > 0) ? sh[w - 1] : i192_zero();
  *total = sh[nw - 1];
  return i192_add(warp_pre, i192_sub(inc, v));
}

// i* (the breakpoint inside plane p*): the first coefficient, in vectorised
// order, at which the tracked error falls to the target.  Three ordered
// first-passage searches, each an exclusive prefix sum over the block, a
// per-entry test and a minimum: over the plane's segment summaries, over the
// per-thread summaries inside the hit segment, then element by element inside
// the hit thread's range.
__global__ void __launch_bounds__(kIstarThreads) istar_kernel(const uint64_t* __restrict__ q, int64_t n, int64_t seg_len,
                                                              const Seg* __restrict__ segs, int nseg, int phi,
                                                              TrackState* st) {
  __shared__ I192 sh[32];
  __shared__ int s_first;
  __shared__ I192 s_pre;
  const int p = st->p_star;
  if (p >= 64) return;
  const I192 T = st->t_int;
  const I192 E1 = st->e_plane;
  if (!st->reachable) return;  // i_star stays -1 (everything encoded)
  const int tid = threadIdx.x;
  I192 tot;
  // 1. the first segment whose largest prefix reaches the target
  Seg sg;
  sg.empty = 1;
  sg.s = sg.m = i192_zero();
  if (tid < nseg) sg = segs[(int64_t)(phi - p) * nseg + tid];
  const I192 pre = i192_block_exscan(sg.empty ? i192_zero() : sg.s, sh, &tot);
  if (tid == 0) s_first = INT_MAX;
  __syncthreads();
  if (tid < nseg && !sg.empty && i192_le(i192_sub(E1, i192_add(pre, sg.m)), T)) atomicMin(&s_first, tid);
  __syncthreads();
  const int b = s_first;
  if (b == INT_MAX) return;  // cannot happen when p_star came from plane_scan_kernel
  if (tid == b) s_pre = pre;
  __syncthreads();
  const I192 seg_pre = s_pre;
  // 2. inside segment b: the first thread range that reaches it
  const int64_t s_lo = b * seg_len;
  const int64_t s_hi = min(n, s_lo + seg_len);
  const int64_t per = (seg_len + blockDim.x - 1) / blockDim.x;
  const int64_t t_lo = min(s_hi, s_lo + tid * per);
  const int64_t t_hi = min(s_hi, t_lo + per);
  const int sh_p = plane_shift(p);
  __int128 xs = 0, xm = acc_lowest<__int128>();
  if (p > 60) {
    for (int64_t i = t_lo; i < t_hi; ++i) {
      xs += plane_factor<__int128>(q[i], p);
      if (xm < xs) xm = xs;
    }
  } else {
    for (int64_t i = t_lo; i < t_hi; ++i) {
      xs += (__int128)plane_factor<int64_t>(q[i], p);
      if (xm < xs) xm = xs;
    }
  }
  Seg a;
  a.empty = t_lo >= t_hi;
  a.s = a.empty ? i192_zero() : i192_from_i128_shl(xs, sh_p);
  a.m = a.empty ? i192_zero() : i192_from_i128_shl(xm, sh_p);
  const I192 pre2 = i192_add(seg_pre, i192_block_exscan(a.empty ? i192_zero() : a.s, sh, &tot));
  if (tid == 0) s_first = INT_MAX;
  __syncthreads();
  if (!a.empty && i192_le(i192_sub(E1, i192_add(pre2, a.m)), T)) atomicMin(&s_first, tid);
  __syncthreads();
  // 3. element by element inside the hit thread's range: the first prefix of
  // factors reaching ceil((E1 - pre2 - T) / 2^(p-1)), which the range's largest
  // prefix does, so the threshold fits the 128-bit sum
  if (tid == s_first) {
    const I192 run0 = i192_sub(E1, pre2);
    const __int128 tau = i192_ceil_shr(i192_sub(run0, T), sh_p);
    __int128 acc = 0;
    for (int64_t i = t_lo; i < t_hi; ++i) {
      acc += (p > 60) ? plane_factor<__int128>(q[i], p) : (__int128)plane_factor<int64_t>(q[i], p);
      if (acc >= tau) {
        st->i_star = i;
        st->e_star = i192_sub(run0, i192_from_i128_shl(acc, sh_p));
        break;
      }
    }
  }
}

// ------------------------------------------------ split truncation (S.3)
// Reduction D_i(p) of the bit of coefficient v on plane p when it belongs to
// category cat of that plane (0 leading: not significant above p, 1 trailing:
// significant above p); zero for the other category and for a coefficient
// still zero through plane p.
__device__ __forceinline__ I192 cat_reduction(uint64_t v, int p, int cat) {
  if ((v >> p) == 0) return i192_zero();
  const int sig = (p == 63) ? 0 : ((v >> (p + 1)) != 0 ? 1 : 0);
  if (sig != cat) return i192_zero();
  return plane_reduction(v, p);
}

template <typename X>
__device__ __forceinline__ X cat_factor(uint64_t v, int p, int cat) {
  if ((v >> p) == 0) return (X)0;
  const int sig = (p == 63) ? 0 : ((v >> (p + 1)) != 0 ? 1 : 0);
  return sig == cat ? plane_factor<X>(v, p) : (X)0;
}

// Per segment of the tracker's segmentation: the ordered summaries of the
// reductions of plane p restricted to each category (prefix maxima taken over
// every prefix, the empty one included: a prefix value at a segment start is
// the running error already tested there), and for the priority the
// order-free totals of plane p + 1 -- the SSE reductions of its leading and
// trailing bits and their counts (leading ones, trailing bits).
struct SplitSeg {
  Seg c[2];
  I192 d[2];
  unsigned long long cnt[2];
};

__device__ Seg block_seg_reduce(Seg a, Seg* wsum) {
  Seg r = warp_seg_reduce(a);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) wsum[warp] = r;
  __syncthreads();
  Seg t = wsum[0];
  for (int w = 1; w < (int)(blockDim.x >> 5); ++w) t = seg_combine(t, wsum[w]);
  return t;  // valid in every thread
}

__device__ I192 warp_i192_sum(I192 e) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    I192 o;
    o.w0 = __shfl_down_sync(0xffffffffu, e.w0, off);
    o.w1 = __shfl_down_sync(0xffffffffu, e.w1, off);
    o.w2 = __shfl_down_sync(0xffffffffu, e.w2, off);
    e = i192_add(e, o);
  }
  return e;  // lane 0 holds the sum (other lanes: partial sums, mod 2^192)
}

template <typename X>
__device__ __forceinline__ void split_stats_range(const uint64_t* __restrict__ q, int64_t t_lo, int64_t t_hi, int p,
                                                  __int128 (&xs)[2], __int128 (&xm)[2], __int128 (&xd)[2],
                                                  unsigned long long (&c)[2]) {
  for (int64_t i = t_lo; i < t_hi; ++i) {
    const uint64_t v = q[i];
    if ((v >> p) == 0) continue;
    const bool sig = p < 63 && (v >> (p + 1)) != 0;
    const __int128 x = (__int128)plane_factor<X>(v, p);
    // only the category the bit belongs to moves; the other keeps its prefix
    if (sig) {
      xs[1] += x;
      if (xm[1] < xs[1]) xm[1] = xs[1];
      // plane p + 1: this coefficient's bit there is leading or trailing
      const __int128 x1 = (__int128)plane_factor<X>(v, p + 1);
      if (p + 1 < 63 && (v >> (p + 2)) != 0) { xd[1] += x1; ++c[1]; }
      else { xd[0] += x1; ++c[0]; }
    } else {
      xs[0] += x;
      if (xm[0] < xs[0]) xm[0] = xs[0];
    }
  }
}

__global__ void __launch_bounds__(kSegThreads) split_stats_kernel(const uint64_t* __restrict__ q, int64_t n,
                                                                   int64_t seg_len, int p, SplitSeg* __restrict__ out) {
  __shared__ Seg wsum[kSegThreads / 32];
  __shared__ I192 wd[2][kSegThreads / 32];
  __shared__ unsigned long long wc[2][kSegThreads / 32];
  const int64_t s_lo = blockIdx.x * seg_len;
  const int64_t s_hi = min(n, s_lo + seg_len);
  const int64_t per = (seg_len + blockDim.x - 1) / blockDim.x;
  const int64_t t_lo = min(s_hi, s_lo + threadIdx.x * per);
  const int64_t t_hi = min(s_hi, t_lo + per);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // factors of plane p per category (sum and largest prefix, the empty prefix
  // included) and of plane p + 1 per category (order-free sums)
  __int128 xs[2] = {0, 0}, xm[2] = {0, 0}, xd[2] = {0, 0};
  unsigned long long c[2] = {0ull, 0ull};
  if (p >= 60) split_stats_range<__int128>(q, t_lo, t_hi, p, xs, xm, xd, c);
  else split_stats_range<int64_t>(q, t_lo, t_hi, p, xs, xm, xd, c);
  Seg a[2];
  I192 d[2];
  for (int k = 0; k < 2; ++k) {
    a[k].empty = 0;
    a[k].s = i192_from_i128_shl(xs[k], plane_shift(p));
    a[k].m = i192_from_i128_shl(xm[k], plane_shift(p));
    d[k] = p <= 62 ? i192_from_i128_shl(xd[k], plane_shift(p + 1)) : i192_zero();
  }
  const Seg l = block_seg_reduce(a[0], wsum);
  const Seg t = block_seg_reduce(a[1], wsum);
  for (int k = 0; k < 2; ++k) {
    const I192 e = warp_i192_sum(d[k]);
    unsigned long long cc = c[k];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) cc += __shfl_down_sync(0xffffffffu, cc, off);
    if (lane == 0) { wd[k][warp] = e; wc[k][warp] = cc; }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    SplitSeg o;
    o.c[0] = l;
    o.c[1] = t;
    for (int k = 0; k < 2; ++k) {
      I192 e = i192_zero();
      unsigned long long cc = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { e = i192_add(e, wd[k][w]); cc += wc[k][w]; }
      o.d[k] = e;
      o.cnt[k] = cc;
    }
    out[blockIdx.x] = o;
  }
}

// 256-bit two's complement: (signed 192-bit) x (unsigned 64-bit), signed compare
struct I256 {
  uint64_t w[4];
};
__device__ I256 i256_mul(I192 a, uint64_t b) {
  const bool neg = (int64_t)a.w2 < 0;
  if (neg) a = i192_neg(a);
  I256 r;
  u128 t = (u128)a.w0 * b;
  r.w[0] = (uint64_t)t;
  t = (u128)a.w1 * b + (uint64_t)(t >> 64);
  r.w[1] = (uint64_t)t;
  t = (u128)a.w2 * b + (uint64_t)(t >> 64);
  r.w[2] = (uint64_t)t;
  r.w[3] = (uint64_t)(t >> 64);
  if (neg) {
    uint64_t carry = 1;
    for (int k = 0; k < 4; ++k) {
      const u128 x = (u128)(~r.w[k]) + carry;
      r.w[k] = (uint64_t)x;
      carry = (uint64_t)(x >> 64);
    }
  }
  return r;
}
__device__ bool i256_ge(const I256& a, const I256& b) {
  if (a.w[3] != b.w[3]) return (int64_t)a.w[3] > (int64_t)b.w[3];
  for (int k = 2; k >= 0; --k)
    if (a.w[k] != b.w[k]) return a.w[k] > b.w[k];
  return true;
}

struct SplitShared {
  I192 sh[32];
  I192 pre;
  int first;
  int hit;
  long long j;
  I192 run;
};

// First bit of category cat of plane p, in coefficient order, at which the
// running error (start minus the reductions so far) is <= T; returns its index
// or -1.  Three ordered first-passage searches as for i_star: over the
// segments' category summaries, over per-thread summaries inside the hit
// segment, then element by element.  *total: the category's whole reduction.
// Every thread of the block calls it.
__device__ int64_t split_first_passage(const uint64_t* __restrict__ q, int64_t n, int64_t seg_len,
                                       const SplitSeg* __restrict__ segs, int nseg, int p, int cat, I192 start, I192 T,
                                       SplitShared* S, I192* err_at, I192* total) {
  const int tid = threadIdx.x;
  Seg g;
  g.empty = 0;
  g.s = g.m = i192_zero();
  if (tid < nseg) g = segs[tid].c[cat];
  I192 tot;
  const I192 pre = i192_block_exscan(g.s, S->sh, &tot);
  *total = tot;
  if (tid == 0) { S->first = INT_MAX; S->hit = 0; }
  __syncthreads();
  if (tid < nseg && i192_le(i192_sub(start, i192_add(pre, g.m)), T)) atomicMin(&S->first, tid);
  __syncthreads();
  const int b = S->first;
  if (b == INT_MAX) return -1;
  if (tid == b) S->pre = pre;
  __syncthreads();
  const I192 seg_pre = S->pre;
  const int64_t s_lo = b * seg_len;
  const int64_t s_hi = min(n, s_lo + seg_len);
  const int64_t per = (seg_len + blockDim.x - 1) / blockDim.x;
  const int64_t t_lo = min(s_hi, s_lo + tid * per);
  const int64_t t_hi = min(s_hi, t_lo + per);
  const int sh_p = plane_shift(p);
  __int128 xs = 0, xm = 0;
  if (p > 60) {
    for (int64_t i = t_lo; i < t_hi; ++i) {
      xs += cat_factor<__int128>(q[i], p, cat);
      if (xm < xs) xm = xs;
    }
  } else {
    for (int64_t i = t_lo; i < t_hi; ++i) {
      xs += (__int128)cat_factor<int64_t>(q[i], p, cat);
      if (xm < xs) xm = xs;
    }
  }
  Seg a;
  a.empty = 0;
  a.s = i192_from_i128_shl(xs, sh_p);
  a.m = i192_from_i128_shl(xm, sh_p);
  I192 tot2;
  const I192 pre2 = i192_add(seg_pre, i192_block_exscan(a.s, S->sh, &tot2));
  if (tid == 0) S->first = INT_MAX;
  __syncthreads();
  if (i192_le(i192_sub(start, i192_add(pre2, a.m)), T)) atomicMin(&S->first, tid);
  __syncthreads();
  if (tid == S->first) {
    // the first prefix of factors reaching ceil((start - pre2 - T) / 2^(p-1))
    const I192 run0 = i192_sub(start, pre2);
    const __int128 tau = i192_ceil_shr(i192_sub(run0, T), sh_p);
    __int128 acc = 0;
    for (int64_t i = t_lo; i < t_hi; ++i) {
      acc += (p > 60) ? cat_factor<__int128>(q[i], p, cat) : (__int128)cat_factor<int64_t>(q[i], p, cat);
      if (acc >= tau) {
        S->j = i;
        S->run = i192_sub(run0, i192_from_i128_shl(acc, sh_p));
        S->hit = 1;
        break;
      }
    }
  }
  __syncthreads();
  if (!S->hit) return -1;  // cannot happen: the hit thread holds the passage
  *err_at = S->run;
  return S->j;
}

// Priority and breakpoints of the last plane (one CTA of kIstarThreads):
// plane p + 1's efficiencies decide which category goes first (exact:
// d_lead * cost_trail >= d_trail * cost_lead, ties and empty categories leading
// first; cost_lead = 8 x its rANS bytes + one sign bit per leading 1,
// cost_trail = one bit per trailing bit); then the walk of the first
// category, and if it does not reach the target, the second one from the end
// of the first.  cost_rs: the rANS bytes of plane p + 1 per block.
__global__ void __launch_bounds__(kIstarThreads) split_kernel(const uint64_t* __restrict__ q, int64_t n, int64_t seg_len,
                                                              const SplitSeg* __restrict__ segs, int nseg, int p,
                                                              const uint32_t* __restrict__ cost_rs, int64_t ncost,
                                                              TrackState* st) {
  __shared__ SplitShared S;
  __shared__ unsigned long long s_rb;
  __shared__ int s_prio;
  const int tid = threadIdx.x;
  if (tid == 0) { s_rb = 0; s_prio = 0; }
  __syncthreads();
  if (p <= 62) {
    unsigned long long rb = 0;
    for (int64_t i = tid; i < ncost; i += blockDim.x) rb += cost_rs[i];
    atomicAdd(&s_rb, rb);
    I192 dl = i192_zero(), dt = i192_zero();
    unsigned long long ones = 0, trail = 0;
    if (tid < nseg) { dl = segs[tid].d[0]; dt = segs[tid].d[1]; ones = segs[tid].cnt[0]; trail = segs[tid].cnt[1]; }
    I192 tl, tt, tmp;
    i192_block_exscan(dl, S.sh, &tl);
    i192_block_exscan(dt, S.sh, &tt);
    i192_block_exscan({ones, 0, 0}, S.sh, &tmp);
    ones = tmp.w0;
    i192_block_exscan({trail, 0, 0}, S.sh, &tmp);
    trail = tmp.w0;
    __syncthreads();
    if (tid == 0) {
      const uint64_t cost_lead = 8ull * s_rb + ones, cost_trail = trail;
      s_prio = i256_ge(i256_mul(tl, cost_trail), i256_mul(tt, cost_lead)) ? 0 : 1;
    }
  }
  __syncthreads();
  const int first = s_prio;
  const int64_t i_std = (st->i_star < 0) ? n - 1 : st->i_star;
  int64_t il = i_std, it = i_std;
  int hit = 0;
  I192 err = st->e_star;
  if (st->reachable) {
    const I192 T = st->t_int, E1 = st->e_plane;
    I192 tot, e;
    const int64_t j1 = split_first_passage(q, n, seg_len, segs, nseg, p, first, E1, T, &S, &e, &tot);
    if (j1 >= 0) {
      hit = 1;
      err = e;
      il = first == 0 ? j1 : -1;
      it = first == 0 ? -1 : j1;
    } else {
      I192 tot2;
      const int64_t j2 = split_first_passage(q, n, seg_len, segs, nseg, p, 1 - first, i192_sub(E1, tot), T, &S, &e, &tot2);
      if (j2 >= 0) {
        hit = 1;
        err = e;
        il = first == 0 ? n - 1 : j2;
        it = first == 0 ? j2 : n - 1;
      }
    }
  }
  if (tid == 0) {
    st->prio = first;
    st->split_hit = hit;
    st->i_lead = il;
    st->i_trail = it;
    st->e_star = err;
  }
}

// -------------------------------------------------------------------- encoder
struct EncParams {
  const uint64_t* q;
  const uint8_t* sg;
  int64_t n;
  int block_size;
  int p_top;                 // first plane (63, or p_star + 1 for the cost of that plane alone)
  int p_star;                // last plane: leading bits up to i_lead, trailing bits up to i_trail
  int64_t i_lead, i_trail;
  int nplanes;
  int64_t nblocks;
  unsigned long long* hist;  // nplanes x 17
  const uint32_t* freq;      // nplanes x 17 (then cum at +nplanes*17)
  uint32_t* rsize;           // nchunks
  uint32_t* wsize;           // nchunks
  const uint64_t* off;       // nchunks + 1 (payload offsets)
  uint8_t* out;              // payload base
  uint32_t* table;           // size table (nblocks x nplanes x 2)
};

__device__ __forceinline__ int bucket_of(uint32_t v) { return 31 - __clz(v + 1u); }

// Warp walk of one (block, plane) chunk: leading bits of coefficients before
// hl, trailing bits of those before ht.  For every run (in order) calls
// on_run(run); raw bits are reported per 32-coefficient group as
// (packed value, count).  Returns via the callbacks only.
template <typename RunF, typename RawF>
__device__ __forceinline__ void chunk_walk(const EncParams& P, int64_t lo, int64_t hl, int64_t ht, int p, RunF on_run,
                                           RawF on_raw) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const int64_t hi = max(hl, ht);
  uint32_t carry = 0;  // zeros since the last 1 (leading subsequence)
  for (int64_t g = lo; g < hi; g += 32) {
    const int64_t j = g + lane;
    const bool in = j < hi;
    uint64_t v = in ? P.q[j] : 0;
    const bool bit = (v >> p) & 1ull;
    const bool sigb = (p == 63) ? false : ((v >> (p + 1)) != 0ull);
    const bool lead = in && !sigb && j < hl;
    const bool trail = in && sigb && j < ht;
    const bool one = lead && bit;
    const bool rawp = trail || one;
    const bool rawv = trail ? bit : (one ? (P.sg[j] != 0) : false);
    const unsigned lead_m = __ballot_sync(0xffffffffu, lead);
    const unsigned one_m = __ballot_sync(0xffffffffu, one);
    const unsigned raw_m = __ballot_sync(0xffffffffu, rawp);
    // raw bits packed in order of position
    const int rank = __popc(raw_m & lt);
    const unsigned packed = __reduce_or_sync(0xffffffffu, (rawp && rawv) ? (1u << rank) : 0u);
    on_raw(packed, __popc(raw_m));
    // runs: each 1 ends a run of the leading zeros since the previous 1
    const unsigned zero_m = lead_m & ~one_m;
    unsigned ones = one_m;
    while (ones) {
      const int l = __ffs(ones) - 1;
      ones &= ones - 1u;
      // zeros strictly before lane l since the previous processed 1 (tracked by carry)
      const unsigned below = (l == 0) ? 0u : ((1u << l) - 1u);
      const unsigned prevmask = one_m & below;
      unsigned from;
      uint32_t run;
      if (prevmask) {
        const int pl = 31 - __clz(prevmask);
        from = (pl == 31) ? 0u : ~((2u << pl) - 1u);
        run = __popc(zero_m & below & from);
      } else {
        run = carry + __popc(zero_m & below);
      }
      on_run(run);
    }
    if (one_m) {
      const int ll = 31 - __clz(one_m);
      const unsigned above = (ll == 31) ? 0u : ~((2u << ll) - 1u);
      carry = __popc(zero_m & above);
    } else {
      carry += __popc(zero_m);
    }
  }
  if (carry > 0) on_run(carry);
}

// end (exclusive) of the coefficients whose bit of plane p is encoded, for a
// breakpoint i of the last plane
__device__ __host__ __forceinline__ int64_t cat_end(int64_t lo, int64_t hi, int p, int p_star, int64_t i) {
  if (p == p_star && hi > i + 1) hi = i + 1;
  return hi < lo ? lo : hi;
}
__device__ __forceinline__ void chunk_range(const EncParams& P, int64_t blk, int p, int64_t* lo, int64_t* hl,
                                            int64_t* ht) {
  const int64_t a = blk * P.block_size, b = min(P.n, a + P.block_size);
  *lo = a;
  *hl = cat_end(a, b, p, P.p_star, P.i_lead);
  *ht = cat_end(a, b, p, P.p_star, P.i_trail);
}

// pass 1: per-plane histograms of run symbols and raw byte counts
__global__ void enc_hist_kernel(EncParams P) {
  const int64_t chunk = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int64_t nchunks = P.nblocks * P.nplanes;
  if (chunk >= nchunks) return;
  const int64_t blk = chunk / P.nplanes;
  const int pi = (int)(chunk % P.nplanes);
  const int p = P.p_top - pi;
  int64_t lo, hl, ht;
  chunk_range(P, blk, p, &lo, &hl, &ht);
  const int lane = threadIdx.x & 31;
  uint64_t rawbits = 0;
  unsigned long long* h = P.hist + pi * kNsym;
  chunk_walk(
      P, lo, hl, ht, p,
      [&](uint32_t run) {
        if (lane == 0) atomicAdd(h + bucket_of(run), 1ull);
      },
      [&](unsigned, int cnt) { rawbits += cnt; });
  if (lane == 0) P.wsize[chunk] = (uint32_t)((rawbits + 7) / 8);
}

// frequency normalisation (12-bit), one thread per plane; writes freq and cum
__global__ void freq_kernel(const unsigned long long* __restrict__ hist, int nplanes, uint32_t* __restrict__ fc) {
  const int pi = blockIdx.x * blockDim.x + threadIdx.x;
  if (pi >= nplanes) return;
  const unsigned long long* c = hist + pi * kNsym;
  uint32_t* f = fc + pi * kNsym;
  uint32_t* cum = fc + nplanes * kNsym + pi * kNsym;
  unsigned long long tot = 0;
  int best = 0;
  for (int i = 0; i < kNsym; ++i) {
    tot += c[i];
    if (c[i] > c[best]) best = i;
  }
  if (tot == 0) {
    for (int i = 0; i < kNsym; ++i) { f[i] = 0; cum[i] = 0; }
    return;
  }
  int64_t sum = 0;
  for (int i = 0; i < kNsym; ++i) {
    uint64_t v = 0;
    if (c[i]) {
      v = (uint64_t)(((u128)c[i] * kM) / tot);
      if (v == 0) v = 1;
    }
    f[i] = (uint32_t)v;
    sum += (int64_t)v;
  }
  f[best] = (uint32_t)((int64_t)f[best] + ((int64_t)kM - sum));
  uint32_t a = 0;
  for (int i = 0; i < kNsym; ++i) { cum[i] = a; a += f[i]; }
}

// rANS of the runs of one chunk, backwards.  `emit` receives bytes in
// emission order (the stream stores them reversed after the 4-byte state).
struct RansEnc {
  uint32_t x;
  uint32_t nbytes;
};

// x / f for x < 2^31 and 1 <= f <= 2^12 by one multiply-high with
// inv = ceil(2^44 / f): the error of x inv / 2^44 is below 2^31 / 2^44 = 2^-13,
// less than the distance 1/f >= 2^-12 of x/f to the next integer when x mod f
// < f - 1, and the floor is exact in every case (Granlund-Montgomery style)
__device__ __forceinline__ uint32_t div_by_inv(uint32_t x, uint64_t inv) {
  return (uint32_t)__umul64hi((uint64_t)x << 20, inv);
}

template <typename EmitF>
__device__ __forceinline__ void rans_put_run(RansEnc& r, uint32_t run, const uint32_t* f, const uint32_t* cum,
                                             const uint64_t* inv, EmitF emit) {
  const int sb = bucket_of(run);
  const uint32_t extra = run + 1u - (1u << sb);
  if (sb > 0) {
    const uint32_t xmax = (kRansL >> sb) << 8;
    while (r.x >= xmax) { emit((uint8_t)(r.x & 0xff)); r.x >>= 8; r.nbytes++; }
    r.x = (r.x << sb) | extra;
  }
  const uint32_t fr = f[sb], c = cum[sb];
  const uint32_t xmax = ((kRansL >> kScaleBits) << 8) * fr;
  while (r.x >= xmax) { emit((uint8_t)(r.x & 0xff)); r.x >>= 8; r.nbytes++; }
  const uint32_t q = div_by_inv(r.x, inv[sb]);
  r.x = (q << kScaleBits) + (r.x - q * fr) + c;
}

constexpr int kMaxRuns = 4097;  // enough for block_size <= 4096; larger blocks use the global spill
constexpr int kEncWarps = 2;  // 2 x 4097 x 4 B of static shared memory

// pass 2 (sizes_only) / pass 3: per chunk, collect runs (forward), rANS them backward.
__global__ void __launch_bounds__(32 * kEncWarps) enc_rans_kernel(EncParams P, int sizes_only, uint32_t* spill) {
  __shared__ uint32_t runs_sm[kEncWarps][kMaxRuns];
  __shared__ uint32_t f_sm[kEncWarps][kNsym], c_sm[kEncWarps][kNsym];
  __shared__ uint64_t i_sm[kEncWarps][kNsym];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t chunk = (int64_t)blockIdx.x * kEncWarps + warp;
  const int64_t nchunks = P.nblocks * P.nplanes;
  if (chunk >= nchunks) return;
  const int64_t blk = chunk / P.nplanes;
  const int pi = (int)(chunk % P.nplanes);
  const int p = P.p_top - pi;
  int64_t lo, hl, ht;
  chunk_range(P, blk, p, &lo, &hl, &ht);
  uint32_t* runs = (P.block_size < kMaxRuns) ? runs_sm[warp] : (spill + chunk * (int64_t)(P.block_size + 1));
  uint32_t nr = 0;
  // raw writer state (lane 0)
  uint64_t acc = 0;
  int nacc = 0;
  uint8_t* rawp = nullptr;
  if (!sizes_only) rawp = P.out + P.off[chunk] + P.rsize[chunk];
  chunk_walk(
      P, lo, hl, ht, p,
      [&](uint32_t run) {
        if (lane == 0) runs[nr] = run;
        nr++;
      },
      [&](unsigned packed, int cnt) {
        if (!sizes_only && lane == 0 && cnt > 0) {
          acc |= (uint64_t)packed << nacc;
          nacc += cnt;
          while (nacc >= 8) { *rawp++ = (uint8_t)(acc & 0xff); acc >>= 8; nacc -= 8; }
        }
      });
  if (lane != 0) return;
  if (!sizes_only && nacc > 0) *rawp = (uint8_t)(acc & 0xff);
  // this plane's table in shared memory, with the division constants
  uint32_t* f = f_sm[warp];
  uint32_t* cum = c_sm[warp];
  uint64_t* inv = i_sm[warp];
  for (int i = 0; i < kNsym; ++i) {
    f[i] = P.freq[pi * kNsym + i];
    cum[i] = P.freq[P.nplanes * kNsym + pi * kNsym + i];
    inv[i] = f[i] ? ((1ull << 44) + f[i] - 1) / f[i] : 0ull;
  }
  RansEnc r = {kRansL, 0};
  if (sizes_only) {
    for (int64_t t = (int64_t)nr - 1; t >= 0; --t) rans_put_run(r, runs[t], f, cum, inv, [](uint8_t) {});
    P.rsize[chunk] = nr ? (r.nbytes + 4) : 0;
  } else {
    if (nr) {
      // bytes are written from the end of the rANS area towards its start
      uint8_t* base = P.out + P.off[chunk];
      uint8_t* end = base + P.rsize[chunk];
      uint8_t* w = end;
      for (int64_t t = (int64_t)nr - 1; t >= 0; --t)
        rans_put_run(r, runs[t], f, cum, inv, [&](uint8_t by) { *--w = by; });
      w -= 4;
      w[0] = (uint8_t)r.x;
      w[1] = (uint8_t)(r.x >> 8);
      w[2] = (uint8_t)(r.x >> 16);
      w[3] = (uint8_t)(r.x >> 24);
    }
    P.table[2 * chunk] = P.rsize[chunk];
    P.table[2 * chunk + 1] = P.wsize[chunk];
  }
}

// ------------------------------------------- block-parallel encoder (n large)
// For blocks of at most kEncBlockMax coefficients.  Pass 1 (enc_block_kernel):
// one CTA per block stages the block's magnitudes and signs in shared memory
// once; the leading-bit position m_j of every coefficient gives each plane's
// run and raw-bit counts (for plane p: a leading 1 is m_j == p, a trailing bit
// m_j > p, a leading zero m_j < p, and a final run exists when a leading zero
// follows the plane's last leading 1), hence the offsets of every (block,
// plane) chunk inside the block's run and raw slots; then each warp walks its
// planes from shared memory (the walk of chunk_walk), writing the runs and the
// packed raw bits and counting the run symbols per plane (a CTA takes blocks
// in turn; groups of 32 coefficients zero through a plane only add leading
// zeros to the current run).  Pass 2 (enc_rans_thread_kernel): one THREAD per
// chunk runs rANS over the chunk's stored runs, writing the bytes in place
// over them, and records the sizes; after the offset scan a copy pass moves
// the bytes, the chunk's raw bytes and its table entry to their final place.
// The split priority's cost pass of plane p* + 1 alone walks a block per warp
// (enc_cost_plane_kernel).
constexpr int kEncBlockMax = 4096;
constexpr int kEncBlockThreads = 256;
constexpr int kEncBlockResident = 8;  // CTAs per SM of the persistent pass 1
int g_enc_nsm = 0;

struct BlockEncParams {
  const uint64_t* q;
  const uint8_t* sg;
  int64_t n;
  int block_size;
  int p_top;       // first plane walked (63, or p_star + 1 for the cost pass of that plane alone)
  int p_star;      // last plane (its leading bits up to i_lead, trailing bits up to i_trail)
  int64_t i_lead, i_trail;
  int nplanes;
  int64_t nblocks;
  int64_t run_slot;            // u32 run slots per block (block_size + nplanes)
  int64_t raw_slot;            // raw bytes per block (nplanes * (block_size / 8 + 1))
  uint32_t* runs;              // nblocks * run_slot
  uint8_t* raw;                // nblocks * raw_slot
  uint32_t* nruns;             // nchunks
  uint32_t* run_off;           // nchunks: first run of the chunk inside its block slot
  uint32_t* raw_off;           // nchunks: first raw byte of the chunk inside its block slot
  uint32_t* wsize;             // nchunks: raw bytes
  unsigned long long* hist;    // nplanes x 17
};

// Pass 1 over the blocks b = blockIdx.x, blockIdx.x + gridDim.x, ... (one
// wave of CTAs, the run-symbol histogram kept in shared memory and added to
// the global one once per CTA).  Dynamic shared memory: the block's
// magnitudes (8 B), signs and leading-bit positions (1 B each), block_size of
// each.
__global__ void __launch_bounds__(kEncBlockThreads) enc_block_kernel(BlockEncParams P) {
  extern __shared__ __align__(16) unsigned char enc_dyn[];
  unsigned long long* qs = reinterpret_cast<unsigned long long*>(enc_dyn);
  uint8_t* ss = enc_dyn + 8 * (size_t)P.block_size;
  signed char* ms = reinterpret_cast<signed char*>(ss + P.block_size);  // leading-bit position, -1 for zero
  signed char* gmax = ms + P.block_size;  // per group of 32: the largest leading-bit position
  __shared__ uint32_t s_cnt[65], s_hpos[65];  // per leading-bit position m + 1: count, last index + 1
  __shared__ uint32_t s_pre[66], s_low[64];   // exclusive prefix sums of s_cnt; prefix maxima of s_hpos
  __shared__ uint32_t s_lastones[2], s_lastlow[2], s_cnt_last[2];  // last plane: [leading 1s/last 1, ...]
  __shared__ uint32_t s_roff[64], s_woff[64];
  __shared__ unsigned s_hist[64 * kNsym];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int np = P.nplanes;
  const int plast = P.p_top - (np - 1);   // == p_star unless this is the single-plane cost pass
  const bool last_split = (plast == P.p_star);
  for (int i = tid; i < np * kNsym; i += kEncBlockThreads) s_hist[i] = 0;
  for (int64_t b = blockIdx.x; b < P.nblocks; b += gridDim.x) {
    const int64_t lo = b * P.block_size, hi_all = min(P.n, lo + P.block_size);
    const int len = (int)(hi_all - lo);
    // the last plane's category bounds inside this block (exclusive, relative to lo)
    const int hl = (int)max((int64_t)0, min((int64_t)len, P.i_lead + 1 - lo));
    const int ht = (int)max((int64_t)0, min((int64_t)len, P.i_trail + 1 - lo));
    for (int i = tid; i < 65; i += kEncBlockThreads) { s_cnt[i] = 0; s_hpos[i] = 0; }
    if (tid < 2) { s_lastones[tid] = 0; s_lastlow[tid] = 0; s_cnt_last[tid] = 0; }
    __syncthreads();
    for (int g = 0; g < len; g += kEncBlockThreads) {
      const int i = g + tid;
      const bool valid = i < len;
      const uint64_t v = valid ? P.q[lo + i] : 0ull;
      const int m = valid ? (v ? 63 - __clzll((long long)v) : -1) : -2;
      if (valid) {
        qs[i] = v;
        ss[i] = P.sg[lo + i];
        ms[i] = (signed char)m;
      }
      // whole planes: a histogram over the leading-bit positions, one atomic pair
      // per distinct position in the warp (count, last index + 1)
      const int gm = __reduce_max_sync(0xffffffffu, m + 2) - 2;  // -2: no coefficient
      if (lane == 0 && g + 32 * warp < len) gmax[(g >> 5) + warp] = (signed char)gm;
      const unsigned peers = __match_any_sync(0xffffffffu, m);
      if (valid && lane == __ffs(peers) - 1) {
        atomicAdd(&s_cnt[m + 1], (uint32_t)__popc(peers));
        atomicMax(&s_hpos[m + 1], (uint32_t)(g + warp * 32 + (31 - __clz(peers)) + 1));
      }
    }
    __syncthreads();
    // the last plane (its category bounds): leading ones and trailing bits in range,
    // the last leading one and the last leading zero in range (warp-aggregated)
    if (last_split) {
      const int p = plast;
      uint32_t n1 = 0, nt = 0, l1 = 0, l0 = 0;
      for (int i = tid; i < len; i += kEncBlockThreads) {
        const int m = ms[i];
        if (m > p && i < ht) ++nt;
        if (m == p && i < hl) { ++n1; l1 = max(l1, (uint32_t)(i + 1)); }
        if (m < p && i < hl) l0 = max(l0, (uint32_t)(i + 1));
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        n1 += __shfl_xor_sync(0xffffffffu, n1, o);
        nt += __shfl_xor_sync(0xffffffffu, nt, o);
        l1 = max(l1, __shfl_xor_sync(0xffffffffu, l1, o));
        l0 = max(l0, __shfl_xor_sync(0xffffffffu, l0, o));
      }
      if (lane == 0) {
        atomicAdd(&s_cnt_last[0], n1);
        atomicAdd(&s_cnt_last[1], nt);
        atomicMax(&s_lastones[0], l1);
        atomicMax(&s_lastlow[0], l0);
      }
    }
    __syncthreads();
    if (warp == 0) {
      // scans over the leading-bit positions t = m + 1 in [0, 64]: lane l holds
      // t = l and l + 32 (t = 64 added after): s_pre[t] = sum_{t' < t} cnt,
      // s_low[p] = max_{t <= p} hpos (last index + 1 of a coefficient with m < p)
      uint32_t c0 = s_cnt[lane], c1 = s_cnt[lane + 32];
      uint32_t h0 = s_hpos[lane], h1 = s_hpos[lane + 32];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t a0 = __shfl_up_sync(0xffffffffu, c0, o), a1 = __shfl_up_sync(0xffffffffu, c1, o);
        const uint32_t g0 = __shfl_up_sync(0xffffffffu, h0, o), g1 = __shfl_up_sync(0xffffffffu, h1, o);
        if (lane >= o) { c0 += a0; c1 += a1; h0 = max(h0, g0); h1 = max(h1, g1); }
      }
      const uint32_t tot0 = __shfl_sync(0xffffffffu, c0, 31), max0 = __shfl_sync(0xffffffffu, h0, 31);
      c1 += tot0;
      h1 = max(h1, max0);
      s_pre[lane + 1] = c0;
      s_pre[lane + 33] = c1;
      if (lane == 0) s_pre[0] = 0;
      if (lane == 31) s_pre[65] = c1 + s_cnt[64];
      s_low[lane] = h0;
      s_low[lane + 32] = h1;
      __syncwarp();
      // per plane pi = lane, lane + 32: runs = leading ones + a final run when a
      // leading zero follows the last leading one; raw bits = ones (signs) +
      // trailing bits; then the chunks' offsets inside the block's slots
      uint32_t nr[2], wb[2];
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const int pi = lane + 32 * k;
        nr[k] = 0;
        wb[k] = 0;
        if (pi < np) {
          const int p = P.p_top - pi;
          uint32_t ones, trail, endrun;
          if (pi == np - 1 && last_split) {
            ones = s_cnt_last[0];
            trail = s_cnt_last[1];
            endrun = (s_lastlow[0] > s_lastones[0]) ? 1u : 0u;
          } else {
            ones = s_cnt[p + 1];
            trail = s_pre[65] - s_pre[p + 2];  // coefficients with m > p
            endrun = (s_low[p] > s_hpos[p + 1]) ? 1u : 0u;
          }
          nr[k] = ones + endrun;
          wb[k] = (ones + trail + 7) / 8;
        }
      }
      uint32_t r0 = nr[0], r1 = nr[1], w0 = wb[0], w1 = wb[1];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t a0 = __shfl_up_sync(0xffffffffu, r0, o), a1 = __shfl_up_sync(0xffffffffu, r1, o);
        const uint32_t b0 = __shfl_up_sync(0xffffffffu, w0, o), b1 = __shfl_up_sync(0xffffffffu, w1, o);
        if (lane >= o) { r0 += a0; r1 += a1; w0 += b0; w1 += b1; }
      }
      r1 += __shfl_sync(0xffffffffu, r0, 31);
      w1 += __shfl_sync(0xffffffffu, w0, 31);
      const uint32_t ro[2] = {r0 - nr[0], r1 - nr[1]}, wo[2] = {w0 - wb[0], w1 - wb[1]};
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const int pi = lane + 32 * k;
        if (pi < np) {
          s_roff[pi] = ro[k];
          s_woff[pi] = wo[k];
          const int64_t chunk = b * np + pi;
          P.nruns[chunk] = nr[k];
          P.run_off[chunk] = ro[k];
          P.raw_off[chunk] = wo[k];
          P.wsize[chunk] = wb[k];
        }
      }
    }
    __syncthreads();
    const unsigned lt = (1u << lane) - 1u;
    for (int pi = warp; pi < np; pi += kEncBlockThreads / 32) {
      const int p = P.p_top - pi;
      const bool lastp = (pi == np - 1) && last_split;
      const int cl = lastp ? hl : len, ct = lastp ? ht : len;  // category bounds of this chunk
      const int clen = max(cl, ct);
      uint32_t* runs = P.runs + b * P.run_slot + s_roff[pi];
      uint8_t* rawp = P.raw + b * P.raw_slot + s_woff[pi];
      unsigned* h = s_hist + pi * kNsym;
      uint32_t nrun = 0, carry = 0;
      uint64_t acc = 0;
      int nacc = 0;
      for (int g = 0; g < clen; g += 32) {
        if (gmax[g >> 5] < p) {
          // every coefficient of the group is zero through plane p: leading zeros
          // only (no run ends here, no raw bit)
          carry += (uint32_t)max(0, min(32, cl - g));
          continue;
        }
        const int i = g + lane;
        const int m = (i < clen) ? ms[i] : -1;
        const bool sig_in = i < ct && m > p;          // an encoded trailing bit
        const bool lead = i < cl && m <= p;            // an encoded leading bit
        const bool one = lead && m == p;
        const bool rawp_b = sig_in || one;
        const bool rawv = sig_in ? ((qs[i] >> p) & 1ull) : (one ? (ss[i] != 0) : false);
        const unsigned lead_m = __ballot_sync(0xffffffffu, lead);
        const unsigned one_m = __ballot_sync(0xffffffffu, one);
        const unsigned raw_m = __ballot_sync(0xffffffffu, rawp_b);
        const int rank = __popc(raw_m & lt);
        const unsigned packed = __reduce_or_sync(0xffffffffu, (rawp_b && rawv) ? (1u << rank) : 0u);
        const int cnt = __popc(raw_m);
        // runs: lane l holding a leading 1 emits the zeros since the previous leading 1
        const unsigned zero_m = lead_m & ~one_m;
        if (one) {
          const unsigned prevmask = one_m & lt;
          uint32_t run;
          if (prevmask) {
            const int pl = 31 - __clz(prevmask);
            const unsigned from = (pl == 31) ? 0u : ~((2u << pl) - 1u);
            run = __popc(zero_m & lt & from);
          } else {
            run = carry + __popc(zero_m & lt);
          }
          runs[nrun + __popc(one_m & lt)] = run;
          atomicAdd(&h[bucket_of(run)], 1u);
        }
        nrun += __popc(one_m);
        if (one_m) {
          const int ll = 31 - __clz(one_m);
          const unsigned above_m = (ll == 31) ? 0u : ~((2u << ll) - 1u);
          carry = __popc(zero_m & above_m);
        } else {
          carry += __popc(zero_m);
        }
        if (lane == 0 && cnt > 0) {
          acc |= (uint64_t)packed << nacc;
          nacc += cnt;
          while (nacc >= 8) { *rawp++ = (uint8_t)(acc & 0xff); acc >>= 8; nacc -= 8; }
        }
      }
      if (lane == 0) {
        if (nacc > 0) *rawp = (uint8_t)(acc & 0xff);
        if (carry > 0) {
          runs[nrun] = carry;
          atomicAdd(&h[bucket_of(carry)], 1u);
        }
      }
    }
    __syncthreads();  // the block's staging and counters are reused by the next block
  }
  for (int i = tid; i < np * kNsym; i += kEncBlockThreads)
    if (s_hist[i]) atomicAdd(&P.hist[i], (unsigned long long)s_hist[i]);
}

// The cost pass of plane p = P.p_top alone (np = 1, no split: plane p_star + 1
// encoded whole): the same runs, run-symbol histogram and chunk sizes as
// enc_block_kernel with np = 1, one WARP per block reading the magnitudes
// straight from global memory (each is used once), so that all eight warps of
// a CTA walk blocks; the raw bits are counted, not written (only sizes are
// taken from this pass).
__global__ void __launch_bounds__(kEncBlockThreads) enc_cost_plane_kernel(BlockEncParams P) {
  __shared__ unsigned s_hist[kNsym];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int p = P.p_top;
  for (int i = threadIdx.x; i < kNsym; i += blockDim.x) s_hist[i] = 0;
  __syncthreads();
  const unsigned lt = (1u << lane) - 1u;
  const int64_t wpc = kEncBlockThreads / 32;
  for (int64_t b = blockIdx.x * wpc + warp; b < P.nblocks; b += (int64_t)gridDim.x * wpc) {
    const int64_t lo = b * P.block_size;
    const int len = (int)(min(P.n, lo + P.block_size) - lo);
    uint32_t* runs = P.runs + b * P.run_slot;
    uint32_t nrun = 0, carry = 0, nraw = 0;
    for (int g = 0; g < len; g += 32) {
      const int i = g + lane;
      const uint64_t v = (i < len) ? __ldg(P.q + lo + i) : 0ull;
      const int m = (i < len) ? (v ? 63 - __clzll((long long)v) : -1) : 64;  // 64: past the block
      const bool sig_in = m > p && m < 64;     // a trailing bit
      const bool lead = m <= p;                // a leading bit
      const bool one = m == p;
      const unsigned lead_m = __ballot_sync(0xffffffffu, lead);
      const unsigned one_m = __ballot_sync(0xffffffffu, one);
      const unsigned raw_m = __ballot_sync(0xffffffffu, sig_in || one);
      nraw += __popc(raw_m);
      const unsigned zero_m = lead_m & ~one_m;
      if (one) {
        const unsigned prevmask = one_m & lt;
        uint32_t run;
        if (prevmask) {
          const int pl = 31 - __clz(prevmask);
          const unsigned from = (pl == 31) ? 0u : ~((2u << pl) - 1u);
          run = __popc(zero_m & lt & from);
        } else {
          run = carry + __popc(zero_m & lt);
        }
        runs[nrun + __popc(one_m & lt)] = run;
        atomicAdd(&s_hist[bucket_of(run)], 1u);
      }
      nrun += __popc(one_m);
      if (one_m) {
        const int ll = 31 - __clz(one_m);
        const unsigned above_m = (ll == 31) ? 0u : ~((2u << ll) - 1u);
        carry = __popc(zero_m & above_m);
      } else {
        carry += __popc(zero_m);
      }
    }
    if (lane == 0) {
      // a final run when a leading zero follows the last leading one
      if (carry > 0) {
        runs[nrun] = carry;
        atomicAdd(&s_hist[bucket_of(carry)], 1u);
        ++nrun;
      }
      P.nruns[b] = nrun;
      P.run_off[b] = 0;
      P.raw_off[b] = 0;
      P.wsize[b] = (nraw + 7) / 8;
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kNsym; i += blockDim.x)
    if (s_hist[i]) atomicAdd(&P.hist[i], (unsigned long long)s_hist[i]);
}

struct RansThreadParams {
  uint32_t* runs;         // the sizes pass writes its bytes over them
  const uint8_t* raw;
  int64_t run_slot, raw_slot;
  const uint32_t* nruns;
  const uint32_t* run_off;
  const uint32_t* raw_off;
  const uint32_t* wsize;
  const uint32_t* freq;   // nplanes x 17, then cum
  int nplanes;
  int64_t nchunks;
  uint32_t* rsize;        // nchunks
  uint32_t* rstate;       // nchunks: final rANS state (sizes pass)
  const uint64_t* off;    // nchunks + 1 (payload offsets), write pass only
  uint8_t* out;           // payload base, write pass only
  uint32_t* table;        // size table, write pass only
};

// one thread per (block, plane) chunk: rANS of its runs, backwards.  The
// sizes pass writes the bytes in place over the chunk's runs, backwards from
// their end (a run puts at most 4 bytes -- at most 2 for its extra bits, 2 for
// its symbol, with the state in [2^23, 2^31) -- so the bytes of runs t + 1 ..
// never reach run t before it is read) and the final state into rstate; the
// write pass copies the 4-byte state, those bytes and the chunk's raw bytes to
// their final place and fills its table entry.
__global__ void enc_rans_thread_kernel(RansThreadParams P, int write) {
  const int64_t chunk = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (write) {
    if (chunk >= P.nchunks) return;
    const int64_t blk = chunk / P.nplanes;
    const uint32_t nr = P.nruns[chunk];
    uint8_t* base = P.out + P.off[chunk];
    const uint32_t rs = P.rsize[chunk];
    if (nr) {
      const uint8_t* src = reinterpret_cast<const uint8_t*>(P.runs + blk * P.run_slot + P.run_off[chunk] + nr) - (rs - 4);
      const uint32_t x = P.rstate[chunk];
      base[0] = (uint8_t)x;
      base[1] = (uint8_t)(x >> 8);
      base[2] = (uint8_t)(x >> 16);
      base[3] = (uint8_t)(x >> 24);
      for (uint32_t k = 0; k < rs - 4; ++k) base[4 + k] = src[k];
    }
    const uint32_t ws = P.wsize[chunk];
    const uint8_t* raw = P.raw + blk * P.raw_slot + P.raw_off[chunk];
    uint8_t* dst = base + rs;
    for (uint32_t k = 0; k < ws; ++k) dst[k] = raw[k];
    P.table[2 * chunk] = rs;
    P.table[2 * chunk + 1] = ws;
    return;
  }
  __shared__ uint32_t f_sm[64 * kNsym], c_sm[64 * kNsym];
  __shared__ uint64_t i_sm[64 * kNsym];
  for (int i = threadIdx.x; i < P.nplanes * kNsym; i += blockDim.x) {
    const uint32_t f = P.freq[i];
    f_sm[i] = f;
    c_sm[i] = P.freq[P.nplanes * kNsym + i];
    i_sm[i] = f ? ((1ull << 44) + f - 1) / f : 0ull;
  }
  __syncthreads();
  if (chunk >= P.nchunks) return;
  const int64_t blk = chunk / P.nplanes;
  const int pi = (int)(chunk - blk * P.nplanes);
  const uint32_t nr = P.nruns[chunk];
  uint32_t* runs = P.runs + blk * P.run_slot + P.run_off[chunk];
  const uint32_t* f = f_sm + pi * kNsym;
  const uint32_t* cum = c_sm + pi * kNsym;
  const uint64_t* inv = i_sm + pi * kNsym;
  RansEnc r = {kRansL, 0};
  uint8_t* w = reinterpret_cast<uint8_t*>(runs + nr);
  // eight runs loaded ahead of their encoding: the bytes of runs t + 1 .. lie
  // in [4 (t + 1), 4 nr), so runs t - 7 .. t are intact when loaded
  int64_t t = (int64_t)nr - 1;
  for (; t >= 7; t -= 8) {
    uint32_t rb[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) rb[u] = runs[t - u];
#pragma unroll
    for (int u = 0; u < 8; ++u) rans_put_run(r, rb[u], f, cum, inv, [&](uint8_t by) { *--w = by; });
  }
  for (; t >= 0; --t) rans_put_run(r, runs[t], f, cum, inv, [&](uint8_t by) { *--w = by; });
  P.rsize[chunk] = nr ? (r.nbytes + 4) : 0;
  P.rstate[chunk] = r.x;
}

// Exclusive prefix sums of item sizes f(i) over many CTAs (the payload
// offsets of the encoder's chunks and of the decoder's blocks): each CTA sums
// a contiguous range, one CTA scans the range sums, then each CTA writes the
// offsets of its range (threads on contiguous sub-ranges, a block scan
// between them).  Sums of u64 are exact, so the offsets equal the sequential ones.
constexpr int kScanThreads = 1024;
struct ChunkBytes {
  const uint32_t* rs;
  const uint32_t* ws;
  __device__ unsigned long long operator()(int64_t i) const { return (unsigned long long)rs[i] + ws[i]; }
};
struct BlockBytes {
  const uint8_t* tab;
  int nplanes;
  __device__ unsigned long long operator()(int64_t b) const {
    unsigned long long t = 0;
    for (int pi = 0; pi < nplanes; ++pi) {
      const uint8_t* e = tab + (b * nplanes + pi) * 8;
      t += (unsigned long long)(e[0] | (e[1] << 8) | (e[2] << 16) | ((uint32_t)e[3] << 24)) +
           (unsigned long long)(e[4] | (e[5] << 8) | (e[6] << 16) | ((uint32_t)e[7] << 24));
    }
    return t;
  }
};
__device__ __forceinline__ unsigned long long block_exscan_u64(unsigned long long v, unsigned long long* sh,
                                                               unsigned long long* total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  unsigned long long inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long u = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += u;
  }
  __syncthreads();
  if (lane == 31) sh[w] = inc;
  __syncthreads();
  if (w == 0) {
    unsigned long long x = (lane < nw) ? sh[lane] : 0ull;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long u = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += u;
    }
    if (lane < nw) sh[lane] = x;
  }
  __syncthreads();
  *total = sh[nw - 1];
  return (w > 0 ? sh[w - 1] : 0ull) + inc - v;
}
template <typename F>
__global__ void __launch_bounds__(kScanThreads) range_sum_kernel(F f, int64_t N, int64_t per_cta,
                                                                 unsigned long long* __restrict__ part) {
  __shared__ unsigned long long sh[32];
  const int64_t c0 = (int64_t)blockIdx.x * per_cta, c1 = min(N, c0 + per_cta);
  unsigned long long v = 0;
  for (int64_t i = c0 + threadIdx.x; i < c1; i += blockDim.x) v += f(i);
  unsigned long long tot;
  block_exscan_u64(v, sh, &tot);
  if (threadIdx.x == 0) part[blockIdx.x] = tot;
}
// part[0..G) -> exclusive prefixes in place (from base); *end = base + the
// total, and *err = 1 if that exceeds limit (err may be null)
__global__ void __launch_bounds__(kScanThreads) range_top_kernel(unsigned long long* __restrict__ part, int G,
                                                                 unsigned long long base, uint64_t* __restrict__ end,
                                                                 unsigned long long limit, int* __restrict__ err) {
  __shared__ unsigned long long sh[32];
  const int per = (G + kScanThreads - 1) / kScanThreads;
  const int t0 = min(G, (int)threadIdx.x * per), t1 = min(G, t0 + per);
  unsigned long long v = 0;
  for (int i = t0; i < t1; ++i) v += part[i];
  unsigned long long tot;
  unsigned long long run = base + block_exscan_u64(v, sh, &tot);
  for (int i = t0; i < t1; ++i) {
    const unsigned long long x = part[i];
    part[i] = run;
    run += x;
  }
  if (threadIdx.x == 0) {
    *end = base + tot;
    if (err && base + tot > limit) atomicExch(err, 1);
  }
}
template <typename F>
__global__ void __launch_bounds__(kScanThreads) range_write_kernel(F f, int64_t N, int64_t per_cta,
                                                                   const unsigned long long* __restrict__ part,
                                                                   uint64_t* __restrict__ out) {
  __shared__ unsigned long long sh[32];
  const int64_t c0 = (int64_t)blockIdx.x * per_cta, c1 = min(N, c0 + per_cta);
  const int64_t per = (per_cta + kScanThreads - 1) / kScanThreads;
  const int64_t t0 = min(c1, c0 + (int64_t)threadIdx.x * per), t1 = min(c1, t0 + per);
  unsigned long long v = 0;
  for (int64_t i = t0; i < t1; ++i) v += f(i);
  unsigned long long tot;
  unsigned long long run = part[blockIdx.x] + block_exscan_u64(v, sh, &tot);
  for (int64_t i = t0; i < t1; ++i) {
    out[i] = run;
    run += f(i);
  }
}
// out[0..N) = exclusive prefixes of f (from base), out[N] = base + the total
// (err set when it exceeds limit); scratch: range_scan_parts(N) u64
int range_scan_parts(int64_t N) {
  const int64_t g = (N + 4095) / 4096;
  return (int)(g < 1 ? 1 : (g > 1216 ? 1216 : g));
}
template <typename F>
int range_scan(F f, int64_t N, unsigned long long base, unsigned long long* scratch, uint64_t* out,
               unsigned long long limit, int* err, cudaStream_t s) {
  const int G = range_scan_parts(N);
  const int64_t per_cta = (N + G - 1) / G;
  range_sum_kernel<F><<<G, kScanThreads, 0, s>>>(f, N, per_cta, scratch);
  range_top_kernel<<<1, kScanThreads, 0, s>>>(scratch, G, base, out + N, limit, err);
  range_write_kernel<F><<<G, kScanThreads, 0, s>>>(f, N, per_cta, scratch, out);
  ATC_LAUNCHED(3);
  return ATC_OK;
}


// ------------------------------------------------------------------- decoder
struct DecParams {
  const uint8_t* sec;   // whole ATCQ section (device copy)
  int64_t nbytes;
  int64_t n;
  int k;
  int block_size;
  int p_star;
  int64_t i_lead, i_trail;  // last plane: leading bits up to i_lead, trailing bits up to i_trail
  int nplanes;
  int64_t nblocks;
  int64_t tab;          // offset of the size table
  const uint64_t* boff; // payload offsets: of block b at boff[b * boff_stride]
  int64_t boff_stride;  // 1 (block offsets) or nplanes (chunk offsets)
  uint64_t* qt;
  uint8_t* sg;
  double* out;
  int* err;
};

// Lowest encoded plane of a decoded coefficient a~ != 0 at index j: p_star when
// it became significant there (its leading 1 is on p_star) or when its trailing
// bit of p_star is encoded (j <= i_trail); p_star + 1 otherwise.
__device__ __forceinline__ int lowest_plane(uint64_t a, int64_t j, int p_star, int64_t i_trail) {
  const bool sig_above = (p_star >= 63) ? false : ((a >> (p_star + 1)) != 0ull);
  return (!sig_above || j <= i_trail) ? p_star : p_star + 1;
}

__device__ __forceinline__ uint32_t rd32(const uint8_t* p) {
  return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}

// One thread per block: planes 63 .. p_star in order, then dequantize.
__global__ void decode_kernel(DecParams D) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= D.nblocks) return;
  if (*D.err) return;
  const int64_t lo = b * D.block_size, hi_all = min(D.n, lo + D.block_size);
  for (int64_t j = lo; j < hi_all; ++j) { D.qt[j] = 0; D.sg[j] = 0; }
  uint64_t pos = D.boff[b * D.boff_stride];
  const uint8_t* ftab = D.sec + kQHdr;
  for (int pi = 0; pi < D.nplanes; ++pi) {
    const int p = 63 - pi;
    const uint8_t* t = D.sec + D.tab + (b * D.nplanes + pi) * 8;
    const uint32_t rl = rd32(t), wl = rd32(t + 4);
    if (pos + rl + wl > (uint64_t)D.nbytes) { atomicExch(D.err, 2); return; }
    const uint8_t* rp = D.sec + pos;
    const uint8_t* rend = rp + rl;
    const uint8_t* raw = D.sec + pos + rl;
    const uint64_t rcap = (uint64_t)wl * 8;
    uint64_t rbit = 0;
    uint32_t x = 0;
    if (rl) {
      if (rl < 4) { atomicExch(D.err, 3); return; }
      x = rd32(rp);
      rp += 4;
    }
    uint32_t f[kNsym], cum[kNsym];
    uint32_t ca = 0;
    for (int i = 0; i < kNsym; ++i) {
      f[i] = (uint32_t)ftab[2 * (pi * kNsym + i)] | ((uint32_t)ftab[2 * (pi * kNsym + i) + 1] << 8);
      cum[i] = ca;
      ca += f[i];
    }
    const int64_t hl = cat_end(lo, hi_all, p, D.p_star, D.i_lead), ht = cat_end(lo, hi_all, p, D.p_star, D.i_trail);
    const int64_t hi = max(hl, ht);
    bool need = true;
    uint32_t left = 0;
    for (int64_t j = lo; j < hi; ++j) {
      if (D.qt[j] != 0 ? (j >= ht) : (j >= hl)) continue;  // this category stops earlier
      if (D.qt[j] != 0) {
        if (rbit >= rcap) { atomicExch(D.err, 4); return; }
        const uint64_t bit = (raw[rbit >> 3] >> (rbit & 7)) & 1u;
        rbit++;
        D.qt[j] |= bit << p;
      } else {
        if (need) {
          if (!rl) { atomicExch(D.err, 5); return; }
          const uint32_t slot = x & (kM - 1);
          int sb = -1;
          for (int i = 0; i < kNsym; ++i)
            if (f[i] && slot >= cum[i] && slot < cum[i] + f[i]) { sb = i; break; }
          if (sb < 0) { atomicExch(D.err, 6); return; }
          x = f[sb] * (x >> kScaleBits) + slot - cum[sb];
          while (x < kRansL) { if (rp >= rend) { atomicExch(D.err, 7); return; } x = (x << 8) | *rp++; }
          uint32_t extra = 0;
          if (sb > 0) {
            extra = x & ((1u << sb) - 1u);
            x >>= sb;
            while (x < kRansL) { if (rp >= rend) { atomicExch(D.err, 8); return; } x = (x << 8) | *rp++; }
          }
          left = (1u << sb) - 1u + extra;
          need = false;
        }
        if (left > 0) {
          left--;
        } else {
          D.qt[j] |= 1ull << p;
          if (rbit >= rcap) { atomicExch(D.err, 9); return; }
          D.sg[j] = (raw[rbit >> 3] >> (rbit & 7)) & 1u;
          rbit++;
          need = true;
        }
      }
    }
    pos += rl + wl;
  }
  for (int64_t j = lo; j < hi_all; ++j) {
    const uint64_t a = D.qt[j];
    if (a == 0) { D.out[j] = 0.0; continue; }
    const int pj = lowest_plane(a, j, D.p_star, D.i_trail);
    const uint64_t v = a + ((pj >= 1) ? (1ull << (pj - 1)) : 0ull);
    const double m = mul_pow2(__ull2double_rn(v), -D.k);
    D.out[j] = D.sg[j] ? -m : m;
  }
}

// Block-parallel decoder (blocks of at most kDecMax coefficients): one CTA per
// block, the block's magnitudes and signs in shared memory.  Per plane the
// run-length symbols are decoded by one thread - there is one symbol per new
// significant coefficient (plus a final run), not one step per coefficient -
// and two block-wide scans place the new leading bits (rank among the
// insignificant coefficients -> index) and the raw bits (trailing bits of
// significant coefficients and signs of new ones, in coefficient order).  The
// result is identical to the sequential walk of the encoder's order.
constexpr int kDecThreads = 256;
constexpr int kDecMax = 4096;
constexpr int kDecPer = kDecMax / kDecThreads;  // 16 consecutive coefficients per thread

// exclusive prefix over the CTA of a per-thread count; *total receives the sum
__device__ __forceinline__ int64_t dec_scan(int64_t v, int64_t* sh, int64_t* total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int64_t inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) sh[w] = inc;
  __syncthreads();
  if (w == 0) {
    int64_t t = (lane < kDecThreads / 32) ? sh[lane] : 0;
    int64_t ti = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t u = __shfl_up_sync(0xffffffffu, ti, o);
      if (lane >= o) ti += u;
    }
    if (lane < kDecThreads / 32) sh[8 + lane] = ti - t;  // exclusive warp offsets
    if (lane == kDecThreads / 32 - 1) sh[16] = ti;
  }
  __syncthreads();
  const int64_t r = sh[8 + w] + inc - v;
  *total = sh[16];
  __syncthreads();
  return r;
}

constexpr int kDecBytes = 16384;  // rANS bytes of one (block, plane) staged in shared memory
constexpr int kDecDyn = 4 * kM + 4 * kDecMax + kDecBytes;
__global__ void __launch_bounds__(kDecThreads) decode_block_kernel(DecParams D) {
  __shared__ unsigned long long qs[kDecMax];
  __shared__ uint8_t ss[kDecMax];
  __shared__ uint32_t newbm[kDecMax / 32];
  __shared__ int64_t scan_sh[24];
  __shared__ int s_err;
  __shared__ uint32_t s_rl, s_wl;
  extern __shared__ uint32_t dyn32[];
  // [kM] slot -> (symbol << 25) | (frequency << 12) | (slot - cumulative), or ~0u for an unused slot
  uint32_t* slot_tab = dyn32;
  int32_t* newpos = reinterpret_cast<int32_t*>(dyn32 + kM);      // [kDecMax] ranks of new leading bits
  uint8_t* rbytes = reinterpret_cast<uint8_t*>(newpos + kDecMax);  // [kDecBytes] this plane's rANS bytes
  __shared__ int s_nnew;
  const int64_t b = blockIdx.x;
  const int tid = threadIdx.x;
  const int64_t lo = b * D.block_size, hi_all = min(D.n, lo + D.block_size);
  for (int i = tid; i < kDecMax; i += kDecThreads) { qs[i] = 0; ss[i] = 0; }
  if (tid == 0) s_err = (*D.err != 0) ? -1 : 0;
  __syncthreads();
  if (s_err) return;
  uint64_t pos = D.boff[b * D.boff_stride];
  const uint8_t* ftab = D.sec + kQHdr;
  const int64_t j0 = lo + (int64_t)tid * kDecPer;  // this thread's first coefficient
  for (int pi = 0; pi < D.nplanes; ++pi) {
    const int p = 63 - pi;
    const int64_t hl = cat_end(lo, hi_all, p, D.p_star, D.i_lead), ht = cat_end(lo, hi_all, p, D.p_star, D.i_trail);
    for (int i = tid; i < kDecMax / 32; i += kDecThreads) newbm[i] = 0u;
    if (tid == 0) {
      const uint8_t* t = D.sec + D.tab + (b * D.nplanes + pi) * 8;
      s_rl = rd32(t);
      s_wl = rd32(t + 4);
      if (pos + s_rl + s_wl > (uint64_t)D.nbytes) s_err = 2;
      else if (s_rl && s_rl < 4) s_err = 3;
    }
    // 1. rank of every insignificant coefficient among the insignificant ones
    // active: a significant coefficient before ht (trailing bit), an
    // insignificant one before hl (leading bit)
    uint32_t sigm = 0, actm = 0;
    for (int u = 0; u < kDecPer; ++u) {
      const int64_t j = j0 + u;
      if (j < hi_all) {
        const bool sg_ = qs[j - lo] != 0;
        if (sg_ ? j < ht : j < hl) {
          actm |= 1u << u;
          if (sg_) sigm |= 1u << u;
        }
      }
    }
    int64_t n_insig = 0;
    const int64_t rank0 = dec_scan(__popc(actm & ~sigm), scan_sh, &n_insig);  // (barriers inside)
    // stage the plane's symbol table (slot -> symbol, 0xff = unused slot) and,
    // when they fit, its rANS bytes in shared memory
    uint32_t f[kNsym], cum[kNsym];
    {
      uint32_t ca = 0;
      for (int i = 0; i < kNsym; ++i) {
        f[i] = (uint32_t)ftab[2 * (pi * kNsym + i)] | ((uint32_t)ftab[2 * (pi * kNsym + i) + 1] << 8);
        cum[i] = ca;
        ca += f[i];
      }
    }
    const bool staged = s_err == 0 && n_insig > 0 && s_rl <= (uint32_t)kDecBytes;
    if (s_err == 0 && n_insig > 0) {
      for (int sl = tid; sl < (int)kM; sl += kDecThreads) {
        uint32_t e = ~0u;
        for (int i = 0; i < kNsym; ++i)
          if (f[i] && (uint32_t)sl >= cum[i] && (uint32_t)sl < cum[i] + f[i]) {
            e = ((uint32_t)i << 25) | (f[i] << 12) | ((uint32_t)sl - cum[i]);
            break;
          }
        slot_tab[sl] = e;
      }
      if (staged)
        for (uint32_t i = tid; i < s_rl; i += kDecThreads) rbytes[i] = __ldg(D.sec + pos + i);
    }
    if (tid == 0) s_nnew = 0;
    __syncthreads();
    // 2. run-length symbols of this plane: one thread
    if (tid == 0 && s_err == 0 && n_insig > 0) {
      const uint32_t rl = s_rl;
      if (!rl) s_err = 5;
      const uint8_t* rp = staged ? rbytes : D.sec + pos;
      const uint8_t* rend = rp + rl;
      uint32_t x = 0;
      if (s_err == 0) { x = rd32(rp); rp += 4; }
      int64_t q = 0;
      int nnew = 0;
      int err = s_err;
      // the next stream bytes wait in a register queue (low byte first), refilled
      // ahead of use so that renormalisation does not wait on memory
      uint64_t bq = 0;
      int bn = 0;
      while (err == 0 && q < n_insig) {
        while (bn <= 4 && rp < rend) { bq |= (uint64_t)(*rp++) << (8 * bn); ++bn; }
        const uint32_t e = slot_tab[x & (kM - 1)];
        if (e == ~0u) { err = 6; break; }
        const int sb = (int)(e >> 25);
        x = ((e >> 12) & 0x1fffu) * (x >> kScaleBits) + (e & 0xfffu);
        while (x < kRansL) {
          if (bn == 0) { err = 7; break; }
          x = (x << 8) | (uint32_t)(bq & 0xffu);
          bq >>= 8;
          --bn;
        }
        if (err) break;
        uint32_t extra = 0;
        if (sb > 0) {
          extra = x & ((1u << sb) - 1u);
          x >>= sb;
          while (x < kRansL) {
            if (bn == 0) { err = 8; break; }
            x = (x << 8) | (uint32_t)(bq & 0xffu);
            bq >>= 8;
            --bn;
          }
          if (err) break;
        }
        q += (int64_t)((1u << sb) - 1u + extra);
        if (q < n_insig) {
          newpos[nnew++] = (int32_t)q;
          ++q;
        }
      }
      s_err = err;
      s_nnew = nnew;
    }
    __syncthreads();
    for (int k = tid; k < s_nnew; k += kDecThreads) {
      const int32_t qq = newpos[k];
      atomicOr(&newbm[qq >> 5], 1u << (qq & 31));
    }
    __syncthreads();
    if (s_err) break;
    // 3. raw bits: one per significant coefficient (a trailing bit) and one per
    //    new significant coefficient (its sign), in coefficient order
    uint32_t newm = 0;
    {
      int64_t r = rank0;
      for (int u = 0; u < kDecPer; ++u)
        if ((actm >> u & 1u) && !(sigm >> u & 1u)) {
          if (newbm[r >> 5] >> (r & 31) & 1u) newm |= 1u << u;
          ++r;
        }
    }
    const uint32_t consm = sigm | newm;
    int64_t ncons = 0;
    const int64_t rb0 = dec_scan(__popc(consm), scan_sh, &ncons);
    const uint64_t rcap = (uint64_t)s_wl * 8;
    if ((uint64_t)ncons > rcap) {
      if (tid == 0) s_err = 4;
    } else {
      const uint8_t* raw = D.sec + pos + s_rl;
      int64_t rbit = rb0;
      for (int u = 0; u < kDecPer; ++u) {
        if (!(consm >> u & 1u)) continue;
        const uint32_t bit = (__ldg(raw + (rbit >> 3)) >> (rbit & 7)) & 1u;
        ++rbit;
        const int64_t jj = j0 + u - lo;
        if (sigm >> u & 1u) qs[jj] |= (unsigned long long)bit << p;
        else { qs[jj] |= 1ull << p; ss[jj] = (uint8_t)bit; }
      }
    }
    pos += s_rl + s_wl;
    __syncthreads();
    if (s_err) break;
  }
  if (s_err) {
    if (tid == 0 && s_err > 0) atomicExch(D.err, s_err);
    return;
  }
  for (int u = 0; u < kDecPer; ++u) {
    const int64_t j = j0 + u;
    if (j >= hi_all) break;
    const uint64_t a = qs[j - lo];
    if (a == 0) { D.out[j] = 0.0; continue; }
    const int pj = lowest_plane(a, j, D.p_star, D.i_trail);
    const uint64_t v = a + ((pj >= 1) ? (1ull << (pj - 1)) : 0ull);
    const double m = mul_pow2(__ull2double_rn(v), -D.k);
    D.out[j] = ss[j - lo] ? -m : m;
  }
}

// Two-phase decoder.  The run-length symbols of a (block, plane) chunk do not
// depend on any other chunk - only their placement does - and a rANS decoder
// ends exactly in the encoder's initial state kRansL with every byte used.
// Phase A (decode_runs_kernel) therefore decodes every chunk's runs in
// parallel, one thread per chunk, until that end state; a plane whose table
// holds a single bucket of probability one with no extra bits carries no
// information and is marked implicit (every remaining run is 0).  Phase B
// (decode_place_kernel, one CTA per block, planes in order) turns the runs
// into positions with a block scan and places the leading and raw bits.
constexpr int kRunsImplicit = -1;

struct RunParams {
  const uint8_t* sec;
  int64_t nbytes, tab;
  int nplanes;
  int64_t nblocks;
  int block_size;
  const uint64_t* coff;  // payload offset of every chunk (nblocks * nplanes + 1)
  uint32_t* runs;  // [chunk][block_size + 2]
  int* nruns;      // [chunk]
  int* err;
};

// payload bytes of one (block, plane) chunk from the size table: rANS + raw
struct TabBytes {
  const uint8_t* tab;
  __device__ unsigned long long operator()(int64_t c) const {
    const uint8_t* e = tab + c * 8;
    return (unsigned long long)(e[0] | (e[1] << 8) | (e[2] << 16) | ((uint32_t)e[3] << 24)) +
           (unsigned long long)(e[4] | (e[5] << 8) | (e[6] << 16) | ((uint32_t)e[7] << 24));
  }
};

// Phase A: the runs of every chunk.  CTA (x, pi) takes plane pi of blocks
// [x * kRunThreads, (x + 1) * kRunThreads), a thread per chunk, so that the
// plane's slot -> symbol table (the 2^12 slots of its frequency table) sits in
// shared memory and a symbol costs one table read instead of a search.
constexpr int kRunThreads = 128;
__global__ void __launch_bounds__(kRunThreads) decode_runs_kernel(RunParams P) {
  __shared__ uint8_t lut[kM];
  __shared__ uint32_t s_f[kNsym], s_c[kNsym];
  __shared__ int s_single;
  const int pi = blockIdx.y;
  const uint8_t* ftab = P.sec + kQHdr + 2 * pi * kNsym;
  if (threadIdx.x == 0) {
    uint32_t ca = 0;
    int single = -1;
    for (int i = 0; i < kNsym; ++i) {
      const uint32_t f = (uint32_t)ftab[2 * i] | ((uint32_t)ftab[2 * i + 1] << 8);
      s_f[i] = f;
      s_c[i] = ca;
      ca += f;
      if (f == kM) single = i;
    }
    s_single = single;
  }
  __syncthreads();
  // slot -> the symbol whose interval [cum, cum + f) holds it (0xff: none)
  for (int sl = threadIdx.x; sl < (int)kM; sl += blockDim.x) {
    int sb = 0xff;
#pragma unroll
    for (int i = 0; i < kNsym; ++i)
      if (s_f[i] && (uint32_t)sl >= s_c[i] && (uint32_t)sl < s_c[i] + s_f[i]) sb = i;
    lut[sl] = (uint8_t)sb;
  }
  __syncthreads();
  const int64_t b = blockIdx.x * (int64_t)kRunThreads + threadIdx.x;
  if (b >= P.nblocks) return;
  const int64_t c = b * P.nplanes + pi;
  const int cap = P.block_size + 2;
  const uint64_t pos = P.coff[c];
  const uint8_t* t = P.sec + P.tab + c * 8;
  const uint32_t rl = rd32(t), wl = rd32(t + 4);
  int* nr = P.nruns + c;
  if (pos + rl + wl > (uint64_t)P.nbytes) { atomicExch(P.err, 2); *nr = 0; return; }
  if (rl == 0) { *nr = 0; return; }
  if (rl < 4) { atomicExch(P.err, 3); *nr = 0; return; }
  if (s_single == 0) { *nr = kRunsImplicit; return; }
  const uint8_t* rp = P.sec + pos;
  const uint8_t* rend = rp + rl;
  uint32_t x = rd32(rp);
  rp += 4;
  uint32_t* out = P.runs + c * (int64_t)cap;
  int k = 0;
  while (!(x == kRansL && rp == rend)) {
    const uint32_t slot = x & (kM - 1);
    const int sb = lut[slot];
    if (sb == 0xff) { atomicExch(P.err, 6); break; }
    x = s_f[sb] * (x >> kScaleBits) + slot - s_c[sb];
    bool bad = false;
    while (x < kRansL) { if (rp >= rend) { bad = true; break; } x = (x << 8) | *rp++; }
    if (bad) { atomicExch(P.err, 7); break; }
    uint32_t extra = 0;
    if (sb > 0) {
      extra = x & ((1u << sb) - 1u);
      x >>= sb;
      while (x < kRansL) { if (rp >= rend) { bad = true; break; } x = (x << 8) | *rp++; }
      if (bad) { atomicExch(P.err, 8); break; }
    }
    if (k >= cap) { atomicExch(P.err, 10); break; }
    out[k++] = (1u << sb) - 1u + extra;
  }
  *nr = k;
}

// Phase B, one CTA per block of at most kDecMax coefficients, 16 consecutive
// coefficients a thread held in registers (magnitudes, significance and sign
// masks: no shared-memory traffic per coefficient and plane).  Per plane: one
// block scan gives both the thread's first rank among the active leading bits
// and its first position in the run list (two 32-bit counts in one 64-bit
// sum); the runs mark the new leading 1s in a shared bit map; a second scan
// places the thread's raw bits, read as one window of at most three bytes.
__global__ void __launch_bounds__(kDecThreads) decode_place_kernel(DecParams D, const uint32_t* __restrict__ runs,
                                                                   const int* __restrict__ nruns) {
  __shared__ uint32_t newbm[kDecMax / 32 + 2];
  __shared__ int64_t scan_sh[24];
  __shared__ int s_err;
  __shared__ uint32_t s_rl[64], s_wl[64], s_po[64];
  __shared__ int s_nr[64];
  constexpr int kRunPer = (kDecMax + 2 + kDecThreads - 1) / kDecThreads;  // runs per thread (17)
  const int64_t b = blockIdx.x;
  const int tid = threadIdx.x;
  const int64_t lo = b * D.block_size, hi_all = min(D.n, lo + D.block_size);
  const int cap = D.block_size + 2;
  if (tid == 0) s_err = (*D.err != 0) ? -1 : 0;
  // size table, run counts and payload offsets of the block's planes
  const uint64_t base = D.boff[b * D.boff_stride];
  if (tid < 32) {
    uint64_t acc = 0;
    for (int p0 = 0; p0 < D.nplanes; p0 += 32) {
      const int pi = p0 + tid;
      uint32_t rl = 0, wl = 0;
      int nr = 0;
      if (pi < D.nplanes) {
        const uint8_t* te = D.sec + D.tab + (b * D.nplanes + pi) * 8;
        rl = rd32(te);
        wl = rd32(te + 4);
        nr = nruns[b * D.nplanes + pi];
      }
      uint64_t inc = (uint64_t)rl + wl;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint64_t t = __shfl_up_sync(0xffffffffu, inc, o);
        if (tid >= o) inc += t;
      }
      if (pi < D.nplanes) {
        s_rl[pi] = rl;
        s_wl[pi] = wl;
        s_nr[pi] = nr;
        s_po[pi] = (uint32_t)(acc + inc - ((uint64_t)rl + wl));
      }
      acc += __shfl_sync(0xffffffffu, inc, 31);
    }
    if (tid == 0 && base + acc > (uint64_t)D.nbytes && s_err == 0) s_err = 2;
  }
  __syncthreads();
  if (s_err) {
    if (tid == 0 && s_err > 0) atomicExch(D.err, s_err);
    return;
  }
  const int64_t j0 = lo + (int64_t)tid * kDecPer;
  const int nvalid = (int)max((int64_t)0, min((int64_t)kDecPer, hi_all - j0));
  uint64_t qv[kDecPer];
#pragma unroll
  for (int u = 0; u < kDecPer; ++u) qv[u] = 0;
  uint32_t sigall = 0, sgn = 0;  // significant so far, sign bits
  const int k0 = tid * kRunPer;
  for (int pi = 0; pi < D.nplanes; ++pi) {
    const int p = 63 - pi;
    const int64_t hl = cat_end(lo, hi_all, p, D.p_star, D.i_lead), ht = cat_end(lo, hi_all, p, D.p_star, D.i_trail);
    for (int i = tid; i < kDecMax / 32 + 2; i += kDecThreads) newbm[i] = 0u;
    // active coefficients: a significant one before ht (trailing bit), an
    // insignificant one before hl (leading bit)
    const int nt = (int)max((int64_t)0, min((int64_t)nvalid, ht - j0));
    const int nl = (int)max((int64_t)0, min((int64_t)nvalid, hl - j0));
    const uint32_t lowt = nt >= 32 ? ~0u : ((1u << nt) - 1u), lowl = nl >= 32 ? ~0u : ((1u << nl) - 1u);
    const uint32_t sigm = sigall & lowt, insm = ~sigall & lowl;
    const int nr = s_nr[pi];
    const uint32_t* rr = runs + (b * D.nplanes + pi) * (int64_t)cap;
    // this thread's runs k0 .. k0 + kend - 1 (read twice from L1/L2: a loop over
    // only the runs there are, instead of kRunPer predicated slots)
    const int kend = (nr == kRunsImplicit) ? 0 : max(0, min(kRunPer, nr - k0));
    int64_t loc = 0;
    for (int u = 0; u < kend; ++u) loc += (int64_t)__ldg(rr + k0 + u) + 1;
    // one scan: (insignificant active count) << 32 | (run-list position)
    int64_t tot = 0;
    const int64_t ex = dec_scan(((int64_t)__popc(insm) << 32) | loc, scan_sh, &tot);
    const int64_t rank0 = ex >> 32, n_insig = tot >> 32;
    int64_t q = ex & 0xffffffffll;
    if (nr == kRunsImplicit) {
      for (int64_t r = tid; r < n_insig; r += kDecThreads) atomicOr(&newbm[r >> 5], 1u << (r & 31));
    } else {
      for (int u = 0; u < kend; ++u) {
        const int k = k0 + u;
        const uint32_t rv = __ldg(rr + k);
        const int64_t at = q + rv;  // rank of this run's 1
        if (k == nr - 1 && !(q < n_insig && n_insig <= q + (int64_t)rv + 1)) s_err = 11;  // symbol count
        if (at < n_insig) atomicOr(&newbm[at >> 5], 1u << (at & 31));
        q += (int64_t)rv + 1;
      }
      if (tid == 0 && nr == 0 && n_insig > 0) s_err = 5;
    }
    __syncthreads();
    if (s_err) break;
    // the thread's leading bits have consecutive ranks rank0 ..: a window of the bit map
    uint32_t newm = 0;
    {
      const uint32_t w0 = newbm[rank0 >> 5], w1 = newbm[(rank0 >> 5) + 1];
      const uint32_t win = (uint32_t)((((uint64_t)w1 << 32) | w0) >> (rank0 & 31));
      int k = 0;
#pragma unroll
      for (int u = 0; u < kDecPer; ++u)
        if (insm >> u & 1u) {
          if (win >> k & 1u) newm |= 1u << u;
          ++k;
        }
    }
    const uint32_t consm = sigm | newm;
    int64_t ncons = 0;
    const int64_t rb0 = dec_scan(__popc(consm), scan_sh, &ncons);
    const uint32_t wl = s_wl[pi];
    if ((uint64_t)ncons > (uint64_t)wl * 8) {
      if (tid == 0) s_err = 4;
    } else if (consm) {
      // this thread's raw bits [rb0, rb0 + popc(consm)), at most 16: three bytes
      const uint8_t* raw = D.sec + base + s_po[pi] + s_rl[pi];
      const int64_t by = rb0 >> 3;
      const int64_t last = (rb0 + __popc(consm) - 1) >> 3;
      uint32_t win = 0;
      for (int64_t t = by; t <= last; ++t) win |= (uint32_t)__ldg(raw + t) << (8 * (int)(t - by));
      win >>= (rb0 & 7);
      int k = 0;
#pragma unroll
      for (int u = 0; u < kDecPer; ++u) {
        if (!(consm >> u & 1u)) continue;
        const uint32_t bit = (win >> k) & 1u;
        ++k;
        if (sigm >> u & 1u) {
          qv[u] |= (uint64_t)bit << p;
        } else {
          qv[u] |= 1ull << p;
          sgn |= bit << u;
          sigall |= 1u << u;
        }
      }
    }
    __syncthreads();
    if (s_err) break;
  }
  if (s_err) {
    if (tid == 0 && s_err > 0) atomicExch(D.err, s_err);
    return;
  }
#pragma unroll
  for (int u = 0; u < kDecPer; ++u) {
    const int64_t j = j0 + u;
    if (u >= nvalid) break;
    const uint64_t a = qv[u];
    if (a == 0) { D.out[j] = 0.0; continue; }
    const int pj = lowest_plane(a, j, D.p_star, D.i_trail);
    const uint64_t v = a + ((pj >= 1) ? (1ull << (pj - 1)) : 0ull);
    const double m = mul_pow2(__ull2double_rn(v), -D.k);
    D.out[j] = (sgn >> u & 1u) ? -m : m;
  }
}

// Blocks of at most 512 coefficients: one WARP per block (16 consecutive
// coefficients a lane, in registers), the placement of decode_place_kernel
// with warp scans instead of block scans, so a plane costs no CTA barrier.
// The block's size table entries, plane offsets and (when it fits) its whole
// payload are staged in shared memory first.  Same result.
constexpr int kWDecPer = 16;
constexpr int kWDecMax = 32 * kWDecPer;
constexpr int kWDecWarps = 4;    // blocks per CTA
constexpr int kWDecStage = 8192; // payload bytes staged per block
__device__ __forceinline__ int64_t warp_exscan64(int64_t v, int64_t* total) {
  const int lane = threadIdx.x & 31;
  int64_t inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  *total = __shfl_sync(0xffffffffu, inc, 31);
  return inc - v;
}

__global__ void __launch_bounds__(32 * kWDecWarps) decode_place_warp_kernel(DecParams D,
                                                                            const uint32_t* __restrict__ runs,
                                                                            const int* __restrict__ nruns) {
  __shared__ uint32_t nb_all[kWDecWarps][kWDecMax / 32 + 2];
  __shared__ uint32_t rl_all[kWDecWarps][64], wl_all[kWDecWarps][64], po_all[kWDecWarps][64];
  __shared__ int nr_all[kWDecWarps][64];
  __shared__ __align__(16) uint8_t pay_all[kWDecWarps][kWDecStage];
  constexpr int kRunPerW = (kWDecMax + 2 + 31) / 32;  // runs per lane (17)
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t b = (int64_t)blockIdx.x * kWDecWarps + w;
  if (b >= D.nblocks) return;  // the whole warp: nothing below synchronises the CTA
  uint32_t* newbm = nb_all[w];
  uint32_t *rlp = rl_all[w], *wlp = wl_all[w], *pop = po_all[w];
  int* nrp = nr_all[w];
  uint8_t* pay = pay_all[w];
  const int64_t lo = b * D.block_size, hi_all = min(D.n, lo + D.block_size);
  const int cap = D.block_size + 2;
  int err = (*D.err != 0) ? -1 : 0;
  err = __reduce_max_sync(0xffffffffu, err);
  if (err) return;
  // size table entries, run counts and payload offsets of this block's planes
  const uint64_t base = D.boff[b * D.boff_stride];
  uint64_t acc = 0;
  for (int p0 = 0; p0 < D.nplanes; p0 += 32) {
    const int pi = p0 + lane;
    uint32_t rl = 0, wl = 0;
    int nr = 0;
    if (pi < D.nplanes) {
      const uint8_t* te = D.sec + D.tab + (b * D.nplanes + pi) * 8;
      rl = rd32(te);
      wl = rd32(te + 4);
      nr = nruns[b * D.nplanes + pi];
    }
    int64_t tot = 0;
    const int64_t ex = warp_exscan64((int64_t)rl + wl, &tot);
    if (pi < D.nplanes) {
      rlp[pi] = rl;
      wlp[pi] = wl;
      nrp[pi] = nr;
      pop[pi] = (uint32_t)(acc + (uint64_t)ex);
    }
    acc += (uint64_t)tot;
  }
  if (base + acc > (uint64_t)D.nbytes) err = 2;
  const bool staged = acc <= (uint64_t)kWDecStage;
  if (staged && !err)
    for (uint32_t i = lane; i < (uint32_t)acc; i += 32) pay[i] = __ldg(D.sec + base + i);
  __syncwarp();
  if (err) {
    if (lane == 0) atomicExch(D.err, err);
    return;
  }
  const int64_t j0 = lo + (int64_t)lane * kWDecPer;
  const int nvalid = (int)max((int64_t)0, min((int64_t)kWDecPer, hi_all - j0));
  uint64_t qv[kWDecPer];
#pragma unroll
  for (int u = 0; u < kWDecPer; ++u) qv[u] = 0;
  uint32_t sigall = 0, sgn = 0;
  const int k0 = lane * kRunPerW;
  for (int pi = 0; pi < D.nplanes; ++pi) {
    const int p = 63 - pi;
    const int64_t hl = cat_end(lo, hi_all, p, D.p_star, D.i_lead), ht = cat_end(lo, hi_all, p, D.p_star, D.i_trail);
    for (int i = lane; i < kWDecMax / 32 + 2; i += 32) newbm[i] = 0u;
    const int nt = (int)max((int64_t)0, min((int64_t)nvalid, ht - j0));
    const int nl = (int)max((int64_t)0, min((int64_t)nvalid, hl - j0));
    const uint32_t lowt = (1u << nt) - 1u, lowl = (1u << nl) - 1u;  // nt, nl <= 16
    const uint32_t sigm = sigall & lowt, insm = ~sigall & lowl;
    const int nr = nrp[pi];
    const uint32_t* rr = runs + (b * D.nplanes + pi) * (int64_t)cap;
    // this lane's runs k0 .. k0 + kend - 1 (a loop over only the runs there are)
    const int kend = (nr == kRunsImplicit) ? 0 : max(0, min(kRunPerW, nr - k0));
    int64_t loc = 0;
    for (int u = 0; u < kend; ++u) loc += (int64_t)__ldg(rr + k0 + u) + 1;
    int64_t tot = 0;
    const int64_t ex = warp_exscan64(((int64_t)__popc(insm) << 32) | loc, &tot);
    const int64_t rank0 = ex >> 32, n_insig = tot >> 32;
    int64_t q = ex & 0xffffffffll;
    __syncwarp();
    if (nr == kRunsImplicit) {
      for (int64_t r = lane; r < n_insig; r += 32) atomicOr(&newbm[r >> 5], 1u << (r & 31));
    } else {
      for (int u = 0; u < kend; ++u) {
        const int k = k0 + u;
        const uint32_t rv = __ldg(rr + k);
        const int64_t at = q + rv;  // rank of this run's 1
        if (k == nr - 1 && !(q < n_insig && n_insig <= q + (int64_t)rv + 1)) err = 11;  // symbol count
        if (at < n_insig) atomicOr(&newbm[at >> 5], 1u << (at & 31));
        q += (int64_t)rv + 1;
      }
      if (nr == 0 && n_insig > 0) err = 5;
    }
    err = __reduce_max_sync(0xffffffffu, err);
    __syncwarp();
    if (err) break;
    uint32_t newm = 0;
    {
      const uint32_t w0 = newbm[rank0 >> 5], w1 = newbm[(rank0 >> 5) + 1];
      const uint32_t win = (uint32_t)((((uint64_t)w1 << 32) | w0) >> (rank0 & 31));
      int k = 0;
#pragma unroll
      for (int u = 0; u < kWDecPer; ++u)
        if (insm >> u & 1u) {
          if (win >> k & 1u) newm |= 1u << u;
          ++k;
        }
    }
    const uint32_t consm = sigm | newm;
    int64_t ncons = 0;
    const int64_t rb0 = warp_exscan64(__popc(consm), &ncons);
    if ((uint64_t)ncons > (uint64_t)wlp[pi] * 8) {
      err = 4;
      break;
    }
    if (consm) {
      const uint32_t roff = pop[pi] + rlp[pi];  // raw bytes of this plane, relative to the block's payload
      const int64_t by = rb0 >> 3, last = (rb0 + __popc(consm) - 1) >> 3;
      uint32_t win = 0;
      for (int64_t t = by; t <= last; ++t)
        win |= (uint32_t)(staged ? pay[roff + (uint32_t)t] : __ldg(D.sec + base + roff + t)) << (8 * (int)(t - by));
      win >>= (rb0 & 7);
      int k = 0;
#pragma unroll
      for (int u = 0; u < kWDecPer; ++u) {
        if (!(consm >> u & 1u)) continue;
        const uint32_t bit = (win >> k) & 1u;
        ++k;
        if (sigm >> u & 1u) {
          qv[u] |= (uint64_t)bit << p;
        } else {
          qv[u] |= 1ull << p;
          sgn |= bit << u;
          sigall |= 1u << u;
        }
      }
    }
    __syncwarp();
  }
  if (err) {
    if (lane == 0 && err > 0) atomicExch(D.err, err);
    return;
  }
#pragma unroll
  for (int u = 0; u < kWDecPer; ++u) {
    if (u >= nvalid) break;
    const int64_t j = j0 + u;
    const uint64_t a = qv[u];
    if (a == 0) { D.out[j] = 0.0; continue; }
    const int pj = lowest_plane(a, j, D.p_star, D.i_trail);
    const uint64_t v = a + ((pj >= 1) ? (1ull << (pj - 1)) : 0ull);
    const double m = mul_pow2(__ull2double_rn(v), -D.k);
    D.out[j] = (sgn >> u & 1u) ? -m : m;
  }
}

static void put32(uint8_t* p, uint32_t v) { for (int i = 0; i < 4; ++i) p[i] = (uint8_t)(v >> (8 * i)); }
static void put64(uint8_t* p, uint64_t v) { for (int i = 0; i < 8; ++i) p[i] = (uint8_t)(v >> (8 * i)); }
static uint32_t get32(const uint8_t* p) { uint32_t v = 0; for (int i = 0; i < 4; ++i) v |= (uint32_t)p[i] << (8 * i); return v; }
static uint64_t get64(const uint8_t* p) { uint64_t v = 0; for (int i = 0; i < 8; ++i) v |= (uint64_t)p[i] << (8 * i); return v; }

double i192_to_double(const I192& v) {
  // v >= 0 assumed
  return (double)v.w2 * 0x1p128 + (double)v.w1 * 0x1p64 + (double)v.w0;
}

}  // namespace

// Pinned host staging for the tracker state and the encoder's small tables:
// copies into it are asynchronous, so each readback costs one stream
// synchronisation and no pageable staging (grow-only, process-wide).
static int quant_pinned(size_t bytes, void** p) {
  static std::mutex mu;
  static void* buf = nullptr;
  static size_t cap = 0;
  std::lock_guard<std::mutex> lk(mu);
  if (cap < bytes) {
    if (buf) {
      ATC_CUDA_TRY(cudaDeviceSynchronize());
      cudaFreeHost(buf);
      buf = nullptr;
      cap = 0;
    }
    ATC_CUDA_TRY(cudaHostAlloc(&buf, bytes, cudaHostAllocPortable));
    cap = bytes;
  }
  *p = buf;
  return ATC_OK;
}

int quantize_encode(const double* core, int64_t n, double target, int block_size, cudaStream_t s, QuantSection* out,
                    QuantResult* res, float* ms_quant, float* ms_encode) {
  if (n < 1) return fail(ATC_EINVAL, "empty core");
  if (block_size < 32 || block_size > 65535 || (block_size % 32)) return fail(ATC_EINVAL, "bad block_size %d", block_size);
  cudaEvent_t e0, e1, e2;
  ATC_CUDA_TRY(cudaEventCreate(&e0));
  ATC_CUDA_TRY(cudaEventCreate(&e1));
  ATC_CUDA_TRY(cudaEventCreate(&e2));
  ATC_CUDA_TRY(cudaEventRecord(e0, s));
  // scratch layout
  uint64_t* q = nullptr;
  uint8_t* sg = nullptr;
  ATC_TRY(Scratch::get(SLOT_Q, sizeof(uint64_t) * n, (void**)&q));
  ATC_TRY(Scratch::get(SLOT_QS, (size_t)n, (void**)&sg));
  const int64_t seg_len = (n + kSegBlocks - 1) / kSegBlocks;
  const int nseg = (int)((n + seg_len - 1) / seg_len);
  uint8_t* small = nullptr;
  const size_t seg_bytes = sizeof(Seg) * (size_t)nseg * kPlaneChunk;
  const size_t ss_off = (4096 + seg_bytes + sizeof(I192) * nseg + 255) & ~(size_t)255;
  const size_t small_bytes = ss_off + sizeof(SplitSeg) * nseg + 256;
  ATC_TRY(Scratch::get(SLOT_QPART, small_bytes, (void**)&small));
  TrackState* st = reinterpret_cast<TrackState*>(small);
  unsigned long long* mx = reinterpret_cast<unsigned long long*>(small + 1024);
  Seg* segs = reinterpret_cast<Seg*>(small + 4096);
  I192* e64s = reinterpret_cast<I192*>(small + 4096 + seg_bytes);
  SplitSeg* sseg = reinterpret_cast<SplitSeg*>(small + ss_off);
  ATC_CUDA_TRY(cudaMemsetAsync(small, 0, 4096, s));
  const int64_t gb = (n + 255) / 256;
  const int grid = (int)(gb < 152 * 8 ? gb : 152 * 8);
  maxabs_kernel<<<grid, 256, 0, s>>>(core, n, mx);
  ATC_LAUNCHED(1);
  scale_exp_kernel<<<1, 32, 0, s>>>(mx, target, st);
  ATC_LAUNCHED(1);
  {
    KTimed kt_(s, "quantize_kernel", (double)n * (8.0 + 8.0 + 1.0));
    quantize_kernel<<<grid, 256, 0, s>>>(core, n, &st->k, q, sg);
  }
  ATC_LAUNCHED(1);
  TrackState* hstp = nullptr;
  ATC_TRY(quant_pinned(sizeof(TrackState) + 16 + sizeof(uint32_t) * 2 * 64 * kNsym, (void**)&hstp));
  TrackState& hst = *hstp;
  int phi = 63;
  bool first = true;
  for (;;) {
    int plo = phi - kPlaneChunk + 1;
    if (plo < 0) plo = 0;
    {
      KTimed kt_(s, "plane_stats_kernel", (double)n * 8.0);
      plane_stats_kernel<<<nseg, kSegThreads, 0, s>>>(q, n, seg_len, plo, phi, first ? 1 : 0, segs, e64s);
    }
    ATC_LAUNCHED(1);
    plane_scan_kernel<<<1, 32 * kPlaneChunk, 0, s>>>(segs, e64s, nseg, plo, phi, first ? 1 : 0, st);
    ATC_LAUNCHED(1);
    ATC_CUDA_TRY(cudaMemcpyAsync(&hst, st, sizeof(hst), cudaMemcpyDeviceToHost, s));
    ATC_CUDA_TRY(cudaStreamSynchronize(s));
    if (hst.nan) return fail(ATC_ENUMERIC, "core contains NaN or Inf");
    first = false;
    if (hst.found) break;
    phi = plo - 1;
    if (phi < 0) return fail(ATC_ECUDA, "tracker did not terminate");
  }
  if (hst.p_star < 64 && hst.reachable) {
    istar_kernel<<<1, kIstarThreads, 0, s>>>(q, n, seg_len, segs, nseg, phi, st);
    ATC_LAUNCHED(1);
  }
  const int k = hst.k;
  const int p_star = hst.p_star;
  const int nplanes = (p_star >= 64) ? 0 : 64 - p_star;
  const int64_t nblocks = (n + block_size - 1) / block_size;
  const int64_t nchunks = nblocks * nplanes;
  const bool block_path = block_size <= kEncBlockMax;
  // encoder scratch for planes 63 .. p_star (the cost pass of plane p_star + 1
  // alone, which sets the split priority, runs in the same buffers first)
  unsigned long long* hist = nullptr;
  uint32_t *fc = nullptr, *rsize = nullptr, *wsize = nullptr;
  uint64_t* off = nullptr;
  uint32_t* spill = nullptr;
  BlockEncParams B;
  RansThreadParams R;
  EncParams P;
  memset(&B, 0, sizeof(B));
  memset(&R, 0, sizeof(R));
  memset(&P, 0, sizeof(P));
  if (nplanes > 0) {
    uint8_t* enc = nullptr;
    const size_t enc_small = sizeof(unsigned long long) * nplanes * kNsym + sizeof(uint32_t) * 2 * nplanes * kNsym +
                             sizeof(uint32_t) * 2 * nchunks + sizeof(uint64_t) * (nchunks + 1) + 1024;
    ATC_TRY(Scratch::get(SLOT_ENC, enc_small, (void**)&enc));
    hist = reinterpret_cast<unsigned long long*>(enc);
    fc = reinterpret_cast<uint32_t*>(hist + nplanes * kNsym);
    rsize = fc + 2 * nplanes * kNsym;
    wsize = rsize + nchunks;
    off = reinterpret_cast<uint64_t*>(((uintptr_t)(wsize + nchunks) + 7) & ~(uintptr_t)7);
    if (block_path) {
      B.q = q; B.sg = sg; B.n = n; B.block_size = block_size; B.p_star = p_star;
      B.nblocks = nblocks;
      B.run_slot = (int64_t)block_size + nplanes;
      B.raw_slot = (int64_t)nplanes * (block_size / 8 + 1);
      uint8_t* work = nullptr;
      const size_t runs_b = sizeof(uint32_t) * (size_t)nblocks * (size_t)B.run_slot;
      const size_t raw_b = ((size_t)nblocks * (size_t)B.raw_slot + 255) & ~(size_t)255;
      const size_t meta_b = sizeof(uint32_t) * 4 * (size_t)nchunks + 256;  // nruns, run_off, raw_off, rstate
      ATC_TRY(Scratch::get(SLOT_SPILL, runs_b + raw_b + meta_b, (void**)&work));
      B.runs = reinterpret_cast<uint32_t*>(work);
      B.raw = work + runs_b;
      B.nruns = reinterpret_cast<uint32_t*>(work + runs_b + raw_b);
      B.run_off = B.nruns + nchunks;
      B.raw_off = B.run_off + nchunks;
      R.rstate = B.raw_off + nchunks;
      B.wsize = wsize;
      B.hist = hist;
      R.runs = B.runs; R.raw = B.raw; R.run_slot = B.run_slot; R.raw_slot = B.raw_slot;
      R.nruns = B.nruns; R.run_off = B.run_off; R.raw_off = B.raw_off; R.wsize = wsize;
      R.freq = fc; R.rsize = rsize; R.off = off;
    } else {
      if (block_size >= kMaxRuns)
        ATC_TRY(Scratch::get(SLOT_SPILL, sizeof(uint32_t) * (size_t)nchunks * (block_size + 1), (void**)&spill));
      P.q = q; P.sg = sg; P.n = n; P.block_size = block_size; P.p_star = p_star;
      P.nblocks = nblocks; P.hist = hist; P.freq = fc; P.rsize = rsize; P.wsize = wsize; P.off = off;
    }
  }
  // passes over `np` planes from p_top: histograms, tables, rANS sizes
  if (g_enc_nsm == 0) {
    int dev = 0;
    ATC_CUDA_TRY(cudaGetDevice(&dev));
    ATC_CUDA_TRY(cudaDeviceGetAttribute(&g_enc_nsm, cudaDevAttrMultiProcessorCount, dev));
  }
  auto size_pass = [&](int p_top, int np, int64_t il, int64_t it) -> int {
    const int64_t nch = nblocks * np;
    ATC_CUDA_TRY(cudaMemsetAsync(hist, 0, sizeof(unsigned long long) * np * kNsym, s));
    if (block_path) {
      B.p_top = p_top; B.nplanes = np; B.i_lead = il; B.i_trail = it;
      const int64_t waves = (int64_t)g_enc_nsm * kEncBlockResident;
      if (np == 1 && p_top != p_star) {
        // the cost pass of plane p_star + 1: a warp per block
        KTimed kt_(s, "enc_cost_plane_kernel", (double)n * 8.0 + (double)nblocks * (double)B.run_slot * 4.0 / nplanes);
        const int64_t ctas = (nblocks + kEncBlockThreads / 32 - 1) / (kEncBlockThreads / 32);
        enc_cost_plane_kernel<<<(unsigned)(ctas < waves ? ctas : waves), kEncBlockThreads, 0, s>>>(B);
      } else {
        KTimed kt_(s, "enc_block_kernel", (double)n * 9.0 + (double)nblocks * (double)B.run_slot * 4.0 * np / nplanes);
        const size_t dyn = (size_t)10 * B.block_size + B.block_size / 32;
        enc_block_kernel<<<(unsigned)(nblocks < waves ? nblocks : waves), kEncBlockThreads, dyn, s>>>(B);
      }
      ATC_LAUNCHED(1);
      freq_kernel<<<(np + 63) / 64, 64, 0, s>>>(hist, np, fc);
      ATC_LAUNCHED(1);
      R.nplanes = np;
      R.nchunks = nch;
      KTimed kt_(s, "enc_rans_thread_kernel(sizes)");
      enc_rans_thread_kernel<<<(unsigned)((nch + 127) / 128), 128, 0, s>>>(R, 0);
    } else {
      P.p_top = p_top; P.nplanes = np; P.i_lead = il; P.i_trail = it;
      const int wpb = 4;
      {
        KTimed kt_(s, "enc_hist_kernel");
        enc_hist_kernel<<<(unsigned)((nch + wpb - 1) / wpb), 32 * wpb, 0, s>>>(P);
      }
      ATC_LAUNCHED(1);
      freq_kernel<<<(np + 63) / 64, 64, 0, s>>>(hist, np, fc);
      ATC_LAUNCHED(1);
      KTimed kt_(s, "enc_rans_kernel(sizes)");
      enc_rans_kernel<<<(unsigned)((nch + kEncWarps - 1) / kEncWarps), 32 * kEncWarps, 0, s>>>(P, 1, spill);
    }
    ATC_LAUNCHED(1);
    return ATC_OK;
  };
  // split truncation of plane p_star (Supplement S.3)
  if (nplanes > 0) {
    {
      KTimed kt_(s, "split_stats_kernel", (double)n * 8.0);
      split_stats_kernel<<<nseg, kSegThreads, 0, s>>>(q, n, seg_len, p_star, sseg);
    }
    ATC_LAUNCHED(1);
    int64_t ncost = 0;
    if (p_star <= 62) {
      ATC_TRY(size_pass(p_star + 1, 1, -1, -1));
      ncost = nblocks;
    }
    {
      KTimed kt_(s, "split_kernel");
      split_kernel<<<1, kIstarThreads, 0, s>>>(q, n, seg_len, sseg, nseg, p_star, rsize, ncost, st);
    }
    ATC_LAUNCHED(1);
  }
  ATC_CUDA_TRY(cudaMemcpyAsync(&hst, st, sizeof(hst), cudaMemcpyDeviceToHost, s));
  ATC_CUDA_TRY(cudaStreamSynchronize(s));
  int prio = 0;
  int64_t i_lead = n - 1, i_trail = n - 1;
  if (nplanes > 0) {
    prio = hst.prio;
    i_lead = hst.i_lead;
    i_trail = hst.i_trail;
  }
  ATC_CUDA_TRY(cudaEventRecord(e1, s));
  // ------------------------------------------------ encoding
  const size_t hdr = kQHdr + (size_t)nplanes * kNsym * 2;
  const size_t tabb = (size_t)nchunks * 8;
  std::vector<uint8_t> head(hdr, 0);
  memcpy(head.data(), "ATCQ", 4);
  put32(head.data() + 4, 2);
  put64(head.data() + 8, (uint64_t)n);
  put32(head.data() + 16, (uint32_t)k);
  put32(head.data() + 20, (uint32_t)block_size);
  put32(head.data() + 24, (uint32_t)p_star);
  put32(head.data() + 28, (uint32_t)prio);
  put64(head.data() + 32, (uint64_t)i_lead);
  put64(head.data() + 40, (uint64_t)i_trail);
  put32(head.data() + 48, (uint32_t)nplanes);
  put32(head.data() + 52, kNsym);
  out->payload = nullptr;
  out->payload_bytes = 0;
  if (nplanes > 0) {
    ATC_TRY(size_pass(63, nplanes, i_lead, i_trail));
    {
      unsigned long long* sc = nullptr;
      ATC_TRY(Scratch::get(SLOT_SCAN, sizeof(unsigned long long) * (range_scan_parts(nchunks) + 8), (void**)&sc));
      ChunkBytes f{rsize, wsize};
      ATC_TRY(range_scan(f, nchunks, 0ull, sc, off, ~0ull, nullptr, s));
    }
    uint64_t* ptotal = reinterpret_cast<uint64_t*>(hstp + 1);
    uint32_t* hfc = reinterpret_cast<uint32_t*>(ptotal + 2);
    ATC_CUDA_TRY(cudaMemcpyAsync(ptotal, off + nchunks, sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
    ATC_CUDA_TRY(cudaMemcpyAsync(hfc, fc, sizeof(uint32_t) * nplanes * kNsym, cudaMemcpyDeviceToHost, s));
    ATC_CUDA_TRY(cudaStreamSynchronize(s));
    const uint64_t total = *ptotal;
    for (int i = 0; i < nplanes * kNsym; ++i) {
      head[kQHdr + 2 * i] = (uint8_t)hfc[i];
      head[kQHdr + 2 * i + 1] = (uint8_t)(hfc[i] >> 8);
    }
    uint8_t* dout = nullptr;
    ATC_TRY(Scratch::get(SLOT_OUT, tabb + total + 64, (void**)&dout));
    if (block_path) {
      R.table = reinterpret_cast<uint32_t*>(dout);
      R.out = dout + tabb;
      KTimed kt_(s, "enc_rans_thread_kernel");
      enc_rans_thread_kernel<<<(unsigned)((nchunks + 127) / 128), 128, 0, s>>>(R, 1);
    } else {
      P.table = reinterpret_cast<uint32_t*>(dout);
      P.out = dout + tabb;
      KTimed kt_(s, "enc_rans_kernel");
      enc_rans_kernel<<<(unsigned)((nchunks + kEncWarps - 1) / kEncWarps), 32 * kEncWarps, 0, s>>>(P, 0, spill);
    }
    ATC_LAUNCHED(1);
    out->payload = dout;
    out->payload_bytes = tabb + total;
  }
  ATC_CUDA_TRY(cudaEventRecord(e2, s));
  ATC_CUDA_TRY(cudaEventSynchronize(e2));
  float a = 0.f, b = 0.f;
  cudaEventElapsedTime(&a, e0, e1);
  cudaEventElapsedTime(&b, e1, e2);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaEventDestroy(e2);
  if (ms_quant) *ms_quant = a;
  if (ms_encode) *ms_encode = b;
  if (res) {
    res->k = k;
    res->p_star = p_star;
    res->prio = prio;
    res->i_lead = i_lead;
    res->i_trail = i_trail;
    res->sse_pred = ldexp(i192_to_double(hst.e_star), -2 * k);
  }
  out->head.swap(head);
  return ATC_OK;
}

namespace {
// Slices of the core that keep a significant coefficient (Section 3.3, the
// paragraph after Table 2): coefficient j of the vectorised core is significant
// when one of its encoded bits is a 1 -- its leading 1 lies above p_star, or on
// p_star with the leading bits of plane p_star encoded through j (j <= i_lead);
// its storage-order index on axis a marks slice idx_a of mode perm[a].  A flag is read before it is set, so a slice costs one
// atomic however many significant coefficients it holds.
struct KeptArgs {
  int d;
  int64_t dim[8];  // storage-order sizes (the vectorisation's row-major shape)
  int off[8];      // first flag of storage axis a
};
__global__ void kept_slices_kernel(const uint64_t* __restrict__ q, int64_t n, int p_star, int64_t i_lead, KeptArgs a,
                                   unsigned* __restrict__ flags) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    const int lo = (j <= i_lead) ? p_star : p_star + 1;
    if (lo >= 64 || (q[j] >> lo) == 0ull) continue;
    int64_t rem = j;
    for (int ax = a.d - 1; ax >= 0; --ax) {
      const int64_t idx = rem % a.dim[ax];
      rem /= a.dim[ax];
      unsigned* f = flags + a.off[ax] + idx;
      if (*reinterpret_cast<volatile unsigned*>(f) == 0u) atomicOr(f, 1u);
    }
  }
}
}  // namespace

// kept[i][c] (host, sum_i ranks[i] bytes, mode-major) for the core most recently
// quantized by quantize_encode on this device (its magnitudes are still in the
// quantizer scratch): 1 where slice c of mode i holds a significant coefficient.
int core_kept_slices(int64_t n, const int64_t* ranks, const int* perm, int d, int p_star, int64_t i_lead,
                     uint8_t* kept_host, cudaStream_t s) {
  if (d < 1 || d > 8) return fail(ATC_EINVAL, "core_kept_slices: ndim %d", d);
  int total = 0, moff[8];
  for (int i = 0; i < d; ++i) {
    moff[i] = total;
    total += (int)ranks[i];
  }
  uint64_t* q = nullptr;
  ATC_TRY(Scratch::get(SLOT_Q, sizeof(uint64_t) * (size_t)n, (void**)&q));
  unsigned* flags = nullptr;
  ATC_TRY(Scratch::get(SLOT_KEPT, sizeof(unsigned) * (size_t)total + 64, (void**)&flags));
  ATC_CUDA_TRY(cudaMemsetAsync(flags, 0, sizeof(unsigned) * (size_t)total, s));
  KeptArgs a;
  a.d = d;
  for (int ax = 0; ax < d; ++ax) {
    a.dim[ax] = ranks[perm[ax]];
    a.off[ax] = moff[perm[ax]];
  }
  if (p_star < 64 && n > 0) {
    const int64_t gb = (n + 255) / 256;
    const int grid = (int)(gb < 152 * 16 ? gb : 152 * 16);
    KTimed kt_(s, "kept_slices_kernel", (double)n * 8.0);
    kept_slices_kernel<<<grid, 256, 0, s>>>(q, n, p_star, i_lead, a, flags);
  }
  ATC_LAUNCHED(1);
  std::vector<unsigned> h((size_t)total);
  ATC_CUDA_TRY(cudaMemcpyAsync(h.data(), flags, sizeof(unsigned) * (size_t)total, cudaMemcpyDeviceToHost, s));
  ATC_CUDA_TRY(cudaStreamSynchronize(s));
  for (int t = 0; t < total; ++t) kept_host[t] = h[t] ? 1 : 0;
  return ATC_OK;
}

int decode_dequantize(const uint8_t* bytes, size_t nbytes, double* core, int64_t n, cudaStream_t s) {
  if (!bytes || nbytes < (size_t)kQHdr) return fail(ATC_ECORRUPT, "core section too short");
  if (memcmp(bytes, "ATCQ", 4) != 0 || get32(bytes + 4) != 2) return fail(ATC_ECORRUPT, "bad core section magic/version");
  DecParams D;
  D.n = (int64_t)get64(bytes + 8);
  D.k = (int)get32(bytes + 16);
  D.block_size = (int)get32(bytes + 20);
  D.p_star = (int)get32(bytes + 24);
  const uint32_t prio = get32(bytes + 28);
  D.i_lead = (int64_t)get64(bytes + 32);
  D.i_trail = (int64_t)get64(bytes + 40);
  D.nplanes = (int)get32(bytes + 48);
  if (D.n != n) return fail(ATC_ECORRUPT, "core size mismatch (%lld vs %lld)", (long long)D.n, (long long)n);
  if (D.block_size < 32 || D.block_size > 65535 || (D.block_size % 32)) return fail(ATC_ECORRUPT, "bad block size");
  if (get32(bytes + 52) != kNsym) return fail(ATC_ECORRUPT, "bad alphabet size");
  if (D.p_star < 0 || D.p_star > 64 || D.nplanes != (D.p_star >= 64 ? 0 : 64 - D.p_star))
    return fail(ATC_ECORRUPT, "bad breakpoint plane");
  if (prio > 1) return fail(ATC_ECORRUPT, "bad split priority");
  // a breakpoint is -1 (nothing of its category on the last plane) .. n - 1
  if (D.i_lead < -1 || D.i_lead >= n || D.i_trail < -1 || D.i_trail >= n)
    return fail(ATC_ECORRUPT, "bad breakpoint index");
  D.nblocks = (n + D.block_size - 1) / D.block_size;
  D.tab = kQHdr + (int64_t)D.nplanes * kNsym * 2;
  if ((uint64_t)D.tab + (uint64_t)D.nblocks * D.nplanes * 8 > nbytes) return fail(ATC_ECORRUPT, "truncated size table");
  for (int pi = 0; pi < D.nplanes; ++pi) {
    uint32_t sum = 0;
    for (int i = 0; i < kNsym; ++i)
      sum += (uint32_t)bytes[kQHdr + 2 * (pi * kNsym + i)] | ((uint32_t)bytes[kQHdr + 2 * (pi * kNsym + i) + 1] << 8);
    if (sum != 0 && sum != kM) return fail(ATC_ECORRUPT, "bad frequency table");
  }
  D.nbytes = (int64_t)nbytes;
  uint8_t* dsec = nullptr;
  ATC_TRY(Scratch::get(SLOT_OUT, nbytes + 64, (void**)&dsec));
  ATC_CUDA_TRY(cudaMemcpyAsync(dsec, bytes, nbytes, cudaMemcpyHostToDevice, s));
  uint64_t* qt = nullptr;
  uint8_t* sg = nullptr;
  ATC_TRY(Scratch::get(SLOT_Q, sizeof(uint64_t) * n, (void**)&qt));
  ATC_TRY(Scratch::get(SLOT_QS, (size_t)n, (void**)&sg));
  uint8_t* small = nullptr;
  const int64_t nchunk = D.nblocks * D.nplanes;
  const bool run_path = D.block_size <= kDecMax && D.nplanes > 0;
  const int64_t noff = run_path ? nchunk : D.nblocks;
  ATC_TRY(Scratch::get(SLOT_ENC, sizeof(uint64_t) * (noff + 1) + 64, (void**)&small));
  int* err = reinterpret_cast<int*>(small);
  uint64_t* boff = reinterpret_cast<uint64_t*>(small + 64);
  ATC_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), s));
  D.sec = dsec; D.qt = qt; D.sg = sg; D.out = core; D.err = err; D.boff = boff;
  {
    // payload offset of every chunk (run path) or block, from the size table
    unsigned long long* sc = nullptr;
    ATC_TRY(Scratch::get(SLOT_SCAN, sizeof(unsigned long long) * (range_scan_parts(noff) + 8), (void**)&sc));
    const unsigned long long base = (unsigned long long)D.tab + (unsigned long long)D.nblocks * D.nplanes * 8;
    if (run_path) {
      TabBytes f{dsec + D.tab};
      ATC_TRY(range_scan(f, nchunk, base, sc, boff, (unsigned long long)D.nbytes, err, s));
      D.boff_stride = D.nplanes;
    } else {
      BlockBytes f{dsec + D.tab, D.nplanes};
      ATC_TRY(range_scan(f, D.nblocks, base, sc, boff, (unsigned long long)D.nbytes, err, s));
      D.boff_stride = 1;
    }
  }
  if (run_path) {
    // phase A: every (block, plane) chunk's runs in parallel; phase B: placement
    RunParams RP;
    RP.sec = dsec; RP.nbytes = D.nbytes; RP.tab = D.tab; RP.nplanes = D.nplanes; RP.nblocks = D.nblocks;
    RP.block_size = D.block_size; RP.coff = boff; RP.err = err;
    uint8_t* rbuf = nullptr;
    ATC_TRY(Scratch::get(SLOT_DEC_RUNS, sizeof(uint32_t) * (size_t)nchunk * (D.block_size + 2) +
                                            sizeof(int) * (size_t)nchunk + 256, (void**)&rbuf));
    RP.runs = reinterpret_cast<uint32_t*>(rbuf);
    RP.nruns = reinterpret_cast<int*>(rbuf + sizeof(uint32_t) * (size_t)nchunk * (D.block_size + 2));
    {
      KTimed kt_(s, "decode_runs_kernel");
      decode_runs_kernel<<<dim3((unsigned)((D.nblocks + kRunThreads - 1) / kRunThreads), (unsigned)D.nplanes),
                           kRunThreads, 0, s>>>(RP);
    }
    if (D.block_size <= kWDecMax) {
      KTimed kt_(s, "decode_place_warp_kernel");
      decode_place_warp_kernel<<<(unsigned)((D.nblocks + kWDecWarps - 1) / kWDecWarps), 32 * kWDecWarps, 0, s>>>(
          D, RP.runs, RP.nruns);
    } else {
      KTimed kt_(s, "decode_place_kernel");
      decode_place_kernel<<<(unsigned)D.nblocks, kDecThreads, 0, s>>>(D, RP.runs, RP.nruns);
    }
    ATC_LAUNCHED(2);
  } else if (D.block_size <= kDecMax) {
    static bool dec_attr = false;
    if (!dec_attr) {
      ATC_CUDA_TRY(cudaFuncSetAttribute(decode_block_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kDecDyn));
      dec_attr = true;
    }
    decode_block_kernel<<<(unsigned)D.nblocks, kDecThreads, kDecDyn, s>>>(D);
    ATC_LAUNCHED(1);
  } else {
    decode_kernel<<<(unsigned)((D.nblocks + 63) / 64), 64, 0, s>>>(D);
    ATC_LAUNCHED(1);
  }
  int herr = 0;
  ATC_CUDA_TRY(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
  ATC_CUDA_TRY(cudaStreamSynchronize(s));
  if (herr) return fail(ATC_ECORRUPT, "corrupt core payload (code %d)", herr);
  return ATC_OK;
}

}  // namespace atc
