// Rayleigh-Ritz step of the subspace iteration (k_subspace.cu): every
// eigenvalue and the leading eigenvectors of the small symmetric matrix
// B = V^T G V (K x K, K <= 64) in ONE CTA of 1024 threads, in double-float
// arithmetic (pairs of FP32: GB300 issues FP64 at 1/64 of the FP32 rate and
// every stage below is a chain of dependent steps), with the whole problem in
// shared memory:
//   1. Householder tridiagonalisation T = Q_T^T B Q_T on the lower triangle
//      (K - 2 steps, two CTA barriers a step: one thread per row forms
//      p = tau A v; warp 0 updates column s+1 and builds the next reflector
//      from it while warps of the other SM sub-partitions apply the rank-2
//      update to the remaining columns).
//   2. All K eigenvalues by Sturm counts (number of sign changes of the leading
//      principal minors of T - x I, one double-float multiply-add pair per row
//      with power-of-two rescaling): one shared round of 1024 geometrically
//      spaced points brackets every eigenvalue within a factor 1.09, then a
//      group of 8 lanes per eigenvalue narrows its bracket 9-fold per round to
//      2^-30 relative (brackets in double-float, points in float).
//   3. The provisional rank from the Ritz values, rp = the smallest r with
//      trace(G) - sum_{j<r} theta_j <= budget (FP64 warp prefix sum), and the
//      convergence test of the subspace, (|theta_K| / theta_rp)^T <= conv; the
//      vector count is nv = rp + extra (at most nmax).
//   4. The leading nv eigenvectors of T by inverse iteration (lane per vector:
//      LU with partial pivoting of T - theta I as selects, two solves), groups
//      of eigenvalues closer than 2^-12 relative re-orthonormalised by
//      Gram-Schmidt applied twice (a warp per group), then the
//      back-transformation Y = Q_T Z (two lanes per vector), normalised,
//      largest entry positive.
// Outputs: theta (K, descending, FP64), decision = {rp, nv (0 unless the
// subspace passed), passed, the tensor-core error word}, Y (K x nv row-major,
// FP64).
#include <math.h>
#include <stdint.h>

#include "atc_internal.cuh"
#include "dd.cuh"

namespace atc {
namespace {

constexpr int kRrThreads = 1024;
constexpr int kRrWarps = kRrThreads / 32;
constexpr int kRrMaxK = 64;
constexpr int kRrGroup = 8;    // multisection points per eigenvalue and round
constexpr int kRrRounds = 10;  // refinement rounds (9^9 > 0.09 * 2^30)
constexpr int kRrVecWarps = 2; // inverse iteration: lane = vector, at most 64 vectors

__device__ __forceinline__ dd rr_shfl(dd a, int o) {
  return dd{__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o)};
}
__device__ __forceinline__ dd rr_wsum(dd a) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) a = dd_add(a, rr_shfl(a, o));
  return a;
}
__device__ __forceinline__ dd rr_scale(dd a, float f) { return dd{a.hi * f, a.lo * f}; }

// Division and square root seeded by the MUFU approximations (about 2^-22
// relative); the exact double-float residual corrections that follow carry the
// result to double-float accuracy, so the IEEE-rounded float operations are not
// needed for the seeds.
__device__ __forceinline__ dd rr_div(dd a, dd b) {
  const float rb = __fdividef(1.0f, b.hi);
  const float q1 = a.hi * rb;
  const dd r = dd_sub(a, dd_mul(b, ddf(q1)));
  const dd q = dd_qts(q1, r.hi * rb);
  const dd r2 = dd_sub(a, dd_mul(b, q));
  return dd_add(q, ddf(r2.hi * rb));
}
__device__ __forceinline__ dd rr_sqrt(dd a) {
  if (a.hi <= 0.f) return dd{0.f, 0.f};
  const float rs = rsqrtf(a.hi);
  const float x = a.hi * rs;
  const dd r = dd_sub(a, dd_mul(ddf(x), ddf(x)));
  return dd_qts(x, r.hi * (0.5f * rs));
}

// Number of eigenvalues of the tridiagonal matrix (d, e2 = e^2) below x: sign
// changes of p_0 = 1, p_i = (d_{i-1} - x) p_{i-1} - e2_{i-2} p_{i-2} (the
// leading principal minors of T - x I; a sign change is a negative pivot of
// its LDL^T factorisation).  An exact zero is replaced by a tiny value of the
// opposite sign (a negative pivot, as the pivmin rule of bisection codes).
// Both kept minors are rescaled by the same power of two, which changes no
// sign or ratio.
__device__ int rr_count(const dd* __restrict__ d, const dd* __restrict__ e2, int K, dd x) {
  const float kPiv = 0x1p-80f;
  dd pm = dd{1.f, 0.f};
  dd pc = dd_sub(d[0], x);
  if (pc.hi == 0.f) pc = dd{-kPiv, 0.f};
  int cnt = pc.hi < 0.f;
  for (int i = 1; i < K; ++i) {
    dd pn = dd_sub(dd_mul(dd_sub(d[i], x), pc), dd_mul(e2[i - 1], pm));
    if (pn.hi == 0.f) pn = dd{-kPiv * pc.hi, 0.f};
    cnt += (pn.hi < 0.f) != (pc.hi < 0.f);
    pm = pc;
    pc = pn;
    const float m = fmaxf(fabsf(pc.hi), fabsf(pm.hi));
    if (m > 0x1p40f) {
      pc = rr_scale(pc, 0x1p-48f);
      pm = rr_scale(pm, 0x1p-48f);
    } else if (m < 0x1p-40f) {
      pc = rr_scale(pc, 0x1p48f);
      pm = rr_scale(pm, 0x1p48f);
    }
  }
  return cnt;
}

// Reflector of tridiagonalisation step s from column s of the lower triangle
// (x_i = A[i][s], i = s+1..K-1, at col[i * P]), one warp: H = I - tau v v^T with
// v_{s+1} = 1 maps x to alpha e_{s+1}; tau = 2 v0^2 / (v0^2 + sig) is computed
// from v itself, so H is orthogonal to working precision whatever the rounding
// of alpha.  e_s = alpha (or x_{s+1} when x is already zero below it, tau = 0).
__device__ void rr_reflector(const dd* __restrict__ col, int P, int s, int K, int lane, dd* __restrict__ v,
                             dd* tau_out, dd* e_out) {
  const dd zero = dd{0.f, 0.f}, one = dd{1.f, 0.f};
  dd part = zero;
  for (int k = s + 2 + lane; k < K; k += 32) part = dd_add(part, dd_mul(col[k * P], col[k * P]));
  const dd sig = rr_wsum(part);
  const dd x0 = col[(s + 1) * P];
  dd tau = zero, alpha = x0, scal = zero;
  if (sig.hi != 0.f) {
    const dd nrm = rr_sqrt(dd_add(dd_mul(x0, x0), sig));
    alpha = dd_neg_sign(x0) ? nrm : dd_neg(nrm);
    const dd v0 = dd_sub(x0, alpha);
    const dd v02 = dd_mul(v0, v0);
    tau = rr_div(dd_add(v02, v02), dd_add(v02, sig));
    scal = rr_div(one, v0);
  }
  for (int k = lane; k < K; k += 32) v[k] = (k == s + 1) ? one : ((k > s + 1) ? dd_mul(col[k * P], scal) : zero);
  if (lane == 0) {
    *tau_out = tau;
    *e_out = alpha;
  }
}

// pseudo-random start vector of inverse iteration, entries of magnitude [0.5, 1)
__device__ __forceinline__ float rr_start(uint32_t j, uint32_t i) {
  uint32_t h = (j + 1u) * 0x9E3779B1u ^ (i + 0x632BE5ABu) * 0x85EBCA77u;
  h ^= h >> 15;
  h *= 0x2C1B3C6Du;
  h ^= h >> 12;
  h *= 0x297A2D39u;
  h ^= h >> 15;
  const float m = 0.5f + (float)(h >> 9) * 0x1p-24f;
  return (h & 1u) ? m : -m;
}

// Inverse iteration for eigenvalue lam of (d, e), one lane per vector (the
// lanes of a warp run the same steps on their own vectors, so the row
// interchanges are selects, not branches): LU factorisation with partial
// pivoting of T - lam I (unit lower factor with multipliers fl and row
// interchanges fp; upper factor with diagonal fd (stored inverted) and two
// superdiagonals fu, fu2), then two solves from a pseudo-random start, each
// followed by a power-of-two rescaling.  Every array holds element i of this
// lane's vector at [i * 32] (conflict-free across the lanes); result in x.
__device__ void rr_invit(const dd* __restrict__ d, const dd* __restrict__ e, int K, dd lam, uint32_t seed,
                         dd* __restrict__ fd, dd* __restrict__ fl, dd* __restrict__ fu, dd* __restrict__ fu2,
                         float* __restrict__ fp, dd* __restrict__ x) {
  const dd zero = dd{0.f, 0.f};
  const float eps_piv = 0x1p-46f;
  for (int i = 0; i < K; ++i) {
    fd[i * 32] = dd_sub(d[i], lam);
    fl[i * 32] = (i < K - 1) ? e[i] : zero;
    fu[i * 32] = fl[i * 32];
    fu2[i * 32] = zero;
    x[i * 32] = ddf(rr_start(seed, (uint32_t)i));
  }
  for (int i = 0; i < K - 1; ++i) {
    const dd a = fd[i * 32], b = fl[i * 32], u1 = fu[i * 32], d1 = fd[(i + 1) * 32];
    const dd u2 = (i < K - 2) ? fu[(i + 1) * 32] : zero;
    const bool sw = fabsf(a.hi) < fabsf(b.hi);
    dd piv = a;
    if (fabsf(piv.hi) < eps_piv) piv = dd{piv.hi < 0.f ? -eps_piv : eps_piv, 0.f};
    const dd den = sw ? b : piv;
    const dd l = rr_div(sw ? a : b, den);
    fd[i * 32] = den;
    fl[i * 32] = l;
    fu[i * 32] = sw ? d1 : u1;
    fd[(i + 1) * 32] = dd_sub(sw ? u1 : d1, dd_mul(l, sw ? d1 : u1));
    if (i < K - 2) {
      fu2[i * 32] = sw ? u2 : zero;
      fu[(i + 1) * 32] = sw ? dd_neg(dd_mul(l, u2)) : u2;
    }
    fp[i * 32] = sw ? 1.f : 0.f;
  }
  for (int i = 0; i < K; ++i) {
    dd v = fd[i * 32];
    if (fabsf(v.hi) < eps_piv) v = dd{v.hi < 0.f ? -eps_piv : eps_piv, 0.f};
    fd[i * 32] = rr_div(dd{1.f, 0.f}, v);
  }
  for (int it = 0; it < 2; ++it) {
    dd xi = x[0];
    for (int i = 0; i < K - 1; ++i) {
      dd xn = x[(i + 1) * 32];
      const bool sw = fp[i * 32] != 0.f;
      const dd lo = sw ? xn : xi, hi = sw ? xi : xn;
      x[i * 32] = lo;
      xi = dd_sub(hi, dd_mul(fl[i * 32], lo));
    }
    x[(K - 1) * 32] = xi;
    float mx = 0.f;
    dd x1 = zero, x2 = zero;
    for (int i = K - 1; i >= 0; --i) {
      const dd v = dd_sub(dd_sub(x[i * 32], dd_mul(fu[i * 32], x1)), dd_mul(fu2[i * 32], x2));
      const dd r = dd_mul(v, fd[i * 32]);
      x[i * 32] = r;
      x2 = x1;
      x1 = r;
      mx = fmaxf(mx, fabsf(r.hi));
    }
    int ex = 0;
    if (mx > 0.f) frexpf(mx, &ex);
    const float sc = ldexpf(1.0f, -ex);
    for (int i = 0; i < K; ++i) x[i * 32] = rr_scale(x[i * 32], sc);
  }
}

// One reflector of the back-transformation on this lane's rows (i0, i0 + 2, ...)
// of vector z; the partner lane (lane ^ 16) holds the other rows.  Restrict-
// qualified: the reflector rows and the vectors are disjoint parts of one
// shared array.
__device__ __forceinline__ void rr_bt_apply(const dd* __restrict__ hs, dd* __restrict__ z, int i0, int K, dd t,
                                            bool act) {
  const dd zero = dd{0.f, 0.f};
  dd a0 = zero, a1 = zero;
  int i = i0;
  for (; i + 2 < K; i += 4) {
    a0 = dd_add(a0, dd_mul(hs[i], z[i]));
    a1 = dd_add(a1, dd_mul(hs[i + 2], z[i + 2]));
  }
  if (i < K) a0 = dd_add(a0, dd_mul(hs[i], z[i]));
  dd dt = dd_add(a0, a1);
  dt = dd_add(dt, rr_shfl(dt, 16));
  const dd f = dd_mul(t, dt);
  if (act) {
    int i2 = i0;
    for (; i2 + 2 < K; i2 += 4) {
      const dd x0 = z[i2], x1 = z[i2 + 2], h0 = hs[i2], h1 = hs[i2 + 2];
      z[i2] = dd_sub(x0, dd_mul(f, h0));
      z[i2 + 2] = dd_sub(x1, dd_mul(f, h1));
    }
    if (i2 < K) z[i2] = dd_sub(z[i2], dd_mul(f, hs[i2]));
  }
}

__global__ void __launch_bounds__(kRrThreads) rr_kernel(const double* __restrict__ B, int K, int n,
                                                        const double* __restrict__ trace_g, double budget, int extra,
                                                        int nmax, double conv, int T, const int* __restrict__ tc_err,
                                                        double* __restrict__ theta_out, int* __restrict__ decision,
                                                        double* __restrict__ Y) {
  extern __shared__ dd sm[];
  const int P = K | 1;                          // odd pitches: row- and column-wise access are conflict-free
  dd* A = sm;                                   // K x P, lower triangle used
  dd* H = A + K * P;                            // reflector s in row s (pitch K)
  dd* Z = H + K * K;                            // nmax x P: vector j in row j
  dd* IV = Z + nmax * P;                        // kRrVecWarps x 5 x K x 32 (fd, fl, fu, fu2, x)
  float* FP = reinterpret_cast<float*>(IV + (size_t)kRrVecWarps * 5 * K * 32);  // kRrVecWarps x K x 32
  __shared__ dd s_d[kRrMaxK], s_e[kRrMaxK], s_e2[kRrMaxK], s_tau[kRrMaxK], s_p[kRrMaxK];
  __shared__ dd s_v[2][kRrMaxK];
  __shared__ dd s_pv[2];
  __shared__ double s_red[kRrWarps];
  __shared__ double s_theta[kRrMaxK];
  __shared__ int s_cnt[kRrThreads];
  __shared__ int s_grp[kRrMaxK + 1];
  __shared__ int s_ngrp, s_nv;
  __shared__ float s_tsc;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const dd zero = dd{0.f, 0.f};

  // ---- 1. load, power-of-two scale (largest |B| in [0.5, 1)), tridiagonalise
  double mx = 0.0;
  for (int e = tid; e < K * K; e += kRrThreads) mx = fmax(mx, fabs(B[e]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) s_red[warp] = mx;
  __syncthreads();
  mx = 0.0;
  for (int q = 0; q < kRrWarps; ++q) mx = fmax(mx, s_red[q]);
  int exb = 0;
  if (mx > 0.0) frexp(mx, &exb);
  const double scb = ldexp(1.0, -exb);
  for (int e = tid; e < K * K; e += kRrThreads) {
    const int i = e / K, k = e - i * K;
    if (k <= i) A[i * P + k] = dd_from(B[e] * scb);
  }
  __syncthreads();
  // Step s (a warp-0 reflector v_s from column s is ready):
  //   P: p_i = tau sum_{k > s} A[i][k] v_k for rows i > s, one thread per row
  //      (symmetric reads from the lower triangle), p . v summed per warp;
  //   U: w = p - (tau/2)(p . v) v, A <- A - v w^T - w v^T on the lower triangle
  //      of rows/columns > s; warp 0 updates column s+1 and builds the next
  //      reflector from it while warps 1..8 update the columns > s+1.
  if (K >= 3) {
    if (warp == 0) {
      rr_reflector(A, P, 0, K, lane, s_v[0], &s_tau[0], &s_e[0]);
      if (lane == 0) s_d[0] = A[0];
    }
    __syncthreads();
    for (int s = 0; s <= K - 3; ++s) {
      const dd* v = s_v[s & 1];
      const dd tau = s_tau[s];
      if (warp == 2) {
        for (int k = lane; k < K; k += 32) H[s * K + k] = v[k];
      } else if (warp < 2) {
        const int i = s + 1 + tid;
        dd pi = zero;
        if (i < K) {
          dd a0 = zero, a1 = zero, a2 = zero, a3 = zero;
          int k = s + 1;
          for (; k + 3 < K; k += 4) {
            a0 = dd_add(a0, dd_mul((k <= i) ? A[i * P + k] : A[k * P + i], v[k]));
            a1 = dd_add(a1, dd_mul((k + 1 <= i) ? A[i * P + k + 1] : A[(k + 1) * P + i], v[k + 1]));
            a2 = dd_add(a2, dd_mul((k + 2 <= i) ? A[i * P + k + 2] : A[(k + 2) * P + i], v[k + 2]));
            a3 = dd_add(a3, dd_mul((k + 3 <= i) ? A[i * P + k + 3] : A[(k + 3) * P + i], v[k + 3]));
          }
          for (; k < K; ++k) a0 = dd_add(a0, dd_mul((k <= i) ? A[i * P + k] : A[k * P + i], v[k]));
          pi = dd_mul(tau, dd_add(dd_add(a0, a1), dd_add(a2, a3)));
          s_p[i] = pi;
        }
        const dd pv = rr_wsum((i < K) ? dd_mul(pi, v[i]) : zero);
        if (lane == 0) s_pv[warp] = pv;
      }
      __syncthreads();
      const dd kc = dd_mul(dd_mul(ddf(0.5f), tau), dd_add(s_pv[0], s_pv[1]));
      if (warp == 0) {
        const int c = s + 1;
        const dd vc = v[c], wc = dd_sub(s_p[c], dd_mul(kc, vc));
        for (int i = c + lane; i < K; i += 32) {
          const dd wi = dd_sub(s_p[i], dd_mul(kc, v[i]));
          A[i * P + c] = dd_sub(dd_sub(A[i * P + c], dd_mul(v[i], wc)), dd_mul(wi, vc));
        }
        __syncwarp();
        if (c <= K - 3) {
          rr_reflector(A + c, P, c, K, lane, s_v[c & 1], &s_tau[c], &s_e[c]);
          if (lane == 0) s_d[c] = A[c * P + c];
        } else if (lane == 0) {
          s_d[c] = A[c * P + c];
          s_e[c] = A[(c + 1) * P + c];
        }
      } else if ((warp & 3) != 0 && warp < 12) {
        // rows i >= s+2, columns s+2 .. i: warps 1-3, 5-7, 9-11 (warp 0 keeps its SM sub-partition)
        const int u = warp - 1 - (warp >> 2);
        for (int i = s + 2 + u; i < K; i += 9) {
          const dd vi = v[i], wi = dd_sub(s_p[i], dd_mul(kc, vi));
          for (int k = s + 2 + lane; k <= i; k += 32) {
            const dd wk = dd_sub(s_p[k], dd_mul(kc, v[k]));
            A[i * P + k] = dd_sub(dd_sub(A[i * P + k], dd_mul(vi, wk)), dd_mul(wi, v[k]));
          }
        }
      }
      __syncthreads();
    }
    if (tid == 0) s_d[K - 1] = A[(K - 1) * P + K - 1];
  } else if (tid == 0) {
    s_d[0] = A[0];
    if (K == 2) {
      s_d[1] = A[P + 1];
      s_e[0] = A[P];
    }
  }
  __syncthreads();

  // ---- 2. eigenvalues: scale T so that its Gershgorin discs lie in [-1, 1]
  if (warp == 0) {
    float g = 0.f;
    for (int i = lane; i < K; i += 32) {
      float r = fabsf(s_d[i].hi);
      if (i > 0) r += fabsf(s_e[i - 1].hi);
      if (i < K - 1) r += fabsf(s_e[i].hi);
      g = fmaxf(g, r);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) g = fmaxf(g, __shfl_xor_sync(0xffffffffu, g, o));
    if (lane == 0) {
      int ex = 0;
      if (g > 0.f) frexpf(g * (1.0f + 0x1p-20f), &ex);
      s_tsc = ldexpf(1.0f, -ex);
    }
  }
  __syncthreads();
  const float tsc = s_tsc;
  for (int i = tid; i < K; i += kRrThreads) {
    s_d[i] = rr_scale(s_d[i], tsc);
    if (i < K - 1) {
      s_e[i] = rr_scale(s_e[i], tsc);
      s_e2[i] = dd_mul(s_e[i], s_e[i]);
    } else {
      s_e[i] = zero;
      s_e2[i] = zero;
    }
  }
  __syncthreads();
  // shared round: point t = 511 is 0, t > 511 runs 2^-64 .. 1, t < 511 runs -2^-64 .. -1
  // (float exponentials: any increasing sequence brackets; no FP64 anywhere in the search)
  auto point = [](int t) -> float {
    if (t == 511) return 0.f;
    if (t > 511) return exp2f(-64.f + (float)(t - 512) * (64.f / 511.f));
    return -exp2f(-64.f + (float)(510 - t) * (64.f / 510.f));
  };
  s_cnt[tid] = rr_count(s_d, s_e2, K, ddf(point(tid)));
  __syncthreads();
  {
    const int j = tid / kRrGroup, q = tid % kRrGroup;
    const int m = K - 1 - j;  // ascending index of the j-th largest eigenvalue
    dd lo = ddf(-1.0f - 0x1p-20f), hi = ddf(1.0f + 0x1p-20f);
    if (j < K) {
      // smallest t with count(x_t) > m (counts are non-decreasing in t)
      int a = 0, b = kRrThreads;
      while (a < b) {
        const int c = (a + b) >> 1;
        if (s_cnt[c] > m) b = c;
        else a = c + 1;
      }
      if (a > 0) lo = ddf(point(a - 1));
      if (a < kRrThreads) hi = ddf(point(a));
    }
    const unsigned gshift = (unsigned)(lane & ~(kRrGroup - 1));
    const dd frac = dd_div(ddf((float)(q + 1)), ddf((float)(kRrGroup + 1)));
    for (int round = 0; round < kRrRounds; ++round) {
      const dd wd = dd_sub(hi, lo);
      const bool done = !(j < K) || (wd.hi <= 0x1p-30f * fmaxf(fabsf(lo.hi), fabsf(hi.hi)) + 0x1p-70f);
      if (__all_sync(0xffffffffu, done)) break;
      const dd xq = dd_add(lo, dd_mul(wd, frac));  // this lane's point
      const int c = (j < K) ? rr_count(s_d, s_e2, K, xq) : 0;
      const unsigned bal = (__ballot_sync(0xffffffffu, c > m) >> gshift) & ((1u << kRrGroup) - 1u);
      // new bracket [x_{f-1}, x_f] from the group's points (x_{-1} = lo, x_G = hi), f = first point above
      const int f = bal ? __ffs(bal) - 1 : kRrGroup;
      const int sl = (int)gshift + (f > 0 ? f - 1 : 0), sh = (int)gshift + (f < kRrGroup ? f : 0);
      const dd xl = dd{__shfl_sync(0xffffffffu, xq.hi, sl), __shfl_sync(0xffffffffu, xq.lo, sl)};
      const dd xh = dd{__shfl_sync(0xffffffffu, xq.hi, sh), __shfl_sync(0xffffffffu, xq.lo, sh)};
      if (!done) {
        if (f > 0) lo = xl;
        if (f < kRrGroup) hi = xh;
      }
    }
    if (j < K && q == 0) s_theta[j] = dd_to(rr_scale(dd_add(lo, hi), 0.5f));
  }
  __syncthreads();

  // ---- 3. provisional rank and convergence test (FP64, unscaled values; warp 0):
  // tail(r) = trace(G) - sum_{j<r} theta_j from a warp prefix sum, rp = first r with tail <= budget
  const double unsc = ldexp(1.0, exb) / (double)tsc;
  for (int j = tid; j < K; j += kRrThreads) theta_out[j] = s_theta[j] * unsc;
  if (warp == 0) {
    const double trs = *trace_g;
    double t0 = (lane < K) ? s_theta[lane] * unsc : 0.0;
    double t1 = (lane + 32 < K) ? s_theta[lane + 32] * unsc : 0.0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const double u0 = __shfl_up_sync(0xffffffffu, t0, o), u1 = __shfl_up_sync(0xffffffffu, t1, o);
      if (lane >= o) {
        t0 += u0;
        t1 += u1;
      }
    }
    t1 += __shfl_sync(0xffffffffu, t0, 31);
    const unsigned b0 = __ballot_sync(0xffffffffu, lane < K && fmax(0.0, trs - t0) <= budget);
    const unsigned b1 = __ballot_sync(0xffffffffu, lane + 32 < K && fmax(0.0, trs - t1) <= budget);
    if (lane == 0) {
      const int rp = b0 ? __ffs(b0) : (b1 ? 32 + __ffs(b1) : -1);
      int ok = 0;
      const int nv = rp + extra;
      if (rp >= 1 && rp < n && nv <= nmax && s_theta[rp - 1] > 0.0) {
        const double ratio = fabs(s_theta[K - 1]) / s_theta[rp - 1];
        double pw = 1.0;
        for (int t = 0; t < T; ++t) pw *= ratio;
        ok = pw <= conv;
      }
      decision[0] = rp;
      decision[1] = ok ? nv : 0;
      decision[2] = ok;
      decision[3] = tc_err ? *tc_err : 0;
      s_nv = ok ? nv : 0;
    }
  }
  __syncthreads();
  const int nv = s_nv;
  if (nv == 0) return;

  // ---- 4. eigenvectors: inverse iteration, lane = vector (warps 0 .. kRrVecWarps-1)
  if (warp < kRrVecWarps && warp * 32 < nv) {
    const int j = warp * 32 + lane;
    dd* f = IV + (size_t)warp * 5 * K * 32 + lane;
    dd* xv = f + 4 * K * 32;
    rr_invit(s_d, s_e, K, dd_from(s_theta[j < nv ? j : nv - 1]), (uint32_t)j, f, f + K * 32, f + 2 * K * 32,
             f + 3 * K * 32, FP + (size_t)warp * K * 32 + lane, xv);
    if (j < nv)
      for (int i = 0; i < K; ++i) Z[(size_t)j * P + i] = xv[i * 32];
  }
  if (tid == 0) {
    int g = 0;
    s_grp[0] = 0;
    for (int j = 1; j < nv; ++j)
      if (s_theta[j - 1] - s_theta[j] > 0x1p-12 * fabs(s_theta[j - 1]) + 0x1p-60) s_grp[++g] = j;
    s_grp[++g] = nv;
    s_ngrp = g;
  }
  __syncthreads();
  // groups of close eigenvalues: classical Gram-Schmidt twice, a warp per group
  for (int g = warp; g < s_ngrp; g += kRrWarps) {
    const int g0 = s_grp[g], g1 = s_grp[g + 1];
    if (g1 - g0 < 2) continue;
    for (int k = g0; k < g1; ++k) {
      dd* zk = Z + (size_t)k * P;
      for (int pass = 0; pass < 2; ++pass)
        for (int a = g0; a < k; ++a) {
          const dd* za = Z + (size_t)a * P;
          dd part = zero;
          for (int i = lane; i < K; i += 32) part = dd_add(part, dd_mul(za[i], zk[i]));
          const dd dt = rr_wsum(part);
          __syncwarp();
          for (int i = lane; i < K; i += 32) zk[i] = dd_sub(zk[i], dd_mul(dt, za[i]));
          __syncwarp();
        }
      dd part = zero;
      for (int i = lane; i < K; i += 32) part = dd_add(part, dd_mul(zk[i], zk[i]));
      const dd inv = rr_div(dd{1.f, 0.f}, rr_sqrt(rr_wsum(part)));
      __syncwarp();
      for (int i = lane; i < K; i += 32) zk[i] = dd_mul(zk[i], inv);
      __syncwarp();
    }
  }
  __syncthreads();
  // back-transformation y = H_0 ... H_{K-3} z: two lanes per vector (lanes l and
  // l + 16 take the rows of even and odd index), one shuffle per reflector
  {
    const int j = warp * 16 + (lane & 15), h = lane >> 4;
    if (warp * 16 < nv) {
      const bool act = j < nv;
      dd* z = Z + (size_t)(act ? j : 0) * P;
      for (int s = K - 3; s >= 0; --s) {
        const dd t = s_tau[s];
        if (t.hi == 0.f) continue;
        rr_bt_apply(H + s * K, z, s + 1 + ((s + 1 + h) & 1), K, t, act);
      }
      // normalise, largest entry positive, write FP64
      dd q = zero;
      float best = -1.f;
      int bidx = K;
      for (int i = h; i < K; i += 2) {
        q = dd_add(q, dd_mul(z[i], z[i]));
        const float a = fabsf(z[i].hi);
        if (a > best) {
          best = a;
          bidx = i;
        }
      }
      q = dd_add(q, rr_shfl(q, 16));
      const float ob = __shfl_xor_sync(0xffffffffu, best, 16);
      const int oi = __shfl_xor_sync(0xffffffffu, bidx, 16);
      if (ob > best || (ob == best && oi < bidx)) {
        best = ob;
        bidx = oi;
      }
      const dd inv = rr_div(dd{1.f, 0.f}, rr_sqrt(q));
      const float sg = (z[bidx].hi < 0.f) ? -1.f : 1.f;
      if (act)
        for (int i = h; i < K; i += 2) Y[(size_t)i * nv + j] = (double)sg * dd_to(dd_mul(z[i], inv));
    }
  }
}

}  // namespace

size_t rr_smem_bytes(int K, int nmax) {
  const size_t P = (size_t)(K | 1);
  return sizeof(dd) * ((size_t)K * P + (size_t)K * K + (size_t)nmax * P + (size_t)kRrVecWarps * 5 * K * 32) +
         sizeof(float) * (size_t)kRrVecWarps * K * 32;
}

int launch_rr_small(const double* B, int K, int n, const double* trace_dev, double budget, int extra, int nmax,
                    double conv, int T, const int* tc_err, double* theta_dev, int* decision_dev, double* Y_dev,
                    cudaStream_t s) {
  if (K < 1 || K > kRrMaxK || nmax < 1 || nmax > K || nmax > 32 * kRrVecWarps)
    return fail(ATC_EINVAL, "Rayleigh-Ritz solver: K = %d, nmax = %d unsupported", K, nmax);
  const size_t smem = rr_smem_bytes(K, nmax);
  if (smem > 180 * 1024) return fail(ATC_EINVAL, "Rayleigh-Ritz solver: K = %d, nmax = %d exceed shared memory", K, nmax);
  static bool attr = false;
  if (!attr) {
    ATC_CUDA_TRY(cudaFuncSetAttribute(rr_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 180 * 1024));
    attr = true;
  }
  rr_kernel<<<1, kRrThreads, smem, s>>>(B, K, n, trace_dev, budget, extra, nmax, conv, T, tc_err, theta_dev,
                                        decision_dev, Y_dev);
  ATC_LAUNCHED(1);
  return ATC_OK;
}

}  // namespace atc
