// Leading eigenpairs of a symmetric positive semi-definite n x n matrix by
// subspace iteration with a final Rayleigh-Ritz step.
//
// The split-precision paths certify every rank from measured residual tails
// (||X - U ._k Y||^2 + sum_{j>=r} ||Y_j||^2), so they need the leading
// r_h (+ margin) eigenvectors of the mode Gram matrix to moderate accuracy and
// its eigenvalues only to pick a provisional rank.  For the smooth fields this
// library targets the Gram spectrum falls by many orders of magnitude within
// the first few dozen eigenvalues, and K = 40 columns of
//     V <- orth(G V)  (T times),  B = V^T G V = Y Theta Y^T,  U = V Y
// reach the leading subspace to the angles the certification needs, with GEMM
// work and short QR chains instead of the n - 2 dependent Householder steps of
// a full tridiagonalisation.  The Rayleigh-Ritz kernel also takes the
// provisional rank and checks the Ritz ratio for convergence; when it is not
// assured the caller falls back to the full eigensolver.
//
// orth() is a blocked Householder QR in double-float (the columns of G V are
// conditioned like lambda_1 / lambda_K, far beyond what a Cholesky QR
// tolerates), one CTA with the block in shared memory; Q is then formed from
// the compact-WY panels, a warp per column.  The start block is orthonormal by
// construction.
#include <math.h>
#include <stdint.h>

#include "atc_internal.cuh"
#include "dd.cuh"

namespace atc {
namespace {

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Start block, orthonormal by construction: column c is the c-th DCT-II basis
// vector of length n (sqrt(1/n) for c = 0, sqrt(2/n) cos(pi (i + 1/2) c / n)
// otherwise) with row i multiplied by a pseudo-random sign s_i (an integer hash
// of i) -- a randomised orthonormal frame, no QR needed.
__global__ void sub_init_kernel(double* __restrict__ V, int n, int K) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n * K; e += gridDim.x * blockDim.x) {
    const int c = e / n, i = e - c * n;
    uint32_t h = (uint32_t)i * 0x9E3779B1u + 0x7F4A7C15u;
    h ^= h >> 15;
    h *= 0x2C1B3C6Du;
    h ^= h >> 12;
    const double sg = (h & 0x10000u) ? -1.0 : 1.0;
    const double v = (c == 0) ? sqrt(1.0 / n) : sqrt(2.0 / n) * cospi((double)(2 * i + 1) * c / (2.0 * n));
    V[e] = sg * v;
  }
}

// *ex = the exponent e with max_i G[i][i] * 2^-e in [0.5, 1) (G is PSD, so it
// bounds |G|; 0 for a zero matrix): the scale of the double-float copy of G V
__global__ void sub_scale_kernel(const double* __restrict__ G, int n, int* __restrict__ ex) {
  double m = 0.0;
  for (int i = threadIdx.x; i < n; i += 32) m = fmax(m, fabs(G[(int64_t)i * n + i]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (threadIdx.x == 0) {
    int e = 0;
    if (m > 0.0) frexp(m, &e);
    *ex = e;
  }
}

// W[c][i] = sum_k G[i][k] V[c][k]: a warp per (i, group of 8 columns c).
// Wd != nullptr: written as double-floats scaled by 2^-(*ex) (|W| <= sqrt(n)
// then, since |G| <= max diag and V has orthonormal columns) for the QR,
// which so needs no FP64 arithmetic; else FP64 into W.
__global__ void __launch_bounds__(256) sub_gemm_kernel(const double* __restrict__ G, int n,
                                                       const double* __restrict__ V, int K, double* __restrict__ W,
                                                       dd* __restrict__ Wd, const int* __restrict__ ex) {
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int ngrp = (K + 7) / 8;
  if (gw >= n * ngrp) return;
  const int i = gw / ngrp, c0 = (gw - i * ngrp) * 8;
  double acc[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) acc[q] = 0.0;
  const double* gi = G + (int64_t)i * n;
  for (int k = lane; k < n; k += 32) {
    const double g = gi[k];
#pragma unroll
    for (int q = 0; q < 8; ++q)
      if (c0 + q < K) acc[q] = fma(g, V[(int64_t)(c0 + q) * n + k], acc[q]);
  }
  const double sc = Wd ? ldexp(1.0, -*ex) : 1.0;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const double v = warp_sum_d(acc[q]);
    if (lane == q && c0 + q < K) {
      if (Wd) Wd[(int64_t)(c0 + q) * n + i] = dd_from(v * sc);
      else W[(int64_t)(c0 + q) * n + i] = v;
    }
  }
}

// B[a][c] = sum_i V[a][i] W[c][i] (symmetric: a warp per a <= c)
__global__ void __launch_bounds__(256) sub_proj_kernel(const double* __restrict__ V, const double* __restrict__ W,
                                                       int n, int K, double* __restrict__ B) {
  const int lane = threadIdx.x & 31;
  const int e = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (e >= K * K) return;
  const int a = e / K, c = e - a * K;
  if (c < a) return;
  double s = 0.0;
  for (int i = lane; i < n; i += 32) s = fma(V[(int64_t)a * n + i], W[(int64_t)c * n + i], s);
  s = warp_sum_d(s);
  if (lane == 0) {
    // symmetrise with the mirrored product: B is V^T G V for symmetric G
    B[a * K + c] = s;
    B[c * K + a] = s;
  }
}

// U[i][j] = sum_a V[a][i] Y[a][j] (U n x m row-major; Y K x m row-major), m = *m_dev
// (the vector count chosen on the device by the Rayleigh-Ritz kernel; 0: nothing)
__global__ void sub_rotate_kernel(const double* __restrict__ V, int n, int K, const double* __restrict__ Y,
                                  const int* __restrict__ m_dev, double* __restrict__ U) {
  const int m = *m_dev;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n * m; e += gridDim.x * blockDim.x) {
    const int i = e / m, j = e - i * m;
    double s0 = 0.0, s1 = 0.0;
    int a = 0;
    for (; a + 1 < K; a += 2) {
      s0 = fma(V[(int64_t)a * n + i], Y[a * m + j], s0);
      s1 = fma(V[(int64_t)(a + 1) * n + i], Y[(a + 1) * m + j], s1);
    }
    if (a < K) s0 = fma(V[(int64_t)a * n + i], Y[a * m + j], s0);
    U[e] = s0 + s1;
  }
}

__global__ void sub_trace_kernel(const double* __restrict__ G, int n, double* __restrict__ out) {
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += 32) s += G[(int64_t)i * n + i];
  s = warp_sum_d(s);
  if (threadIdx.x == 0) *out = s;
}

// Blocked Householder QR of the K columns of W (n x K, column c at W + c n,
// K <= 64 <= ... n), one CTA, in double-float (FP64 issues at 2 lanes per
// clock per SM on GB300; the pair arithmetic runs on the FP32 pipes).  The
// columns are taken in panels of kQrNb: inside a panel a pivot updates only
// the remaining panel columns (a warp each; the warp updating the next column
// also sums its squares below the diagonal, so the next pivot needs no block
// reduction), then the panel's reflectors are gathered in compact WY form
// H_p0 ... H_p1-1 = I - V T V^T (T upper triangular, from V^T V) and applied
// to every trailing column at once (a warp per column: V^T a, T^T, update).
// Outputs: the reflectors Vg (column j: 0 above row j, 1 at row j, v below)
// and the panels' T blocks Tg (kQrNb x kQrNb each), from which
// sub_qform_kernel forms Q column by column.
constexpr int kQrThreads = 512;
constexpr int kQrNb = 8;

__device__ __forceinline__ dd dd_warp_sum_l(dd a) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
    a = dd_add(a, dd{__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o)});
  return a;
}
__device__ dd dd_block_sum(dd v, dd* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = dd_warp_sum_l(v);
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  dd t = dd{0.f, 0.f};
  for (int q = 0; q < nw; ++q) t = dd_add(t, red[q]);
  return t;
}

// Division and square root seeded by the MUFU approximations (about 2^-22
// relative); the exact double-float residual corrections carry the results to
// double-float accuracy.
__device__ __forceinline__ dd qr_div(dd a, dd b) {
  const float rb = __fdividef(1.0f, b.hi);
  const float q1 = a.hi * rb;
  const dd r = dd_sub(a, dd_mul(b, ddf(q1)));
  const dd q = dd_qts(q1, r.hi * rb);
  const dd r2 = dd_sub(a, dd_mul(b, q));
  return dd_add(q, ddf(r2.hi * rb));
}
__device__ __forceinline__ dd qr_sqrt(dd a) {
  if (a.hi <= 0.f) return dd{0.f, 0.f};
  const float rs = rsqrtf(a.hi);
  const float x = a.hi * rs;
  const dd r = dd_sub(a, dd_mul(ddf(x), ddf(x)));
  return dd_qts(x, r.hi * (0.5f * rs));
}

// column j of the reflector block: v_j = (1 at row j, a_j[i] / (x0 - alpha) below)
// (R is never used: the entries above row j are cleared, so the trailing
// updates can run over whole columns without row predicates)
__device__ __forceinline__ void qr_finalize(dd* __restrict__ aj, int j, int n, dd inv, dd tau, int lane) {
  const dd zero = dd{0.f, 0.f};
  for (int i = lane; i < n; i += 32)
    aj[i] = (i < j) ? zero : ((i == j) ? dd{1.f, 0.f} : ((tau.hi != 0.f) ? dd_mul(aj[i], inv) : zero));
}

__global__ void __launch_bounds__(kQrThreads) sub_qr_kernel(const dd* __restrict__ W, int n, int K,
                                                            dd* __restrict__ Vg, dd* __restrict__ Tg) {
  extern __shared__ dd A[];
  __shared__ dd red[32];
  __shared__ dd s_tau[64], s_inv[64];
  __shared__ dd s_sig[2], s_x0[2];
  __shared__ dd s_S[kQrNb * kQrNb], s_T[kQrNb * kQrNb];
  __shared__ float smx[32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  const dd zero = dd{0.f, 0.f}, one = dd{1.f, 0.f};
  // power-of-two scale: |entries| <= 1 keeps every pair product far from the float range limits
  float mx = 0.f;
  for (int e = tid; e < n * K; e += blockDim.x) mx = fmaxf(mx, fabsf(W[e].hi));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) smx[warp] = mx;
  __syncthreads();
  mx = 0.f;
  for (int q = 0; q < nw; ++q) mx = fmaxf(mx, smx[q]);
  int ex = 0;
  if (mx > 0.f) frexpf(mx, &ex);
  const float sc = ldexpf(1.0f, -ex);
  for (int e = tid; e < n * K; e += blockDim.x) {
    const dd w = W[e];
    A[e] = dd{w.hi * sc, w.lo * sc};
  }
  __syncthreads();
  for (int p0 = 0; p0 < K; p0 += kQrNb) {
    const int p1 = min(p0 + kQrNb, K), nb = p1 - p0;
    {
      const dd* a = A + (size_t)p0 * n;
      dd part = zero;
      for (int i = p0 + 1 + tid; i < n; i += blockDim.x) part = dd_add(part, dd_mul(a[i], a[i]));
      const dd sig = dd_block_sum(part, red);
      if (tid == 0) { s_sig[p0 & 1] = sig; s_x0[p0 & 1] = a[p0]; }
      for (int e = tid; e < kQrNb * kQrNb; e += blockDim.x) s_T[e] = zero;
      __syncthreads();
    }
    for (int j = p0; j < p1; ++j) {
      // only the warps that use the reflector form it (warp 0 stores tau and 1/v0)
      const int c = j + 1 + warp;
      const bool uses = c < p1 || warp == 0 || warp == nw - 1;
      const dd sig = s_sig[j & 1], x0 = s_x0[j & 1];
      dd tj = zero, inv = one;
      if (uses && sig.hi != 0.f) {
        const dd nrm = qr_sqrt(dd_add(dd_mul(x0, x0), sig));
        const dd alpha = dd_neg_sign(x0) ? nrm : dd_neg(nrm);
        const dd v0 = dd_sub(x0, alpha);
        const dd v02 = dd_mul(v0, v0);
        tj = qr_div(dd_add(v02, v02), dd_add(v02, sig));
        inv = qr_div(one, v0);
      }
      if (tid == 0) { s_tau[j] = tj; s_inv[j] = inv; }
      const dd* aj = A + (size_t)j * n;
      if (c < p1) {
        dd* ac = A + (size_t)c * n;
        if (tj.hi != 0.f) {
          // d = tau (a_c[j] + sum_{i>j} v_i a_c[i]) with v_i = inv a_j[i]
          dd s0 = zero, s1 = zero, s2 = zero, s3 = zero;
          int i = j + 1 + lane;
          for (; i + 96 < n; i += 128) {
            s0 = dd_add(s0, dd_mul(aj[i], ac[i]));
            s1 = dd_add(s1, dd_mul(aj[i + 32], ac[i + 32]));
            s2 = dd_add(s2, dd_mul(aj[i + 64], ac[i + 64]));
            s3 = dd_add(s3, dd_mul(aj[i + 96], ac[i + 96]));
          }
          for (; i < n; i += 32) s0 = dd_add(s0, dd_mul(aj[i], ac[i]));
          const dd sdot = dd_warp_sum_l(dd_add(dd_add(s0, s1), dd_add(s2, s3)));
          const dd acj = ac[j];
          const dd d = dd_mul(tj, dd_add(acj, dd_mul(inv, sdot)));
          const dd dv = dd_mul(d, inv);
          __syncwarp();
          if (lane == 0) ac[j] = dd_sub(acj, d);
          dd q = zero;
          for (int i2 = j + 1 + lane; i2 < n; i2 += 32) {
            const dd v = dd_sub(ac[i2], dd_mul(dv, aj[i2]));
            ac[i2] = v;
            if (i2 > j + 1) q = dd_add(q, dd_mul(v, v));
          }
          if (c == j + 1) {
            q = dd_warp_sum_l(q);
            if (lane == 0) { s_sig[(j + 1) & 1] = q; s_x0[(j + 1) & 1] = ac[j + 1]; }
          }
        } else if (c == j + 1) {
          dd q = zero;
          for (int i2 = j + 2 + lane; i2 < n; i2 += 32) q = dd_add(q, dd_mul(ac[i2], ac[i2]));
          q = dd_warp_sum_l(q);
          if (lane == 0) { s_sig[(j + 1) & 1] = q; s_x0[(j + 1) & 1] = ac[j + 1]; }
        }
      }
      // column j-1 is no longer read by the panel: scale it into its reflector
      if (warp == nw - 1 && j > p0) qr_finalize(A + (size_t)(j - 1) * n, j - 1, n, s_inv[j - 1], s_tau[j - 1], lane);
      __syncthreads();
    }
    if (warp == nw - 1) qr_finalize(A + (size_t)(p1 - 1) * n, p1 - 1, n, s_inv[p1 - 1], s_tau[p1 - 1], lane);
    __syncthreads();
    // S[a][b] = v_a . v_b for a < b (v_b is 0 above row p0 + b)
    for (int e = warp; e < nb * nb; e += nw) {
      const int a = e / nb, b = e - a * nb;
      if (a >= b) continue;
      const dd* va = A + (size_t)(p0 + a) * n;
      const dd* vb = A + (size_t)(p0 + b) * n;
      dd s0 = zero;
      for (int i = p0 + b + lane; i < n; i += 32) s0 = dd_add(s0, dd_mul(va[i], vb[i]));
      s0 = dd_warp_sum_l(s0);
      if (lane == 0) s_S[a * kQrNb + b] = s0;
    }
    __syncthreads();
    // T: T[b][b] = tau_b, T[0:b, b] = -tau_b T[0:b, 0:b] S[0:b, b]
    if (warp == 0) {
      for (int b = 0; b < nb; ++b) {
        const dd tb = s_tau[p0 + b];
        dd t = zero;
        if (lane < b)
          for (int c2 = lane; c2 < b; ++c2) t = dd_add(t, dd_mul(s_T[lane * kQrNb + c2], s_S[c2 * kQrNb + b]));
        __syncwarp();
        if (lane < b) s_T[lane * kQrNb + b] = dd_neg(dd_mul(tb, t));
        if (lane == b) s_T[b * kQrNb + b] = tb;
        __syncwarp();
      }
    }
    __syncthreads();
    for (int e = tid; e < kQrNb * kQrNb; e += blockDim.x) Tg[(size_t)(p0 / kQrNb) * kQrNb * kQrNb + e] = s_T[e];
    // trailing columns: a_c -= V (T^T (V^T a_c)), a warp per column
    for (int c = p1 + warp; c < K; c += nw) {
      dd* ac = A + (size_t)c * n;
      dd y[kQrNb];
#pragma unroll
      for (int a = 0; a < kQrNb; ++a) y[a] = zero;
      for (int i = p0 + lane; i < n; i += 32) {
        const dd x = ac[i];
#pragma unroll
        for (int a = 0; a < kQrNb; ++a)
          if (a < nb) y[a] = dd_add(y[a], dd_mul(A[(size_t)(p0 + a) * n + i], x));
      }
#pragma unroll
      for (int a = 0; a < kQrNb; ++a) y[a] = dd_warp_sum_l(y[a]);
      // z = T^T y: lane a < kQrNb forms z_a, then every lane takes all of them
      dd za = zero;
#pragma unroll
      for (int b = 0; b < kQrNb; ++b)
        if (b <= lane) za = dd_add(za, dd_mul(s_T[b * kQrNb + (lane & (kQrNb - 1))], y[b]));
      dd z[kQrNb];
#pragma unroll
      for (int a = 0; a < kQrNb; ++a)
        z[a] = dd{__shfl_sync(0xffffffffu, za.hi, a), __shfl_sync(0xffffffffu, za.lo, a)};
      __syncwarp();
      for (int i = p0 + lane; i < n; i += 32) {
        dd x = ac[i];
#pragma unroll
        for (int a = 0; a < kQrNb; ++a)
          if (a < nb) x = dd_sub(x, dd_mul(A[(size_t)(p0 + a) * n + i], z[a]));
        ac[i] = x;
      }
    }
    __syncthreads();
  }
  for (int e = tid; e < n * K; e += blockDim.x) Vg[e] = A[e];
}

// Q = H_0 H_1 ... H_{K-1} [I_K; 0] from the panels' WY blocks, a warp per
// column c: q = e_c, then q <- q - V_p (T_p (V_p^T q)) for the panels p from
// the one holding c down to the first (later panels leave e_c unchanged).  A
// CTA holds the kQrNb columns of one panel, so its warps walk the same panels:
// each panel's reflectors and T are staged in shared memory once per CTA.
constexpr int kQfWarps = kQrNb;
__global__ void __launch_bounds__(kQfWarps * 32) sub_qform_kernel(const dd* __restrict__ Vg, const dd* __restrict__ Tg,
                                                                  int n, int K, double* __restrict__ Q) {
  extern __shared__ dd qs[];
  __shared__ dd sT[kQrNb * kQrNb];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int c = blockIdx.x * kQfWarps + w;
  const bool active = c < K;
  const dd zero = dd{0.f, 0.f};
  dd* Vs = qs;                            // kQrNb x n
  dd* q = qs + (size_t)(kQrNb + w) * n;   // this warp's column
  for (int i = lane; i < n; i += 32) q[i] = (i == c) ? dd{1.f, 0.f} : zero;
  for (int p = (int)blockIdx.x; p >= 0; --p) {
    const int p0 = p * kQrNb, nb = min(kQrNb, K - p0);
    __syncthreads();
    for (int e = threadIdx.x; e < nb * n; e += blockDim.x) Vs[e] = Vg[(size_t)p0 * n + e];
    for (int e = threadIdx.x; e < kQrNb * kQrNb; e += blockDim.x) sT[e] = Tg[(size_t)p * kQrNb * kQrNb + e];
    __syncthreads();
    if (!active) continue;
    dd y[kQrNb];
#pragma unroll
    for (int a = 0; a < kQrNb; ++a) y[a] = zero;
    for (int i = p0 + lane; i < n; i += 32) {
      const dd x = q[i];
#pragma unroll
      for (int a = 0; a < kQrNb; ++a)
        if (a < nb) y[a] = dd_add(y[a], dd_mul(Vs[(size_t)a * n + i], x));
    }
#pragma unroll
    for (int a = 0; a < kQrNb; ++a) y[a] = dd_warp_sum_l(y[a]);
    dd z[kQrNb];
#pragma unroll
    for (int a = 0; a < kQrNb; ++a) {
      dd t = zero;
#pragma unroll
      for (int b = a; b < kQrNb; ++b)
        if (b < nb) t = dd_add(t, dd_mul(sT[a * kQrNb + b], y[b]));
      z[a] = t;
    }
    __syncwarp();
    for (int i = p0 + lane; i < n; i += 32) {
      dd x = q[i];
#pragma unroll
      for (int a = 0; a < kQrNb; ++a)
        if (a < nb) x = dd_sub(x, dd_mul(Vs[(size_t)a * n + i], z[a]));
      q[i] = x;
    }
    __syncwarp();
  }
  if (active)
    for (int i = lane; i < n; i += 32) Q[(size_t)c * n + i] = dd_to(q[i]);
}

}  // namespace

bool subspace_supported(int n, int K) {
  return K >= 5 && K <= 64 && K <= n && (size_t)n * K * sizeof(dd) <= 200 * 1024 &&
         (size_t)2 * kQrNb * n * sizeof(dd) <= 200 * 1024 && rr_smem_bytes(K, K - 4) <= 180 * 1024;
}

int subspace_solve(const double* G, int n, int K, int T, double budget, int extra, int nmax, double conv,
                   double* U_dev, double* theta_host, double* trace_host, int* decision_host, cudaStream_t s) {
  if (!subspace_supported(n, K)) return fail(ATC_EINVAL, "subspace_solve: unsupported n = %d, K = %d", n, K);
  if (nmax < 1 || nmax > K || T < 1) return fail(ATC_EINVAL, "subspace_solve: nmax = %d, T = %d", nmax, T);
  const size_t nk = (size_t)n * K;
  const int npan = (K + kQrNb - 1) / kQrNb;
  const size_t nd = 2 * nk + (size_t)K * K + K + 8 + nk + (size_t)npan * kQrNb * kQrNb + (size_t)K * nmax + 8;
  // (the last 8 doubles: decision ints and the scale exponent)
  double* base = nullptr;
  ATC_TRY(Scratch::get(SLOT_SUBSPACE, sizeof(double) * nd, (void**)&base));
  double* V = base;
  double* W = V + nk;
  double* B = W + nk;
  double* th = B + (size_t)K * K;
  double* tr = th + K;
  dd* Vg = reinterpret_cast<dd*>(tr + 8);
  dd* Tg = Vg + nk;
  double* Y = reinterpret_cast<double*>(Tg + (size_t)npan * kQrNb * kQrNb);
  int* dec = reinterpret_cast<int*>(Y + (size_t)K * nmax);
  int* gex = dec + 4;
  dd* Wd = reinterpret_cast<dd*>(W);  // the double-float copy of G V reuses the FP64 block
  const size_t qsm = sizeof(dd) * nk;
  const size_t fsm = sizeof(dd) * 2 * kQrNb * (size_t)n;
  static bool attr = false;
  if (!attr) {
    ATC_CUDA_TRY(cudaFuncSetAttribute(sub_qr_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    ATC_CUDA_TRY(cudaFuncSetAttribute(sub_qform_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    attr = true;
  }
  const int blocks = (int)((nk + 255) / 256 < 1024 ? (nk + 255) / 256 : 1024);
  sub_init_kernel<<<blocks, 256, 0, s>>>(V, n, K);
  sub_scale_kernel<<<1, 32, 0, s>>>(G, n, gex);
  ATC_LAUNCHED(2);
  const int gemm_blocks = (int)(((int64_t)n * ((K + 7) / 8) * 32 + 255) / 256);
  for (int t = 0; t < T; ++t) {
    sub_gemm_kernel<<<gemm_blocks, 256, 0, s>>>(G, n, V, K, nullptr, Wd, gex);
    ATC_LAUNCHED(1);
    sub_qr_kernel<<<1, kQrThreads, qsm, s>>>(Wd, n, K, Vg, Tg);
    ATC_LAUNCHED(1);
    sub_qform_kernel<<<(K + kQfWarps - 1) / kQfWarps, kQfWarps * 32, fsm, s>>>(Vg, Tg, n, K, V);
    ATC_LAUNCHED(1);
  }
  sub_gemm_kernel<<<gemm_blocks, 256, 0, s>>>(G, n, V, K, W, nullptr, gex);
  ATC_LAUNCHED(1);
  sub_proj_kernel<<<(K * K * 32 + 255) / 256, 256, 0, s>>>(V, W, n, K, B);
  sub_trace_kernel<<<1, 32, 0, s>>>(G, n, tr);
  ATC_LAUNCHED(2);
  // Rayleigh-Ritz on the K x K matrix B (one CTA), provisional rank and vector count on the device
  ATC_TRY(launch_rr_small(B, K, n, tr, budget, extra, nmax, conv, T, th, dec, Y, s));
  const int rblocks = (int)(((size_t)n * nmax + 255) / 256 < 1024 ? ((size_t)n * nmax + 255) / 256 : 1024);
  sub_rotate_kernel<<<rblocks, 256, 0, s>>>(V, n, K, Y, dec + 1, U_dev);
  ATC_LAUNCHED(1);
  ATC_CUDA_TRY(cudaMemcpyAsync(theta_host, th, sizeof(double) * K, cudaMemcpyDeviceToHost, s));
  ATC_CUDA_TRY(cudaMemcpyAsync(trace_host, tr, sizeof(double), cudaMemcpyDeviceToHost, s));
  ATC_CUDA_TRY(cudaMemcpyAsync(decision_host, dec, sizeof(int) * 3, cudaMemcpyDeviceToHost, s));
  return ATC_OK;
}

}  // namespace atc
