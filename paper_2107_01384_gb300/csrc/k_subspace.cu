// Leading eigenpairs of a symmetric positive semi-definite n x n matrix by
// subspace iteration with a final Rayleigh-Ritz step.
//
// The split-precision paths certify every rank from measured residual tails
// (||X - U ._k Y||^2 + sum_{j>=r} ||Y_j||^2), so they need the leading
// r_h (+ margin) eigenvectors of the mode Gram matrix to moderate accuracy and
// its eigenvalues only to pick a provisional rank.  For the smooth fields this
// library targets the Gram spectrum falls by many orders of magnitude within
// the first few dozen eigenvalues, and K = 32 columns of
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

// W = G V (G n x n symmetric, V K columns of n): CTA (x, c) computes rows
// [32 x, 32 x + 32) of column c; its eight warps take eight consecutive k
// ranges (four FMA chains a lane), then warp 0 adds the eight parts in warp
// order.  Wd != nullptr: the result as double-floats scaled by 2^-(*ex)
// (|W| <= sqrt(n) then, since |G| <= max diag and V has orthonormal columns),
// so that the QR needs no FP64 arithmetic; else FP64 into W.
constexpr int kGemmWarps = 8;
// trace != nullptr (the first product of a solve): from the diagonal of G
// every CTA also takes the exponent e with max_i G_ii 2^-e in [0.5, 1) (G is
// PSD, so its diagonal bounds |G|; 0 for a zero matrix) for its own scaling,
// and CTA (0, 0) stores e and trace(G).
__global__ void __launch_bounds__(32 * kGemmWarps) sub_gemm_kernel(const double* __restrict__ G, int n,
                                                                  const double* __restrict__ V, double* __restrict__ W,
                                                                  dd* __restrict__ Wd, int* __restrict__ ex,
                                                                  double* __restrict__ trace) {
  __shared__ double red[kGemmWarps][32];
  __shared__ int s_ex;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (trace && warp == kGemmWarps - 1) {
    double m = 0.0, t = 0.0;
    for (int i = lane; i < n; i += 32) {
      const double g = G[(int64_t)i * n + i];
      m = fmax(m, fabs(g));
      t += g;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
      t += __shfl_xor_sync(0xffffffffu, t, o);
    }
    if (lane == 0) {
      int e = 0;
      if (m > 0.0) frexp(m, &e);
      s_ex = e;
      if (blockIdx.x == 0 && blockIdx.y == 0) {
        *ex = e;
        *trace = t;
      }
    }
  }
  const int i = blockIdx.x * 32 + lane;
  const int c = blockIdx.y;
  const int k0 = (int)((int64_t)n * warp / kGemmWarps), k1 = (int)((int64_t)n * (warp + 1) / kGemmWarps);
  const double* vc = V + (int64_t)c * n;
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
  if (i < n) {
    int k = k0;
    for (; k + 3 < k1; k += 4) {
      a0 = fma(__ldg(G + (int64_t)k * n + i), __ldg(vc + k), a0);
      a1 = fma(__ldg(G + (int64_t)(k + 1) * n + i), __ldg(vc + k + 1), a1);
      a2 = fma(__ldg(G + (int64_t)(k + 2) * n + i), __ldg(vc + k + 2), a2);
      a3 = fma(__ldg(G + (int64_t)(k + 3) * n + i), __ldg(vc + k + 3), a3);
    }
    for (; k < k1; ++k) a0 = fma(__ldg(G + (int64_t)k * n + i), __ldg(vc + k), a0);
  }
  red[warp][lane] = (a0 + a1) + (a2 + a3);
  __syncthreads();
  if (warp == 0 && i < n) {
    double v = red[0][lane];
#pragma unroll
    for (int w = 1; w < kGemmWarps; ++w) v += red[w][lane];
    const int64_t e = (int64_t)c * n + i;
    if (Wd) Wd[e] = dd_from(v * __longlong_as_double((long long)(1023 - (trace ? s_ex : *ex)) << 52));  // v 2^-ex
    else W[e] = v;
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
                                  const int* __restrict__ m_dev, double* __restrict__ U, int ldu) {
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
    U[(int64_t)i * ldu + j] = s0 + s1;
  }
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

// Inner loops of the QR as helpers with restrict-qualified operands (the
// reflector columns and the columns they update are disjoint parts of one
// shared array, which the compiler cannot see through the offsets).
// d = tau (c[j] + inv sum_{i>j} a[i] c[i]), four accumulators, warp-summed
__device__ __forceinline__ dd qr_pivot_dot(const dd* __restrict__ a, const dd* __restrict__ c, int j, int n,
                                           int lane) {
  const dd zero = dd{0.f, 0.f};
  dd s0 = zero, s1 = zero, s2 = zero, s3 = zero;
  int i = j + 1 + lane;
  for (; i + 96 < n; i += 128) {
    s0 = dd_add(s0, dd_mul(a[i], c[i]));
    s1 = dd_add(s1, dd_mul(a[i + 32], c[i + 32]));
    s2 = dd_add(s2, dd_mul(a[i + 64], c[i + 64]));
    s3 = dd_add(s3, dd_mul(a[i + 96], c[i + 96]));
  }
  for (; i < n; i += 32) s0 = dd_add(s0, dd_mul(a[i], c[i]));
  return dd_warp_sum_l(dd_add(dd_add(s0, s1), dd_add(s2, s3)));
}
// c[i] -= dv a[i] for i > j; returns the lane's sum of the new c[i]^2 for i > j + 1
__device__ __forceinline__ dd qr_pivot_update(const dd* __restrict__ a, dd* __restrict__ c, dd dv, int j, int n,
                                              int lane) {
  const dd zero = dd{0.f, 0.f};
  dd q0 = zero, q1 = zero;
  int i = j + 1 + lane;
  for (; i + 32 < n; i += 64) {
    const dd x0 = c[i], x1 = c[i + 32], y0 = a[i], y1 = a[i + 32];
    const dd v0 = dd_sub(x0, dd_mul(dv, y0)), v1 = dd_sub(x1, dd_mul(dv, y1));
    c[i] = v0;
    c[i + 32] = v1;
    if (i > j + 1) q0 = dd_add(q0, dd_mul(v0, v0));
    q1 = dd_add(q1, dd_mul(v1, v1));
  }
  if (i < n) {
    const dd v0 = dd_sub(c[i], dd_mul(dv, a[i]));
    c[i] = v0;
    if (i > j + 1) q0 = dd_add(q0, dd_mul(v0, v0));
  }
  return dd_add(q0, q1);
}
// trailing column c <- c - V (T^T (V^T c)) for the panel's reflectors V (column a at V + a n)
__device__ __forceinline__ void qr_trailing(const dd* __restrict__ V, dd* __restrict__ c, const dd* __restrict__ T,
                                            int p0, int n, int nb, int lane) {
  const dd zero = dd{0.f, 0.f};
  dd y[kQrNb];
#pragma unroll
  for (int a = 0; a < kQrNb; ++a) y[a] = zero;
  for (int i = p0 + lane; i < n; i += 32) {
    const dd x = c[i];
#pragma unroll
    for (int a = 0; a < kQrNb; ++a)
      if (a < nb) y[a] = dd_add(y[a], dd_mul(V[(size_t)a * n + i], x));
  }
#pragma unroll
  for (int a = 0; a < kQrNb; ++a) y[a] = dd_warp_sum_l(y[a]);
  // z = T^T y: lane a < kQrNb forms z_a, then every lane takes all of them
  dd za = zero;
#pragma unroll
  for (int b = 0; b < kQrNb; ++b)
    if (b <= lane) za = dd_add(za, dd_mul(T[b * kQrNb + (lane & (kQrNb - 1))], y[b]));
  dd z[kQrNb];
#pragma unroll
  for (int a = 0; a < kQrNb; ++a) z[a] = dd{__shfl_sync(0xffffffffu, za.hi, a), __shfl_sync(0xffffffffu, za.lo, a)};
  __syncwarp();
  for (int i = p0 + lane; i < n; i += 32) {
    dd x = c[i];
#pragma unroll
    for (int a = 0; a < kQrNb; ++a)
      if (a < nb) x = dd_sub(x, dd_mul(V[(size_t)a * n + i], z[a]));
    c[i] = x;
  }
}
// warp that takes panel column offset o = c - j - 1 (0 .. kQrNb-2): the critical
// column (o = 0) gets warp 0 alone on its SM sub-partition (warp % 4 == 0);
// the others go to warps of the other three sub-partitions
__device__ __forceinline__ int qr_col_warp(int o) { return o == 0 ? 0 : o + (o - 1) / 3; }
constexpr int kQrFinWarp = 9;  // finalises the previous reflector column

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
      // the panel column this warp updates (if any); only those warps form the reflector
      int o = -1;
      for (int t = 0; t < p1 - j - 1; ++t)
        if (qr_col_warp(t) == warp) o = t;
      const int c = j + 1 + o;
      const bool uses = o >= 0 || warp == 0;
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
      if (o >= 0) {
        dd* ac = A + (size_t)c * n;
        if (tj.hi != 0.f) {
          const dd sdot = qr_pivot_dot(aj, ac, j, n, lane);
          const dd acj = ac[j];
          const dd d = dd_mul(tj, dd_add(acj, dd_mul(inv, sdot)));
          const dd dv = dd_mul(d, inv);
          __syncwarp();
          if (lane == 0) ac[j] = dd_sub(acj, d);
          dd q = qr_pivot_update(aj, ac, dv, j, n, lane);
          if (o == 0) {
            q = dd_warp_sum_l(q);
            if (lane == 0) { s_sig[(j + 1) & 1] = q; s_x0[(j + 1) & 1] = ac[j + 1]; }
          }
        } else if (o == 0) {
          dd q = zero;
          for (int i2 = j + 2 + lane; i2 < n; i2 += 32) q = dd_add(q, dd_mul(ac[i2], ac[i2]));
          q = dd_warp_sum_l(q);
          if (lane == 0) { s_sig[(j + 1) & 1] = q; s_x0[(j + 1) & 1] = ac[j + 1]; }
        }
      }
      // column j-1 is no longer read by the panel: scale it into its reflector
      if (warp == kQrFinWarp && j > p0)
        qr_finalize(A + (size_t)(j - 1) * n, j - 1, n, s_inv[j - 1], s_tau[j - 1], lane);
      __syncthreads();
    }
    if (warp == kQrFinWarp) qr_finalize(A + (size_t)(p1 - 1) * n, p1 - 1, n, s_inv[p1 - 1], s_tau[p1 - 1], lane);
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
    for (int c = p1 + warp; c < K; c += nw) qr_trailing(A + (size_t)p0 * n, A + (size_t)c * n, s_T, p0, n, nb, lane);
    __syncthreads();
  }
  for (int e = tid; e < n * K; e += blockDim.x) Vg[e] = A[e];
}

// Householder QR of the K <= 32 columns of W (n x K, n <= 256), one CTA of
// 1024 threads in double-float, for the mode lengths of the smooth fields:
// warp c owns column c with its n entries in registers (kQcRpl rows per lane,
// row = lane + 32 t).  Pivot j: warp j sums the squares below the diagonal
// (warp butterfly), forms the reflector H_j = I - tau v v^T (v_j = 1, tau =
// 2 v0^2 / (v0^2 + sigma) from v itself, so H_j is orthogonal to working
// precision) and publishes v in shared memory; after one CTA barrier every warp
// c > j applies H_j to its column (dot product by butterfly, update in
// registers).  Warp j + 1 then pivots at once while the others still apply
// H_j, so each pivot costs one barrier and no CTA-wide reduction.  The panels'
// compact-WY blocks T (kQrNb columns each) are formed at the end for
// sub_qform_kernel; the outputs match sub_qr_kernel's.
constexpr int kQcRpl = 8;          // rows per lane: n <= 32 * kQcRpl
constexpr int kQcThreads = 1024;   // 32 warps, one per column

__global__ void __launch_bounds__(kQcThreads, 1) qr_col_kernel(const dd* __restrict__ W, int n, int K,
                                                                dd* __restrict__ Vg, dd* __restrict__ Tg) {
  extern __shared__ dd Vs[];  // K x n: column j = reflector j
  __shared__ dd s_tau[32];
  __shared__ dd s_S[4][kQrNb * kQrNb], s_T[4][kQrNb * kQrNb];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const dd zero = dd{0.f, 0.f}, one = dd{1.f, 0.f};
  dd a[kQcRpl];
#pragma unroll
  for (int t = 0; t < kQcRpl; ++t) {
    const int row = lane + 32 * t;
    a[t] = (warp < K && row < n) ? W[(size_t)warp * n + row] : zero;
  }
  // sigma_j = sum_{row > j} a_row^2 of the next pivot column, accumulated by
  // its warp while it applies the previous reflector (column 0: here)
  dd sig_next = zero;
  if (warp == 0) {
    dd q0 = zero, q1 = zero;
#pragma unroll
    for (int t = 0; t < kQcRpl; ++t) {
      const int row = lane + 32 * t;
      if (row > 0 && row < n) {
        if (t & 1) q1 = dd_add(q1, dd_mul(a[t], a[t]));
        else q0 = dd_add(q0, dd_mul(a[t], a[t]));
      }
    }
    sig_next = dd_add(q0, q1);
  }
  for (int j = 0; j < K; ++j) {
    if (warp == j) {
      const dd sig = dd_warp_sum_l(sig_next);
      // a at row j: lane j % 32, register group j / 32
      dd xl = zero;
#pragma unroll
      for (int t = 0; t < kQcRpl; ++t)
        if (t == (j >> 5)) xl = a[t];
      const dd x0 = dd{__shfl_sync(0xffffffffu, xl.hi, j & 31), __shfl_sync(0xffffffffu, xl.lo, j & 31)};
      dd tau = zero, inv = zero;
      if (sig.hi != 0.f) {
        const dd nrm = qr_sqrt(dd_add(dd_mul(x0, x0), sig));
        const dd alpha = dd_neg_sign(x0) ? nrm : dd_neg(nrm);
        const dd v0 = dd_sub(x0, alpha);
        const dd v02 = dd_mul(v0, v0);
        tau = qr_div(dd_add(v02, v02), dd_add(v02, sig));
        inv = qr_div(one, v0);
      }
#pragma unroll
      for (int t = 0; t < kQcRpl; ++t) {
        const int row = lane + 32 * t;
        if (row < n) Vs[(size_t)j * n + row] = (row < j) ? zero : ((row == j) ? one : dd_mul(a[t], inv));
      }
      if (lane == 0) s_tau[j] = tau;
    }
    __syncthreads();
    if (warp > j && warp < K) {
      const dd tau = s_tau[j];
      const bool next = warp == j + 1;  // the next pivot: also sums its squares below row j + 1
      if (tau.hi != 0.f) {
        dd v[kQcRpl];
        dd s0 = zero, s1 = zero;
#pragma unroll
        for (int t = 0; t < kQcRpl; ++t) {
          const int row = lane + 32 * t;
          v[t] = zero;
          if (32 * t + 32 > j) {  // groups entirely above row j hold zeros of v
            v[t] = (row < n) ? Vs[(size_t)j * n + row] : zero;
            if (t & 1) s1 = dd_add(s1, dd_mul(v[t], a[t]));
            else s0 = dd_add(s0, dd_mul(v[t], a[t]));
          }
        }
        const dd dv = dd_mul(tau, dd_warp_sum_l(dd_add(s0, s1)));
        dd q0 = zero, q1 = zero;
#pragma unroll
        for (int t = 0; t < kQcRpl; ++t) {
          if (32 * t + 32 > j) a[t] = dd_sub(a[t], dd_mul(dv, v[t]));
          if (next) {
            const int row = lane + 32 * t;
            if (row > j + 1 && row < n) {
              if (t & 1) q1 = dd_add(q1, dd_mul(a[t], a[t]));
              else q0 = dd_add(q0, dd_mul(a[t], a[t]));
            }
          }
        }
        if (next) sig_next = dd_add(q0, q1);
      } else if (next) {
        dd q0 = zero, q1 = zero;
#pragma unroll
        for (int t = 0; t < kQcRpl; ++t) {
          const int row = lane + 32 * t;
          if (row > j + 1 && row < n) {
            if (t & 1) q1 = dd_add(q1, dd_mul(a[t], a[t]));
            else q0 = dd_add(q0, dd_mul(a[t], a[t]));
          }
        }
        sig_next = dd_add(q0, q1);
      }
    }
  }
  __syncthreads();
  // reflectors out; S[a][b] = v_a . v_b (a < b) inside each panel, a warp per pair
  for (int e = tid; e < K * n; e += kQcThreads) Vg[e] = Vs[e];
  const int npan = (K + kQrNb - 1) / kQrNb;
  for (int item = warp; item < npan * kQrNb * kQrNb; item += kQcThreads / 32) {
    const int p = item / (kQrNb * kQrNb), ab = item - p * kQrNb * kQrNb, aa = ab / kQrNb, bb = ab - aa * kQrNb;
    const int ca = p * kQrNb + aa, cb = p * kQrNb + bb;
    if (aa >= bb || cb >= K) continue;
    dd sp = zero;
    for (int row = cb + lane; row < n; row += 32) sp = dd_add(sp, dd_mul(Vs[(size_t)ca * n + row], Vs[(size_t)cb * n + row]));
    sp = dd_warp_sum_l(sp);
    if (lane == 0) s_S[p][aa * kQrNb + bb] = sp;
  }
  for (int e = tid; e < 4 * kQrNb * kQrNb; e += kQcThreads) (&s_T[0][0])[e] = zero;
  __syncthreads();
  // T (upper triangular): T[b][b] = tau_b, T[0:b, b] = -tau_b T[0:b, 0:b] S[0:b, b]
  if (warp < npan) {
    const int p = warp, p0 = p * kQrNb, nb = min(kQrNb, K - p0);
    for (int b = 0; b < nb; ++b) {
      const dd tb = s_tau[p0 + b];
      dd t = zero;
      if (lane < b)
        for (int c2 = lane; c2 < b; ++c2) t = dd_add(t, dd_mul(s_T[p][lane * kQrNb + c2], s_S[p][c2 * kQrNb + b]));
      __syncwarp();
      if (lane < b) s_T[p][lane * kQrNb + b] = dd_neg(dd_mul(tb, t));
      if (lane == b) s_T[p][b * kQrNb + b] = tb;
      __syncwarp();
    }
    for (int e = lane; e < kQrNb * kQrNb; e += 32) Tg[(size_t)p * kQrNb * kQrNb + e] = s_T[p][e];
  }
}

// Q = H_0 H_1 ... H_{K-1} [I_K; 0] from the panels' WY blocks, one CTA per
// column c (threads over rows): q = e_c, then q <- q - V_p (T_p (V_p^T q)) for
// the panels p from the one holding c down to the first (later panels leave
// e_c unchanged); per panel one CTA reduction of the kQrNb dot products, z = T y
// in warp 0, and the update of the thread's rows.
constexpr int kQfThreads = 256;
constexpr int kQfRows = 3;  // rows per thread: n <= 768
__global__ void __launch_bounds__(kQfThreads) sub_qform_kernel(const dd* __restrict__ Vg, const dd* __restrict__ Tg,
                                                               int n, int K, double* __restrict__ Q) {
  __shared__ dd part[kQfThreads / 32][kQrNb];
  __shared__ dd zs[kQrNb];
  const int c = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const dd zero = dd{0.f, 0.f};
  dd q[kQfRows];
#pragma unroll
  for (int r = 0; r < kQfRows; ++r) q[r] = (tid + r * kQfThreads == c) ? dd{1.f, 0.f} : zero;
  for (int p = c / kQrNb; p >= 0; --p) {
    const int p0 = p * kQrNb, nb = min(kQrNb, K - p0);
    const dd* V = Vg + (size_t)p0 * n;
    const dd* T = Tg + (size_t)p * kQrNb * kQrNb;
    dd y[kQrNb];
#pragma unroll
    for (int a = 0; a < kQrNb; ++a) y[a] = zero;
#pragma unroll
    for (int r = 0; r < kQfRows; ++r) {
      const int i = tid + r * kQfThreads;
      if (i >= p0 && i < n)
#pragma unroll
        for (int a = 0; a < kQrNb; ++a)
          if (a < nb) y[a] = dd_add(y[a], dd_mul(V[(size_t)a * n + i], q[r]));
    }
#pragma unroll
    for (int a = 0; a < kQrNb; ++a) y[a] = dd_warp_sum_l(y[a]);
    if (lane == 0)
#pragma unroll
      for (int a = 0; a < kQrNb; ++a) part[warp][a] = y[a];
    __syncthreads();
    if (warp == 0) {
      dd ya = zero;
      if (lane < kQrNb)
        for (int w = 0; w < kQfThreads / 32; ++w) ya = dd_add(ya, part[w][lane]);
      dd za = zero;
#pragma unroll
      for (int b = 0; b < kQrNb; ++b) {
        const dd yb = dd{__shfl_sync(0xffffffffu, ya.hi, b), __shfl_sync(0xffffffffu, ya.lo, b)};
        if (lane < nb && b >= lane && b < nb) za = dd_add(za, dd_mul(T[lane * kQrNb + b], yb));
      }
      if (lane < kQrNb) zs[lane] = za;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kQfRows; ++r) {
      const int i = tid + r * kQfThreads;
      if (i >= p0 && i < n)
#pragma unroll
        for (int a = 0; a < kQrNb; ++a)
          if (a < nb) q[r] = dd_sub(q[r], dd_mul(V[(size_t)a * n + i], zs[a]));
    }
  }
#pragma unroll
  for (int r = 0; r < kQfRows; ++r) {
    const int i = tid + r * kQfThreads;
    if (i < n) Q[(size_t)c * n + i] = dd_to(q[r]);
  }
}

}  // namespace

bool subspace_supported(int n, int K) {
  return K >= 5 && K <= 64 && K <= n && n <= kQfThreads * kQfRows && (size_t)n * K * sizeof(dd) <= 200 * 1024 &&
         rr_smem_bytes(K, K - 4) <= 180 * 1024;
}

int subspace_solve(const double* G, int n, int K, int T, double budget, int extra, int nmax, double conv,
                   const int* tc_err, double* U_dev, int* decision_host, cudaStream_t s) {
  if (!subspace_supported(n, K)) return fail(ATC_EINVAL, "subspace_solve: unsupported n = %d, K = %d", n, K);
  if (nmax < 1 || nmax > K || T < 1) return fail(ATC_EINVAL, "subspace_solve: nmax = %d, T = %d", nmax, T);
  const size_t nk = (size_t)n * K;
  const int npan = (K + kQrNb - 1) / kQrNb;
  // V, W, B, theta, trace (8), Vg, Tg, Y, decision + exponent (8)
  const size_t nd = 2 * nk + (size_t)K * K + K + 8 + nk + (size_t)npan * kQrNb * kQrNb + (size_t)K * nmax + 8;
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
  // the start frame depends on (n, K) only: kept in its own slot per device
  double* V0 = nullptr;
  ATC_TRY(Scratch::get(SLOT_SUB_V0, sizeof(double) * nk, (void**)&V0));
  {
    static int c_dev = -1, c_n = -1, c_K = -1;
    static long long c_serial = -1;
    int dev = 0;
    ATC_CUDA_TRY(cudaGetDevice(&dev));
    if (dev != c_dev || n != c_n || K != c_K || g_scratch_serial != c_serial) {
      const int blocks = (int)((nk + 255) / 256 < 1024 ? (nk + 255) / 256 : 1024);
      sub_init_kernel<<<blocks, 256, 0, s>>>(V0, n, K);
      ATC_LAUNCHED(1);
      c_dev = dev;
      c_n = n;
      c_K = K;
      c_serial = g_scratch_serial;
    }
  }
  static bool attr = false;
  if (!attr) {
    ATC_CUDA_TRY(cudaFuncSetAttribute(sub_qr_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    ATC_CUDA_TRY(cudaFuncSetAttribute(qr_col_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)(sizeof(dd) * 32 * 32 * kQcRpl)));
    attr = true;
  }
  // column-owner QR for n <= 256 (K <= 32 warps), the blocked one-CTA QR above
  const bool qr_col = n <= 32 * kQcRpl && K <= 32;
  const dim3 ggrid((n + 31) / 32, K);
  for (int t = 0; t < T; ++t) {
    { KTimed kt_(s, "sub_gemm_kernel", (double)n * n * 8.0 + 2.0 * (double)nk * 8.0, 2.0 * (double)n * n * K); sub_gemm_kernel<<<ggrid, 32 * kGemmWarps, 0, s>>>(G, n, t == 0 ? V0 : V, nullptr, Wd, gex, t == 0 ? tr : nullptr); }
    ATC_LAUNCHED(1);
    {
      KTimed kt_(s, qr_col ? "qr_col_kernel" : "sub_qr_kernel", 2.0 * (double)nk * 8.0, 2.0 * (double)n * K * K - 2.0 / 3.0 * (double)K * K * K);
      if (qr_col) qr_col_kernel<<<1, kQcThreads, sizeof(dd) * nk, s>>>(Wd, n, K, Vg, Tg);
      else sub_qr_kernel<<<1, kQrThreads, sizeof(dd) * nk, s>>>(Wd, n, K, Vg, Tg);
    }
    ATC_LAUNCHED(1);
    { KTimed kt_(s, "sub_qform_kernel", 2.0 * (double)nk * 8.0, 2.0 * (double)n * K * K); sub_qform_kernel<<<K, kQfThreads, 0, s>>>(Vg, Tg, n, K, V); }
    ATC_LAUNCHED(1);
  }
  { KTimed kt_(s, "sub_gemm_kernel", (double)n * n * 8.0 + 2.0 * (double)nk * 8.0, 2.0 * (double)n * n * K); sub_gemm_kernel<<<ggrid, 32 * kGemmWarps, 0, s>>>(G, n, V, W, nullptr, gex, nullptr); }
  ATC_LAUNCHED(1);
  { KTimed kt_(s, "sub_proj_kernel"); sub_proj_kernel<<<(K * K * 32 + 255) / 256, 256, 0, s>>>(V, W, n, K, B); }
  ATC_LAUNCHED(1);
  // Rayleigh-Ritz on the K x K matrix B (one CTA), provisional rank and vector count on the device
  ATC_TRY(launch_rr_small(B, K, n, tr, budget, extra, nmax, conv, T, tc_err, th, dec, Y, s));
  const int rblocks = (int)(((size_t)n * nmax + 255) / 256 < 1024 ? ((size_t)n * nmax + 255) / 256 : 1024);
  { KTimed kt_(s, "sub_rotate_kernel"); sub_rotate_kernel<<<rblocks, 256, 0, s>>>(V, n, K, Y, dec + 1, U_dev, nmax); }
  ATC_LAUNCHED(1);
  ATC_CUDA_TRY(cudaMemcpyAsync(decision_host, dec, sizeof(int) * 4, cudaMemcpyDeviceToHost, s));
  return ATC_OK;
}

}  // namespace atc
