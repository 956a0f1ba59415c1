// Leading eigenpairs of a symmetric positive semi-definite n x n matrix by
// subspace iteration with a final Rayleigh-Ritz step (FP64).
//
// The split-precision paths certify every rank from measured residual tails
// (||X - U ._k Y||^2 + sum_{j>=r} ||Y_j||^2), so they need the leading
// r_h (+ margin) eigenvectors of the mode Gram matrix to moderate accuracy and
// its eigenvalues only to pick a provisional rank.  For the smooth fields this
// library targets the Gram spectrum falls by many orders of magnitude within
// the first few dozen eigenvalues, and K = 48 columns of
//     V <- orth(G V)  (T times),  B = V^T G V = Y Theta Y^T,  U = V Y
// reach the leading subspace to the angles the certification needs, with GEMM
// work and two short QR chains instead of the n - 2 dependent Householder steps
// of a full tridiagonalisation.  The caller checks the Ritz ratio and falls
// back to the full eigensolver when convergence is not assured.
//
// orth() is a Householder QR (the columns of G V are conditioned like
// lambda_1 / lambda_K, far beyond what a Cholesky QR tolerates), one CTA with
// the block in shared memory: a warp per trailing column, a block reduction per
// pivot column.  The start block is orthonormal by construction, and the K x K
// Rayleigh-Ritz problem goes to the double-float eigensolver, which computes
// only the eigenvectors asked for.
#include <math.h>
#include <stdint.h>

#include "atc_internal.cuh"
#include "dd.cuh"

namespace atc {
namespace {

constexpr int kSubThreads = 512;

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

// W[c][i] = sum_k G[i][k] V[c][k]: a warp per (i, group of 8 columns c)
__global__ void __launch_bounds__(256) sub_gemm_kernel(const double* __restrict__ G, int n,
                                                       const double* __restrict__ V, int K, double* __restrict__ W) {
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
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const double v = warp_sum_d(acc[q]);
    if (lane == 0 && c0 + q < K) W[(int64_t)(c0 + q) * n + i] = v;
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

// U[i][j] = sum_a V[a][i] Y[a][j] (U n x m row-major; Y K x m row-major)
__global__ void sub_rotate_kernel(const double* __restrict__ V, int n, int K, const double* __restrict__ Y, int m,
                                  double* __restrict__ U) {
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

__device__ double block_sum_d(double v, double* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum_d(v);
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  for (int q = 0; q < nw; ++q) t += red[q];
  return t;
}

// Householder QR of the K columns W[c][.] (length n, K <= n) in shared
// memory, one CTA, in double-float (FP64 issues at 2 lanes per clock per SM on
// GB300; the pair arithmetic runs on the FP32 pipes): Q (K orthonormal columns
// spanning the same space) is formed in place from the reflectors (stored below
// the diagonal, v_j(j) = 1 implicit) by applying them backwards, and written
// to Q in FP64.  Column c of the working array holds element (row i, column c)
// at A[c * n + i].
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
// sum_{i >= i0} a[i] b[i] over a warp, two interleaved accumulators
__device__ __forceinline__ dd dd_dot_from(const dd* __restrict__ a, const dd* __restrict__ b, int i0, int n, int lane) {
  dd d0 = dd{0.f, 0.f}, d1 = dd{0.f, 0.f}, d2 = dd{0.f, 0.f}, d3 = dd{0.f, 0.f};
  int i = i0 + lane;
  for (; i + 96 < n; i += 128) {
    d0 = dd_add(d0, dd_mul(a[i], b[i]));
    d1 = dd_add(d1, dd_mul(a[i + 32], b[i + 32]));
    d2 = dd_add(d2, dd_mul(a[i + 64], b[i + 64]));
    d3 = dd_add(d3, dd_mul(a[i + 96], b[i + 96]));
  }
  for (; i < n; i += 32) d0 = dd_add(d0, dd_mul(a[i], b[i]));
  return dd_warp_sum_l(dd_add(dd_add(d0, d1), dd_add(d2, d3)));
}
// c[i] -= d * v[i] for i > j, c[j] -= d (v_j = 1)
__device__ __forceinline__ void dd_reflect(dd* __restrict__ c, const dd* __restrict__ v, dd d, int j, int n, int lane) {
  if (lane == 0) c[j] = dd_sub(c[j], d);
  for (int i = j + 1 + lane; i < n; i += 32) c[i] = dd_sub(c[i], dd_mul(d, v[i]));
}
__global__ void __launch_bounds__(kSubThreads) sub_hqr_kernel(const double* __restrict__ W, int n, int K,
                                                              double* __restrict__ Q) {
  extern __shared__ dd A[];
  __shared__ dd red[32];
  __shared__ dd tau[64];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  // power-of-two scale: |entries| <= 1 keeps every pair product far from the float range limits
  double mx = 0.0;
  for (int e = tid; e < n * K; e += blockDim.x) mx = fmax(mx, fabs(W[e]));
  {
    __shared__ double smx[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) smx[warp] = mx;
    __syncthreads();
    mx = 0.0;
    for (int q = 0; q < nw; ++q) mx = fmax(mx, smx[q]);
  }
  int ex = 0;
  if (mx > 0.0) frexp(mx, &ex);
  const double sc = ldexp(1.0, -ex);
  for (int e = tid; e < n * K; e += blockDim.x) A[e] = dd_from(W[e] * sc);
  __syncthreads();
  const dd zero = dd{0.f, 0.f}, one = dd{1.f, 0.f};
  for (int j = 0; j < K; ++j) {
    dd* aj = A + (int64_t)j * n;
    dd part = zero;
    for (int i = j + 1 + tid; i < n; i += blockDim.x) part = dd_add(part, dd_mul(aj[i], aj[i]));
    const dd sig = dd_block_sum(part, red);
    const dd x0 = aj[j];
    dd tj = zero, v0 = one, alpha = x0;
    if (sig.hi != 0.f) {
      const dd nrm = dd_sqrt(dd_add(dd_mul(x0, x0), sig));
      alpha = dd_neg_sign(x0) ? nrm : dd_neg(nrm);
      v0 = dd_sub(x0, alpha);
      const dd v02 = dd_mul(v0, v0);
      tj = dd_div(dd_add(v02, v02), dd_add(v02, sig));
    }
    __syncthreads();
    if (tid == 0) {
      tau[j] = tj;
      aj[j] = alpha;  // R_jj
    }
    if (tj.hi != 0.f) {
      const dd inv = dd_div(one, v0);
      for (int i = j + 1 + tid; i < n; i += blockDim.x) aj[i] = dd_mul(aj[i], inv);
    } else {
      for (int i = j + 1 + tid; i < n; i += blockDim.x) aj[i] = zero;
    }
    __syncthreads();
    if (tj.hi != 0.f)
      for (int c = j + 1 + warp; c < K; c += nw) {
        dd* ac = A + (int64_t)c * n;
        const dd d = dd_mul(dd_add(ac[j], dd_dot_from(aj, ac, j + 1, n, lane)), tj);
        dd_reflect(ac, aj, d, j, n, lane);
      }
    __syncthreads();
  }
  // Q in place, backwards: column j becomes H_j e_j after H_j has acted on the later columns
  for (int j = K - 1; j >= 0; --j) {
    dd* aj = A + (int64_t)j * n;
    const dd tj = tau[j];
    if (tj.hi != 0.f)
      for (int c = j + 1 + warp; c < K; c += nw) {
        dd* ac = A + (int64_t)c * n;
        const dd d = dd_mul(dd_add(ac[j], dd_dot_from(aj, ac, j + 1, n, lane)), tj);
        dd_reflect(ac, aj, d, j, n, lane);
      }
    __syncthreads();
    for (int i = tid; i < n; i += blockDim.x) {
      if (i < j) aj[i] = zero;
      else if (i == j) aj[i] = dd_sub(one, tj);
      else aj[i] = dd_neg(dd_mul(tj, aj[i]));
    }
    __syncthreads();
  }
  for (int e = tid; e < n * K; e += blockDim.x) Q[e] = dd_to(A[e]);
}

}  // namespace

bool subspace_supported(int n, int K) { return K >= 1 && K <= 64 && K <= n && (size_t)n * K * sizeof(dd) <= 200 * 1024; }

int subspace_values(const double* G, int n, int K, int T, double* theta_host, double* trace_host, cudaStream_t s) {
  if (!subspace_supported(n, K)) return fail(ATC_EINVAL, "subspace_values: unsupported n = %d, K = %d", n, K);
  double* base = nullptr;
  const size_t nk = (size_t)n * K;
  ATC_TRY(Scratch::get(SLOT_SUBSPACE, sizeof(double) * (2 * nk + (size_t)K * K + K + 8), (void**)&base));
  double* V = base;
  double* W = V + nk;
  double* B = W + nk;
  double* th = B + (size_t)K * K;
  double* tr = th + K;
  const size_t hsm = sizeof(dd) * nk;
  static bool attr = false;
  if (!attr) {
    ATC_CUDA_TRY(cudaFuncSetAttribute(sub_hqr_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    attr = true;
  }
  const int blocks = (int)((nk + 255) / 256 < 1024 ? (nk + 255) / 256 : 1024);
  sub_init_kernel<<<blocks, 256, 0, s>>>(V, n, K);
  ATC_LAUNCHED(1);
  const int gemm_blocks = (int)(((int64_t)n * ((K + 7) / 8) * 32 + 255) / 256);
  for (int t = 0; t < T; ++t) {
    sub_gemm_kernel<<<gemm_blocks, 256, 0, s>>>(G, n, V, K, W);
    sub_hqr_kernel<<<1, kSubThreads, hsm, s>>>(W, n, K, V);
    ATC_LAUNCHED(2);
  }
  sub_gemm_kernel<<<gemm_blocks, 256, 0, s>>>(G, n, V, K, W);
  sub_proj_kernel<<<(K * K * 32 + 255) / 256, 256, 0, s>>>(V, W, n, K, B);
  sub_trace_kernel<<<1, 32, 0, s>>>(G, n, tr);
  ATC_LAUNCHED(3);
  // Rayleigh-Ritz on the K x K matrix B with the double-float solver
  ATC_TRY(launch_eig_tridiag(B, K, tr + 1, s, true));  // tr + 1: trace of B (unused)
  ATC_TRY(launch_eig_more(K, K, th, s));
  ATC_CUDA_TRY(cudaMemcpyAsync(theta_host, th, sizeof(double) * K, cudaMemcpyDeviceToHost, s));
  ATC_CUDA_TRY(cudaMemcpyAsync(trace_host, tr, sizeof(double), cudaMemcpyDeviceToHost, s));
  return ATC_OK;
}

int subspace_vectors(int n, int K, int nvec, double* U_dev, cudaStream_t s) {
  double* base = nullptr;
  const size_t nk = (size_t)n * K;
  ATC_TRY(Scratch::get(SLOT_SUBSPACE, sizeof(double) * (2 * nk + (size_t)K * K + K + 8), (void**)&base));
  double* V = base;
  double* Y = base + nk;  // the W block is free again
  ATC_TRY(launch_eig_vectors(K, nvec, Y, s));
  const int blocks = (int)(((size_t)n * nvec + 255) / 256 < 1024 ? ((size_t)n * nvec + 255) / 256 : 1024);
  sub_rotate_kernel<<<blocks, 256, 0, s>>>(V, n, K, Y, nvec, U_dev);
  ATC_LAUNCHED(1);
  return ATC_OK;
}

}  // namespace atc
