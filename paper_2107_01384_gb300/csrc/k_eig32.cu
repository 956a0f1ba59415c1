// FP64-accurate symmetric eigensolver built for GB300's arithmetic mix.
//
// GB300 runs FP32 at ~64x its FP64 rate, and FP64 latency chains are long, so
// the eigen-decomposition of a mode Gram matrix (Algorithm 1: eigenvectors /
// eigenvalues of G = B_(k) B_(k)^T are the left singular vectors / squared
// singular values of the unfolding) is done in two stages:
//
//  1. FP32 stage, latency bound, one CTA:
//     * Householder tridiagonalisation of the scaled G held as a packed lower
//       triangle in shared memory (one fused update + matrix-vector sweep per
//       step, row and column contributions in the same pass);
//     * all eigenvalues of T by 32-way multisection on Sturm counts;
//     * eigenvectors of T for the q "significant" eigenvalues only (those
//       above eta * lambda_m, where m columns are to be refined) by inverse
//       iteration, re-orthogonalised inside groups of close eigenvalues, then
//       back-transformed with the stored reflectors.
//  2. FP64 stage, GEMM shaped (parallel over the whole GPU): a refinement of
//     the top-m eigenpairs after Ogita and Aishima ("Iterative refinement for
//     symmetric eigenvalue decomposition", 2018), restricted to m columns:
//       W = G X_J,  S = X_JK^T W,  Q = X_JK^T X_J,  R = I - Q,
//       lambda~_j = S_jj / (1 - R_jj),
//       E_ij = (S_ij + lambda~_j R_ij) / (lambda~_j - lambda~_i)  (or R_ij / 2 for close pairs),
//     and the eigenvalues below eta * lambda_m (not computed explicitly) are
//     handled as one invariant subspace with eigenvalue 0, which folds their
//     correction into  x_j' = W_j / lambda~_j + X_JK F_j,
//       F = E - (S - Q diag(lambda~)) diag(1 / lambda~).
//     Two passes take FP32 accuracy to FP64 accuracy for separated eigenvalues.
// The tail energy used by the rank rule is trace(G) - sum of refined top
// eigenvalues, all in FP64.
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

#include <algorithm>
#include <vector>

#include "atc_internal.cuh"

namespace atc {
namespace {

constexpr int kTri = 1024;     // threads of the tridiagonalisation CTA
constexpr int kMaxN32 = 256;   // packed FP32 lower triangle must fit in shared memory

__device__ __forceinline__ float wsum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double wsumd(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
// deterministic block sum (all threads get the result)
__device__ float bsum(float v, float* red) {
  v = wsum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  float t = 0.f;
  const int nw = blockDim.x >> 5;
  for (int i = 0; i < nw; ++i) t += red[i];
  return t;
}

__device__ __forceinline__ int poff(int i, int j) { return (i * (i + 1)) / 2 + j; }  // j <= i

struct E32 {
  float* d;     // n  (scaled)
  float* e;     // n
  float* tau;   // n
  float* hv;    // n x n reflectors, row s = v_s
  float* lam;   // n eigenvalues of T, descending (scaled)
  float* z;     // q x n eigenvectors of T (row j = vector j)
  float* lu;    // 5 x n x q
  double* x;    // n x q  back-transformed (FP64, row-major, column j = vector j)
  double* w;    // n x m
  double* s;    // q x m
  double* qm;   // q x m
  double* f;    // q x m
  double* lt;   // m refined eigenvalues (unscaled)
  double* gpart;  // split-K partials of the FP64 GEMMs
  double* misc;   // [0] scale (float in double), [1] trace, [2] delta ...
  int* grp;       // group starts
  int n, q, m;
  int lumped;     // 1: eigenvalues beyond q are folded in as one eigenvalue-0 subspace
};

// ------------------------------------------------------ tridiagonalisation
__global__ void __launch_bounds__(kTri, 1) tri32_kernel(const double* __restrict__ G, int n, E32 st) {
  extern __shared__ float sm[];
  const int npk = n * (n + 1) / 2;
  float* Ap = sm;
  float* vp = Ap + ((npk + 31) & ~31);  // v_{s-1}
  float* wp = vp + kMaxN32;             // w_{s-1}
  float* vc = wp + kMaxN32;             // v_s
  float* row = vc + kMaxN32;            // row s of A^(s)
  float* pv = row + kMaxN32;            // p_s
  float* prow = pv + kMaxN32;           // row contributions
  float* colp = prow + kMaxN32;         // 32 x kMaxN32 column partials
  float* red = colp + 32 * kMaxN32;     // 32
  __shared__ float s_tau_prev, s_tau, s_scale;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // power-of-two scale: max |G| -> [0.5, 1)
  {
    double m = 0.0;
    for (int idx = tid; idx < n * n; idx += kTri) m = fmax(m, fabs(G[idx]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    __shared__ double redd[32];
    if (lane == 0) redd[warp] = m;
    __syncthreads();
    if (tid == 0) {
      double mm = 0.0;
      for (int i = 0; i < kTri / 32; ++i) mm = fmax(mm, redd[i]);
      int ex = 0;
      if (mm > 0.0) frexp(mm, &ex);
      s_scale = ldexpf(1.0f, -ex);
      st.misc[0] = (double)s_scale;
    }
    __syncthreads();
  }
  const float sc = s_scale;
  for (int i = warp; i < n; i += 32)
    for (int j = lane; j <= i; j += 32) Ap[poff(i, j)] = (float)(G[(int64_t)i * n + j] * (double)sc);
  for (int i = tid; i < kMaxN32; i += kTri) { vp[i] = 0.f; wp[i] = 0.f; vc[i] = 0.f; pv[i] = 0.f; }
  if (tid == 0) { s_tau_prev = 0.f; s_tau = 0.f; }
  __syncthreads();
  if (n == 1) {
    if (tid == 0) { st.d[0] = Ap[0]; st.e[0] = 0.f; st.tau[0] = 0.f; }
    return;
  }
  for (int s = 0; s <= n - 2; ++s) {
    if (s >= 1) {
      float part = 0.f;
      for (int i = s + tid; i < n; i += kTri) part += pv[i] * vp[i];
      const float dot = bsum(part, red);
      const float K = 0.5f * s_tau_prev * dot;
      for (int i = tid; i < n; i += kTri) wp[i] = (i >= s) ? pv[i] - K * vp[i] : 0.f;
      __syncthreads();
    }
    {
      const float vs = vp[s], ws = wp[s];
      for (int j = s + tid; j < n; j += kTri) row[j] = Ap[poff(j, s)] - vs * wp[j] - ws * vp[j];
      __syncthreads();
    }
    if (s <= n - 3) {
      float part = 0.f;
      for (int j = s + 2 + tid; j < n; j += kTri) part += row[j] * row[j];
      const float sig2 = bsum(part, red);
      const float x0 = row[s + 1];
      float alpha, tau, scal;
      if (sig2 == 0.f) {
        tau = 0.f; alpha = x0; scal = 0.f;
      } else {
        const float nrm = sqrtf(x0 * x0 + sig2);
        alpha = (x0 >= 0.f) ? -nrm : nrm;
        tau = (alpha - x0) / alpha;
        scal = 1.f / (x0 - alpha);
      }
      for (int j = tid; j < n; j += kTri) vc[j] = (j == s + 1) ? 1.f : ((j > s + 1) ? row[j] * scal : 0.f);
      if (tid == 0) s_tau = tau;
      __syncthreads();
      for (int j = tid; j < n; j += kTri) st.hv[(int64_t)s * n + j] = vc[j];
      if (tid == 0) { st.d[s] = row[s]; st.e[s] = alpha; st.tau[s] = tau; }
      // fused update of the trailing block (lower triangle) and p_s = tau A^(s) v_s
      float cacc[kMaxN32 / 32];
#pragma unroll
      for (int t = 0; t < kMaxN32 / 32; ++t) cacc[t] = 0.f;
      for (int i = s + 1 + warp; i < n; i += 32) {
        const float vi = vp[i], wi = wp[i], vci = vc[i];
        float racc = 0.f;
#pragma unroll
        for (int t = 0; t < kMaxN32 / 32; ++t) {
          const int j = s + 1 + lane + 32 * t;
          if (j <= i) {
            float* ap = Ap + poff(i, j);
            const float a = *ap - vi * wp[j] - wi * vp[j];
            *ap = a;
            racc = fmaf(a, vc[j], racc);
            if (j < i) cacc[t] = fmaf(a, vci, cacc[t]);
          }
        }
        racc = wsum(racc);
        if (lane == 0) prow[i] = racc;
      }
#pragma unroll
      for (int t = 0; t < kMaxN32 / 32; ++t) {
        const int j = s + 1 + lane + 32 * t;
        if (j < n) colp[warp * kMaxN32 + j] = cacc[t];
      }
      __syncthreads();
      for (int j = s + 1 + tid; j < n; j += kTri) {
        float p = prow[j];
        for (int w = 0; w < 32; ++w) p += colp[w * kMaxN32 + j];
        pv[j] = tau * p;
      }
      for (int j = tid; j < n; j += kTri) vp[j] = vc[j];
      if (tid == 0) s_tau_prev = s_tau;
      __syncthreads();
    } else {
      if (tid == 0) {
        st.d[s] = row[s];
        st.e[s] = row[s + 1];
        st.tau[s] = 0.f;
        st.d[n - 1] = Ap[poff(n - 1, n - 1)] - 2.f * vp[n - 1] * wp[n - 1];
        st.e[n - 1] = 0.f;
        st.tau[n - 1] = 0.f;
      }
    }
  }
}

// ------------------------------------------------ eigenvalues (multisection)
__device__ __forceinline__ int count32(const float* __restrict__ d, const float* __restrict__ e2, int n, float sig,
                                       float pivmin) {
  float q = d[0] - sig;
  if (fabsf(q) < pivmin) q = -pivmin;
  int c = (q < 0.f);
  for (int i = 1; i < n; ++i) {
    q = (d[i] - sig) - e2[i - 1] / q;
    if (fabsf(q) < pivmin) q = -pivmin;
    c += (q < 0.f);
  }
  return c;
}

// one warp per eigenvalue (index j = j-th largest); 32 probes per round
__global__ void bis32_kernel(E32 st) {
  extern __shared__ float smb[];
  const int n = st.n;
  float* d = smb;
  float* e2 = smb + n;
  __shared__ float s_g;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    d[i] = st.d[i];
    e2[i] = (i < n - 1) ? st.e[i] * st.e[i] : 0.f;
  }
  if (threadIdx.x == 0) {
    float g = 0.f;
    for (int i = 0; i < n; ++i)
      g = fmaxf(g, fabsf(st.d[i]) + (i > 0 ? fabsf(st.e[i - 1]) : 0.f) + (i < n - 1 ? fabsf(st.e[i]) : 0.f));
    s_g = g * 1.001f + 1e-30f;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (j >= n) return;
  const int m = n - 1 - j;  // m-th smallest
  const float pivmin = 1e-36f + 1e-30f * s_g * s_g;
  float lo = -s_g, hi = s_g;
  for (int round = 0; round < 8; ++round) {
    const float p = lo + (hi - lo) * (float)(lane + 1) / 33.f;
    const int c = count32(d, e2, n, p, pivmin);
    const unsigned above = __ballot_sync(0xffffffffu, c > m);
    float nlo, nhi;
    if (above == 0u) {
      nlo = __shfl_sync(0xffffffffu, p, 31);
      nhi = hi;
    } else {
      const int f = __ffs(above) - 1;
      nhi = __shfl_sync(0xffffffffu, p, f);
      nlo = (f == 0) ? lo : __shfl_sync(0xffffffffu, p, f - 1 < 0 ? 0 : f - 1);
    }
    lo = nlo;
    hi = nhi;
    if (hi - lo <= 2.5e-7f * fmaxf(fabsf(lo), fabsf(hi)) + 1e-30f) break;
  }
  if (lane == 0) st.lam[j] = 0.5f * (lo + hi);
}

// ------------------------------------------- inverse iteration (FP32, q vectors)
__device__ __forceinline__ float hash01(uint32_t a, uint32_t b) {
  uint32_t h = a * 0x9E3779B1u ^ (b + 0x7F4A7C15u) * 0x85EBCA77u;
  h ^= h >> 15;
  h *= 0x2C1B3C6Du;
  h ^= h >> 12;
  h *= 0x297A2D39u;
  h ^= h >> 15;
  return 0.5f + (float)(h >> 8) * (1.0f / 16777216.0f);
}

__global__ void invit32_kernel(E32 st) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = st.n;
  if (j >= st.q) return;
  float* fl = st.lu + (int64_t)j * 5 * n;
  float* fd = fl + n;
  float* fu = fd + n;
  float* fu2 = fu + n;
  float* fp = fu2 + n;
  float* x = st.z + (int64_t)j * n;
  const float lam = st.lam[j];
  float g = 0.f;
  for (int i = 0; i < n; ++i) g = fmaxf(g, fabsf(st.d[i]) + fabsf(st.e[i]));
  const float eps_piv = 1.2e-7f * g + 1e-30f;
  for (int i = 0; i < n; ++i) {
    fd[i] = st.d[i] - lam;
    fl[i] = (i < n - 1) ? st.e[i] : 0.f;
    fu[i] = (i < n - 1) ? st.e[i] : 0.f;
    fu2[i] = 0.f;
    fp[i] = 0.f;
  }
  for (int i = 0; i < n - 1; ++i) {
    if (fabsf(fd[i]) >= fabsf(fl[i])) {
      float piv = fd[i];
      if (fabsf(piv) < eps_piv) { piv = (piv < 0.f) ? -eps_piv : eps_piv; fd[i] = piv; }
      const float l = fl[i] / piv;
      fl[i] = l;
      fd[i + 1] -= l * fu[i];
      fp[i] = 0.f;
    } else {
      const float l = fd[i] / fl[i];
      fd[i] = fl[i];
      fl[i] = l;
      const float t = fu[i];
      fu[i] = fd[i + 1];
      fd[i + 1] = t - l * fd[i + 1];
      if (i < n - 2) { fu2[i] = fu[i + 1]; fu[i + 1] = -l * fu[i + 1]; }
      fp[i] = 1.f;
    }
  }
  for (int i = 0; i < n; ++i)
    if (fabsf(fd[i]) < eps_piv) fd[i] = (fd[i] < 0.f) ? -eps_piv : eps_piv;
  // random start (deterministic hash), then three solves with normalisation
  for (int i = 0; i < n; ++i) x[i] = hash01((uint32_t)j, (uint32_t)i) * ((i & 1) ? 1.f : -1.f);
  for (int it = 0; it < 3; ++it) {
    for (int i = 0; i < n - 1; ++i) {
      if (fp[i] != 0.f) { const float t = x[i]; x[i] = x[i + 1]; x[i + 1] = t; }
      x[i + 1] -= fl[i] * x[i];
    }
    for (int i = n - 1; i >= 0; --i) {
      float v = x[i];
      if (i + 1 < n) v -= fu[i] * x[i + 1];
      if (i + 2 < n) v -= fu2[i] * x[i + 2];
      x[i] = v / fd[i];
    }
    float nr = 0.f, mx = 0.f;
    for (int i = 0; i < n; ++i) mx = fmaxf(mx, fabsf(x[i]));
    const float inv_mx = (mx > 0.f) ? 1.f / mx : 1.f;
    for (int i = 0; i < n; ++i) { x[i] *= inv_mx; nr += x[i] * x[i]; }
    const float inv = (nr > 0.f) ? rsqrtf(nr) : 0.f;
    for (int i = 0; i < n; ++i) x[i] *= inv;
  }
}

// groups of consecutive eigenvalues closer than tol * |T| (descending order)
__global__ void group32_kernel(E32 st, int* ngrp) {
  if (threadIdx.x != 0) return;
  float g = 0.f;
  for (int i = 0; i < st.n; ++i) g = fmaxf(g, fabsf(st.lam[i]));
  const float tol = 1e-3f * g;
  int k = 0;
  st.grp[0] = 0;
  for (int j = 1; j < st.q; ++j)
    if (st.lam[j - 1] - st.lam[j] > tol) st.grp[++k] = j;
  st.grp[++k] = st.q;
  *ngrp = k;
}

// modified Gram-Schmidt inside each group of size > 1 (one CTA per group)
__global__ void mgs32_kernel(E32 st, const int* __restrict__ ngrp) {
  __shared__ float red[32];
  if ((int)blockIdx.x >= *ngrp) return;
  const int g0 = st.grp[blockIdx.x], g1 = st.grp[blockIdx.x + 1];
  if (g1 - g0 < 2) return;
  const int n = st.n;
  for (int k = g0; k < g1; ++k) {
    float* xk = st.z + (int64_t)k * n;
    for (int pass = 0; pass < 2; ++pass) {
      for (int i0 = g0; i0 < k; ++i0) {
        const float* y = st.z + (int64_t)i0 * n;
        float part = 0.f;
        for (int i = threadIdx.x; i < n; i += blockDim.x) part += y[i] * xk[i];
        const float dot = bsum(part, red);
        for (int i = threadIdx.x; i < n; i += blockDim.x) xk[i] -= dot * y[i];
        __syncthreads();
      }
    }
    float part = 0.f;
    for (int i = threadIdx.x; i < n; i += blockDim.x) part += xk[i] * xk[i];
    const float nr = bsum(part, red);
    const float inv = (nr > 0.f) ? rsqrtf(nr) : 0.f;
    for (int i = threadIdx.x; i < n; i += blockDim.x) xk[i] *= inv;
    __syncthreads();
  }
}

// X = H_0 ... H_{n-3} Z, one warp per column; FP64 output x[i * q + j]
__global__ void bt32_kernel(E32 st) {
  const int n = st.n;
  const int lane = threadIdx.x & 31;
  const int col = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (col >= st.q) return;
  constexpr int PER = kMaxN32 / 32;
  float z[PER];
  const float* zc = st.z + (int64_t)col * n;
#pragma unroll
  for (int t = 0; t < PER; ++t) {
    const int i = lane + 32 * t;
    z[t] = (i < n) ? zc[i] : 0.f;
  }
  for (int s = n - 3; s >= 0; --s) {
    const float ta = st.tau[s];
    if (ta == 0.f) continue;
    const float* hv = st.hv + (int64_t)s * n;
    float part = 0.f;
#pragma unroll
    for (int t = 0; t < PER; ++t) {
      const int i = lane + 32 * t;
      if (i > s && i < n) part = fmaf(hv[i], z[t], part);
    }
    const float dot = wsum(part) * ta;
#pragma unroll
    for (int t = 0; t < PER; ++t) {
      const int i = lane + 32 * t;
      if (i > s && i < n) z[t] -= dot * hv[i];
    }
  }
  // renormalise in FP64
  double nr = 0.0;
#pragma unroll
  for (int t = 0; t < PER; ++t) nr += (double)z[t] * (double)z[t];
  nr = wsumd(nr);
  const double inv = (nr > 0.0) ? 1.0 / sqrt(nr) : 0.0;
#pragma unroll
  for (int t = 0; t < PER; ++t) {
    const int i = lane + 32 * t;
    if (i < n) st.x[(int64_t)i * st.q + col] = (double)z[t] * inv;
  }
}

// ------------------------------------------------------------ FP64 GEMM
// C[M x N] = op(A) B, A row-major M x K (lda) or, with TA, stored K x M (lda);
// B row-major K x N (ldb).  Split-K partials part[ks][M][N], summed in order.
constexpr int GT = 32;
__global__ void __launch_bounds__(256) dgemm_kernel(const double* __restrict__ A, int lda, int TA,
                                                    const double* __restrict__ B, int ldb, int M, int N, int K,
                                                    int kchunk, double* __restrict__ part) {
  __shared__ double As[GT][GT + 1];
  __shared__ double Bs[GT][GT + 1];
  const int m0 = blockIdx.y * GT, n0 = blockIdx.x * GT;
  const int kb = blockIdx.z * kchunk, ke = min(K, kb + kchunk);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;  // 16 x 16 threads, 2 x 2 outputs each
  double acc[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
  for (int k0 = kb; k0 < ke; k0 += GT) {
    for (int idx = threadIdx.x; idx < GT * GT; idx += 256) {
      const int r = idx / GT, c = idx % GT;
      // As[kk][mm]
      int kk, mm;
      if (TA) { kk = r; mm = c; } else { mm = r; kk = c; }
      const int gm = m0 + mm, gk = k0 + kk;
      double av = 0.0;
      if (gm < M && gk < ke) av = TA ? A[(int64_t)gk * lda + gm] : A[(int64_t)gm * lda + gk];
      As[kk][mm] = av;
      const int bk = k0 + r, bn = n0 + c;
      Bs[r][c] = (bk < ke && bn < N) ? B[(int64_t)bk * ldb + bn] : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < GT; ++kk) {
      const double a0 = As[kk][ty], a1 = As[kk][ty + 16];
      const double b0 = Bs[kk][tx], b1 = Bs[kk][tx + 16];
      acc[0][0] = fma(a0, b0, acc[0][0]);
      acc[0][1] = fma(a0, b1, acc[0][1]);
      acc[1][0] = fma(a1, b0, acc[1][0]);
      acc[1][1] = fma(a1, b1, acc[1][1]);
    }
    __syncthreads();
  }
  double* out = part + (int64_t)blockIdx.z * M * N;
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const int gm = m0 + ty + 16 * a, gn = n0 + tx + 16 * b;
      if (gm < M && gn < N) out[(int64_t)gm * N + gn] = acc[a][b];
    }
}

__global__ void dgemm_reduce(const double* __restrict__ part, int ks, int M, int N, double* __restrict__ C, int ldc) {
  const int64_t tot = (int64_t)M * N;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < tot; idx += (int64_t)gridDim.x * blockDim.x) {
    double a = 0.0;
    for (int s = 0; s < ks; ++s) a += part[(int64_t)s * tot + idx];
    C[(idx / N) * ldc + (idx % N)] = a;
  }
}

// ---------------------------------------------- refinement: lambda~, delta, F
__global__ void oa_coef_kernel(E32 st, double lam_scale_inv, double gnorm) {
  // one CTA; q x m blocks S, Q (row i in [0,q), column j in [0,m))
  __shared__ double red[64];
  const int q = st.q, m = st.m;
  double* lt = st.lt;
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    const double Sjj = st.s[(int64_t)j * m + j];
    const double Rjj = 1.0 - st.qm[(int64_t)j * m + j];
    lt[j] = Sjj / (1.0 - Rjj);
  }
  __syncthreads();
  double offS = 0.0, nR = 0.0;
  for (int64_t idx = threadIdx.x; idx < (int64_t)q * m; idx += blockDim.x) {
    const int i = (int)(idx / m), j = (int)(idx % m);
    const double R = ((i == j) ? 1.0 : 0.0) - st.qm[idx];
    const double S = st.s[idx] - ((i == j) ? lt[j] : 0.0);
    offS += S * S;
    nR += R * R;
  }
  offS = wsumd(offS);
  nR = wsumd(nR);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) { red[w] = offS; red[32 + w] = nR; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) { a += red[i]; b += red[32 + i]; }
    st.misc[2] = 2.0 * (sqrt(a) + gnorm * sqrt(b));
  }
  __syncthreads();
  const double delta = st.misc[2];
  for (int64_t idx = threadIdx.x; idx < (int64_t)q * m; idx += blockDim.x) {
    const int i = (int)(idx / m), j = (int)(idx % m);
    const double R = ((i == j) ? 1.0 : 0.0) - st.qm[idx];
    const double lj = lt[j];
    const double li = (i < m) ? lt[i] : (double)st.lam[i] * lam_scale_inv;
    double E;
    if (i == j) E = 0.5 * R;
    else if (fabs(lj - li) > delta) E = (st.s[idx] + lj * R) / (lj - li);
    else E = 0.5 * R;
    // F = E - (S - Q diag(l)) diag(1/l); the eigenvalue-0 complement is folded into W / l
    if (st.lumped) {
      const double c = st.s[idx] - st.qm[idx] * lj;
      st.f[idx] = E - c / lj;
    } else {
      st.f[idx] = E;
    }
  }
}

// x_j' = W_j / lambda~_j + (X_JK F)_j   (C holds X_JK F on entry, written back into x[:, j])
__global__ void oa_update_kernel(E32 st, const double* __restrict__ xf) {
  const int n = st.n, q = st.q, m = st.m;
  const int64_t tot = (int64_t)n * m;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < tot; idx += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx / m), j = (int)(idx % m);
    double* xp = st.x + (int64_t)i * q + j;
    *xp = st.lumped ? st.w[idx] / st.lt[j] + xf[idx] : *xp + xf[idx];
  }
}

// output: eigenvalues (unscaled FP64), top-nvec vectors with the sign convention
__global__ void eig32_out_kernel(E32 st, double lam_scale_inv, double* __restrict__ lam_out, double* __restrict__ v,
                                 int nvec) {
  const int n = st.n;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
    lam_out[j] = (j < st.m) ? st.lt[j] : (double)st.lam[j] * lam_scale_inv;
  if (!v) return;
  const int lane = threadIdx.x & 31;
  const int col = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (col >= nvec) return;
  double best = -1.0, bval = 0.0;
  int bidx = n;
  for (int i = lane; i < n; i += 32) {
    const double a = st.x[(int64_t)i * st.q + col];
    if (fabs(a) > best) { best = fabs(a); bidx = i; bval = a; }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double ob = __shfl_xor_sync(0xffffffffu, best, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bidx, o);
    const double ov = __shfl_xor_sync(0xffffffffu, bval, o);
    if (ob > best || (ob == best && oi < bidx)) { best = ob; bidx = oi; bval = ov; }
  }
  // normalise in FP64 as well
  double nr = 0.0;
  for (int i = lane; i < n; i += 32) { const double a = st.x[(int64_t)i * st.q + col]; nr += a * a; }
  nr = wsumd(nr);
  const double sg = ((bval < 0.0) ? -1.0 : 1.0) / sqrt(nr);
  for (int i = lane; i < n; i += 32) v[(int64_t)i * nvec + col] = sg * st.x[(int64_t)i * st.q + col];
}

__global__ void trace_kernel(const double* __restrict__ G, int n, double* __restrict__ out) {
  double a = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) a += G[(int64_t)i * n + i];
  a = wsumd(a);
  __shared__ double red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
    *out = t;
  }
}

// ----------------------------------------------------------------- host side
E32 g32;
const double* g_G = nullptr;
std::vector<float> g_lam32;
double g_scale = 1.0, g_trace = 0.0;

int dgemm(const double* A, int lda, int TA, const double* B, int ldb, int M, int N, int K, double* C, int ldc,
          cudaStream_t s) {
  const int tm = (M + GT - 1) / GT, tn = (N + GT - 1) / GT;
  int ks = (2 * 152 + tm * tn - 1) / (tm * tn);
  const int maxks = (K + GT - 1) / GT;
  if (ks > maxks) ks = maxks;
  if (ks < 1) ks = 1;
  int kchunk = (K + ks - 1) / ks;
  kchunk = (kchunk + GT - 1) / GT * GT;
  ks = (K + kchunk - 1) / kchunk;
  if ((size_t)ks * M * N > (size_t)4 * 1024 * 1024) return fail(ATC_EUNSUP, "refinement GEMM too large");
  dgemm_kernel<<<dim3(tn, tm, ks), 256, 0, s>>>(A, lda, TA, B, ldb, M, N, K, kchunk, g32.gpart);
  const int64_t tot = (int64_t)M * N;
  dgemm_reduce<<<(int)((tot + 255) / 256 < 1024 ? (tot + 255) / 256 : 1024), 256, 0, s>>>(g32.gpart, ks, M, N, C, ldc);
  ATC_LAUNCHED(2);
  return ATC_OK;
}

}  // namespace

bool eig32_supported(int n) { return n >= 1 && n <= kMaxN32; }

// Experimental (ATC_EIG32=1): the FP32 first stage cannot resolve eigenvectors
// whose eigenvalues lie below ~1e-7 of the largest, where rank cuts at small
// rel_eps fall, so the default solver is the FP64 one.
bool eig32_enabled() {
  static int v = -1;
  if (v < 0) {
    const char* e = getenv("ATC_EIG32");
    v = (e && e[0] == '1') ? 1 : 0;
  }
  return v == 1;
}

// Stage 1a: scaled FP32 tridiagonalisation + all eigenvalues.  lam_host
// receives the n FP32-accurate eigenvalues (unscaled, descending) and
// *trace the FP64 trace of G.  Synchronises the stream.
int eig32_values(const double* G, int n, std::vector<double>* lam_host, double* trace, cudaStream_t s) {
  if (!eig32_supported(n)) return fail(ATC_EUNSUP, "eig32: n = %d", n);
  E32 st{};
  st.n = n;
  float* fbuf = nullptr;
  ATC_TRY(Scratch::get(SLOT_EIG_V, sizeof(float) * ((size_t)n * n + 8 * n + 64), (void**)&fbuf));
  st.hv = fbuf;
  st.d = fbuf + (size_t)n * n;
  st.e = st.d + n;
  st.tau = st.e + n;
  st.lam = st.tau + n;
  double* misc = nullptr;
  ATC_TRY(Scratch::get(SLOT_EIG_VEC, sizeof(double) * 64, (void**)&misc));
  st.misc = misc;
  const int npk = n * (n + 1) / 2;
  const size_t smem = sizeof(float) * (((npk + 31) & ~31) + 6 * kMaxN32 + 32 * kMaxN32 + 64);
  static bool attr = false;
  if (!attr) {
    ATC_CUDA_TRY(cudaFuncSetAttribute(tri32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 225 * 1024));
    attr = true;
  }
  if (smem > 225 * 1024) return fail(ATC_EUNSUP, "eig32: shared memory");
  tri32_kernel<<<1, kTri, smem, s>>>(G, n, st);
  ATC_LAUNCHED(1);
  const int wpb = 8;
  bis32_kernel<<<(n + wpb - 1) / wpb, 32 * wpb, sizeof(float) * 2 * n, s>>>(st);
  ATC_LAUNCHED(1);
  trace_kernel<<<1, 256, 0, s>>>(G, n, misc + 1);
  ATC_LAUNCHED(1);
  std::vector<float> lam(n);
  double mh[2];
  ATC_CUDA_TRY(cudaMemcpyAsync(lam.data(), st.lam, sizeof(float) * n, cudaMemcpyDeviceToHost, s));
  ATC_CUDA_TRY(cudaMemcpyAsync(mh, misc, sizeof(double) * 2, cudaMemcpyDeviceToHost, s));
  ATC_CUDA_TRY(cudaStreamSynchronize(s));
  g_scale = mh[0];
  g_trace = mh[1];
  g32 = st;
  g_G = G;
  g_lam32 = lam;
  lam_host->resize(n);
  for (int j = 0; j < n; ++j) (*lam_host)[j] = (double)lam[j] / g_scale;
  *trace = g_trace;
  return ATC_OK;
}

// Stage 1b + 2: eigenvectors of the top q (chosen from m and eta), FP64
// refinement of the top m.  lam_dev (n) receives eigenvalues (refined for
// j < m), v_dev (n x nvec, nvec <= m) the refined vectors.  lam_host gets the
// refined top m.  Synchronises the stream.
int eig32_refine(int m, double* lam_dev, double* v_dev, int nvec, std::vector<double>* lam_top, cudaStream_t s) {
  E32 st = g32;
  const int n = st.n;
  if (m < 1) m = 1;
  if (m > n) m = n;
  // q: every eigenvalue above eta * lambda_{m-1} gets an explicit vector
  const double eta = 1e-3;
  const float thr = (float)(eta * (double)g_lam32[m - 1]);
  int q = m;
  while (q < n && g_lam32[q] > thr && g_lam32[q] > 0.f) ++q;
  if (g_lam32[m - 1] <= 0.f) q = n;
  st.q = q;
  st.m = m;
  st.lumped = (q < n) ? 1 : 0;
  uint8_t* buf = nullptr;
  const size_t zf = (size_t)q * n * 6 + 64;                 // z + lu (floats)
  const size_t db = (size_t)n * q + 2 * (size_t)n * m + 3 * (size_t)q * m + m + 64;  // doubles
  ATC_TRY(Scratch::get(SLOT_EIG_Z, sizeof(float) * zf + sizeof(double) * db + sizeof(int) * (q + 8) + 1024, (void**)&buf));
  st.z = reinterpret_cast<float*>(buf);
  st.lu = st.z + (size_t)q * n;
  double* dptr = reinterpret_cast<double*>(buf + ((sizeof(float) * zf + 255) & ~(size_t)255));
  st.x = dptr;
  st.w = st.x + (size_t)n * q;
  double* xf = st.w + (size_t)n * m;
  st.s = xf + (size_t)n * m;
  st.qm = st.s + (size_t)q * m;
  st.f = st.qm + (size_t)q * m;
  st.lt = st.f + (size_t)q * m;
  st.grp = reinterpret_cast<int*>(st.lt + m + 8);
  int* ngrp = st.grp + q + 2;
  ATC_TRY(Scratch::get(SLOT_GRAM_PART, sizeof(double) * 4 * 1024 * 1024, (void**)&st.gpart));
  g32 = st;
  invit32_kernel<<<(q + 63) / 64, 64, 0, s>>>(st);
  ATC_LAUNCHED(1);
  group32_kernel<<<1, 32, 0, s>>>(st, ngrp);
  ATC_LAUNCHED(1);
  mgs32_kernel<<<q, 128, 0, s>>>(st, ngrp);
  ATC_LAUNCHED(1);
  bt32_kernel<<<(q + 3) / 4, 128, 0, s>>>(st);
  ATC_LAUNCHED(1);
  const double inv_sc = 1.0 / g_scale;
  const double gnorm = (double)g_lam32[0] * inv_sc;
  for (int pass = 0; pass < 2; ++pass) {
    ATC_TRY(dgemm(g_G, n, 0, st.x, q, n, m, n, st.w, m, s));         // W = G X_J
    ATC_TRY(dgemm(st.x, q, 1, st.w, m, q, m, n, st.s, m, s));        // S = X_JK^T W
    ATC_TRY(dgemm(st.x, q, 1, st.x, q, q, m, n, st.qm, m, s));       // Q = X_JK^T X_J
    oa_coef_kernel<<<1, 256, 0, s>>>(st, inv_sc, gnorm);
    ATC_LAUNCHED(1);
    ATC_TRY(dgemm(st.x, q, 0, st.f, m, n, m, q, xf, m, s));          // X_JK F
    oa_update_kernel<<<(int)(((int64_t)n * m + 255) / 256), 256, 0, s>>>(st, xf);
    ATC_LAUNCHED(1);
  }
  eig32_out_kernel<<<(std::max(n, nvec * 32) + 127) / 128, 128, 0, s>>>(st, inv_sc, lam_dev, v_dev, nvec);
  ATC_LAUNCHED(1);
  lam_top->resize(m);
  ATC_CUDA_TRY(cudaMemcpyAsync(lam_top->data(), st.lt, sizeof(double) * m, cudaMemcpyDeviceToHost, s));
  ATC_CUDA_TRY(cudaStreamSynchronize(s));
  return ATC_OK;
}

double eig32_trace() { return g_trace; }

}  // namespace atc
