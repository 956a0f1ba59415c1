// FP64 symmetric eigensolver for the mode Gram matrices (Algorithm 1: the
// left singular vectors / squared singular values of the unfolding are the
// eigenvectors / eigenvalues of G = B_(k) B_(k)^T), and the rank choice of
// Section 4.1.3.
//
// GB300 has a small FP64 rate (about 2 DFMA lanes per clock per SM), so the
// solver keeps FP64 work proportional to n^3 only where unavoidable and spreads
// it over many SMs:
//   1. Householder tridiagonalisation T = Q^T G Q: rows dealt cyclically to the
//      CTAs; each step re-forms the next reflector redundantly in every CTA and
//      fuses the two-sided update of step s-1 with the matrix-vector product of
//      step s, so a step costs ONE barrier.  For n <= 512 the CTAs form one
//      thread-block cluster (16, else 8): the rows live in shared memory, row s
//      and the vector p are read from the owners through distributed shared
//      memory, and the barrier is the hardware cluster barrier.  Larger n use a
//      cooperative grid with the rows in global memory and a bounded software
//      grid barrier (on time-out an error flag is raised and every CTA returns).
//   2. Eigenvalues of T by bisection on Sturm counts; the count uses the
//      three-term recurrence of the leading principal minors (one dependent
//      FMA per row) with power-of-two rescaling instead of a division per row.
//   3. Eigenvectors of T for the largest eigenvalues by inverse iteration
//      (LU with partial pivoting of T - lambda I), one CTA per group of close
//      eigenvalues, re-orthogonalised within the group.
//   4. Back-transformation X = Q Z, a warp per column, then the sign
//      convention (largest-magnitude entry positive).
#include <math.h>
#include <stdio.h>
#include <stdint.h>

#include <cooperative_groups.h>

#include <vector>

#include "atc_internal.cuh"
#include "dd.cuh"

namespace cg = cooperative_groups;

namespace atc {
namespace {

constexpr int kTriThreads = 256;
constexpr unsigned kSpinLimit = 1u << 22;  // about 0.3 s of nanosleep(64) polling

struct EigState {
  double* a;      // n x n working copy
  double* hv;     // (n) x n Householder vectors, row s holds v_s (v_s[s+1] = 1)
  double* d;      // n diagonal of T (scaled after eig_values)
  double* e;      // n off-diagonal of T (e[s] couples s, s+1)
  double* tau;    // n
  double* pbuf;   // 2 x n
  double* lam;    // n eigenvalues of T, descending (scaled)
  double* z;      // n x nvec tridiagonal eigenvectors (column j contiguous: z[j*n + i])
  double* lu;     // 5 x n x nvec LU scratch
  int* flags;     // [0] barrier count, [1] barrier generation, [2] error, [3] spare
  double* scale;  // [0] power-of-two scale applied to T
  int n;
};
EigState g_state = {};  // host-side copy of the scratch layout (single-stream use per device)
bool g_state_dd = false;  // the current tridiagonal matrix came from the double-float solver

__device__ __forceinline__ double ldcg(const double* p) { return __ldcg(p); }

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Grid-wide barrier for a cooperative launch with a bounded wait.
// Returns false if any CTA gave up (error flag raised).
__device__ bool grid_barrier(int* flags) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned* count = reinterpret_cast<unsigned*>(flags);
    unsigned* gen = reinterpret_cast<unsigned*>(flags + 1);
    volatile int* err = flags + 2;
    unsigned g = ld_acquire(gen);
    __threadfence();
    unsigned arrived = atomicAdd(count, 1u) + 1u;
    int ok = 1;
    if (arrived == gridDim.x) {
      atomicExch(count, 0u);
      __threadfence();
      st_release(gen, g + 1u);
    } else {
      unsigned it = 0;
      while (ld_acquire(gen) == g) {
        if (*err) { ok = 0; break; }
        if (++it > kSpinLimit) { atomicExch(flags + 2, 1); ok = 0; break; }
        __nanosleep(64);
      }
    }
    __threadfence();
    if (*err) ok = 0;
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Deterministic block sum (identical result in every CTA for identical input).
__device__ double block_sum(double v, double* red) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  const int nw = blockDim.x >> 5;
  for (int i = 0; i < nw; ++i) t += red[i];
  return t;
}

// ------------------------------------------------------------ tridiagonalisation
// Iteration s (0 <= s <= n-2):
//   phase 1 (s >= 1): w_{s-1} = p_{s-1} - (tau_{s-1}/2)(p_{s-1}.v_{s-1}) v_{s-1}
//   phase 2: row s of A^(s) = stored row s - v_{s-1}[s] w_{s-1} - w_{s-1}[s] v_{s-1};
//            d_s = its diagonal; reflector v_s, tau_s from its entries s+1..n-1; e_s = alpha.
//   phase 3 (s <= n-3): owned rows i >= s+1: A^(s) = A^(s-1) - v w^T - w v^T on columns
//            >= s+1, stored; p_s[i] = tau_s * (A^(s) row i) . v_s
//   grid barrier
__global__ void __launch_bounds__(kTriThreads) tridiag_kernel(EigState st) {
  extern __shared__ double sm[];
  const int n = st.n;
  double* v_prev = sm;          // v_{s-1}
  double* w_prev = sm + n;      // w_{s-1}
  double* v_cur = sm + 2 * n;   // v_s
  double* row = sm + 3 * n;     // row s of A^(s)
  double* red = sm + 4 * n;     // 32 doubles
  __shared__ double s_tau_prev, s_tau;
  const int tid = threadIdx.x;
  const int P = gridDim.x, b = blockIdx.x;
  const int lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
  for (int i = tid; i < n; i += blockDim.x) { v_prev[i] = 0.0; w_prev[i] = 0.0; v_cur[i] = 0.0; }
  if (tid == 0) { s_tau_prev = 0.0; s_tau = 0.0; }
  __syncthreads();
  for (int s = 0; s <= n - 2; ++s) {
    // phase 1
    if (s >= 1) {
      const double* p = st.pbuf + ((s - 1) & 1) * n;
      double part = 0.0;
      for (int i = s + tid; i < n; i += blockDim.x) part += ldcg(p + i) * v_prev[i];
      double dot = block_sum(part, red);
      double K = 0.5 * s_tau_prev * dot;
      for (int i = tid; i < n; i += blockDim.x) w_prev[i] = (i >= s) ? ldcg(p + i) - K * v_prev[i] : 0.0;
      __syncthreads();
    }
    // phase 2: row s of A^(s)
    {
      const double vs = v_prev[s], ws = w_prev[s];
      for (int j = s + tid; j < n; j += blockDim.x)
        row[j] = ldcg(st.a + (int64_t)s * n + j) - vs * w_prev[j] - ws * v_prev[j];
      __syncthreads();
    }
    double alpha = 0.0, tau = 0.0;
    if (s <= n - 3) {
      double part = 0.0;
      for (int j = s + 2 + tid; j < n; j += blockDim.x) part += row[j] * row[j];
      double sig2 = block_sum(part, red);
      const double x0 = row[s + 1];
      double scal = 0.0;
      if (sig2 == 0.0) {
        tau = 0.0; alpha = x0; scal = 0.0;
      } else {
        double nrm = sqrt(x0 * x0 + sig2);
        alpha = (x0 >= 0.0) ? -nrm : nrm;
        tau = (alpha - x0) / alpha;
        scal = 1.0 / (x0 - alpha);
      }
      for (int j = tid; j < n; j += blockDim.x) {
        double v = 0.0;
        if (j == s + 1) v = 1.0;
        else if (j > s + 1) v = row[j] * scal;
        v_cur[j] = v;
      }
      if (tid == 0) s_tau = tau;
      __syncthreads();
      if (b == 0) {
        for (int j = tid; j < n; j += blockDim.x) st.hv[(int64_t)s * n + j] = v_cur[j];
        if (tid == 0) { st.d[s] = row[s]; st.e[s] = alpha; st.tau[s] = tau; }
      }
      // phase 3: fused update of rows >= s+1 and p_s
      double* pout = st.pbuf + (s & 1) * n;
      for (int i = s + 1 + ((b - (s + 1)) % P + P) % P + warp * P; i < n; i += P * nwarp) {
        const double vi = v_prev[i], wi = w_prev[i];
        double* arow = st.a + (int64_t)i * n;
        double acc = 0.0;
        for (int j = s + 1 + lane; j < n; j += 32) {
          double a = ldcg(arow + j) - vi * w_prev[j] - wi * v_prev[j];
          arow[j] = a;
          acc = fma(a, v_cur[j], acc);
        }
        acc = warp_sum(acc);
        if (lane == 0) pout[i] = tau * acc;
      }
      if (!grid_barrier(st.flags)) return;
      // rotate v/w
      for (int i = tid; i < n; i += blockDim.x) v_prev[i] = v_cur[i];
      if (tid == 0) s_tau_prev = s_tau;
      __syncthreads();
    } else {
      // s == n-2: last 2x2 block
      if (b == 0 && tid == 0) {
        st.d[s] = row[s];
        st.e[s] = row[s + 1];
        double a11 = ldcg(st.a + (int64_t)(n - 1) * n + (n - 1));
        st.d[n - 1] = a11 - 2.0 * v_prev[n - 1] * w_prev[n - 1];
        st.tau[s] = 0.0;
      }
    }
  }
}

// Same iteration as tridiag_kernel, on one cluster of C CTAs with the rows in
// shared memory: CTA b owns rows i == b (mod C), stored at local index i / C.
// Thread t handles index j = s + t of the step's vectors, so the gathered p,
// w and row s never need a barrier of their own; a step has two block
// reductions, one block barrier and one cluster barrier.  Every CTA runs the
// same number of cluster barriers (no early exit).
constexpr int kTriCThreads = 512;  // launch uses 256 for n <= 256 (one thread per index)

// sum over the CTA, identical in every thread: warp sums, then warp 0 sums the
// partials (fixed tree) and publishes the total.  Warps whose lanes all carry
// zero skip their FP64 work (the FP64 pipe is the scarce resource).
__device__ __forceinline__ double block_reduce(double v, double* red, bool warp_active) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (warp_active) v = warp_sum(v);
  if (lane == 0) red[warp] = warp_active ? v : 0.0;
  __syncthreads();
  if (warp == 0) {
    double t = (lane < nw) ? red[lane] : 0.0;
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) red[16] = t;
  }
  __syncthreads();
  return red[16];
}

template <int NPER>
__global__ void __launch_bounds__(kTriCThreads) tridiag_cluster_kernel(EigState st, const double* __restrict__ g) {
  extern __shared__ double sm[];
  cg::cluster_group cl = cg::this_cluster();
  const int n = st.n;
  const int C = (int)cl.num_blocks(), b = (int)cl.block_rank();
  const int rows = (n + C - 1) / C;
  double* vprev = sm;           // v_{s-1}
  double* vcur = sm + n;        // v_s
  double* wv = sm + 2 * n;      // w_{s-1}
  double* red1 = sm + 3 * n;    // 16 partials + total
  double* red2 = red1 + 24;     // 16 partials + total
  double* sx = red2 + 24;       // [0] row_s[s+1], [1] row_s[s]
  double* pfull = sx + 16;      // [2][n] p_s, written into every CTA by the row owners
  double* A = pfull + 2 * n;    // [rows][n]
  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
  for (int li = 0; li < rows; ++li) {
    const int i = li * C + b;
    for (int j = tid; j < n; j += blockDim.x) A[(int64_t)li * n + j] = (i < n) ? g[(int64_t)i * n + j] : 0.0;
  }
  for (int i = tid; i < n; i += blockDim.x) {
    vprev[i] = 0.0; vcur[i] = 0.0; wv[i] = 0.0; pfull[i] = 0.0; pfull[n + i] = 0.0;
  }
  double tau_prev = 0.0;
  cl.sync();
  for (int s = 0; s <= n - 2; ++s) {
    const int j = s + tid;
    const bool has = j < n;
    const bool wact = s + (tid & ~31) < n;  // some lane of this warp has j < n
    // w_{s-1} = p_{s-1} - K v_{s-1}, K = (tau_{s-1} / 2) p_{s-1} . v_{s-1}
    double pj = 0.0, ps = 0.0, K = 0.0;
    const double vj = has ? vprev[j] : 0.0, vs = vprev[s];
    if (s >= 1) {
      const double* pb = pfull + ((s - 1) & 1) * n;
      if (has) pj = pb[j];
      ps = pb[s];
      K = 0.5 * tau_prev * block_reduce(pj * vj, red1, wact);
    }
    const double wj = pj - K * vj, ws = ps - K * vs;
    // row s of A^(s), entries j >= s, read from the owner of row s
    double rowj = 0.0;
    if (has) rowj = *cl.map_shared_rank(A + (int64_t)(s / C) * n + j, s % C) - vs * wj - ws * vj;
    if (s <= n - 3) {
      if (tid == 1) sx[0] = rowj;
      if (tid == 0) sx[1] = rowj;
      const double sig2 = block_reduce((j >= s + 2 && has) ? rowj * rowj : 0.0, red2, wact);
      const double x0 = sx[0], ds = sx[1];
      double alpha, tau, scal;
      if (sig2 == 0.0) {
        tau = 0.0; alpha = x0; scal = 0.0;
      } else {
        const double nrm = sqrt(x0 * x0 + sig2);
        alpha = (x0 >= 0.0) ? -nrm : nrm;
        tau = (alpha - x0) / alpha;
        scal = 1.0 / (x0 - alpha);
      }
      if (has) {
        wv[j] = wj;
        vcur[j] = (j == s + 1) ? 1.0 : ((j > s + 1) ? rowj * scal : 0.0);
      }
      __syncthreads();
      if (b == 0) {
        for (int q = tid; q < n; q += blockDim.x) st.hv[(int64_t)s * n + q] = (q > s) ? vcur[q] : 0.0;
        if (tid == 0) { st.d[s] = ds; st.e[s] = alpha; st.tau[s] = tau; }
      }
      // fused update of the owned rows >= s+1 and p_s, a warp per row, the
      // lane's slice of the vectors in registers
      double vp[NPER], wq[NPER], vc[NPER];
#pragma unroll
      for (int q = 0; q < NPER; ++q) {
        const int jj = s + 1 + lane + 32 * q;
        const bool ok = jj < n;
        vp[q] = ok ? vprev[jj] : 0.0;
        wq[q] = ok ? wv[jj] : 0.0;
        vc[q] = ok ? vcur[jj] : 0.0;
      }
      double* pout = pfull + (s & 1) * n;
      const int li0 = (s + 1 - b + C - 1) / C;  // first local row with global index >= s+1
      for (int li = li0 + warp; li < rows; li += nwarp) {
        const int i = li * C + b;
        if (i >= n) break;
        const double vi = vprev[i], wi = wv[i];
        double* arow = A + (int64_t)li * n + s + 1 + lane;
        double a[NPER];
#pragma unroll
        for (int q = 0; q < NPER; ++q) a[q] = (s + 1 + lane + 32 * q < n) ? arow[32 * q] : 0.0;
#pragma unroll
        for (int q = 0; q < NPER; ++q) {
          a[q] = fma(-vi, wq[q], fma(-wi, vp[q], a[q]));
          if (s + 1 + lane + 32 * q < n) arow[32 * q] = a[q];
          a[q] *= vc[q];
        }
#pragma unroll
        for (int w = 1; w < NPER; w <<= 1)
#pragma unroll
          for (int q = 0; q + w < NPER; q += 2 * w) a[q] += a[q + w];
        const double acc = warp_sum(a[0]);
        // p_s[i] into every CTA of the cluster (remote stores, visible after the barrier)
        if (lane < C) *cl.map_shared_rank(pout + i, lane) = tau * acc;
      }
      cl.sync();
      double* t = vprev;
      vprev = vcur;
      vcur = t;
      tau_prev = tau;
    } else {
      // s == n-2: the last 2 x 2 block
      if (b == 0 && tid == 0) { st.d[s] = rowj; st.tau[s] = 0.0; }
      if (b == 0 && tid == 1) {
        st.e[s] = rowj;
        const double a11 = *cl.map_shared_rank(A + (int64_t)((n - 1) / C) * n + (n - 1), (n - 1) % C);
        st.d[n - 1] = a11 - 2.0 * vj * wj;
      }
    }
  }
  // no CTA may leave while another can still read its shared memory
  cl.sync();
}

__global__ void tridiag_small_kernel(EigState st) {
  // n == 1
  if (threadIdx.x == 0) { st.d[0] = st.a[0]; st.e[0] = 0.0; }
}

// ------------------------------------------------------------------ eigenvalues
// Scale T by a power of two so that the Gershgorin disc radius is <= 1.
__global__ void scale_kernel(EigState st) {
  __shared__ double red[32];
  const int n = st.n;
  double m = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double r = fabs(st.d[i]) + (i > 0 ? fabs(st.e[i - 1]) : 0.0) + (i < n - 1 ? fabs(st.e[i]) : 0.0);
    m = fmax(m, r);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double mm = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) mm = fmax(mm, red[i]);
    int ex = 0;
    if (mm > 0.0) frexp(mm, &ex);
    red[0] = ldexp(1.0, -ex);  // mm * scale in [0.5, 1)
    st.scale[0] = red[0];
  }
  __syncthreads();
  const double sc = red[0];
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    st.d[i] *= sc;
    if (i < n - 1) st.e[i] *= sc;
  }
}

// Number of eigenvalues of T (scaled, |entries| <= 1) smaller than sigma: sign
// changes of the leading principal minors p_0 = 1, p_1, ..., p_n.  The
// recurrence p_i = (d_i - sigma) p_{i-1} - e_{i-1}^2 p_{i-2} is one dependent
// FMA per row (e^2 p_{i-2} and d_i - sigma are ready a step early); the
// power-of-two rescaling only selects, so it adds no FP64 latency.
__device__ int sturm_count(const double* __restrict__ d, const double* __restrict__ e2, int n, double sigma) {
  double pp = 1.0, p = d[0] - sigma;
  const double tiny = 0x1p-900;
  if (p == 0.0) p = -tiny;
  int cnt = (p < 0.0);
  int i = 1;
  while (i < n) {
    const int i1 = min(n, i + 4);
    for (; i < i1; ++i) {
      const double t = e2[i - 1] * pp;
      const double dm = d[i] - sigma;
      double q = fma(dm, p, -t);
      const long long qb = __double_as_longlong(q), pb = __double_as_longlong(p);
      // an exact zero continues with the sign opposite to p (a sign change)
      if ((qb & 0x7fffffffffffffffll) == 0) q = (pb < 0) ? tiny : -tiny;
      cnt += (int)(((unsigned long long)(__double_as_longlong(q) ^ pb)) >> 63);
      pp = p;
      p = q;
    }
    // rescale by 2^-500 / 2^500 when max(|p|, |pp|) leaves [2^-500, 2^500]: a
    // row grows the pair at most 3-fold (|entries| <= 1) and shrinks it at most
    // by e^2 >= 2^-120 (the floor applied when e2 is built), so between checks
    // it stays within [2^-980, 2^507]
    const int ex = (__double2hiint(p) >> 20) & 0x7ff;
    const int ex2 = (__double2hiint(pp) >> 20) & 0x7ff;
    const int mx = max(ex, ex2);
    if (mx > 1023 + 500) { p *= 0x1p-500; pp *= 0x1p-500; }
    else if (mx < 1023 - 500) { p *= 0x1p500; pp *= 0x1p500; }
  }
  return cnt;
}

__global__ void bisect_kernel(EigState st) {
  extern __shared__ double sm[];
  const int n = st.n;
  double* d = sm;
  double* e2 = sm + n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    d[i] = st.d[i];
    e2[i] = (i < n - 1) ? fmax(st.e[i] * st.e[i], 0x1p-120) : 0.0;
  }
  __syncthreads();
  const int j = blockIdx.x * blockDim.x + threadIdx.x;  // j-th largest
  if (j >= n) return;
  const int m = n - 1 - j;  // m-th smallest (0-based)
  double lo = -1.0, hi = 1.0;  // Gershgorin radius <= 1 after scaling
  for (int it = 0; it < 200; ++it) {
    double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (sturm_count(d, e2, n, mid) <= m) lo = mid; else hi = mid;
    if (hi - lo <= 0x1p-54) break;
  }
  st.lam[j] = 0.5 * (lo + hi);
}

// ----------------------------------------------------------------- eigenvectors
// Inverse iteration for the eigenvalues of one group (consecutive indices with
// gaps below the grouping threshold); thread 0 runs the O(n) recurrences,
// the block does the re-orthogonalisation against earlier vectors of the group.
__global__ void invit_kernel(EigState st, const int* __restrict__ grp_start, const int* __restrict__ ngrp, int nvec) {
  __shared__ double red[32];
  const int n = st.n;
  if ((int)blockIdx.x >= *ngrp) return;
  const int g0 = grp_start[blockIdx.x], g1 = grp_start[blockIdx.x + 1];
  const double* dd = st.d;
  const double* ee = st.e;
  for (int j = g0; j < g1 && j < nvec; ++j) {
    double* x = st.z + (int64_t)j * n;
    double* ld_ = st.lu + (int64_t)j * 5 * n;  // dl, d, du, du2, piv
    double* fl = ld_;
    double* fd = ld_ + n;
    double* fu = ld_ + 2 * n;
    double* fu2 = ld_ + 3 * n;
    double* fp = ld_ + 4 * n;
    const double lam = st.lam[j];
    const double eps_piv = 0x1p-52;  // |T| <= 1 after scaling
    if (threadIdx.x == 0) {
      // LU with partial pivoting of T - lam I (rows i, i+1 may swap)
      for (int i = 0; i < n; ++i) {
        fd[i] = dd[i] - lam;
        fl[i] = (i < n - 1) ? ee[i] : 0.0;
        fu[i] = (i < n - 1) ? ee[i] : 0.0;
        fu2[i] = 0.0;
        fp[i] = 0.0;
      }
      for (int i = 0; i < n - 1; ++i) {
        if (fabs(fd[i]) >= fabs(fl[i])) {
          double piv = fd[i];
          if (piv == 0.0) { piv = eps_piv; fd[i] = piv; }
          double l = fl[i] / piv;
          fl[i] = l;
          fd[i + 1] -= l * fu[i];
          fp[i] = 0.0;
        } else {
          double l = fd[i] / fl[i];
          fd[i] = fl[i];
          fl[i] = l;
          double t = fu[i];
          fu[i] = fd[i + 1];
          fd[i + 1] = t - l * fd[i + 1];
          if (i < n - 2) { fu2[i] = fu[i + 1]; fu[i + 1] = -l * fu[i + 1]; }
          fp[i] = 1.0;
        }
      }
      if (fd[n - 1] == 0.0) fd[n - 1] = eps_piv;
      for (int i = 0; i < n; ++i) if (fabs(fd[i]) < eps_piv) fd[i] = (fd[i] < 0.0) ? -eps_piv : eps_piv;
      // start vector: U x = (1, ..., 1) (first step skips L, as usual)
      for (int i = n - 1; i >= 0; --i) {
        double v = 1.0;
        if (i + 1 < n) v -= fu[i] * x[i + 1];
        if (i + 2 < n) v -= fu2[i] * x[i + 2];
        x[i] = v / fd[i];
      }
    }
    __syncthreads();
    for (int iter = 0; iter < 3; ++iter) {
      // orthogonalise against earlier vectors of the group, then normalise
      for (int k = g0; k < j; ++k) {
        const double* y = st.z + (int64_t)k * n;
        double part = 0.0;
        for (int i = threadIdx.x; i < n; i += blockDim.x) part += y[i] * x[i];
        double dot = block_sum(part, red);
        for (int i = threadIdx.x; i < n; i += blockDim.x) x[i] -= dot * y[i];
        __syncthreads();
      }
      double part = 0.0;
      for (int i = threadIdx.x; i < n; i += blockDim.x) part += x[i] * x[i];
      double nr = block_sum(part, red);
      double inv = (nr > 0.0) ? 1.0 / sqrt(nr) : 0.0;
      for (int i = threadIdx.x; i < n; i += blockDim.x) x[i] *= inv;
      __syncthreads();
      if (iter == 2) break;
      if (threadIdx.x == 0) {
        // solve P L U y = x: apply L^-1 (with the row swaps), then U^-1
        for (int i = 0; i < n - 1; ++i) {
          if (fp[i] != 0.0) { double t = x[i]; x[i] = x[i + 1]; x[i + 1] = t; }
          x[i + 1] -= fl[i] * x[i];
        }
        for (int i = n - 1; i >= 0; --i) {
          double v = x[i];
          if (i + 1 < n) v -= fu[i] * x[i + 1];
          if (i + 2 < n) v -= fu2[i] * x[i + 2];
          x[i] = v / fd[i];
        }
      }
      __syncthreads();
    }
  }
}

// X = H_0 H_1 ... H_{n-3} Z, one warp per column; then the sign convention and
// the transpose into v (n x nvec row-major).
template <int NPER>
__global__ void backtransform_kernel(EigState st, int nvec, double* __restrict__ v) {
  const int n = st.n;
  const int lane = threadIdx.x & 31;
  const int col = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (col >= nvec) return;
  constexpr int MAXPER = NPER;  // n <= 32 * NPER
  double z[MAXPER], h[MAXPER];
  const double* zc = st.z + (int64_t)col * n;
#pragma unroll
  for (int q = 0; q < MAXPER; ++q) {
    int i = lane + 32 * q;
    z[q] = (i < n) ? zc[i] : 0.0;
  }
  // reflector s acts on entries i > s; the next one is prefetched while the
  // current one is applied (the loop is a chain of dependent reductions)
  auto load_h = [&](int s) {
    const double* hv = st.hv + (int64_t)s * n;
#pragma unroll
    for (int q = 0; q < MAXPER; ++q) {
      const int i = lane + 32 * q;
      h[q] = (i > s && i < n) ? __ldg(hv + i) : 0.0;
    }
  };
  if (n >= 3) load_h(n - 3);
  for (int s = n - 3; s >= 0; --s) {
    const double t = st.tau[s];
    double hc[MAXPER];
#pragma unroll
    for (int q = 0; q < MAXPER; ++q) hc[q] = h[q];
    if (s > 0) load_h(s - 1);
    if (t == 0.0) continue;
    // pairwise dot product (tree depth log2(MAXPER)) and warp reduction
    double pr[MAXPER];
#pragma unroll
    for (int q = 0; q < MAXPER; ++q) pr[q] = hc[q] * z[q];
#pragma unroll
    for (int w = 1; w < MAXPER; w <<= 1)
#pragma unroll
      for (int q = 0; q + w < MAXPER; q += 2 * w) pr[q] += pr[q + w];
    const double dot = warp_sum(pr[0]) * t;
#pragma unroll
    for (int q = 0; q < MAXPER; ++q) z[q] = fma(-dot, hc[q], z[q]);
  }
  // sign: entry of largest magnitude (first on ties) positive
  double best = -1.0;
  int bidx = n;
  double bval = 0.0;
#pragma unroll
  for (int q = 0; q < MAXPER; ++q) {
    int i = lane + 32 * q;
    if (i < n) {
      double a = fabs(z[q]);
      if (a > best) { best = a; bidx = i; bval = z[q]; }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    double ob = __shfl_xor_sync(0xffffffffu, best, o);
    int oi = __shfl_xor_sync(0xffffffffu, bidx, o);
    double ov = __shfl_xor_sync(0xffffffffu, bval, o);
    if (ob > best || (ob == best && oi < bidx)) { best = ob; bidx = oi; bval = ov; }
  }
  const double sg = (bval < 0.0) ? -1.0 : 1.0;
#pragma unroll
  for (int q = 0; q < MAXPER; ++q) {
    int i = lane + 32 * q;
    if (i < n) v[(int64_t)i * nvec + col] = sg * z[q];
  }
}

// lam_out[j] = lam_scaled[j] / scale (exact power of two)
__global__ void unscale_kernel(EigState st, double* __restrict__ lam_out, int K) {
  const double inv = 1.0 / st.scale[0];
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < K; j += gridDim.x * blockDim.x)
    lam_out[j] = st.lam[j] * inv;
}

// Group consecutive eigenvalues (descending, scaled) whose gap is below tol.
__global__ void group_kernel(EigState st, int nvec, int* grp_start, int* ngrp) {
  if (threadIdx.x != 0) return;
  const double tol = 0x1p-10;  // |T| <= 1: gaps below ~1e-3 |T| are re-orthogonalised (as in LAPACK stein)
  int g = 0;
  grp_start[0] = 0;
  for (int j = 1; j < nvec; ++j) {
    if (st.lam[j - 1] - st.lam[j] > tol) grp_start[++g] = j;
  }
  grp_start[++g] = nvec;
  *ngrp = g;
}

// 32-way multisection: one warp per eigenvalue (j-th largest, j < K), each
// lane evaluates a Sturm count at one of 32 interior points per round, so a
// round narrows the bracket 33-fold (5 bits).  One warp per CTA spreads the
// FP64 work over many SMs.
// Multisection: kMsThreads Sturm counts per round at equally spaced points of
// the current bracket of eigenvalue j (descending order), one CTA per
// eigenvalue; every thread derives the new bracket from the same ballots.
constexpr int kMsThreads = 64;
__global__ void __launch_bounds__(kMsThreads) msect_kernel(EigState st, int K) {
  const int j = blockIdx.x;
  if (j >= K) return;
  const int n = st.n;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  extern __shared__ double smd[];
  __shared__ unsigned masks[kMsThreads / 32];
  double* d = smd;
  double* e2 = smd + n;
  for (int i = tid; i < n; i += kMsThreads) {
    d[i] = st.d[i];
    // floor 2^-120 on e^2 (changes eigenvalues by <= 2^-60): bounds the decay of the recurrence
    e2[i] = (i < n - 1) ? fmax(st.e[i] * st.e[i], 0x1p-120) : 0.0;
  }
  __syncthreads();
  const int m = n - 1 - j;
  const double inv = 1.0 / (double)(kMsThreads + 1);
  double lo = -1.0, hi = 1.0;  // Gershgorin radius < 1 after scaling
  for (int round = 0; round < 16; ++round) {
    const double p = lo + (hi - lo) * (double)(tid + 1) * inv;
    const int c = sturm_count(d, e2, n, p);
    const unsigned above = __ballot_sync(0xffffffffu, c > m);
    if (lane == 0) masks[warp] = above;
    __syncthreads();
    int f = kMsThreads;  // first point above eigenvalue j
    for (int w = 0; w < kMsThreads / 32; ++w)
      if (masks[w]) { f = 32 * w + __ffs(masks[w]) - 1; break; }
    const double nlo = (f == 0) ? lo : lo + (hi - lo) * (double)f * inv;
    const double nhi = (f == kMsThreads) ? hi : lo + (hi - lo) * (double)(f + 1) * inv;
    lo = nlo;
    hi = nhi;
    __syncthreads();
    // stop at (about) one ulp: adjacent doubles satisfy the relative test
    if (hi - lo <= 0x1p-52 * fmax(fabs(lo), fabs(hi)) + 0x1p-60) break;
  }
  if (tid == 0) st.lam[j] = 0.5 * (lo + hi);
}

__device__ __forceinline__ double hash_start(uint32_t a, uint32_t b) {
  uint32_t h = a * 0x9E3779B1u ^ (b + 0x7F4A7C15u) * 0x85EBCA77u;
  h ^= h >> 15;
  h *= 0x2C1B3C6Du;
  h ^= h >> 12;
  h *= 0x297A2D39u;
  h ^= h >> 15;
  return (0.5 + (double)(h >> 8) * (1.0 / 16777216.0)) * ((b & 1u) ? 1.0 : -1.0);
}

// Inverse iteration for every requested eigenvalue in parallel (one thread per
// vector, one vector per CTA to spread the FP64 recurrences over the SMs);
// deterministic pseudo-random start vectors, three solves.  The LU factors and
// the iterate live in shared memory: the recurrences are sequential, so every
// access sits on the critical path.  Close eigenvalues are re-orthogonalised
// afterwards (CholQR2 per group, block Gram-Schmidt for large groups).
__global__ void __launch_bounds__(32) invit_par_kernel(EigState st, int nvec) {
  extern __shared__ double smi[];
  const int j = blockIdx.x;
  if (j >= nvec) return;
  const int n = st.n;
  double* fl = smi;
  double* fd = fl + n;
  double* fu = fd + n;
  double* fu2 = fu + n;
  double* fp = fu2 + n;
  double* x = fp + n;
  const double lam = st.lam[j];
  for (int i = threadIdx.x; i < n; i += 32) {
    fd[i] = st.d[i] - lam;
    fl[i] = (i < n - 1) ? st.e[i] : 0.0;
    fu[i] = (i < n - 1) ? st.e[i] : 0.0;
    fu2[i] = 0.0;
    fp[i] = 0.0;
    x[i] = hash_start((uint32_t)j, (uint32_t)i);
  }
  __syncwarp();
  if (threadIdx.x == 0) {
    const double eps_piv = 0x1p-52;
    for (int i = 0; i < n - 1; ++i) {
      if (fabs(fd[i]) >= fabs(fl[i])) {
        double piv = fd[i];
        if (fabs(piv) < eps_piv) { piv = (piv < 0.0) ? -eps_piv : eps_piv; fd[i] = piv; }
        const double l = fl[i] / piv;
        fl[i] = l;
        fd[i + 1] -= l * fu[i];
      } else {
        const double l = fd[i] / fl[i];
        fd[i] = fl[i];
        fl[i] = l;
        const double t = fu[i];
        fu[i] = fd[i + 1];
        fd[i + 1] = t - l * fd[i + 1];
        if (i < n - 2) { fu2[i] = fu[i + 1]; fu[i + 1] = -l * fu[i + 1]; }
        fp[i] = 1.0;
      }
    }
  }
  __syncwarp();
  // pivot clamp and reciprocals: independent per entry, done by the whole warp
  for (int i = threadIdx.x; i < n; i += 32) {
    double v = fd[i];
    if (fabs(v) < 0x1p-52) v = (v < 0.0) ? -0x1p-52 : 0x1p-52;
    fd[i] = 1.0 / v;
    if (i + 2 >= n) fu2[i] = 0.0;
  }
  __syncwarp();
  for (int it = 0; it < 3; ++it) {
    if (threadIdx.x == 0) {
      for (int i = 0; i < n - 1; ++i) {
        if (fp[i] != 0.0) { const double t = x[i]; x[i] = x[i + 1]; x[i + 1] = t; }
        x[i + 1] -= fl[i] * x[i];
      }
      for (int i = n - 1; i >= 0; --i) {
        double v = x[i];
        if (i + 1 < n) v -= fu[i] * x[i + 1];
        if (i + 2 < n) v -= fu2[i] * x[i + 2];
        x[i] = v * fd[i];
      }
    }
    __syncwarp();
    double mx = 0.0;
    for (int i = threadIdx.x; i < n; i += 32) mx = fmax(mx, fabs(x[i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    const double inv = (mx > 0.0) ? 1.0 / mx : 1.0;
    for (int i = threadIdx.x; i < n; i += 32) x[i] *= inv;
    __syncwarp();
  }
  double* xo = st.z + (int64_t)j * n;
  for (int i = threadIdx.x; i < n; i += 32) xo[i] = x[i];
}

// Orthonormalisation of every group of close eigenvalues by CholQR2: the
// vectors of inverse iteration are already nearly orthonormal (well
// conditioned), so two passes of  W = Z^T Z,  W = R^T R,  Z <- Z R^-1
// reach orthonormality to rounding level, with parallel dot products instead
// of a chain of Gram-Schmidt reductions.  One CTA per group of at most
// kQrMax vectors; larger groups are cut into blocks of kQrMax that are
// orthonormalised in turn (block classical Gram-Schmidt, two passes, against
// the earlier blocks, then CholQR2 inside the block across the GPU).
constexpr int kQrMax = 48;
// CholQR2 of the g <= kQrMax vectors Z + c * n (c < g), one CTA.
__device__ void cholqr_block(double* __restrict__ Z, int g, int n, double* __restrict__ W) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  for (int pass = 0; pass < 2; ++pass) {
    // W = Z^T Z (upper triangle), a warp per entry
    for (int e = warp; e < g * g; e += nw) {
      const int a = e / g, c = e % g;
      if (c < a) continue;
      const double* za = Z + (int64_t)a * n;
      const double* zc = Z + (int64_t)c * n;
      double part = 0.0;
      for (int i = lane; i < n; i += 32) part = fma(za[i], zc[i], part);
      part = warp_sum(part);
      if (lane == 0) { W[a * kQrMax + c] = part; W[c * kQrMax + a] = part; }
    }
    __syncthreads();
    // Cholesky W = R^T R (R upper, stored in the upper triangle of W); one warp
    if (warp == 0) {
      for (int k = 0; k < g; ++k) {
        const double dkk = sqrt(fmax(W[k * kQrMax + k], 1e-300));
        const double inv = 1.0 / dkk;
        __syncwarp();
        for (int c = k + 1 + lane; c < g; c += 32) W[k * kQrMax + c] *= inv;
        if (lane == 0) W[k * kQrMax + k] = dkk;
        __syncwarp();
        for (int e = lane; e < (g - k - 1) * (g - k - 1); e += 32) {
          const int a = k + 1 + e / (g - k - 1), c = k + 1 + e % (g - k - 1);
          if (c >= a) W[a * kQrMax + c] -= W[k * kQrMax + a] * W[k * kQrMax + c];
        }
        __syncwarp();
      }
    }
    __syncthreads();
    // Z <- Z R^-1, a thread per row: forward substitution y R = z
    for (int i = tid; i < n; i += blockDim.x) {
      double y[kQrMax];
      for (int c = 0; c < g; ++c) {
        double v = Z[(int64_t)c * n + i];
        for (int a = 0; a < c; ++a) v -= y[a] * W[a * kQrMax + c];
        y[c] = v / W[c * kQrMax + c];
      }
      for (int c = 0; c < g; ++c) Z[(int64_t)c * n + i] = y[c];
    }
    __syncthreads();
  }
}

// One CTA per group of at most gmax vectors.
__global__ void __launch_bounds__(256) cholqr_group_kernel(EigState st, const int* __restrict__ grp_start,
                                                           const int* __restrict__ ngrp, int gmax) {
  __shared__ double W[kQrMax * kQrMax];
  if ((int)blockIdx.x >= *ngrp) return;
  const int g0 = grp_start[blockIdx.x], g1 = grp_start[blockIdx.x + 1];
  const int g = g1 - g0;
  if (g > gmax) return;
  cholqr_block(st.z + (int64_t)g0 * st.n, g, st.n, W);
}


// The same CholQR2 of one block of a large group spread over the GPU (the
// block Gram-Schmidt of a large cluster runs its blocks in turn, so a one-CTA
// block leaves the other SMs idle through a long FP64 chain): W = Z^T Z by
// blk_dot_kernel (a warp per entry), the Cholesky factor by one CTA
// (cholqr_chol_kernel), Z <- Z R^-1 a warp per row (cholqr_trsm_kernel).
// Every value is formed as in cholqr_block, in the same order.
constexpr int kCholThreads = 256;
__global__ void __launch_bounds__(kCholThreads) cholqr_chol_kernel(const double* __restrict__ Wg, int g,
                                                                  double* __restrict__ Rg) {
  // right-looking: every entry takes its updates in the order k = 0, 1, ...
  // with the same expressions as cholqr_block (the threads of the CTA share
  // the trailing update of each step)
  __shared__ double W[kQrMax * kQrMax];
  const int tid = threadIdx.x;
  for (int e = tid; e < g * g; e += kCholThreads) W[(e / g) * kQrMax + (e % g)] = Wg[e];
  __syncthreads();
  for (int k = 0; k < g; ++k) {
    const double dkk = sqrt(fmax(W[k * kQrMax + k], 1e-300));
    const double inv = 1.0 / dkk;
    __syncthreads();
    for (int c = k + 1 + tid; c < g; c += kCholThreads) W[k * kQrMax + c] *= inv;
    if (tid == 0) W[k * kQrMax + k] = dkk;
    __syncthreads();
    const int m = g - k - 1;
    for (int e = tid; e < m * m; e += kCholThreads) {
      const int a = k + 1 + e / m, c = k + 1 + e % m;
      if (c >= a) W[a * kQrMax + c] -= W[k * kQrMax + a] * W[k * kQrMax + c];
    }
    __syncthreads();
  }
  for (int e = tid; e < kQrMax * kQrMax; e += kCholThreads) Rg[e] = W[e];
}
constexpr int kTrsmWarps = 8;  // rows per CTA: a warp per row, a lane per column (two when g > 32)
__global__ void __launch_bounds__(32 * kTrsmWarps) cholqr_trsm_kernel(double* __restrict__ Z, int g, int n,
                                                                       const double* __restrict__ Rg) {
  __shared__ double R[kQrMax * kQrMax];
  // the upper triangle of the g x g factor is all the solve reads
  for (int e = threadIdx.x; e < g * g; e += blockDim.x) {
    const int c = e / g, d = e - c * g;
    if (d >= c) R[c * kQrMax + d] = Rg[c * kQrMax + d];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * kTrsmWarps + (threadIdx.x >> 5);
  if (i >= n) return;
  // forward substitution y R = z for row i, right-looking: pivot c divides
  // y_c (its lane), broadcasts it, and every later y_d takes its term; for each
  // y_d the terms are subtracted in the order c = 0, 1, ..., as in cholqr_block
  const int d0 = lane, d1 = lane + 32;
  double y0 = (d0 < g) ? Z[(int64_t)d0 * n + i] : 0.0;
  double y1 = (d1 < g) ? Z[(int64_t)d1 * n + i] : 0.0;
  for (int c = 0; c < g; ++c) {
    const bool lo = c < 32;
    if (lane == (c & 31)) {
      if (lo) y0 = y0 / R[c * kQrMax + c];
      else y1 = y1 / R[c * kQrMax + c];
    }
    const double yc = __shfl_sync(0xffffffffu, lo ? y0 : y1, c & 31);
    if (d0 > c && d0 < g) y0 -= yc * R[c * kQrMax + d0];
    if (d1 > c && d1 < g) y1 -= yc * R[c * kQrMax + d1];
  }
  if (d0 < g) Z[(int64_t)d0 * n + i] = y0;
  if (d1 < g) Z[(int64_t)d1 * n + i] = y1;
}

// Block Gram-Schmidt step against the earlier vectors g0 .. g0+np-1 of a group:
// W[p][b] = <z_{g0+p}, z_{k0+b}> (a warp per entry, FP64) ...
__global__ void __launch_bounds__(256) blk_dot_kernel(const double* __restrict__ z, int n, int g0, int np, int k0,
                                                      int nb, double* __restrict__ W) {
  const int lane = threadIdx.x & 31;
  const int e = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (e >= np * nb) return;
  const int p = e / nb, b = e - p * nb;
  const double* zp = z + (int64_t)(g0 + p) * n;
  const double* zb = z + (int64_t)(k0 + b) * n;
  double part = 0.0;
  for (int i = lane; i < n; i += 32) part = fma(zp[i], zb[i], part);
  part = warp_sum(part);
  if (lane == 0) W[e] = part;
}
// ... then z_{k0+b} -= sum_p z_{g0+p} W[p][b] (a thread per entry of the block).
__global__ void __launch_bounds__(256) blk_update_kernel(double* __restrict__ z, int n, int g0, int np, int k0,
                                                         int nb, const double* __restrict__ W) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)nb * n) return;
  const int b = (int)(idx / n), i = (int)(idx - (int64_t)b * n);
  double acc = z[(int64_t)(k0 + b) * n + i];
  for (int p = 0; p < np; ++p) acc = fma(-z[(int64_t)(g0 + p) * n + i], W[p * nb + b], acc);
  z[(int64_t)(k0 + b) * n + i] = acc;
}

__global__ void trace_g_kernel(const double* __restrict__ G, int n, double* __restrict__ out) {
  __shared__ double red[32];
  double a = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) a += G[(int64_t)i * n + i];
  const double t = block_sum(a, red);
  if (threadIdx.x == 0) *out = t;
}

// Rank choice: clamp at 0, tail sums from the smallest value, smallest r >= 1
// with t[r] <= budget (Section 4.1.3).
__global__ void rank_kernel(const double* __restrict__ lam, int n, double budget, int* r_out, double* disc_out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double acc = 0.0;
  int r = n;
  double disc = 0.0;
  // t[r] for r = n .. 1: t[n] = 0
  if (0.0 <= budget) { r = n; disc = 0.0; }
  for (int j = n - 1; j >= 1; --j) {
    acc += fmax(lam[j], 0.0);  // acc = t[j]
    if (acc <= budget) { r = j; disc = acc; }
    else break;  // t[j] is non-increasing in j: once over budget, smaller r are too
  }
  *r_out = r;
  *disc_out = disc;
}

// ===================================================== double-float (FP32 pairs): dd.cuh
__device__ __forceinline__ dd dd_shfl_xor(dd a, int o) {
  return dd{__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o)};
}
__device__ __forceinline__ dd dd_warp_sum(dd a) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) a = dd_add(a, dd_shfl_xor(a, o));
  return a;
}
// CTA sum identical in every thread (warp sums, then warp 0 over the partials)
__device__ __forceinline__ dd dd_block_reduce(dd v, dd* red, bool warp_active) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (warp_active) v = dd_warp_sum(v);
  if (lane == 0) red[warp] = warp_active ? v : dd{0.f, 0.f};
  __syncthreads();
  if (warp == 0) {
    dd t = (lane < nw) ? red[lane] : dd{0.f, 0.f};
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) t = dd_add(t, dd_shfl_xor(t, o));
    if (lane == 0) red[16] = t;
  }
  __syncthreads();
  return red[16];
}

// Householder tridiagonalisation in double-float on one cluster (the
// iteration of tridiag_cluster_kernel).  G is scaled by 2^-sh (diag max ->
// [0.5, 1)) on load; d and e are written back unscaled in FP64, the reflectors
// as float pairs (row s of hv holds v_s).
template <int NPER>
__global__ void __launch_bounds__(kTriCThreads) tridiag_cluster_dd_kernel(EigState st, const double* __restrict__ g) {
  extern __shared__ dd smdd[];
  __shared__ double s_scale[2];
  cg::cluster_group cl = cg::this_cluster();
  const int n = st.n;
  const int C = (int)cl.num_blocks(), b = (int)cl.block_rank();
  const int rows = (n + C - 1) / C;
  dd* vprev = smdd;
  dd* vcur = smdd + n;
  dd* wv = smdd + 2 * n;
  dd* red1 = smdd + 3 * n;  // 17 used
  dd* red2 = red1 + 24;
  dd* sx = red2 + 24;
  dd* pfull = sx + 16;      // [2][n]
  dd* A = pfull + 2 * n;    // [rows][n]
  dd* hvo = reinterpret_cast<dd*>(st.hv);
  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
  // power-of-two scale from the largest diagonal entry (G is PSD: it bounds |G|)
  if (warp == 0) {
    double m = 0.0;
    for (int i = lane; i < n; i += 32) m = fmax(m, fabs(g[(int64_t)i * n + i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) {
      int ex = 0;
      if (m > 0.0) frexp(m, &ex);
      s_scale[0] = ldexp(1.0, -ex);
      s_scale[1] = ldexp(1.0, ex);
    }
  }
  __syncthreads();
  const double sc = s_scale[0], usc = s_scale[1];
  for (int li = 0; li < rows; ++li) {
    const int i = li * C + b;
    for (int j = tid; j < n; j += blockDim.x)
      A[(int64_t)li * n + j] = (i < n) ? dd_from(g[(int64_t)i * n + j] * sc) : dd{0.f, 0.f};
  }
  for (int i = tid; i < n; i += blockDim.x) {
    vprev[i] = dd{0.f, 0.f}; vcur[i] = dd{0.f, 0.f}; wv[i] = dd{0.f, 0.f};
    pfull[i] = dd{0.f, 0.f}; pfull[n + i] = dd{0.f, 0.f};
  }
  dd tau_prev = dd{0.f, 0.f};
  const dd zero = dd{0.f, 0.f};
  cl.sync();
  for (int s = 0; s <= n - 2; ++s) {
    const int j = s + tid;
    const bool has = j < n;
    const bool wact = s + (tid & ~31) < n;
    dd pj = zero, ps = zero, K = zero;
    const dd vj = has ? vprev[j] : zero, vs = vprev[s];
    if (s >= 1) {
      const dd* pb = pfull + ((s - 1) & 1) * n;
      if (has) pj = pb[j];
      ps = pb[s];
      const dd dot = dd_block_reduce(has ? dd_mul(pj, vj) : zero, red1, wact);
      K = dd_mul(dd_mul(ddf(0.5f), tau_prev), dot);
    }
    const dd wj = dd_sub(pj, dd_mul(K, vj)), ws = dd_sub(ps, dd_mul(K, vs));
    dd rowj = zero;
    if (has) {
      const dd a = *cl.map_shared_rank(A + (int64_t)(s / C) * n + j, s % C);
      rowj = dd_sub(dd_sub(a, dd_mul(vs, wj)), dd_mul(ws, vj));
    }
    if (s <= n - 3) {
      if (tid == 1) sx[0] = rowj;
      if (tid == 0) sx[1] = rowj;
      const dd sig2 = dd_block_reduce((j >= s + 2 && has) ? dd_mul(rowj, rowj) : zero, red2, wact);
      const dd x0 = sx[0], ds = sx[1];
      dd alpha, tau, scal;
      if (sig2.hi == 0.f) {
        tau = zero; alpha = x0; scal = zero;
      } else {
        const dd nrm = dd_sqrt(dd_add(dd_mul(x0, x0), sig2));
        alpha = dd_neg_sign(x0) ? nrm : dd_neg(nrm);
        tau = dd_div(dd_sub(alpha, x0), alpha);
        scal = dd_div(ddf(1.0f), dd_sub(x0, alpha));
      }
      if (has) {
        wv[j] = wj;
        vcur[j] = (j == s + 1) ? ddf(1.0f) : ((j > s + 1) ? dd_mul(rowj, scal) : zero);
      }
      __syncthreads();
      if (b == 0) {
        for (int q = tid; q < n; q += blockDim.x) hvo[(int64_t)s * n + q] = (q > s) ? vcur[q] : zero;
        if (tid == 0) { st.d[s] = dd_to(ds) * usc; st.e[s] = dd_to(alpha) * usc; st.tau[s] = dd_to(tau); }
      }
      dd vp[NPER], wq[NPER], vc[NPER];
#pragma unroll
      for (int q = 0; q < NPER; ++q) {
        const int jj = s + 1 + lane + 32 * q;
        const bool ok = jj < n;
        vp[q] = ok ? vprev[jj] : zero;
        wq[q] = ok ? wv[jj] : zero;
        vc[q] = ok ? vcur[jj] : zero;
      }
      dd* pout = pfull + (s & 1) * n;
      const int li0 = (s + 1 - b + C - 1) / C;
      for (int li = li0 + warp; li < rows; li += nwarp) {
        const int i = li * C + b;
        if (i >= n) break;
        const dd vi = vprev[i], wi = wv[i];
        dd* arow = A + (int64_t)li * n + s + 1 + lane;
        dd a[NPER];
#pragma unroll
        for (int q = 0; q < NPER; ++q) a[q] = (s + 1 + lane + 32 * q < n) ? arow[32 * q] : zero;
#pragma unroll
        for (int q = 0; q < NPER; ++q) {
          a[q] = dd_sub(dd_sub(a[q], dd_mul(vi, wq[q])), dd_mul(wi, vp[q]));
          if (s + 1 + lane + 32 * q < n) arow[32 * q] = a[q];
          a[q] = dd_mul(a[q], vc[q]);
        }
#pragma unroll
        for (int w = 1; w < NPER; w <<= 1)
#pragma unroll
          for (int q = 0; q + w < NPER; q += 2 * w) a[q] = dd_add(a[q], a[q + w]);
        const dd acc = dd_mul(tau, dd_warp_sum(a[0]));
        if (lane < C) *cl.map_shared_rank(pout + i, lane) = acc;
      }
      cl.sync();
      dd* t = vprev;
      vprev = vcur;
      vcur = t;
      tau_prev = tau;
    } else {
      if (b == 0 && tid == 0) { st.d[s] = dd_to(rowj) * usc; st.tau[s] = 0.0; }
      if (b == 0 && tid == 1) {
        st.e[s] = dd_to(rowj) * usc;
        const dd a11 = *cl.map_shared_rank(A + (int64_t)((n - 1) / C) * n + (n - 1), (n - 1) % C);
        st.d[n - 1] = dd_to(dd_sub(a11, dd_mul(ddf(2.0f), dd_mul(vj, wj)))) * usc;
      }
    }
  }
  cl.sync();
}

// Sturm count in double-float with the LDL^T recurrence
// q_i = (d_i - sigma) - e_{i-1}^2 / q_{i-1}, |q| floored at pivmin (as in
// bisection codes of LAPACK's dstebz); T scaled to |entries| < 1.
__device__ int sturm_count_dd(const dd* __restrict__ d, const dd* __restrict__ e2, int n, dd sigma) {
  const float pivmin = 0x1p-90f;
  dd q = dd_sub(d[0], sigma);
  if (fabsf(q.hi) < pivmin) q = dd{-pivmin, 0.f};
  int cnt = dd_neg_sign(q);
  for (int i = 1; i < n; ++i) {
    q = dd_sub(dd_sub(d[i], sigma), dd_div(e2[i - 1], q));
    if (fabsf(q.hi) < pivmin) q = dd{-pivmin, 0.f};
    cnt += dd_neg_sign(q);
  }
  return cnt;
}

__global__ void __launch_bounds__(kMsThreads) msect_dd_kernel(EigState st, int K) {
  const int j = blockIdx.x;
  if (j >= K) return;
  const int n = st.n;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  extern __shared__ dd smm[];
  __shared__ unsigned masks[kMsThreads / 32];
  dd* d = smm;
  dd* e2 = smm + n;
  for (int i = tid; i < n; i += kMsThreads) {
    d[i] = dd_from(st.d[i]);
    e2[i] = (i < n - 1) ? dd_from(st.e[i] * st.e[i]) : dd{0.f, 0.f};
  }
  __syncthreads();
  const int m = n - 1 - j;
  const double inv = 1.0 / (double)(kMsThreads + 1);
  double lo = -1.0, hi = 1.0;  // Gershgorin radius < 1 after scaling
  // round 0 is geometric: points 0 and 2^-62 .. 2^0 (increasing), so that the
  // bracket of a small eigenvalue (T comes from a PSD Gram matrix) is within a
  // factor two after one round; later rounds are linear
  for (int round = 0; round < 16; ++round) {
    const double p = (round == 0) ? ((tid == 0) ? 0.0 : ldexp(1.0, tid - (kMsThreads - 1)))
                                  : lo + (hi - lo) * (double)(tid + 1) * inv;
    const int c = sturm_count_dd(d, e2, n, dd_from(p));
    const unsigned above = __ballot_sync(0xffffffffu, c > m);
    if (lane == 0) masks[warp] = above;
    __syncthreads();
    int f = kMsThreads;
    for (int w = 0; w < kMsThreads / 32; ++w)
      if (masks[w]) { f = 32 * w + __ffs(masks[w]) - 1; break; }
    double nlo, nhi;
    if (round == 0) {
      // point t is 0 (t = 0) or 2^(t-63); kMsThreads points, the last is 1
      auto pt = [&](int t) { return (t == 0) ? 0.0 : ldexp(1.0, t - (kMsThreads - 1)); };
      nlo = (f == 0) ? lo : pt(f - 1);
      nhi = (f == kMsThreads) ? hi : pt(f);
    } else {
      nlo = (f == 0) ? lo : lo + (hi - lo) * (double)f * inv;
      nhi = (f == kMsThreads) ? hi : lo + (hi - lo) * (double)(f + 1) * inv;
    }
    lo = nlo;
    hi = nhi;
    __syncthreads();
    // the split paths use these values for inverse-iteration shifts and a
    // provisional rank only (ranks are certified from residuals): 2^-30
    // relative (or 2^-70 absolute) is ample
    if (hi - lo <= 0x1p-30 * fmax(fabs(lo), fabs(hi)) + 0x1p-70) break;
  }
  if (tid == 0) st.lam[j] = 0.5 * (lo + hi);
}

// Inverse iteration in double-float (the iteration of invit_par_kernel).
__global__ void __launch_bounds__(32) invit_dd_kernel(EigState st, int nvec) {
  extern __shared__ dd smv[];
  const int j = blockIdx.x;
  if (j >= nvec) return;
  const int n = st.n;
  dd* fl = smv;
  dd* fd = fl + n;
  dd* fu = fd + n;
  dd* fu2 = fu + n;
  dd* x = fu2 + n;
  uint8_t* fp = reinterpret_cast<uint8_t*>(x + n);
  const dd lam = dd_from(st.lam[j]);
  const dd zero = dd{0.f, 0.f};
  for (int i = threadIdx.x; i < n; i += 32) {
    fd[i] = dd_sub(dd_from(st.d[i]), lam);
    fl[i] = (i < n - 1) ? dd_from(st.e[i]) : zero;
    fu[i] = fl[i];
    fu2[i] = zero;
    fp[i] = 0;
    x[i] = dd_from(hash_start((uint32_t)j, (uint32_t)i));
  }
  __syncwarp();
  const float eps_piv = 0x1p-46f;
  if (threadIdx.x == 0) {
    for (int i = 0; i < n - 1; ++i) {
      if (fabsf(fd[i].hi) >= fabsf(fl[i].hi)) {
        dd piv = fd[i];
        if (fabsf(piv.hi) < eps_piv) { piv = dd{piv.hi < 0.f ? -eps_piv : eps_piv, 0.f}; fd[i] = piv; }
        const dd l = dd_div(fl[i], piv);
        fl[i] = l;
        fd[i + 1] = dd_sub(fd[i + 1], dd_mul(l, fu[i]));
      } else {
        const dd l = dd_div(fd[i], fl[i]);
        fd[i] = fl[i];
        fl[i] = l;
        const dd t = fu[i];
        fu[i] = fd[i + 1];
        fd[i + 1] = dd_sub(t, dd_mul(l, fd[i + 1]));
        if (i < n - 2) { fu2[i] = fu[i + 1]; fu[i + 1] = dd_neg(dd_mul(l, fu[i + 1])); }
        fp[i] = 1;
      }
    }
  }
  __syncwarp();
  for (int i = threadIdx.x; i < n; i += 32) {
    dd v = fd[i];
    if (fabsf(v.hi) < eps_piv) v = dd{v.hi < 0.f ? -eps_piv : eps_piv, 0.f};
    fd[i] = dd_div(ddf(1.0f), v);
    if (i + 2 >= n) fu2[i] = zero;
  }
  __syncwarp();
  // two solves: the shifts come from multisection to ~2^-44 relative
  for (int it = 0; it < 2; ++it) {
    if (threadIdx.x == 0) {
      for (int i = 0; i < n - 1; ++i) {
        if (fp[i]) { const dd t = x[i]; x[i] = x[i + 1]; x[i + 1] = t; }
        x[i + 1] = dd_sub(x[i + 1], dd_mul(fl[i], x[i]));
      }
      for (int i = n - 1; i >= 0; --i) {
        dd v = x[i];
        if (i + 1 < n) v = dd_sub(v, dd_mul(fu[i], x[i + 1]));
        if (i + 2 < n) v = dd_sub(v, dd_mul(fu2[i], x[i + 2]));
        x[i] = dd_mul(v, fd[i]);
      }
    }
    __syncwarp();
    float mx = 0.f;
    for (int i = threadIdx.x; i < n; i += 32) mx = fmaxf(mx, fabsf(x[i].hi));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    // scale by a power of two near 1/max (exact)
    int ex = 0;
    if (mx > 0.f) frexpf(mx, &ex);
    const float sc = ldexpf(1.0f, -ex);
    for (int i = threadIdx.x; i < n; i += 32) x[i] = dd{x[i].hi * sc, x[i].lo * sc};
    __syncwarp();
  }
  double* xo = st.z + (int64_t)j * n;
  for (int i = threadIdx.x; i < n; i += 32) xo[i] = dd_to(x[i]);
}

// Back-transformation X = Q Z with the double-float reflectors of
// tridiag_cluster_dd_kernel (a warp per column; next reflector prefetched).
template <int NPER>
__global__ void backtransform_dd_kernel(EigState st, int nvec, double* __restrict__ v) {
  const int n = st.n;
  const int lane = threadIdx.x & 31;
  const int col = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (col >= nvec) return;
  const dd* hvd = reinterpret_cast<const dd*>(st.hv);
  const dd zero = dd{0.f, 0.f};
  dd z[NPER], h[NPER];
  const double* zc = st.z + (int64_t)col * n;
#pragma unroll
  for (int q = 0; q < NPER; ++q) {
    const int i = lane + 32 * q;
    z[q] = (i < n) ? dd_from(zc[i]) : zero;
  }
  auto load_h = [&](int s) {
    const dd* hv = hvd + (int64_t)s * n;
#pragma unroll
    for (int q = 0; q < NPER; ++q) {
      const int i = lane + 32 * q;
      h[q] = (i > s && i < n) ? hv[i] : zero;
    }
  };
  if (n >= 3) load_h(n - 3);
  for (int s = n - 3; s >= 0; --s) {
    const dd t = dd_from(st.tau[s]);
    dd hc[NPER];
#pragma unroll
    for (int q = 0; q < NPER; ++q) hc[q] = h[q];
    if (s > 0) load_h(s - 1);
    if (t.hi == 0.f) continue;
    dd pr[NPER];
#pragma unroll
    for (int q = 0; q < NPER; ++q) pr[q] = dd_mul(hc[q], z[q]);
#pragma unroll
    for (int w = 1; w < NPER; w <<= 1)
#pragma unroll
      for (int q = 0; q + w < NPER; q += 2 * w) pr[q] = dd_add(pr[q], pr[q + w]);
    const dd dot = dd_mul(dd_warp_sum(pr[0]), t);
#pragma unroll
    for (int q = 0; q < NPER; ++q) z[q] = dd_sub(z[q], dd_mul(dot, hc[q]));
  }
  // sign: entry of largest magnitude (first on ties) positive; write FP64
  double zz[NPER];
#pragma unroll
  for (int q = 0; q < NPER; ++q) zz[q] = dd_to(z[q]);
  double best = -1.0;
  int bidx = n;
  double bval = 0.0;
#pragma unroll
  for (int q = 0; q < NPER; ++q) {
    const int i = lane + 32 * q;
    if (i < n) {
      const double a = fabs(zz[q]);
      if (a > best) { best = a; bidx = i; bval = zz[q]; }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double ob = __shfl_xor_sync(0xffffffffu, best, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bidx, o);
    const double ov = __shfl_xor_sync(0xffffffffu, bval, o);
    if (ob > best || (ob == best && oi < bidx)) { best = ob; bidx = oi; bval = ov; }
  }
  const double sg = (bval < 0.0) ? -1.0 : 1.0;
#pragma unroll
  for (int q = 0; q < NPER; ++q) {
    const int i = lane + 32 * q;
    if (i < n) v[(int64_t)i * nvec + col] = sg * zz[q];
  }
}

int setup_state(int n, int nvec_max) {
  EigState st;
  st.n = n;
  size_t nn = (size_t)n * n;
  ATC_TRY(Scratch::get(SLOT_EIG_A, sizeof(double) * nn, (void**)&st.a));
  ATC_TRY(Scratch::get(SLOT_EIG_V, sizeof(double) * nn, (void**)&st.hv));
  double* vec = nullptr;
  const size_t nv = (size_t)n * 8 + 64;
  ATC_TRY(Scratch::get(SLOT_EIG_VEC, sizeof(double) * nv + 4096, (void**)&vec));
  st.d = vec;
  st.e = vec + n;
  st.tau = vec + 2 * n;
  st.pbuf = vec + 3 * n;  // 2n
  st.lam = vec + 5 * n;
  st.scale = vec + 6 * n;
  st.flags = reinterpret_cast<int*>(vec + 6 * n + 8);
  st.z = nullptr;
  st.lu = nullptr;
  (void)nvec_max;
  g_state = st;
  return ATC_OK;
}

}  // namespace

constexpr int kClusterMaxN = 512;

size_t tri_cluster_smem(int n, int C) {
  const int rows = (n + C - 1) / C;
  return sizeof(double) * ((size_t)5 * n + 64 + (size_t)rows * n);
}

template <int NPER>
int tri_cluster_attr() {
  if (cudaFuncSetAttribute(tridiag_cluster_kernel<NPER>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024) !=
          cudaSuccess ||
      cudaFuncSetAttribute(tridiag_cluster_kernel<NPER>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
          cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return 1;
}

template <int NPER>
int tri_cluster_dd_attr() {
  if (cudaFuncSetAttribute(tridiag_cluster_dd_kernel<NPER>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024) !=
          cudaSuccess ||
      cudaFuncSetAttribute(tridiag_cluster_dd_kernel<NPER>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
          cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return 1;
}

// Cluster size of the shared-memory tridiagonalisation for this n (16 if the
// device schedules such clusters with this much shared memory, else 8), or 0.
int cluster_size_for(int n) {
  static int attr_ok = -1;
  static int last_n = -1, last_c = 0;
  if (n == last_n) return last_c;
  if (attr_ok < 0) attr_ok = tri_cluster_attr<8>() && tri_cluster_attr<16>() && tri_cluster_dd_attr<8>() &&
                              tri_cluster_dd_attr<16>();
  int found = 0;
  for (int C : {16, 8}) {
    if (!attr_ok) break;
    const size_t smem = tri_cluster_smem(n, C);
    if (smem > 200 * 1024) continue;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C);
    cfg.blockDim = dim3(kTriCThreads);  // the larger of the two launch shapes
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nclusters = 0;
    const cudaError_t oe = (n <= 256) ? cudaOccupancyMaxActiveClusters(&nclusters, tridiag_cluster_kernel<8>, &cfg)
                                      : cudaOccupancyMaxActiveClusters(&nclusters, tridiag_cluster_kernel<16>, &cfg);
    if (trace_enabled())
      fprintf(stderr, "[atc] tridiag cluster n=%d C=%d smem=%zu: %s, %d clusters\n", n, C, smem, cudaGetErrorString(oe),
              nclusters);
    if (oe == cudaSuccess && nclusters > 0) {
      found = C;
      break;
    }
    cudaGetLastError();
  }
  if (trace_enabled() && !attr_ok) fprintf(stderr, "[atc] tridiag cluster attributes rejected\n");
  last_n = n;
  last_c = found;
  return found;
}

int launch_eig_values_impl(const double* g, int n, cudaStream_t s, bool use_dd = false) {
  if (n < 1 || n > 1024) return fail(ATC_EUNSUP, "eigensolver supports 1 <= n <= 1024 (n = %d)", n);
  ATC_TRY(setup_state(n, n));
  EigState st = g_state;
  g_state_dd = use_dd && n >= 3 && n <= kClusterMaxN && cluster_size_for(n) > 0;
  ATC_CUDA_TRY(cudaMemcpyAsync(st.a, g, sizeof(double) * n * n, cudaMemcpyDeviceToDevice, s));
  ATC_CUDA_TRY(cudaMemsetAsync(st.flags, 0, 4 * sizeof(int), s));
  ATC_CUDA_TRY(cudaMemsetAsync(st.d, 0, sizeof(double) * 3 * n, s));
  if (n == 1) {
    tridiag_small_kernel<<<1, 32, 0, s>>>(st);
    ATC_LAUNCHED(1);
  } else if (n <= kClusterMaxN && cluster_size_for(n) > 0) {
    const int C = cluster_size_for(n);
    const int rows = (n + C - 1) / C;
    const size_t smem = tri_cluster_smem(n, C);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C);
    cfg.blockDim = dim3(n <= 256 ? 256 : kTriCThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (g_state_dd) {
      if (n <= 256)
        ATC_CUDA_TRY(cudaLaunchKernelEx(&cfg, tridiag_cluster_dd_kernel<8>, st, g));
      else
        ATC_CUDA_TRY(cudaLaunchKernelEx(&cfg, tridiag_cluster_dd_kernel<16>, st, g));
    } else if (n <= 256) {
      ATC_CUDA_TRY(cudaLaunchKernelEx(&cfg, tridiag_cluster_kernel<8>, st, g));
    } else {
      ATC_CUDA_TRY(cudaLaunchKernelEx(&cfg, tridiag_cluster_kernel<16>, st, g));
    }
    ATC_LAUNCHED(1);
  } else {
    static int max_blocks = -1;
    const size_t smem = sizeof(double) * (4 * n + 32);
    if (max_blocks < 0) {
      int dev = 0, nsm = 0, per = 0;
      ATC_CUDA_TRY(cudaGetDevice(&dev));
      ATC_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
      ATC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, tridiag_kernel, kTriThreads,
                                                                 sizeof(double) * (4 * 1024 + 32)));
      max_blocks = nsm * (per > 0 ? 1 : 0);
      if (max_blocks <= 0) return fail(ATC_ECUDA, "tridiagonalisation kernel cannot be resident");
    }
    // about 4 rows per CTA, at most one CTA per SM
    int P = (n + 3) / 4;
    if (P > max_blocks) P = max_blocks;
    if (P > 128) P = 128;
    if (P < 1) P = 1;
    void* args[] = {(void*)&st};
    {
      KTimed kt_(s, "tridiag_kernel");
      ATC_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)tridiag_kernel, dim3(P), dim3(kTriThreads), args, smem, s));
    }
    __atomic_add_fetch(&g_kernel_launches, 1, __ATOMIC_RELAXED);
  }
  scale_kernel<<<1, 256, 0, s>>>(st);
  ATC_LAUNCHED(1);
  return ATC_OK;
}

int launch_eig_more(int n, int K, double* lam, cudaStream_t s);

int launch_eig_values(const double* g, int n, double* lam, cudaStream_t s) {
  ATC_TRY(launch_eig_values_impl(g, n, s));
  ATC_TRY(launch_eig_more(n, n, lam, s));
  return ATC_OK;
}

// (Re)compute the K largest eigenvalues of the current tridiagonal matrix
// (FP64 multisection) into lam[0..K) (unscaled).
int launch_eig_more(int n, int K, double* lam, cudaStream_t s) {
  if (g_state.n != n) return fail(ATC_EINVAL, "eigenvalues requested without a tridiagonal matrix");
  if (K > n) K = n;
  EigState st = g_state;
  {
    KTimed kt_(s, "msect_kernel");
    if (g_state_dd) msect_dd_kernel<<<K, kMsThreads, sizeof(dd) * 2 * n, s>>>(st, K);
    else msect_kernel<<<K, kMsThreads, sizeof(double) * 2 * n, s>>>(st, K);
  }
  ATC_LAUNCHED(1);
  if (lam) {
    unscale_kernel<<<(K + 255) / 256, 256, 0, s>>>(st, lam, K);
    ATC_LAUNCHED(1);
  }
  return ATC_OK;
}

// Tridiagonalise G and return trace(G) (device scalar *trace_dev).
int launch_eig_tridiag(const double* g, int n, double* trace_dev, cudaStream_t s, bool use_dd) {
  ATC_TRY(launch_eig_values_impl(g, n, s, use_dd));
  trace_g_kernel<<<1, 256, 0, s>>>(g, n, trace_dev);
  ATC_LAUNCHED(1);
  return ATC_OK;
}

int launch_eig_vectors(int n, int nvec, double* v, cudaStream_t s) {
  if (nvec <= 0) return ATC_OK;
  if (g_state.n != n) return fail(ATC_EINVAL, "eigenvectors requested without matching eigenvalues");
  EigState st = g_state;
  const size_t zlen = (size_t)n * nvec * 6 + 2 * (size_t)nvec + 64;
  ATC_TRY(Scratch::get(SLOT_EIG_Z, sizeof(double) * (zlen + 2 * kQrMax * kQrMax), (void**)&st.z));
  st.lu = st.z + (size_t)n * nvec;
  int* grp = reinterpret_cast<int*>(st.lu + (size_t)5 * n * nvec);
  int* ngrp = grp + nvec + 2;
  group_kernel<<<1, 32, 0, s>>>(st, nvec, grp, ngrp);
  ATC_LAUNCHED(1);
  std::vector<int> hg((size_t)nvec + 2);
  ATC_CUDA_TRY(cudaMemcpyAsync(hg.data(), grp, sizeof(int) * (nvec + 2), cudaMemcpyDeviceToHost, s));
  {
    KTimed kt_(s, "invit_kernel");
    if (g_state_dd) invit_dd_kernel<<<nvec, 32, (sizeof(dd) * 5 + 1) * n, s>>>(st, nvec);
    else invit_par_kernel<<<nvec, 32, sizeof(double) * 6 * n, s>>>(st, nvec);
  }
  ATC_LAUNCHED(1);
  // CholQR2 for the groups of <= kQrMax vectors (one CTA each) ...
  { KTimed kt_(s, "cholqr_group_kernel"); cholqr_group_kernel<<<nvec, 256, 0, s>>>(st, grp, ngrp, kQrMax); }
  ATC_LAUNCHED(1);
  // ... and block Gram-Schmidt (two passes) + CholQR2 per block for the larger ones
  int hn = 0;
  ATC_CUDA_TRY(cudaMemcpyAsync(&hn, ngrp, sizeof(int), cudaMemcpyDeviceToHost, s));
  ATC_CUDA_TRY(cudaStreamSynchronize(s));
  double* W = st.lu;  // the LU scratch of inverse iteration is free again (stream order)
  double* Wq = st.z + zlen;  // CholQR Gram and factor of one block
  double* Rq = Wq + kQrMax * kQrMax;
  for (int q = 0; q < hn && q < nvec; ++q) {
    const int g0 = hg[q], g1 = hg[q + 1];
    if (g1 - g0 <= kQrMax) continue;
    for (int k0 = g0; k0 < g1; k0 += kQrMax) {
      const int nb = std::min(kQrMax, g1 - k0), np = k0 - g0;
      for (int pass = 0; pass < 2; ++pass) {
        if (np > 0) {
          { KTimed kt_(s, "blk_dot_kernel"); blk_dot_kernel<<<(np * nb + 7) / 8, 256, 0, s>>>(st.z, n, g0, np, k0, nb, W); }
          { KTimed kt_(s, "blk_update_kernel"); blk_update_kernel<<<(int)(((int64_t)nb * n + 255) / 256), 256, 0, s>>>(st.z, n, g0, np, k0, nb, W); }
          ATC_LAUNCHED(2);
        }
        // CholQR2 of the block across the GPU (two passes, as cholqr_block)
        for (int cq = 0; cq < 2; ++cq) {
          { KTimed kt_(s, "blk_dot_kernel"); blk_dot_kernel<<<(nb * nb + 7) / 8, 256, 0, s>>>(st.z, n, k0, nb, k0, nb, Wq); }
          { KTimed kt_(s, "cholqr_chol_kernel"); cholqr_chol_kernel<<<1, kCholThreads, 0, s>>>(Wq, nb, Rq); }
          {
            KTimed kt_(s, "cholqr_trsm_kernel");
            cholqr_trsm_kernel<<<(n + kTrsmWarps - 1) / kTrsmWarps, 32 * kTrsmWarps, 0, s>>>(
                st.z + (int64_t)k0 * n, nb, n, Rq);
          }
          ATC_LAUNCHED(3);
        }
      }
    }
  }
  {
    KTimed kt_(s, "backtransform_kernel");
    if (g_state_dd) {
      if (n <= 256) backtransform_dd_kernel<8><<<nvec, 32, 0, s>>>(st, nvec, v);
      else backtransform_dd_kernel<16><<<nvec, 32, 0, s>>>(st, nvec, v);
    } else if (n <= 256) {
      backtransform_kernel<8><<<nvec, 32, 0, s>>>(st, nvec, v);
    } else if (n <= 512) {
      backtransform_kernel<16><<<nvec, 32, 0, s>>>(st, nvec, v);
    } else {
      backtransform_kernel<32><<<nvec, 32, 0, s>>>(st, nvec, v);
    }
  }
  ATC_LAUNCHED(1);
  return ATC_OK;
}

int launch_eig_sym(const double* g, int n, double* lam, double* v, int nvec, cudaStream_t s) {
  g_state.flags = nullptr;
  ATC_TRY(launch_eig_values(g, n, lam, s));
  ATC_TRY(launch_eig_vectors(n, nvec, v, s));
  return ATC_OK;
}

int launch_rank_select(const double* lam, int n, double budget, int* r_dev, double* disc_dev, cudaStream_t s) {
  rank_kernel<<<1, 32, 0, s>>>(lam, n, budget, r_dev, disc_dev);
  ATC_LAUNCHED(1);
  return ATC_OK;
}

int* eig_error_flag_dev() { return g_state.flags ? g_state.flags + 2 : nullptr; }

int eig_read_error(int* err) {
  *err = 0;
  if (!g_state.flags) return ATC_OK;  // the FP64 tridiagonalisation has not run on this device
  return cudaMemcpy(err, g_state.flags + 2, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess ? ATC_OK : ATC_ECUDA;
}

}  // namespace atc
