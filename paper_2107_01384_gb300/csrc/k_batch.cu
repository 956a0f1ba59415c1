// Batched ST-HOSVD: many small, unevenly shaped tensors in one persistent
// launch (Algorithm 1 for every tensor; Section 4.1 rank rule and mode order).
//
// A CTA takes whole tensors from an atomic queue (largest estimated cost
// first) and runs the full mode loop of each one on the SM, with the n x n
// working matrices in shared memory:
//
//   scale    X is read with a power-of-two scale so that max|x| lies in
//            [0.5, 1) (exact; undone on the eigenvalues and the core);
//   Gram     G = B_(m) B_(m)^T from float products made exact with an FMA
//            (p + e = a*b), summed as double-float (FP32 pairs) and flushed
//            into FP64 every kFlushEvery terms: FP64-class accuracy at FP32
//            pipe rates (FP64 issues at 1/64 of the FP32 rate on GB300);
//   eigen    cyclic Jacobi in double-float on the Gram matrix (round-robin
//            ordering: n/2 disjoint rotations per round, one CTA barrier per
//            round), eigenvectors accumulated in double-float;
//   rank     eigenvalues sorted descending and clamped at 0; tails
//            t[r] = sum_{j>=r} lambda_j in FP64 from the smallest upward; the
//            smallest r >= 1 with t[r] <= budget (static or adaptive rule);
//   project  Y = U^T ._m B in double-float, stored as FP32 for the next mode
//            (FP64 for the last mode: the core).
//
// The register tile of the Gram (TM x TM entries per thread) is chosen per
// mode length from a table that batch_tune() measures on the device.

#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "atc_internal.cuh"
#include "dd.cuh"

namespace atc {

namespace {

constexpr int kBThreads = 512;
constexpr int kBMaxN = 112;        // 16 n^2 bytes of shared memory (G and V in double-float)
constexpr int kBMaxD = 8;
constexpr int kGramKC = 64;        // staged columns per Gram chunk
constexpr int kFlushEvery = 128;   // double-float terms per FP64 flush
constexpr int kMaxSweeps = 40;
constexpr int kMaxPairs = kBMaxN / 2;
constexpr int kMaxBlocks = kMaxPairs * (kMaxPairs + 1) / 2;

}  // namespace

struct BatchTensor {
  int64_t nelem;
  int dims[kBMaxD];
  int order[kBMaxD];
  double eps;
  int64_t core_off;           // doubles into the core pool (capacity nelem)
  int64_t fac_off[kBMaxD];    // doubles into the factor pool (capacity n_k^2)
};

struct BatchOut {
  int ranks[kBMaxD];
  int sweeps[kBMaxD];
  double discarded[kBMaxD];
  double norm2;
  double sse_trunc;
  int status;                 // 0 ok, 1 NaN/Inf in the input, 2 Jacobi did not converge
  int rounds[kBMaxD];         // Jacobi rounds that rotated, per mode
  long long cycles[4];        // SM clocks in scale+Gram, Jacobi, rank+factor, projection
};

struct BatchArgs {
  const BatchTensor* t;
  BatchOut* out;
  const float* const* x;      // device table of input pointers
  const int* sched;           // processing order of the tensors (largest first)
  int count;
  int d;
  int* counter;               // work-queue head (zeroed before each launch)
  float* scratch;             // per CTA: two FP32 buffers of `half` floats
  int64_t half;
  double* core_pool;
  double* fac_pool;
  double rtmss;
  int adaptive;
  const int* tm_of_n;         // Gram register tile per mode length (0..kBMaxN)
};

// ------------------------------------------------------------ double-float
__device__ __forceinline__ void dd_acc_prod(float& hi, float& lo, float a, float b) {
  const float p = a * b;
  const float e = fmaf(a, b, -p);  // a*b = p + e exactly
  const float s = hi + p;
  const float bp = s - hi;
  const float err = (hi - (s - bp)) + (p - bp);  // hi + p = s + err exactly
  const float l = lo + (err + e);
  hi = s + l;
  lo = l - (hi - s);
}
// (hi, lo) += u * b, u double-float, b float
__device__ __forceinline__ void dd_acc_prod2(float& hi, float& lo, dd u, float b) {
  const float p = u.hi * b;
  float e = fmaf(u.hi, b, -p);
  e = fmaf(u.lo, b, e);
  const float s = hi + p;
  const float bp = s - hi;
  const float err = (hi - (s - bp)) + (p - bp);
  const float l = lo + (err + e);
  hi = s + l;
  lo = l - (hi - s);
}

// --------------------------------------------------------------- staging
// Chunk c of the K = L*R columns of the (L, n, R) view, staged as
// stage[kk * cs + i * rs] (kk < cnt, i < n).  For R >= kc a chunk is a run of
// kc consecutive columns inside one l; for R < kc it is max(1, kc / R) whole
// l-slices, copied in memory order (coalesced).
struct ChunkPlan {
  int64_t L, R;
  int n, kc;
  bool small_r;
  int64_t cpl;     // chunks per l (R >= kc)
  int64_t lc;      // l-slices per chunk (R < kc)
  int64_t nchunks;
};
__device__ __forceinline__ ChunkPlan chunk_plan(int64_t L, int n, int64_t R, int kc) {
  ChunkPlan p;
  p.L = L;
  p.R = R;
  p.n = n;
  p.kc = kc;
  p.small_r = R < kc;
  if (!p.small_r) {
    p.cpl = (R + kc - 1) / kc;
    p.lc = 1;
    p.nchunks = L * p.cpl;
  } else {
    p.cpl = 1;
    p.lc = kc / R;
    if (p.lc < 1) p.lc = 1;
    p.nchunks = (L + p.lc - 1) / p.lc;
  }
  return p;
}
// Stage chunk c; returns the number of columns staged.
__device__ __forceinline__ int stage_chunk(const ChunkPlan& p, int64_t c, const float* __restrict__ src, float scl,
                                           float* __restrict__ stage, int cs, int rs) {
  const int n = p.n;
  if (!p.small_r) {
    const int64_t l = c / p.cpl;
    const int64_t r0 = (c - l * p.cpl) * p.kc;
    const int cnt = (int)((p.R - r0 < p.kc) ? (p.R - r0) : (int64_t)p.kc);
    const float* base = src + (l * n) * p.R + r0;
    const int tot = n * p.kc;
    for (int e = threadIdx.x; e < tot; e += blockDim.x) {
      const int i = e / p.kc, kk = e - i * p.kc;
      const float v = (kk < cnt) ? __ldg(base + (int64_t)i * p.R + kk) * scl : 0.f;
      stage[kk * cs + i * rs] = v;
    }
    return cnt;
  }
  const int64_t l0 = c * p.lc;
  const int nl = (int)((p.L - l0 < p.lc) ? (p.L - l0) : p.lc);
  const int nr = n * (int)p.R;
  const int tot = nl * nr;
  const float* base = src + l0 * nr;
  for (int e = threadIdx.x; e < tot; e += blockDim.x) {
    const int lr = e / nr;
    const int rem = e - lr * nr;
    const int i = rem / (int)p.R;
    const int rho = rem - i * (int)p.R;
    stage[(lr * (int)p.R + rho) * cs + i * rs] = __ldg(base + e) * scl;
  }
  return nl * (int)p.R;
}

// ------------------------------------------------------------------- Gram
// Ad (n x n FP64, shared) = B_(m) B_(m)^T, full symmetric on return.
template <int TM>
__device__ void batch_gram(const float* __restrict__ src, float scl, int64_t L, int n, int64_t R,
                           double* __restrict__ Ad, float* __restrict__ stage) {
  const int T = (n + TM - 1) / TM;
  const int U = T * (T + 1) / 2;
  const int SP = T * TM;  // stage row stride (rows >= n stay zero)
  // k-split groups: as many as the CTA has threads for, at most 16, and as
  // many as their FP64 partials fit beside the stage in the second region
  int KS = (int)blockDim.x / U;
  const int room = (int)(((size_t)8 * kBMaxN * kBMaxN - (size_t)4 * (kGramKC * SP + 2)) / ((size_t)8 * U * TM * TM));
  if (KS > room) KS = room;
  if (KS > 16) KS = 16;
  if (KS < 1) KS = 1;
  const int tid = threadIdx.x;
  for (int e = tid; e < n * n; e += blockDim.x) Ad[e] = 0.0;
  for (int e = tid; e < kGramKC * SP; e += blockDim.x) stage[e] = 0.f;
  int ti = 0, tj = 0, ks = 0;
  const bool active = tid < U * KS;  // threads past the tile set only stage data
  if (active) {
    int u = tid % U;
    ks = tid / U;
    while (u >= T - ti) {
      u -= T - ti;
      ++ti;
    }
    tj = ti + u;
  }
  // k-split groups (KS > 1) keep FP64 partials per thread after the stage and
  // add them in group order at the end, so the result does not depend on timing
  double* part = reinterpret_cast<double*>(stage + ((kGramKC * SP + 1) & ~1));
  if (KS > 1)
    for (int e = tid; e < U * KS * TM * TM; e += blockDim.x) part[e] = 0.0;
  float hi[TM][TM], lo[TM][TM];
#pragma unroll
  for (int a = 0; a < TM; ++a)
#pragma unroll
    for (int b = 0; b < TM; ++b) hi[a][b] = lo[a][b] = 0.f;
  int nacc = 0;
  auto flush = [&]() {
#pragma unroll
    for (int a = 0; a < TM; ++a)
#pragma unroll
      for (int b = 0; b < TM; ++b) {
        const double v = (double)hi[a][b] + (double)lo[a][b];
        if (KS > 1) {
          part[tid * TM * TM + a * TM + b] += v;
        } else {
          const int i = ti * TM + a, j = tj * TM + b;
          if (i < n && j < n && i <= j) Ad[i * n + j] += v;
        }
        hi[a][b] = lo[a][b] = 0.f;
      }
    nacc = 0;
  };
  __syncthreads();
  const ChunkPlan cp = chunk_plan(L, n, R, kGramKC);
  for (int64_t c = 0; c < cp.nchunks; ++c) {
    const int cnt = stage_chunk(cp, c, src, scl, stage, SP, 1);
    __syncthreads();
    if (active) {
      for (int kk = ks; kk < cnt; kk += KS) {
        const float* row = stage + kk * SP;
        float av[TM], bv[TM];
#pragma unroll
        for (int a = 0; a < TM; ++a) av[a] = row[ti * TM + a];
#pragma unroll
        for (int b = 0; b < TM; ++b) bv[b] = row[tj * TM + b];
#pragma unroll
        for (int a = 0; a < TM; ++a)
#pragma unroll
          for (int b = 0; b < TM; ++b) dd_acc_prod(hi[a][b], lo[a][b], av[a], bv[b]);
        if (++nacc == kFlushEvery) flush();
      }
    }
    __syncthreads();
  }
  if (active) flush();
  __syncthreads();
  if (KS > 1) {
    // thread slot (ks * U + u) holds group ks's partial of tile u
    for (int e = tid; e < U * TM * TM; e += blockDim.x) {
      int u = e / (TM * TM);
      const int ab = e - u * TM * TM;
      const int a = ab / TM, b = ab - a * TM;
      int ri = 0;
      while (u >= T - ri) {
        u -= T - ri;
        ++ri;
      }
      const int i = ri * TM + a, j = (ri + u) * TM + b;
      if (i < n && j < n && i <= j) {
        double v = 0.0;
        for (int g = 0; g < KS; ++g) v += part[(g * U + e / (TM * TM)) * TM * TM + ab];
        Ad[i * n + j] = v;
      }
    }
    __syncthreads();
  }
  for (int e = tid; e < n * n; e += blockDim.x) {
    const int i = e / n, j = e - i * n;
    if (i > j) Ad[e] = Ad[j * n + i];
  }
  __syncthreads();
}

// A TM is usable when its upper-triangular tile set fits the CTA (one tile per thread).
__host__ __device__ __forceinline__ bool gram_tm_fits(int tm, int n, int threads) {
  const int T = (n + tm - 1) / tm;
  return T * (T + 1) / 2 <= threads;
}

__device__ void batch_gram_dispatch(int tm, const float* src, float scl, int64_t L, int n, int64_t R, double* Ad,
                                    float* stage) {
  while (tm < 5 && !gram_tm_fits(tm, n, blockDim.x)) ++tm;
  switch (tm) {
    case 2: batch_gram<2>(src, scl, L, n, R, Ad, stage); break;
    case 3: batch_gram<3>(src, scl, L, n, R, Ad, stage); break;
    case 5: batch_gram<5>(src, scl, L, n, R, Ad, stage); break;
    default: batch_gram<4>(src, scl, L, n, R, Ad, stage); break;
  }
}

// ----------------------------------------------------------------- Jacobi
struct JacobiShared {
  dd c[kMaxPairs], s[kMaxPairs];
  int p[kMaxPairs], q[kMaxPairs];
  unsigned short blk[kMaxBlocks];
};

// Cyclic Jacobi on A (n x n, double-float, symmetric) with V accumulating the
// rotations (V = I on entry).  Round r of a sweep pairs the indices by the
// circle method (m = n rounded up to even; index m-1 fixed, the rest
// rotating; a pair with index n is idle for odd n), so each round applies
// m/2 disjoint rotations A <- J^T A J, V <- V J.  A rotation is skipped when
// |a_pq| <= 2^-40 sqrt(|a_pp a_qq|) or |a_pq| <= 2^-44 trace(A); the sweeps
// stop after one with no rotation.  Returns the sweeps run (negative if the
// limit was hit).
__device__ int batch_jacobi(dd* __restrict__ A, dd* __restrict__ V, int n, JacobiShared& js, float trace,
                            int* nrounds) {
  const int tid = threadIdx.x;
  const int m = n + (n & 1);
  const int np = m / 2;
  const int nblk = np * (np + 1) / 2;
  for (int b = tid; b < nblk; b += blockDim.x) {
    int ki = 0, u = b;
    while (u >= np - ki) {
      u -= np - ki;
      ++ki;
    }
    js.blk[b] = (unsigned short)((ki << 8) | (ki + u));
  }
  const float floor_abs = 0x1p-44f * trace;
  __syncthreads();
  for (int sweep = 0; sweep < kMaxSweeps; ++sweep) {
    int rotated = 0;
    for (int r = 0; r < m - 1; ++r) {
      int flag = 0;
      if (tid < np) {
        int a = (tid == 0) ? (m - 1) : (r + tid) % (m - 1);
        int b = (tid == 0) ? r : (r - tid + m - 1) % (m - 1);
        const int p = min(a, b), q = max(a, b);
        dd c = ddf(1.f), s = ddf(0.f);
        if (q < n) {
          const dd app = A[p * n + p], aqq = A[q * n + q], apq = A[p * n + q];
          const float mag = fabsf(apq.hi);
          if (mag > 0x1p-40f * sqrtf(fabsf(app.hi) * fabsf(aqq.hi)) && mag > floor_abs) {
            // t = sign(th) / (|th| + sqrt(th^2 + 1)), th = (a_qq - a_pp) / (2 a_pq)
            const dd th = dd_div(dd_sub(aqq, app), dd_add(apq, apq));
            const bool neg = dd_neg_sign(th);
            const dd ath = neg ? dd_neg(th) : th;
            dd t;
            if (ath.hi > 1e18f) {
              t = dd_div(ddf(0.5f), ath);
            } else {
              t = dd_div(ddf(1.f), dd_add(ath, dd_sqrt(dd_add(dd_mul(ath, ath), ddf(1.f)))));
            }
            if (neg) t = dd_neg(t);
            c = dd_div(ddf(1.f), dd_sqrt(dd_add(dd_mul(t, t), ddf(1.f))));
            s = dd_mul(t, c);
            flag = 1;
          }
        }
        js.c[tid] = c;
        js.s[tid] = s;
        js.p[tid] = p;
        js.q[tid] = q;
      }
      if (!__syncthreads_or(flag)) continue;
      rotated = 1;
      ++*nrounds;
      // A <- J^T A J over the 2x2 blocks (ki <= kj; the mirror is written too)
      for (int b = tid; b < nblk; b += blockDim.x) {
        const int ki = js.blk[b] >> 8, kj = js.blk[b] & 0xff;
        const int p1 = js.p[ki], q1 = js.q[ki], p2 = js.p[kj], q2 = js.q[kj];
        const dd c1 = js.c[ki], s1 = js.s[ki], c2 = js.c[kj], s2 = js.s[kj];
        const bool v1 = q1 < n, v2 = q2 < n;
        const dd z0 = ddf(0.f);
        const dd xpp = A[p1 * n + p2];
        const dd xpq = v2 ? A[p1 * n + q2] : z0;
        const dd xqp = v1 ? A[q1 * n + p2] : z0;
        const dd xqq = (v1 && v2) ? A[q1 * n + q2] : z0;
        // rows: y_p = c1 x_p - s1 x_q, y_q = s1 x_p + c1 x_q
        const dd ypp = dd_sub(dd_mul(c1, xpp), dd_mul(s1, xqp));
        const dd ypq = dd_sub(dd_mul(c1, xpq), dd_mul(s1, xqq));
        const dd yqp = dd_add(dd_mul(s1, xpp), dd_mul(c1, xqp));
        const dd yqq = dd_add(dd_mul(s1, xpq), dd_mul(c1, xqq));
        // columns: z_.p = c2 y_.p - s2 y_.q, z_.q = s2 y_.p + c2 y_.q
        dd zpp = dd_sub(dd_mul(c2, ypp), dd_mul(s2, ypq));
        dd zpq = dd_add(dd_mul(s2, ypp), dd_mul(c2, ypq));
        dd zqp = dd_sub(dd_mul(c2, yqp), dd_mul(s2, yqq));
        dd zqq = dd_add(dd_mul(s2, yqp), dd_mul(c2, yqq));
        if (ki == kj) {
          if (v1 && (s1.hi != 0.f)) zpq = zqp = z0;  // annihilated pair
          A[p1 * n + p1] = zpp;
          if (v1) {
            A[p1 * n + q1] = zpq;
            A[q1 * n + p1] = zqp;
            A[q1 * n + q1] = zqq;
          }
        } else {
          A[p1 * n + p2] = zpp;
          A[p2 * n + p1] = zpp;
          if (v2) {
            A[p1 * n + q2] = zpq;
            A[q2 * n + p1] = zpq;
          }
          if (v1) {
            A[q1 * n + p2] = zqp;
            A[p2 * n + q1] = zqp;
          }
          if (v1 && v2) {
            A[q1 * n + q2] = zqq;
            A[q2 * n + q1] = zqq;
          }
        }
      }
      // V <- V J
      for (int e = tid; e < n * np; e += blockDim.x) {
        const int i = e / np, k = e - i * np;
        const int p = js.p[k], q = js.q[k];
        if (q >= n || js.s[k].hi == 0.f) continue;
        const dd c = js.c[k], s = js.s[k];
        const dd vp = V[i * n + p], vq = V[i * n + q];
        V[i * n + p] = dd_sub(dd_mul(c, vp), dd_mul(s, vq));
        V[i * n + q] = dd_add(dd_mul(s, vp), dd_mul(c, vq));
      }
      __syncthreads();
    }
    if (!rotated) return sweep + 1;
  }
  return -kMaxSweeps;
}

// -------------------------------------------------------------------- TTM
// dst (L, r, R) = U^T ._m src with U (n x r, double-float, row stride rp) in
// shared memory; FP32 output, or FP64 times `unscale` when dst64 is set.
constexpr int kTR = 4, kTC = 4;
__device__ void batch_ttm(const float* __restrict__ src, float scl, int64_t L, int n, int64_t R,
                          const dd* __restrict__ Us, int r, int rp, float* __restrict__ stage, int stage_cap,
                          float* __restrict__ dst32, double* __restrict__ dst64, double unscale) {
  const int tid = threadIdx.x;
  const int JB = (r + kTR - 1) / kTR;
  int kc = kTC * ((int)blockDim.x / JB);
  if (kc < kTC) kc = kTC;
  int cap = (stage_cap / n) / kTC * kTC;
  if (kc > cap) kc = cap;
  const int KB = kc / kTC;
  const bool active = tid < JB * KB;
  const int jb = active ? tid / KB : 0, kb = active ? tid % KB : 0;
  const ChunkPlan cp = chunk_plan(L, n, R, kc);
  for (int64_t c = 0; c < cp.nchunks; ++c) {
    const int cnt = stage_chunk(cp, c, src, scl, stage, 1, kc);
    __syncthreads();
    if (active && kb * kTC < cnt) {
      float hi[kTR][kTC], lo[kTR][kTC];
#pragma unroll
      for (int a = 0; a < kTR; ++a)
#pragma unroll
        for (int b = 0; b < kTC; ++b) hi[a][b] = lo[a][b] = 0.f;
      for (int i = 0; i < n; ++i) {
        dd u[kTR];
        float bv[kTC];
#pragma unroll
        for (int a = 0; a < kTR; ++a) u[a] = Us[i * rp + jb * kTR + a];
#pragma unroll
        for (int b = 0; b < kTC; ++b) bv[b] = stage[i * kc + kb * kTC + b];
#pragma unroll
        for (int a = 0; a < kTR; ++a)
#pragma unroll
          for (int b = 0; b < kTC; ++b) dd_acc_prod2(hi[a][b], lo[a][b], u[a], bv[b]);
      }
      // column kk of the chunk -> (l, rho)
      int64_t lbase, rbase;
      if (!cp.small_r) {
        lbase = c / cp.cpl;
        rbase = (c - lbase * cp.cpl) * cp.kc;
      } else {
        lbase = c * cp.lc;
        rbase = 0;
      }
#pragma unroll
      for (int b = 0; b < kTC; ++b) {
        const int kk = kb * kTC + b;
        if (kk >= cnt) continue;
        int64_t l, rho;
        if (!cp.small_r) {
          l = lbase;
          rho = rbase + kk;
        } else {
          l = lbase + kk / R;
          rho = kk % R;
        }
#pragma unroll
        for (int a = 0; a < kTR; ++a) {
          const int j = jb * kTR + a;
          if (j >= r) continue;
          const int64_t o = (l * r + j) * R + rho;
          if (dst64)
            dst64[o] = ((double)hi[a][b] + (double)lo[a][b]) * unscale;
          else
            dst32[o] = hi[a][b] + lo[a][b];
        }
      }
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------- the kernel
__device__ __forceinline__ float block_max(float v, float* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  float m = 0.f;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) m = fmaxf(m, red[i]);
  return m;
}

__global__ void __launch_bounds__(kBThreads) batch_sthosvd_kernel(BatchArgs a) {
  extern __shared__ __align__(16) unsigned char bsm[];
  __shared__ JacobiShared js;
  __shared__ double s_lam[kBMaxN];
  __shared__ double s_tail[kBMaxN + 1];
  __shared__ int s_perm[kBMaxN];
  __shared__ float s_sign[kBMaxN];
  __shared__ float s_red[32];
  __shared__ int s_job, s_bad, s_r;
  __shared__ double s_sc[4];
  const int tid = threadIdx.x;
  const int nmax = kBMaxN;
  (void)nmax;
  float* buf0 = a.scratch + (int64_t)blockIdx.x * 2 * a.half;
  float* buf1 = buf0 + a.half;
  for (;;) {
    if (tid == 0) s_job = atomicAdd(a.counter, 1);
    __syncthreads();
    const int job = s_job;
    __syncthreads();
    if (job >= a.count) break;
    const int t = a.sched[job];
    const BatchTensor& T = a.t[t];
    BatchOut* O = a.out + t;
    const float* x = a.x[t];
    const int d = a.d;
    int cur[kBMaxD];
    for (int i = 0; i < d; ++i) cur[i] = T.dims[i];
    // power-of-two scale of the input; NaN / Inf check
    if (tid == 0) s_bad = 0;
    __syncthreads();
    float mx = 0.f;
    int bad = 0;
    for (int64_t e = tid; e < T.nelem; e += blockDim.x) {
      const float v = fabsf(__ldg(x + e));
      if (!(v <= 3.4028235e38f)) bad = 1;
      mx = fmaxf(mx, v);
    }
    if (bad) s_bad = 1;
    mx = block_max(mx, s_red);
    __syncthreads();
    if (s_bad) {
      if (tid == 0) O->status = 1;
      continue;
    }
    int ex = 0;
    if (mx > 0.f) frexpf(mx, &ex);
    ex = max(-100, min(100, ex));
    const float scl = ldexpf(1.f, -ex);
    const double unscale = ldexp(1.0, ex), unscale2 = ldexp(1.0, 2 * ex);
    const float* src = x;
    float src_scl = scl;
    double norm2 = 0.0, used = 0.0, budget_total = 0.0;
    int status = 0;
    long long cyc[4] = {0, 0, 0, 0};
    long long t0 = clock64();
    for (int step = 0; step < d; ++step) {
      const int m = T.order[step];
      int64_t L = 1, R = 1;
      for (int i = 0; i < m; ++i) L *= cur[i];
      for (int i = m + 1; i < d; ++i) R *= cur[i];
      const int n = cur[m];
      double* Ad = reinterpret_cast<double*>(bsm);
      dd* A = reinterpret_cast<dd*>(bsm);
      unsigned char* reg1 = bsm + (size_t)8 * kBMaxN * kBMaxN;
      dd* V = reinterpret_cast<dd*>(reg1);
      float* stage = reinterpret_cast<float*>(reg1);
      batch_gram_dispatch(a.tm_of_n[n], src, src_scl, L, n, R, Ad, stage);
      // trace (FP64), then the working copy in double-float (same storage)
      if (tid == 0) {
        double tr = 0.0;
        for (int i = 0; i < n; ++i) tr += Ad[i * n + i];
        s_sc[0] = tr;
      }
      __syncthreads();
      const double trace = s_sc[0];
      if (step == 0) {
        norm2 = trace * unscale2;
        budget_total = a.rtmss * T.eps * T.eps * norm2;
      }
      for (int e = tid; e < n * n; e += blockDim.x) {
        const double v = Ad[e];
        A[e] = dd_from(v);
      }
      for (int e = tid; e < n * n; e += blockDim.x) {
        const int i = e / n, j = e - i * n;
        V[e] = ddf(i == j ? 1.f : 0.f);
      }
      __syncthreads();
      long long t1 = clock64();
      cyc[0] += t1 - t0;
      t0 = t1;
      int nrounds = 0;
      const int sw = batch_jacobi(A, V, n, js, (float)trace, &nrounds);
      t1 = clock64();
      cyc[1] += t1 - t0;
      t0 = t1;
      if (sw < 0) status = 2;
      // eigenvalues (clamped at 0, unscaled), descending order, ties by index
      for (int i = tid; i < n; i += blockDim.x) s_lam[i] = fmax(dd_to(A[i * n + i]), 0.0) * unscale2;
      __syncthreads();
      for (int i = tid; i < n; i += blockDim.x) {
        const double li = s_lam[i];
        int pos = 0;
        for (int j = 0; j < n; ++j) {
          const double lj = s_lam[j];
          pos += (lj > li) || (lj == li && j < i);
        }
        s_perm[pos] = i;
      }
      __syncthreads();
      if (tid == 0) {
        double acc = 0.0;
        s_tail[n] = 0.0;
        for (int j = n - 1; j >= 0; --j) {
          acc += s_lam[s_perm[j]];
          s_tail[j] = acc;
        }
        const double budget = a.adaptive ? (budget_total - used) / (double)(d - step) : budget_total / d;
        int r = n;
        for (int rr = 1; rr <= n; ++rr)
          if (s_tail[rr] <= budget) {
            r = rr;
            break;
          }
        s_r = r;
        O->ranks[m] = r;
        O->sweeps[m] = sw;
        O->rounds[m] = nrounds;
        O->discarded[m] = s_tail[r];
      }
      __syncthreads();
      const int r = s_r;
      used += s_tail[r];
      // sign of each kept column: its entry of largest magnitude (first on ties) positive
      {
        const int lane = tid & 31, w = tid >> 5, nw = blockDim.x >> 5;
        for (int j = w; j < r; j += nw) {
          const int col = s_perm[j];
          float best = -1.f;
          int bi = 0;
          for (int i = lane; i < n; i += 32) {
            const float vf = (float)fabs(dd_to(V[i * n + col]));
            if (vf > best) {
              best = vf;
              bi = i;
            }
          }
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            const float ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ob > best || (ob == best && oi < bi)) {
              best = ob;
              bi = oi;
            }
          }
          if (lane == 0) s_sign[j] = dd_neg_sign(V[bi * n + col]) ? -1.f : 1.f;
        }
      }
      __syncthreads();
      // factor (FP64, n x r row-major) and U in double-float over the G storage
      double* fac = a.fac_pool + T.fac_off[m];
      const int rp = ((r + kTR - 1) / kTR) * kTR;
      dd* Us = A;
      for (int e = tid; e < n * rp; e += blockDim.x) {
        const int i = e / rp, j = e - i * rp;
        dd u = ddf(0.f);
        if (j < r) {
          u = V[i * n + s_perm[j]];
          if (s_sign[j] < 0.f) u = dd_neg(u);
          fac[i * r + j] = dd_to(u);
        }
        Us[e] = u;
      }
      __syncthreads();
      const bool last = (step == d - 1);
      float* dst32 = (step & 1) ? buf1 : buf0;
      double* dst64 = last ? a.core_pool + T.core_off : nullptr;
      const int cap = (int)((size_t)8 * kBMaxN * kBMaxN / sizeof(float));
      t1 = clock64();
      cyc[2] += t1 - t0;
      t0 = t1;
      batch_ttm(src, src_scl, L, n, R, Us, r, rp, stage, cap, dst32, dst64, unscale);
      __syncthreads();
      t1 = clock64();
      cyc[3] += t1 - t0;
      t0 = t1;
      src = dst32;
      src_scl = 1.f;
      cur[m] = r;
    }
    if (tid == 0) {
      O->norm2 = norm2;
      O->sse_trunc = used;
      O->status = status;
      for (int i = 0; i < 4; ++i) O->cycles[i] = cyc[i];
    }
    __syncthreads();
  }
}

// Gram timing probe for the tile table: every CTA forms the Gram of the same
// (1, n, K) slab with tile TM; `sink` keeps the result live.
template <int TM>
__global__ void __launch_bounds__(kBThreads) batch_gram_probe_kernel(const float* x, int n, int64_t K, double* sink) {
  extern __shared__ __align__(16) unsigned char bsm[];
  double* Ad = reinterpret_cast<double*>(bsm);
  float* stage = reinterpret_cast<float*>(bsm + (size_t)8 * kBMaxN * kBMaxN);
  batch_gram<TM>(x, 1.f, 1, n, K, Ad, stage);
  if (threadIdx.x == 0) sink[blockIdx.x] = Ad[0] + Ad[n * n - 1];
}

// ------------------------------------------------------------------ host
static size_t batch_smem_bytes() { return (size_t)16 * kBMaxN * kBMaxN; }

static int g_tm_table[kBMaxN + 1];
static bool g_tm_tuned = false;

static void default_tm_table(int* tab) {
  for (int n = 0; n <= kBMaxN; ++n) tab[n] = n <= 24 ? 2 : n <= 40 ? 3 : n <= 72 ? 4 : 5;
}

int batch_sm_count(int* sms) {
  int dev = 0;
  ATC_CUDA_TRY(cudaGetDevice(&dev));
  ATC_CUDA_TRY(cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, dev));
  return ATC_OK;
}

template <int TM>
static int probe_one(const float* x, int n, int64_t K, double* sink, int grid, cudaStream_t s, float* ms) {
  const size_t smem = batch_smem_bytes();
  ATC_CUDA_TRY(cudaFuncSetAttribute(batch_gram_probe_kernel<TM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem));
  cudaEvent_t e0, e1;
  ATC_CUDA_TRY(cudaEventCreate(&e0));
  ATC_CUDA_TRY(cudaEventCreate(&e1));
  batch_gram_probe_kernel<TM><<<grid, kBThreads, smem, s>>>(x, n, K, sink);  // warm-up
  ATC_LAUNCHED(1);
  ATC_CUDA_TRY(cudaEventRecord(e0, s));
  batch_gram_probe_kernel<TM><<<grid, kBThreads, smem, s>>>(x, n, K, sink);
  ATC_LAUNCHED(1);
  ATC_CUDA_TRY(cudaEventRecord(e1, s));
  ATC_CUDA_TRY(cudaEventSynchronize(e1));
  ATC_CUDA_TRY(cudaEventElapsedTime(ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return ATC_OK;
}

// Measures the Gram tile per mode length (buckets of 8) on this device.
int batch_tune(cudaStream_t s, int* table_out) {
  int sms = 0;
  ATC_TRY(batch_sm_count(&sms));
  const int64_t K = 4096;
  float* x = nullptr;
  double* sink = nullptr;
  ATC_TRY(Scratch::get(SLOT_BATCH_TUNE, sizeof(float) * (size_t)kBMaxN * K + sizeof(double) * 4096, (void**)&x));
  sink = reinterpret_cast<double*>(x + (size_t)kBMaxN * K);
  ATC_CUDA_TRY(cudaMemsetAsync(x, 0, sizeof(float) * (size_t)kBMaxN * K, s));
  int tab[kBMaxN + 1];
  default_tm_table(tab);
  const int grid = std::min(sms, 4096);
  for (int nb = 16; nb <= kBMaxN; nb += 8) {
    float best = 1e30f;
    int bt = tab[nb];
    for (int tm : {2, 3, 4, 5}) {
      if (!gram_tm_fits(tm, nb, kBThreads)) continue;
      float ms = 0.f;
      int rc = ATC_OK;
      switch (tm) {
        case 2: rc = probe_one<2>(x, nb, K, sink, grid, s, &ms); break;
        case 3: rc = probe_one<3>(x, nb, K, sink, grid, s, &ms); break;
        case 4: rc = probe_one<4>(x, nb, K, sink, grid, s, &ms); break;
        default: rc = probe_one<5>(x, nb, K, sink, grid, s, &ms); break;
      }
      if (rc) return rc;
      if (ms < best) {
        best = ms;
        bt = tm;
      }
    }
    for (int n = std::max(0, nb - 7); n <= nb; ++n) tab[n] = bt;
  }
  for (int n = 0; n < 9; ++n) tab[n] = tab[16];
  std::copy(tab, tab + kBMaxN + 1, g_tm_table);
  g_tm_tuned = true;
  if (table_out) std::copy(tab, tab + kBMaxN + 1, table_out);
  return ATC_OK;
}

}  // namespace atc

// ====================================================================== ABI
using namespace atc;

struct atc_batch {
  int count = 0, d = 0;
  std::vector<int64_t> dims;
  std::vector<BatchTensor> ht;
  std::vector<BatchOut> hout;
  BatchTensor* dt = nullptr;
  BatchOut* dout = nullptr;
  BatchOut* hout_pinned = nullptr;
  const float** xtab_dev = nullptr;
  const float** xtab_host = nullptr;  // pinned
  int* sched = nullptr;
  int* counter = nullptr;
  int* tm_dev = nullptr;
  float* scratch = nullptr;
  double* core_pool = nullptr;
  double* fac_pool = nullptr;
  int64_t half = 0;
  int grid = 0;
  double rtmss = 0.5;
  int adaptive = 0;
  cudaStream_t cap_stream = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  float last_ms = 0.f;
};

static void batch_release(atc_batch* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  for (void* p : {(void*)b->dt, (void*)b->dout, (void*)b->xtab_dev, (void*)b->sched, (void*)b->counter,
                  (void*)b->tm_dev, (void*)b->scratch, (void*)b->core_pool, (void*)b->fac_pool})
    if (p) cudaFree(p);
  for (void* p : {(void*)b->hout_pinned, (void*)b->xtab_host})
    if (p) cudaFreeHost(p);
  delete b;
}

extern "C" int atc_batch_create(int count, int ndim, const int64_t* dims, int dtype, const double* rel_eps,
                                const atc_options* opt_in, atc_batch** out) {
  if (!out || !dims || !rel_eps || count < 1 || ndim < 1 || ndim > kBMaxD)
    return fail(ATC_EINVAL, "atc_batch_create: bad arguments");
  *out = nullptr;
  if (dtype != ATC_F32) return fail(ATC_EUNSUP, "atc_batch_create: the batched path takes float32 tensors");
  atc_options opt;
  atc_default_options(&opt);
  if (opt_in) opt = *opt_in;
  if (!(opt.rtmss >= 0.0 && opt.rtmss <= 1.0)) return fail(ATC_EINVAL, "atc_batch_create: rtmss not in [0, 1]");
  if (opt.rank_rule != ATC_RANK_STATIC && opt.rank_rule != ATC_RANK_ADAPTIVE)
    return fail(ATC_EINVAL, "atc_batch_create: unknown rank rule");
  if (opt.mode_order) {
    std::vector<int> seen(ndim, 0);
    for (int i = 0; i < ndim; ++i) {
      const int v = opt.mode_order[i];
      if (v < 0 || v >= ndim || seen[v]++) return fail(ATC_EINVAL, "atc_batch_create: mode_order is not a permutation");
    }
  }
  atc_batch* b = new (std::nothrow) atc_batch;
  if (!b) return fail(ATC_ENOMEM, "atc_batch_create: host allocation failed");
  b->count = count;
  b->d = ndim;
  b->rtmss = opt.rtmss;
  b->adaptive = opt.rank_rule == ATC_RANK_ADAPTIVE;
  b->dims.assign(dims, dims + (size_t)count * ndim);
  b->ht.resize(count);
  b->hout.resize(count);
  int64_t maxn_elem = 0, core_tot = 0, fac_tot = 0;
  std::vector<double> cost(count);
  for (int t = 0; t < count; ++t) {
    BatchTensor& T = b->ht[t];
    memset(&T, 0, sizeof(T));
    if (!(rel_eps[t] > 0.0 && rel_eps[t] <= 1.0)) {
      batch_release(b);
      return fail(ATC_EINVAL, "atc_batch_create: rel_eps[%d] not in (0, 1]", t);
    }
    T.eps = rel_eps[t];
    int64_t N = 1;
    for (int i = 0; i < ndim; ++i) {
      const int64_t n = dims[(size_t)t * ndim + i];
      if (n < 1) {
        batch_release(b);
        return fail(ATC_EINVAL, "atc_batch_create: dims of tensor %d must be positive", t);
      }
      if (n > kBMaxN) {
        batch_release(b);
        return fail(ATC_EUNSUP, "atc_batch_create: mode length %lld > %d (use atc_compress)", (long long)n, kBMaxN);
      }
      T.dims[i] = (int)n;
      N *= n;
    }
    if (N > (int64_t)1 << 31) {
      batch_release(b);
      return fail(ATC_EUNSUP, "atc_batch_create: tensor %d too large for the batched path", t);
    }
    T.nelem = N;
    std::vector<int> ord(ndim);
    for (int i = 0; i < ndim; ++i) ord[i] = opt.mode_order ? opt.mode_order[i] : i;
    if (!opt.mode_order)
      std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return T.dims[x] < T.dims[y]; });
    for (int i = 0; i < ndim; ++i) T.order[i] = ord[i];
    T.core_off = core_tot;
    core_tot += N;
    double c = 0.0;
    for (int i = 0; i < ndim; ++i) {
      T.fac_off[i] = fac_tot;
      fac_tot += (int64_t)T.dims[i] * T.dims[i];
      c += 22.0 * T.dims[i] * (double)N + 600.0 * (double)T.dims[i] * T.dims[i] * T.dims[i];
    }
    cost[t] = c;
    maxn_elem = std::max(maxn_elem, N);
  }
  std::vector<int> sched(count);
  for (int t = 0; t < count; ++t) sched[t] = t;
  std::stable_sort(sched.begin(), sched.end(), [&](int x, int y) { return cost[x] > cost[y]; });
  int sms = 0, rc = batch_sm_count(&sms);
  if (rc) {
    batch_release(b);
    return rc;
  }
  const size_t smem = batch_smem_bytes();
  int occ = 0;
  if (cudaFuncSetAttribute(batch_sthosvd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
          cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, batch_sthosvd_kernel, kBThreads, smem) != cudaSuccess ||
      occ < 1) {
    batch_release(b);
    return fail(ATC_ECUDA, "atc_batch_create: kernel cannot be resident (%d)", occ);
  }
  b->grid = std::min(count, sms * occ);
  b->half = (maxn_elem + 63) / 64 * 64;
  cudaStream_t us = (cudaStream_t)opt.stream;
  if (!g_tm_tuned) {
    const char* env = getenv("ATC_BATCH_TUNE");
    if (env && env[0] == '0') {
      default_tm_table(g_tm_table);
    } else {
      rc = batch_tune(us, nullptr);
      if (rc) {
        batch_release(b);
        return rc;
      }
    }
  }
  bool ok = cudaMalloc(&b->dt, sizeof(BatchTensor) * count) == cudaSuccess &&
            cudaMalloc(&b->dout, sizeof(BatchOut) * count) == cudaSuccess &&
            cudaMallocHost(&b->hout_pinned, sizeof(BatchOut) * count) == cudaSuccess &&
            cudaMalloc(&b->xtab_dev, sizeof(float*) * count) == cudaSuccess &&
            cudaMallocHost(&b->xtab_host, sizeof(float*) * count) == cudaSuccess &&
            cudaMalloc(&b->sched, sizeof(int) * count) == cudaSuccess &&
            cudaMalloc(&b->counter, sizeof(int)) == cudaSuccess &&
            cudaMalloc(&b->tm_dev, sizeof(int) * (kBMaxN + 1)) == cudaSuccess &&
            cudaMalloc(&b->scratch, sizeof(float) * (size_t)b->grid * 2 * b->half) == cudaSuccess &&
            cudaMalloc(&b->core_pool, sizeof(double) * (size_t)core_tot) == cudaSuccess &&
            cudaMalloc(&b->fac_pool, sizeof(double) * (size_t)fac_tot) == cudaSuccess;
  if (!ok) {
    batch_release(b);
    cudaGetLastError();
    return fail(ATC_ENOMEM, "atc_batch_create: device allocation failed");
  }
  ok = cudaMemcpy(b->dt, b->ht.data(), sizeof(BatchTensor) * count, cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemcpy(b->sched, sched.data(), sizeof(int) * count, cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemcpy(b->tm_dev, g_tm_table, sizeof(int) * (kBMaxN + 1), cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemset(b->dout, 0, sizeof(BatchOut) * count) == cudaSuccess;
  if (!ok) {
    batch_release(b);
    return fail(ATC_ECUDA, "atc_batch_create: upload failed");
  }
  // the graph: pointer table upload, queue reset, the persistent launch, results readback
  BatchArgs ba;
  ba.t = b->dt;
  ba.out = b->dout;
  ba.x = b->xtab_dev;
  ba.sched = b->sched;
  ba.count = count;
  ba.d = ndim;
  ba.counter = b->counter;
  ba.scratch = b->scratch;
  ba.half = b->half;
  ba.core_pool = b->core_pool;
  ba.fac_pool = b->fac_pool;
  ba.rtmss = b->rtmss;
  ba.adaptive = b->adaptive;
  ba.tm_of_n = b->tm_dev;
  if (cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    batch_release(b);
    return fail(ATC_ECUDA, "atc_batch_create: stream creation failed");
  }
  cudaStream_t cs = b->cap_stream;
  ok = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
  if (ok) {
    cudaMemcpyAsync(b->xtab_dev, b->xtab_host, sizeof(float*) * count, cudaMemcpyHostToDevice, cs);
    cudaMemsetAsync(b->counter, 0, sizeof(int), cs);
    batch_sthosvd_kernel<<<b->grid, kBThreads, smem, cs>>>(ba);
    cudaMemcpyAsync(b->hout_pinned, b->dout, sizeof(BatchOut) * count, cudaMemcpyDeviceToHost, cs);
    ok = cudaStreamEndCapture(cs, &b->graph) == cudaSuccess &&
         cudaGraphInstantiate(&b->exec, b->graph, 0) == cudaSuccess;
  }
  if (!ok) {
    batch_release(b);
    return fail(ATC_ECUDA, "atc_batch_create: graph capture failed: %s", cudaGetErrorString(cudaGetLastError()));
  }
  *out = b;
  return ATC_OK;
}

extern "C" int atc_batch_run(atc_batch* b, const void* const* tensors_dev, void* stream) {
  if (!b || !tensors_dev) return fail(ATC_EINVAL, "atc_batch_run: bad arguments");
  for (int t = 0; t < b->count; ++t) {
    if (!tensors_dev[t]) return fail(ATC_EINVAL, "atc_batch_run: tensor %d is NULL", t);
    b->xtab_host[t] = (const float*)tensors_dev[t];
  }
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  ATC_CUDA_TRY(cudaEventCreate(&e0));
  ATC_CUDA_TRY(cudaEventCreate(&e1));
  ATC_CUDA_TRY(cudaEventRecord(e0, s));
  ATC_CUDA_TRY(cudaGraphLaunch(b->exec, s));
  ATC_LAUNCHED(1);
  ATC_CUDA_TRY(cudaEventRecord(e1, s));
  ATC_CUDA_TRY(cudaEventSynchronize(e1));
  cudaEventElapsedTime(&b->last_ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  std::copy(b->hout_pinned, b->hout_pinned + b->count, b->hout.begin());
  for (int t = 0; t < b->count; ++t) {
    if (b->hout[t].status == 1) return fail(ATC_ENUMERIC, "atc_batch_run: tensor %d holds NaN or Inf", t);
  }
  return ATC_OK;
}

extern "C" int atc_batch_get_ranks(const atc_batch* b, int index, int64_t* ranks) {
  if (!b || !ranks || index < 0 || index >= b->count) return fail(ATC_EINVAL, "atc_batch_get_ranks: bad arguments");
  for (int i = 0; i < b->d; ++i) ranks[i] = b->hout[index].ranks[i];
  return ATC_OK;
}

extern "C" int atc_batch_get_core(const atc_batch* b, int index, const double** core_dev) {
  if (!b || !core_dev || index < 0 || index >= b->count) return fail(ATC_EINVAL, "atc_batch_get_core: bad arguments");
  *core_dev = b->core_pool + b->ht[index].core_off;
  return ATC_OK;
}

extern "C" int atc_batch_get_factor(const atc_batch* b, int index, int mode, const double** u_dev) {
  if (!b || !u_dev || index < 0 || index >= b->count || mode < 0 || mode >= b->d)
    return fail(ATC_EINVAL, "atc_batch_get_factor: bad arguments");
  *u_dev = b->fac_pool + b->ht[index].fac_off[mode];
  return ATC_OK;
}

extern "C" int atc_batch_get_stats(const atc_batch* b, int index, double* norm2, double* sse_trunc, int* sweeps,
                                   int* status) {
  if (!b || index < 0 || index >= b->count) return fail(ATC_EINVAL, "atc_batch_get_stats: bad arguments");
  const BatchOut& o = b->hout[index];
  if (norm2) *norm2 = o.norm2;
  if (sse_trunc) *sse_trunc = o.sse_trunc;
  if (sweeps)
    for (int i = 0; i < b->d; ++i) sweeps[i] = o.sweeps[i];
  if (status) *status = o.status;
  return ATC_OK;
}

extern "C" int atc_batch_get_profile(const atc_batch* b, int index, int64_t* cycles, int* rounds) {
  if (!b || index < 0 || index >= b->count) return fail(ATC_EINVAL, "atc_batch_get_profile: bad arguments");
  const BatchOut& o = b->hout[index];
  if (cycles)
    for (int i = 0; i < 4; ++i) cycles[i] = o.cycles[i];
  if (rounds)
    for (int i = 0; i < b->d; ++i) rounds[i] = o.rounds[i];
  return ATC_OK;
}

extern "C" float atc_batch_last_ms(const atc_batch* b) { return b ? b->last_ms : 0.f; }

extern "C" int atc_batch_tune(void* stream, int* table_out) { return batch_tune((cudaStream_t)stream, table_out); }

extern "C" void atc_batch_free(atc_batch* b) { batch_release(b); }
