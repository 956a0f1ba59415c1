// Rayleigh-Ritz step of the subspace iteration (k_subspace.cu): the
// eigenpairs of the small symmetric matrix B = Q^T G Q (K x K, K <= 32) in ONE
// CTA of 1024 threads, one thread per matrix entry.
//
// B is graded: Q comes from the Householder QR of G V, so column j of Q leans
// on the j-th eigen-direction of G and B_ij ~ sqrt(B_ii B_jj) with diagonal
// entries falling over ~16 orders of magnitude.  Two-sided Jacobi with the
// relative off-diagonal test |b_pq| <= u sqrt(|b_pp b_qq|) resolves the
// eigenvalues and eigenvectors of such a matrix to relative accuracy (Demmel and
// Veselic, SIAM J. Matrix Anal. Appl. 13, 1992), so the rotations run in FP32
// (GB300 issues FP64 at 1/64 of the FP32 rate and every round depends on the
// previous one):
//   1. cyclic Jacobi in FP32 on B scaled by a power of two, parallel ordering
//      (circle method: 16 disjoint rotations a round, 31 rounds a sweep), each
//      round an update of all 32 x 32 entries of B and of the accumulated
//      rotations Y by the first 16 warps (warps 0-7 four entries of B a
//      thread, warps 8-15 four entries of Y, one named barrier of 512 threads:
//      the rounds are a chain, and fewer warps at each barrier shorten it; each
//      thread loads all its inputs before it stores, so its four entries are
//      independent chains), ping-pong buffers in shared memory; four sweeps
//      (fewer when a sweep rotates nothing);
//   2. Ritz values sorted descending (rank by comparison, ties by index);
//   3. one first-order correction Y <- Y (I + F), F_ij = (Y^T B Y)_ij / (theta_j
//      - theta_i) for Ritz values more than 1 % apart (FP32): what the remaining
//      sweeps would add, in three small products;
//   4. Y re-orthonormalised by two Newton-Schulz steps Y <- Y - Y (Y^T Y - I)/2
//      (Y^T Y in double-float, the small correction in FP32): the tail
//      trace(G) - sum_{j<r} theta_j is a small difference of large sums, so the
//      columns must be orthonormal to ~1e-15, not to FP32 level;
//   5. Ritz values as Rayleigh quotients theta_j = y_j^T B y_j in double-float
//      from the FP64 B (FP32 Jacobi values are only relative-accurate);
//   6. the provisional rank rp = the smallest r with trace(G) - sum_{j<r}
//      theta_j <= budget (FP64 warp prefix sum) and the convergence test of the
//      subspace, (|theta_K| / theta_rp)^T <= conv; the vector count is
//      nv = rp + extra (at most nmax).
// Outputs: theta (K, descending, FP64), decision = {rp, nv (0 unless the
// subspace passed), passed, the tensor-core error word}, Y (K x nv row-major,
// FP64).
#include <math.h>
#include <stdint.h>

#include "atc_internal.cuh"
#include "dd.cuh"

namespace atc {
namespace {

constexpr int kJ = 32;        // padded order (entries beyond K are zero rows / columns)
constexpr int kJP = kJ + 1;   // shared-memory pitch (floats)
constexpr int kJThreads = kJ * kJ;
constexpr int kJSweeps = 4;  // at most (earlier when a sweep rotates nothing); a first-order correction follows
constexpr float kJTol = 0x1p-23f;  // relative off-diagonal threshold (FP32 unit roundoff x 2)

// partner of index i in round r of the circle-method ordering of 32 indices:
// index 31 stays fixed, the others rotate; every round is a perfect matching
// and each pair meets once in 31 rounds
__device__ __forceinline__ int jac_partner(int i, int r) {
  if (i == kJ - 1) return r;
  if (i == r) return kJ - 1;
  int p = 2 * r - i;
  p = p < 0 ? p + (kJ - 1) : p;
  return p >= kJ - 1 ? p - (kJ - 1) : p;
}

struct JacShared {
  float A[2][kJ][kJP];
  float Y[2][kJ][kJP];
  float2 cs[kJ];               // per index: (cos, signed coefficient of the partner)
  float t[kJ];                 // per index: signed tan (0: no rotation)
  dd Yd[kJ][kJ];               // refined vectors (column j = Ritz vector j, sorted)
  dd Md[kJ][kJ];               // Y^T Y, then B Y
  dd Bd[kJ][kJ];               // B scaled, double-float
  double theta[kJ];
  int perm[kJ];
  int rot[2];
  int nv;
  int buf;                     // the ping-pong buffer holding the Jacobi result
};

constexpr int kJacThreads = 512;  // threads of the Jacobi rounds (warps 0-7: B, 8-15: Y)
__device__ __forceinline__ void jac_bar() { asm volatile("bar.sync 1, 512;" ::: "memory"); }

// 2^e as a double for |e| < 1022, by its bit pattern (ldexp is a long FP64
// routine, and FP64 issues at 1/64 of the FP32 rate on this GPU)
__device__ __forceinline__ double pow2d(int e) { return __longlong_as_double((long long)(1023 + e) << 52); }

__device__ __forceinline__ dd jd_shfl(dd a, int o) {
  return dd{__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o)};
}

__global__ void __launch_bounds__(kJThreads, 1)
    rr_jacobi_kernel(const double* __restrict__ B, int K, int n, const double* __restrict__ trace_g, double budget,
                     int extra, int nmax, double conv, int T, const int* __restrict__ tc_err,
                     double* __restrict__ theta_out, int* __restrict__ decision, double* __restrict__ Y_out) {
  extern __shared__ __align__(16) uint8_t rr_smem[];
  JacShared& S = *reinterpret_cast<JacShared*>(rr_smem);
  __shared__ int s_ex;
  const int tid = threadIdx.x, i = tid >> 5, j = tid & 31, lane = j, warp = i;
  // power-of-two scale from the largest diagonal entry (B is PSD up to rounding)
  if (warp == 0) {
    double m = (lane < K) ? fabs(B[(size_t)lane * K + lane]) : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) {
      int e = 0;
      if (m > 0.0) frexp(m, &e);
      s_ex = e;
    }
  }
  __syncthreads();
  const int ex = s_ex;
  const double bij = (i < K && j < K) ? B[(size_t)i * K + j] * pow2d(-ex) : 0.0;
  S.A[0][i][j] = (float)bij;
  S.Bd[i][j] = dd_from(bij);
  S.Y[0][i][j] = (i == j) ? 1.f : 0.f;
  // ---- 1. cyclic Jacobi, parallel ordering.  Lanes 0..15 of warp 0 form the
  // round's 16 rotations (MUFU reciprocal / square roots: the rotations only
  // need c^2 + s^2 = 1 to FP32 level, the vectors are re-orthonormalised below),
  // then the threads of warps 0-7 update four entries of A and of Y each.
  __syncthreads();  // B and Y initialised by all 1024 threads
  if (tid < kJacThreads) {
    int buf = 0;
    const int wj = (tid >> 5) & 7;  // this thread's rows: wj, wj + 8, wj + 16, wj + 24 (column j = lane)
    for (int sweep = 0; sweep < kJSweeps; ++sweep) {
      if (tid == 0) S.rot[sweep & 1] = 0;
      jac_bar();
      for (int r = 0; r < kJ - 1; ++r) {
        if (tid < kJ / 2) {
          // pair k of round r: (r, 31) for k = 0, (r + k, r - k) mod 31 otherwise
          int p = r, q = kJ - 1;
          if (tid > 0) {
            p = r + tid;
            p = p >= kJ - 1 ? p - (kJ - 1) : p;
            q = r - tid;
            q = q < 0 ? q + (kJ - 1) : q;
          }
          const int lo = min(p, q), hi = max(p, q);
          const float app = S.A[buf][lo][lo], aqq = S.A[buf][hi][hi], apq = S.A[buf][lo][hi];
          float c = 1.f, ss = 0.f, tt = 0.f;
          // the relative test |apq| > u sqrt(|app aqq|) squared; the rotation from
          // MUFU reciprocals and square roots (FP32 level is all it needs)
          if (apq != 0.f && apq * apq > (kJTol * kJTol) * fabsf(app * aqq)) {
            const float zeta = __fdividef(aqq - app, 2.f * apq);
            const float y = fmaf(zeta, zeta, 1.f);
            tt = copysignf(__fdividef(1.f, fabsf(zeta) + y * rsqrtf(y)), zeta);
            c = rsqrtf(fmaf(tt, tt, 1.f));
            ss = tt * c;
            S.rot[sweep & 1] = 1;
          }
          // per index: (c, signed coefficient of the partner); t signed so that the
          // diagonal update is a_ii + t_i a_{lo,hi} for both members of the pair
          S.cs[lo] = make_float2(c, -ss);
          S.cs[hi] = make_float2(c, ss);
          S.t[lo] = -tt;
          S.t[hi] = tt;
        }
        jac_bar();
        const int pj = jac_partner(j, r);
        const float2 csj = S.cs[j];
        if (tid >= kJacThreads / 2) {
          // Y <- Y J: column j mixes with its partner's
          float y0[kJ / 8], y1[kJ / 8];
#pragma unroll
          for (int k = 0; k < kJ / 8; ++k) {
            y0[k] = S.Y[buf][wj + 8 * k][j];
            y1[k] = S.Y[buf][wj + 8 * k][pj];
          }
#pragma unroll
          for (int k = 0; k < kJ / 8; ++k) S.Y[buf ^ 1][wj + 8 * k][j] = fmaf(csj.x, y0[k], csj.y * y1[k]);
        } else {
          const float(*Ab)[kJP] = S.A[buf];
          float aij[kJ / 8], aipj[kJ / 8], apij[kJ / 8], apipj[kJ / 8], ti[kJ / 8];
          float2 csi[kJ / 8];
          int pi[kJ / 8];
#pragma unroll
          for (int k = 0; k < kJ / 8; ++k) {
            const int ii = wj + 8 * k;
            pi[k] = jac_partner(ii, r);
            csi[k] = S.cs[ii];
            ti[k] = S.t[ii];
            aij[k] = Ab[ii][j];
            aipj[k] = Ab[ii][pj];
            apij[k] = Ab[pi[k]][j];
            apipj[k] = Ab[pi[k]][pj];
          }
#pragma unroll
          for (int k = 0; k < kJ / 8; ++k) {
            const int ii = wj + 8 * k;
            // general entry of J^T A J; the two entries of a rotated pair's 2 x 2 block
            // on the diagonal take the accurate update a_ii + t_i a_lo,hi, the
            // off-diagonal pair entries become 0 (branch-free selects)
            const float gen = csi[k].x * (csj.x * aij[k] + csj.y * aipj[k]) +
                              csi[k].y * (csj.x * apij[k] + csj.y * apipj[k]);
            const float apq = (ii < pi[k]) ? aipj[k] : apij[k];  // a_{lo,hi} of ii's pair, used when ii == j
            float anew = (ii == j) ? fmaf(ti[k], apq, aij[k]) : gen;
            anew = (j == pi[k] && ti[k] != 0.f) ? 0.f : anew;
            S.A[buf ^ 1][ii][j] = anew;
          }
        }
        buf ^= 1;
        jac_bar();
      }
      if (S.rot[sweep & 1] == 0) break;
    }
    if (tid == 0) S.buf = buf;
  }
  __syncthreads();
  const int buf = S.buf;
  // ---- 2. sort the Ritz values (descending; padding last)
  if (tid < kJ) {
    const float th = (tid < K) ? S.A[buf][tid][tid] : -INFINITY;
    int rank = 0;
    for (int k = 0; k < kJ; ++k) {
      const float tk = (k < K) ? S.A[buf][k][k] : -INFINITY;
      rank += (tk > th) || (tk == th && k < tid);
    }
    S.perm[rank] = tid;
  }
  __syncthreads();
  // ---- 3. one first-order correction of the vectors (FP32): with Y sorted,
  // B' = Y^T B Y, F_ij = B'_ij / (B'_jj - B'_ii) for pairs whose Ritz values
  // differ by more than 1 % (closer pairs only mix inside the pair), Y <- Y (I + F).
  // After kJSweeps sweeps the off-diagonal of B' is ~1e-4 of its graded scale, so
  // one correction brings the vectors to what further sweeps would give.
  {
    const int pjx = S.perm[j];
    S.A[buf ^ 1][i][j] = (i < K && j < K) ? S.Y[buf][i][pjx] : 0.f;  // sorted Y (FP32) in the spare buffer
  }
  __syncthreads();
  float (*Ys)[kJP] = S.A[buf ^ 1];
  float (*Zs)[kJP] = S.Y[buf ^ 1];
  {
    float z = 0.f;  // (B Y)_ij
    for (int k = 0; k < K; ++k) z = fmaf(S.Bd[i][k].hi, Ys[k][j], z);
    Zs[i][j] = z;
  }
  __syncthreads();
  {
    float bp = 0.f;  // (Y^T B Y)_ij
    for (int k = 0; k < K; ++k) bp = fmaf(Ys[k][i], Zs[k][j], bp);
    S.Y[buf][i][j] = bp;  // the unsorted Y is no longer needed
  }
  __syncthreads();
  {
    float (*Bp)[kJP] = S.Y[buf];
    const float di = Bp[i][i], dj = Bp[j][j];
    float f = 0.f;
    if (i != j && i < K && j < K && fabsf(dj - di) > 1e-2f * fmaxf(fabsf(di), fabsf(dj))) f = Bp[i][j] / (dj - di);
    __syncthreads();
    Zs[i][j] = f;  // F
  }
  __syncthreads();
  {
    float y = Ys[i][j];
    for (int k = 0; k < K; ++k) y = fmaf(Ys[i][k], Zs[k][j], y);
    S.Yd[i][j] = (i < K && j < K) ? ddf(y) : ddf(0.f);
  }
  __syncthreads();
  // ---- 4. Newton-Schulz: Y <- Y - Y E / 2, E = Y^T Y - I in double-float
  for (int it = 0; it < 2; ++it) {
    // E_ij = sum_k y_ki y_kj - delta_ij (thread (i, j))
    dd e = ddf(0.f);
    if (i < K && j < K) {
      for (int k = 0; k < K; ++k) e = dd_add(e, dd_mul(S.Yd[k][i], S.Yd[k][j]));
      if (i == j) e = dd_sub(e, ddf(1.f));
    }
    S.Md[i][j] = e;
    __syncthreads();
    // y_ij -= (sum_k y_ik E_kj) / 2 in FP32 (the correction is ~1e-6 of y, then ~1e-12)
    float corr = 0.f;
    if (i < K && j < K)
      for (int k = 0; k < K; ++k) corr = fmaf(S.Yd[i][k].hi, S.Md[k][j].hi, corr);
    __syncthreads();
    if (i < K && j < K) S.Yd[i][j] = dd_sub(S.Yd[i][j], ddf(0.5f * corr));
    __syncthreads();
  }
  // ---- 5. Rayleigh quotients theta_j = y_j^T B y_j (B scaled, double-float)
  {
    dd z = ddf(0.f);
    if (i < K && j < K)
      for (int k = 0; k < K; ++k) z = dd_add(z, dd_mul(S.Bd[i][k], S.Yd[k][j]));
    S.Md[i][j] = z;  // (B Y)_ij
  }
  __syncthreads();
  {
    // warp w sums column w over the rows (lane = row)
    dd q = (lane < K && warp < K) ? dd_mul(S.Yd[lane][warp], S.Md[lane][warp]) : ddf(0.f);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) q = dd_add(q, jd_shfl(q, o));
    if (lane == 0) S.theta[warp] = (warp < K) ? dd_to(q) * pow2d(ex) : 0.0;
  }
  __syncthreads();
  // ---- 6. provisional rank and convergence test (FP64, warp 0)
  if (tid < K) theta_out[tid] = S.theta[tid];
  if (warp == 0) {
    const double trs = *trace_g;
    double t0 = (lane < K) ? S.theta[lane] : 0.0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const double u0 = __shfl_up_sync(0xffffffffu, t0, o);
      if (lane >= o) t0 += u0;
    }
    const unsigned b0 = __ballot_sync(0xffffffffu, lane < K && fmax(0.0, trs - t0) <= budget);
    if (lane == 0) {
      const int rp = b0 ? __ffs(b0) : -1;
      int ok = 0;
      const int nv = rp + extra;
      if (rp >= 1 && rp < n && nv <= nmax && S.theta[rp - 1] > 0.0) {
        const double ratio = fabs(S.theta[K - 1]) / S.theta[rp - 1];
        double pw = 1.0;
        for (int t = 0; t < T; ++t) pw *= ratio;
        ok = pw <= conv;
      }
      decision[0] = rp;
      decision[1] = ok ? nv : 0;
      decision[2] = ok;
      decision[3] = tc_err ? *tc_err : 0;
      S.nv = ok ? nv : 0;
    }
  }
  __syncthreads();
  const int nv = S.nv;
  if (i < K && j < nv) Y_out[(size_t)i * nv + j] = dd_to(S.Yd[i][j]);
}

}  // namespace

size_t rr_smem_bytes(int K, int nmax) {
  (void)K;
  (void)nmax;
  return sizeof(JacShared);
}

int launch_rr_small(const double* B, int K, int n, const double* trace_dev, double budget, int extra, int nmax,
                    double conv, int T, const int* tc_err, double* theta_dev, int* decision_dev, double* Y_dev,
                    cudaStream_t s) {
  if (K < 1 || K > kJ || nmax < 1 || nmax > K)
    return fail(ATC_EINVAL, "Rayleigh-Ritz solver: K = %d, nmax = %d unsupported", K, nmax);
  const size_t smem = sizeof(JacShared);
  static bool attr = false;
  if (!attr) {
    ATC_CUDA_TRY(cudaFuncSetAttribute(rr_jacobi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr = true;
  }
  // work of a K x K symmetric eigendecomposition with vectors, ~9 K^3 FLOPs
  KTimed kt_(s, "rr_jacobi_kernel", (double)K * K * 8.0 * 2.0, 9.0 * (double)K * K * K);
  rr_jacobi_kernel<<<1, kJThreads, smem, s>>>(B, K, n, trace_dev, budget, extra, nmax, conv, T, tc_err, theta_dev,
                                              decision_dev, Y_dev);
  ATC_LAUNCHED(1);
  return ATC_OK;
}

}  // namespace atc
