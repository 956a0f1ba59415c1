// Plain FP64 SIMT contractions: the mode Gram matrix and the mode-k product.
//
// These are the "plain FP64" path: every product and every sum in FP64 (DFMA).
// Both read the tensor through the (L, n, R) view of Section 3.1 -- the
// mode-k unfolding is formed by index arithmetic, never by a transpose.
//
//   Gram:  G[i][j] = sum_{l,c} X[l][i][c] X[l][j][c]      (only i-tile <= j-tile
//          is computed; split-K partials are summed in a fixed order)
//   TTM :  Y[l][a][c] = sum_b W[a][b] X[l][b][c]          (W = U^T or U)
#include <stdint.h>

#include <mutex>

#include "atc_internal.cuh"

namespace atc {
namespace {

constexpr int TM = 64, TN = 64, TK = 16;
constexpr int kThreads = 256;

template <typename T>
__device__ __forceinline__ double ld(const T* p) { return (double)__ldg(p); }

// Element (row i, column kappa) of the mode unfolding of an (L, n, R) tensor.
__device__ __forceinline__ int64_t unfold_off(int64_t i, int64_t kappa, int64_t n, int64_t R) {
  int64_t l = kappa / R, c = kappa - l * R;
  return (l * n + i) * R + c;
}

template <typename T>
__global__ void __launch_bounds__(kThreads) gram_fp64_kernel(const T* __restrict__ x, int64_t n, int64_t R,
                                                             int64_t K, int64_t kchunk, int ntile,
                                                             double* __restrict__ part) {
  __shared__ double As[TK][TM + 1];
  __shared__ double Bs[TK][TN + 1];
  // decode the upper-triangular tile pair (ti <= tj)
  int t = blockIdx.x, ti = 0;
  while (t >= ntile - ti) { t -= ntile - ti; ++ti; }
  const int tj = ti + t;
  const int64_t i0 = (int64_t)ti * TM, j0 = (int64_t)tj * TN;
  const int64_t k_begin = (int64_t)blockIdx.y * kchunk;
  const int64_t k_end = min(K, k_begin + kchunk);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
  const bool kfast = R >= TK;
  for (int64_t k0 = k_begin; k0 < k_end; k0 += TK) {
#pragma unroll
    for (int e = 0; e < (TM * TK) / kThreads; ++e) {
      int idx = threadIdx.x + e * kThreads;
      int rr, kk;
      if (kfast) { kk = idx % TK; rr = idx / TK; } else { rr = idx % TM; kk = idx / TM; }
      int64_t kappa = k0 + kk;
      double va = 0.0, vb = 0.0;
      if (kappa < k_end) {
        if (i0 + rr < n) va = ld(x + unfold_off(i0 + rr, kappa, n, R));
        if (j0 + rr < n) vb = ld(x + unfold_off(j0 + rr, kappa, n, R));
      }
      As[kk][rr] = va;
      Bs[kk][rr] = vb;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) { a[q] = As[kk][ty + 16 * q]; b[q] = Bs[kk][tx + 16 * q]; }
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] = fma(a[p], b[q], acc[p][q]);
    }
    __syncthreads();
  }
  double* out = part + (int64_t)blockIdx.y * n * n;
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    int64_t i = i0 + ty + 16 * p;
    if (i >= n) continue;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int64_t j = j0 + tx + 16 * q;
      if (j < n) out[i * n + j] = acc[p][q];
    }
  }
}

// G[i][j] = G[j][i] = sum_s part[s][min-tile entry], summed in split order.
__global__ void gram_reduce_kernel(const double* __restrict__ part, int nsplit, int64_t n, double* __restrict__ g) {
  int64_t total = n * n;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = idx / n, j = idx - i * n;
    // the computed entry lives in the upper tile (tile(i) <= tile(j)) -- pick the
    // orientation whose row tile is <= its column tile
    int64_t si = i, sj = j;
    if (i / TM > j / TN) { si = j; sj = i; }
    double acc = 0.0;
    for (int s = 0; s < nsplit; ++s) acc += part[(int64_t)s * n * n + si * n + sj];
    g[idx] = acc;
  }
}

template <typename TX, typename TY>
__global__ void __launch_bounds__(kThreads) ttm_fp64_kernel(const TX* __restrict__ x, const double* __restrict__ w,
                                                            int64_t wsa, int64_t wsb, int64_t A, int64_t B,
                                                            int64_t R, int64_t N, TY* __restrict__ y) {
  __shared__ double Ws[TK][TM + 1];
  __shared__ double Xs[TK][TN + 1];
  const int64_t a0 = (int64_t)blockIdx.y * TM, g0 = (int64_t)blockIdx.x * TN;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[4][4];
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[p][q] = 0.0;
  for (int64_t b0 = 0; b0 < B; b0 += TK) {
#pragma unroll
    for (int e = 0; e < (TM * TK) / kThreads; ++e) {
      int idx = threadIdx.x + e * kThreads;
      // W tile: rows a, columns b
      int aa = idx / TK, bb = idx % TK;
      double wv = 0.0;
      if (a0 + aa < A && b0 + bb < B) wv = w[(a0 + aa) * wsa + (b0 + bb) * wsb];
      Ws[bb][aa] = wv;
      // X tile: rows b, columns gamma (gamma fastest for coalescing)
      int gg = idx % TN, bx = idx / TN;
      double xv = 0.0;
      int64_t gamma = g0 + gg, b = b0 + bx;
      if (gamma < N && b < B) {
        int64_t l = gamma / R, c = gamma - l * R;
        xv = (double)__ldg(x + (l * B + b) * R + c);
      }
      Xs[bx][gg] = xv;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) { a[q] = Ws[kk][ty + 16 * q]; b[q] = Xs[kk][tx + 16 * q]; }
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] = fma(a[p], b[q], acc[p][q]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    int64_t a = a0 + ty + 16 * p;
    if (a >= A) continue;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int64_t gamma = g0 + tx + 16 * q;
      if (gamma >= N) continue;
      int64_t l = gamma / R, c = gamma - l * R;
      y[(l * A + a) * R + c] = (TY)acc[p][q];
    }
  }
}

// Cross Gram of two tensors that share all modes but one:
//   C[i][j] = sum_{l,c} A[l][i][c] B[l][j][c],   A viewed (L, n, R), B viewed (L, m, R)
// (the factor gradient of the Tucker expansion).  Full n x m tiling, split-K
// partials in part[split][n][m], FP64 accumulation.
template <typename TA, typename TB>
__global__ void __launch_bounds__(kThreads) cross_gram_fp64_kernel(const TA* __restrict__ a, const TB* __restrict__ b,
                                                                   int64_t n, int64_t m, int64_t R, int64_t K,
                                                                   int64_t kchunk, int ntm, double* __restrict__ part) {
  __shared__ double As[TK][TM + 1];
  __shared__ double Bs[TK][TN + 1];
  const int ti = blockIdx.x / ntm, tj = blockIdx.x % ntm;
  const int64_t i0 = (int64_t)ti * TM, j0 = (int64_t)tj * TN;
  const int64_t k_begin = (int64_t)blockIdx.y * kchunk;
  const int64_t k_end = min(K, k_begin + kchunk);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[4][4];
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[p][q] = 0.0;
  const bool kfast = R >= TK;
  for (int64_t k0 = k_begin; k0 < k_end; k0 += TK) {
#pragma unroll
    for (int e = 0; e < (TM * TK) / kThreads; ++e) {
      const int idx = threadIdx.x + e * kThreads;
      int rr, kk;
      if (kfast) { kk = idx % TK; rr = idx / TK; } else { rr = idx % TM; kk = idx / TM; }
      const int64_t kappa = k0 + kk;
      double va = 0.0, vb = 0.0;
      if (kappa < k_end) {
        if (i0 + rr < n) va = ld(a + unfold_off(i0 + rr, kappa, n, R));
        if (j0 + rr < m) vb = ld(b + unfold_off(j0 + rr, kappa, m, R));
      }
      As[kk][rr] = va;
      Bs[kk][rr] = vb;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
      double av[4], bv[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) { av[q] = As[kk][ty + 16 * q]; bv[q] = Bs[kk][tx + 16 * q]; }
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] = fma(av[p], bv[q], acc[p][q]);
    }
    __syncthreads();
  }
  double* out = part + (int64_t)blockIdx.y * n * m;
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const int64_t i = i0 + ty + 16 * p;
    if (i >= n) continue;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int64_t j = j0 + tx + 16 * q;
      if (j < m) out[i * m + j] = acc[p][q];
    }
  }
}

__global__ void sum_splits_kernel(const double* __restrict__ part, int nsplit, int64_t total, double* __restrict__ c) {
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int s = 0; s < nsplit; ++s) acc += part[(int64_t)s * total + idx];
    c[idx] = acc;
  }
}

}  // namespace

int launch_gram_fp64(const void* x, int dtype, int64_t L, int64_t n, int64_t R, double* g, cudaStream_t s) {
  const int64_t K = L * R;
  const int ntile = (int)((n + TM - 1) / TM);
  const int npairs = ntile * (ntile + 1) / 2;
  // split K so that the grid covers the GPU a few times over
  int64_t nsplit = (4 * 152 + npairs - 1) / npairs;
  int64_t maxsplit = (K + 255) / 256;
  if (nsplit > maxsplit) nsplit = maxsplit;
  // keep the partial buffer within 64 MB
  while (nsplit > 1 && nsplit * n * n * 8 > (64ll << 20)) nsplit--;
  if (nsplit < 1) nsplit = 1;
  int64_t kchunk = (K + nsplit - 1) / nsplit;
  kchunk = (kchunk + TK - 1) / TK * TK;
  nsplit = (K + kchunk - 1) / kchunk;
  if (nsplit < 1) nsplit = 1;
  double* part = nullptr;
  ATC_TRY(Scratch::get(SLOT_GRAM_PART, sizeof(double) * nsplit * n * n, (void**)&part));
  dim3 grid(npairs, (unsigned)nsplit);
  {
    KTimed kt_(s, "gram_fp64_kernel", (double)n * (double)K * (dtype == ATC_F32 ? 4.0 : 8.0) +
                                          (double)nsplit * (double)n * (double)n * 8.0,
               (double)n * (double)n * (double)K);
    if (dtype == ATC_F32)
      gram_fp64_kernel<float><<<grid, kThreads, 0, s>>>((const float*)x, n, R, K, kchunk, ntile, part);
    else
      gram_fp64_kernel<double><<<grid, kThreads, 0, s>>>((const double*)x, n, R, K, kchunk, ntile, part);
  }
  ATC_LAUNCHED(1);
  int64_t tot = n * n;
  int blocks = (int)((tot + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  gram_reduce_kernel<<<blocks, 256, 0, s>>>(part, (int)nsplit, n, g);
  ATC_LAUNCHED(1);
  return ATC_OK;
}

int launch_cross_gram_fp64(const void* a, int adt, const void* b, int bdt, int64_t L, int64_t n, int64_t m,
                           int64_t R, double* c, cudaStream_t s) {
  const int64_t K = L * R;
  const int ntn = (int)((n + TM - 1) / TM), ntm = (int)((m + TN - 1) / TN);
  const int ntiles = ntn * ntm;
  int64_t nsplit = (4 * 152 + ntiles - 1) / ntiles;
  const int64_t maxsplit = (K + 255) / 256;
  if (nsplit > maxsplit) nsplit = maxsplit;
  while (nsplit > 1 && nsplit * n * m * 8 > (64ll << 20)) nsplit--;
  if (nsplit < 1) nsplit = 1;
  int64_t kchunk = (K + nsplit - 1) / nsplit;
  kchunk = (kchunk + TK - 1) / TK * TK;
  if (kchunk < TK) kchunk = TK;
  nsplit = (K + kchunk - 1) / kchunk;
  if (nsplit < 1) nsplit = 1;
  double* part = nullptr;
  ATC_TRY(Scratch::get(SLOT_GRAM_PART, sizeof(double) * nsplit * n * m + 64, (void**)&part));
  const dim3 grid((unsigned)ntiles, (unsigned)nsplit);
  if (adt == ATC_F32 && bdt == ATC_F32)
    cross_gram_fp64_kernel<float, float><<<grid, kThreads, 0, s>>>((const float*)a, (const float*)b, n, m, R, K, kchunk, ntm, part);
  else if (adt == ATC_F32)
    cross_gram_fp64_kernel<float, double><<<grid, kThreads, 0, s>>>((const float*)a, (const double*)b, n, m, R, K, kchunk, ntm, part);
  else if (bdt == ATC_F32)
    cross_gram_fp64_kernel<double, float><<<grid, kThreads, 0, s>>>((const double*)a, (const float*)b, n, m, R, K, kchunk, ntm, part);
  else
    cross_gram_fp64_kernel<double, double><<<grid, kThreads, 0, s>>>((const double*)a, (const double*)b, n, m, R, K, kchunk, ntm, part);
  ATC_LAUNCHED(1);
  const int64_t tot = n * m;
  int blocks = (int)((tot + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  sum_splits_kernel<<<blocks, 256, 0, s>>>(part, (int)nsplit, tot, c);
  ATC_LAUNCHED(1);
  return ATC_OK;
}

int launch_ttm_fp64(const void* x, int xdtype, int64_t L, int64_t n, int64_t R, const double* u, int64_t r,
                    int expand, void* y, int ydtype, cudaStream_t s) {
  // project: A = r, B = n, W[a][b] = U[b][a]  -> wsa = 1, wsb = r
  // expand : A = n, B = r, W[a][b] = U[a][b]  -> wsa = r, wsb = 1
  const int64_t A = expand ? n : r, B = expand ? r : n;
  const int64_t wsa = expand ? r : 1, wsb = expand ? 1 : r;
  const int64_t N = L * R;
  if (N == 0 || A == 0) return ATC_OK;
  dim3 grid((unsigned)((N + TN - 1) / TN), (unsigned)((A + TM - 1) / TM));
  if (grid.y > 65535) return fail(ATC_EUNSUP, "ttm: output mode too large");
  KTimed kt_(s, "ttm_fp64_kernel",
             (double)N * (double)B * (xdtype == ATC_F32 ? 4.0 : 8.0) + (double)N * (double)A * (ydtype == ATC_F32 ? 4.0 : 8.0) +
                 (double)A * (double)B * 8.0,
             2.0 * (double)N * (double)A * (double)B);
  if (xdtype == ATC_F32 && ydtype == ATC_F32)
    ttm_fp64_kernel<float, float><<<grid, kThreads, 0, s>>>((const float*)x, u, wsa, wsb, A, B, R, N, (float*)y);
  else if (xdtype == ATC_F32 && ydtype == ATC_F64)
    ttm_fp64_kernel<float, double><<<grid, kThreads, 0, s>>>((const float*)x, u, wsa, wsb, A, B, R, N, (double*)y);
  else if (xdtype == ATC_F64 && ydtype == ATC_F32)
    ttm_fp64_kernel<double, float><<<grid, kThreads, 0, s>>>((const double*)x, u, wsa, wsb, A, B, R, N, (float*)y);
  else
    ttm_fp64_kernel<double, double><<<grid, kThreads, 0, s>>>((const double*)x, u, wsa, wsb, A, B, R, N, (double*)y);
  ATC_LAUNCHED(1);
  return ATC_OK;
}


// ---------------------------------------------------------------------------
// Gram matrix without any device allocation.
//
// Some callers cannot call cudaMalloc: real-time paths that must not block on
// the device allocator (cudaMalloc can synchronise the device), or hosts that
// hand this library a fixed memory budget and account for every byte it may
// take.  For them the split-K partial sums of the FP64 Gram kernel live in the
// file-scope device array below instead of the cached scratch arena.  Every
// GPU that loads this library holds the array (4 MiB) until the process exits.
namespace {
constexpr size_t kNoAllocDoubles = (size_t)1 << 19;  // 4 MiB of FP64 partial sums
constexpr int64_t kNoAllocMaxN = 724;                // largest n with n * n <= kNoAllocDoubles
static_assert(kNoAllocMaxN * kNoAllocMaxN <= (int64_t)kNoAllocDoubles &&
                  (kNoAllocMaxN + 1) * (kNoAllocMaxN + 1) > (int64_t)kNoAllocDoubles,
              "no-allocation limit");
__device__ __align__(256) double g_noalloc_part[kNoAllocDoubles];
constexpr int kMaxDevices = 64;
double* g_noalloc_ptr[kMaxDevices] = {};  // device address of g_noalloc_part, per device
std::mutex g_noalloc_mu;
}  // namespace

// Forget the looked-up address of the no-allocation array on `dev` (called
// where the library drops its per-device state: after a device reset the
// module is loaded again and the array may sit at another address).
void noalloc_forget(int dev) {
  if (dev < 0 || dev >= kMaxDevices) return;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  g_noalloc_ptr[dev] = nullptr;
}

}  // namespace atc

extern "C" int atc_gram_fp64_noalloc(const void* x_dev, int dtype, int64_t L, int64_t n, int64_t R, double* g_dev,
                                     void* stream) {
  using namespace atc;
  if (!x_dev || !g_dev || L < 1 || n < 1 || R < 1 || (dtype != ATC_F32 && dtype != ATC_F64))
    return fail(ATC_EINVAL, "atc_gram_fp64_noalloc: bad arguments");
  // n is checked on its own before any product is formed (n * n could wrap)
  if (n > kNoAllocMaxN)
    return fail(ATC_EINVAL, "atc_gram_fp64_noalloc: n = %lld exceeds the no-allocation maximum (n <= %lld)",
                (long long)n, (long long)kNoAllocMaxN);
  // every element index l n R + i R + c must fit in int64
  if (L > INT64_MAX / R || L * R > (INT64_MAX / 2) / n)
    return fail(ATC_EINVAL, "atc_gram_fp64_noalloc: L * n * R overflows");
  int dev = 0;
  ATC_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(ATC_EUNSUP, "atc_gram_fp64_noalloc: device index %d", dev);
  double* part = nullptr;
  {
    // one-time set-up per device, with that device current: the host-side
    // name of the array is not a device address, so ask the runtime for it
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_part);
      if (e != cudaSuccess)
        return fail(ATC_ECUDA, "cudaGetSymbolAddress(no-allocation scratch): %s", cudaGetErrorString(e));
      g_noalloc_ptr[dev] = static_cast<double*>(p);
    }
    part = g_noalloc_ptr[dev];
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t K = L * R;
  const int ntile = (int)((n + TM - 1) / TM);
  const int npairs = ntile * (ntile + 1) / 2;
  int64_t nsplit = (4 * 152 + npairs - 1) / npairs;
  const int64_t maxsplit = (K + 255) / 256;
  if (nsplit > maxsplit) nsplit = maxsplit;
  const int64_t cap = (int64_t)(kNoAllocDoubles / ((size_t)n * (size_t)n));
  if (nsplit > cap) nsplit = cap;
  if (nsplit < 1) nsplit = 1;
  int64_t kchunk = (K + nsplit - 1) / nsplit;
  kchunk = (kchunk + TK - 1) / TK * TK;
  nsplit = (K + kchunk - 1) / kchunk;
  if (nsplit < 1) nsplit = 1;
  // every entry the reduction reads (upper tiles of each split) is written by
  // the Gram kernel of this call, so the array needs no clearing
  dim3 grid(npairs, (unsigned)nsplit);
  if (dtype == ATC_F32)
    gram_fp64_kernel<float><<<grid, kThreads, 0, s>>>((const float*)x_dev, n, R, K, kchunk, ntile, part);
  else
    gram_fp64_kernel<double><<<grid, kThreads, 0, s>>>((const double*)x_dev, n, R, K, kchunk, ntile, part);
  ATC_LAUNCHED(1);
  const int64_t tot = n * n;
  int blocks = (int)((tot + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  gram_reduce_kernel<<<blocks, 256, 0, s>>>(part, (int)nsplit, n, g_dev);
  ATC_LAUNCHED(1);
  return ATC_OK;
}

