// Norms, conversions and the core permutation.
//
// ||X||^2 (Section 3.1, Euclidean norm) is accumulated in FP64 with a fixed
// grid and a fixed reduction tree, so the result does not depend on timing.
#include <stdint.h>

#include "atc_internal.cuh"

namespace atc {
namespace {

constexpr int kNormBlocks = 1216;  // 8 x 152 SMs
constexpr int kNormThreads = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double block_sum(double v, double* sh) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  if (w == 0) {
    t = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : 0.0;
    t = warp_sum(t);
  }
  __syncthreads();
  return t;
}

// exact square of an FP32 value as a float pair, added to the double-float (hi, lo)
__device__ __forceinline__ void sq_acc(float v, float& hi, float& lo) {
  const float p = v * v;
  const float e = fmaf(v, v, -p);
  const float s = hi + p;
  const float bp = s - hi;
  lo += ((hi - (s - bp)) + (p - bp)) + e;
  hi = s;
}

// Partial sums of x^2 per CTA; with mx_bits != nullptr also max |x| (as float
// bits, atomicMax: non-negative floats order like their bit patterns), the
// slice scale of the same tensor in the same pass.
template <typename T>
__global__ void __launch_bounds__(kNormThreads) norm2_partial(const T* __restrict__ x, int64_t n,
                                                               double* __restrict__ part, unsigned* __restrict__ mx_bits) {
  __shared__ double sh[32];
  double acc = 0.0;
  float mx = 0.f;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t done = 0;
  if (sizeof(T) == 4 && ((uintptr_t)x & 15) == 0) {
    // FP32 input: every square is exact as a float pair (v*v, fma(v, v, -v*v)).
    // Four float4 loads in flight a thread; their sixteen squares are summed as
    // a double-float on the FP32 pipes and each group of sixteen is added into
    // the FP64 accumulator (GB300 issues FP64 at 1/64 of the FP32 rate, which
    // would otherwise bound this HBM pass).
    const int64_t n4 = n / 4;
    const float4* x4 = reinterpret_cast<const float4*>(x);
    int64_t i = t0;
    for (; i + 3 * stride < n4; i += 4 * stride) {
      float4 v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) v[u] = __ldg(x4 + i + u * stride);
      float hi = 0.f, lo = 0.f;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        sq_acc(v[u].x, hi, lo);
        sq_acc(v[u].y, hi, lo);
        sq_acc(v[u].z, hi, lo);
        sq_acc(v[u].w, hi, lo);
        mx = fmaxf(mx, fmaxf(fmaxf(fabsf(v[u].x), fabsf(v[u].y)), fmaxf(fabsf(v[u].z), fabsf(v[u].w))));
      }
      acc += (double)hi + (double)lo;
    }
    for (; i < n4; i += stride) {
      const float4 v = __ldg(x4 + i);
      float hi = 0.f, lo = 0.f;
      sq_acc(v.x, hi, lo);
      sq_acc(v.y, hi, lo);
      sq_acc(v.z, hi, lo);
      sq_acc(v.w, hi, lo);
      mx = fmaxf(mx, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
      acc += (double)hi + (double)lo;
    }
    done = n4 * 4;
  }
  for (int64_t i = done + t0; i < n; i += stride) {
    const double v = (double)x[i];
    acc = fma(v, v, acc);
    mx = fmaxf(mx, fabsf((float)x[i]));
  }
  if (mx_bits) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) atomicMax(mx_bits, __float_as_uint(mx));
  }
  double t = block_sum(acc, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

__global__ void __launch_bounds__(kNormThreads) sum_partials(const double* __restrict__ part, int np,
                                                             double* __restrict__ out) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) acc += part[i];
  double t = block_sum(acc, sh);
  if (threadIdx.x == 0) *out = t;
}

template <typename T>
__global__ void to_f64(const T* __restrict__ x, int64_t n, double* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = (double)x[i];
}

__global__ void f64_to_f32(const double* __restrict__ x, int64_t n, float* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = (float)x[i];
}

struct PermDesc {
  int ndim;
  int64_t dims[8];     // source dims
  int64_t sstride[8];  // source strides
  int64_t dstride[8];  // destination stride of source axis a
};

// y[dest(idx)] = x[idx]: walk the source in order, scatter with per-axis strides.
__global__ void permute_kernel(const double* __restrict__ x, int64_t total, PermDesc pd, double* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    int64_t rem = i, dst = 0;
    for (int a = pd.ndim - 1; a >= 0; --a) {
      int64_t c = rem % pd.dims[a];
      rem /= pd.dims[a];
      dst += c * pd.dstride[a];
    }
    y[dst] = x[i];
  }
}

int grid_for(int64_t n, int threads) {
  int64_t b = (n + threads - 1) / threads;
  if (b > 152 * 16) b = 152 * 16;
  if (b < 1) b = 1;
  return (int)b;
}

// Rayleigh quotients rho_j = u_j^T G u_j of the columns of U (n x rh,
// row-major) and, in out[rh], trace(G): one CTA per column j stages u_j in
// shared memory; a warp forms (G u_j)_i for one row i at a time (lanes over
// the contiguous row, a fixed butterfly), then a fixed-order block sum.  FP64
// throughout, the same order on every run.
constexpr int kRayThreads = 256;
constexpr int kRayMaxN = 1024;
// CTA (j, c): the part of u_j^T G u_j from rows [c * chunk, (c + 1) * chunk)
// of G, i.e. sum_i u_ij (G u_j)_i over the chunk; CTA (rh, c) sums the
// chunk's diagonal of G instead.  out[j * nsplit + c]; the caller adds the
// nsplit parts of each j in order.
__global__ void __launch_bounds__(kRayThreads) rayleigh_kernel(const double* __restrict__ G, int n,
                                                               const double* __restrict__ U, int rh, int chunk,
                                                               double* __restrict__ out) {
  __shared__ double uj[kRayMaxN];
  __shared__ double sh[32];
  const int j = blockIdx.x, c = blockIdx.y;
  const int r0 = c * chunk, r1 = min(n, r0 + chunk);
  double acc = 0.0;
  if (j == rh) {
    for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) acc += G[(int64_t)i * n + i];
  } else {
    for (int i = threadIdx.x; i < n; i += blockDim.x) uj[i] = U[(int64_t)i * rh + j];
    __syncthreads();
    // four rows per warp at a time: independent FMA chains hide the FP64
    // latency (GB300 issues FP64 at a low rate with a long pipeline)
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int i0 = r0 + 4 * (threadIdx.x >> 5); i0 < r1; i0 += 4 * nw) {
      double w[4] = {0.0, 0.0, 0.0, 0.0};
      for (int k = lane; k < n; k += 32) {
        const double u = uj[k];
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (i0 + q < r1) w[q] = fma(G[(int64_t)(i0 + q) * n + k], u, w[q]);
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const double t = warp_sum(w[q]);
        if (lane == 0 && i0 + q < r1) acc = fma(uj[i0 + q], t, acc);
      }
    }
  }
  const double t = block_sum(acc, sh);
  if (threadIdx.x == 0) out[(int64_t)j * gridDim.y + c] = t;
}

}  // namespace

int rayleigh_splits(int64_t n, int rh) {
  // about two CTAs per SM over the (rh + 1) x nsplit grid, chunks of >= 16 rows
  int ns = (int)((2 * 152 + rh) / (rh + 1));
  const int by_rows = (int)((n + 15) / 16);
  if (ns > by_rows) ns = by_rows;
  if (ns > kRaySplitMax) ns = kRaySplitMax;
  return ns < 1 ? 1 : ns;
}

int launch_rayleigh(const double* G, int64_t n, const double* U, int rh, double* out, cudaStream_t s) {
  if (n < 1 || n > kRayMaxN || rh < 0) return fail(ATC_EINVAL, "launch_rayleigh: bad sizes");
  const int ns = rayleigh_splits(n, rh);
  const int chunk = (int)((n + ns - 1) / ns);
  {
    KTimed kt_(s, "rayleigh_kernel", (double)n * (double)n * 8.0 + (double)n * rh * 8.0,
               2.0 * (double)n * (double)n * rh);
    rayleigh_kernel<<<dim3(rh + 1, ns), kRayThreads, 0, s>>>(G, (int)n, U, rh, chunk, out);
  }
  ATC_LAUNCHED(1);
  return ATC_OK;
}

int launch_norm2(const void* x, int dtype, int64_t n, double* out, cudaStream_t s, unsigned* mx_bits) {
  double* part = nullptr;
  ATC_TRY(Scratch::get(SLOT_SMALL, sizeof(double) * (kNormBlocks + 64), (void**)&part));
  if (dtype == ATC_F32)
    { KTimed kt_(s, "norm2_partial", (double)n * 4.0); norm2_partial<float><<<kNormBlocks, kNormThreads, 0, s>>>((const float*)x, n, part, mx_bits); }
  else
    { KTimed kt_(s, "norm2_partial", (double)n * 8.0); norm2_partial<double><<<kNormBlocks, kNormThreads, 0, s>>>((const double*)x, n, part, mx_bits); }
  ATC_LAUNCHED(1);
  sum_partials<<<1, kNormThreads, 0, s>>>(part, kNormBlocks, out);
  ATC_LAUNCHED(1);
  return ATC_OK;
}

int launch_convert_to_f64(const void* x, int dtype, int64_t n, double* y, cudaStream_t s) {
  if (dtype == ATC_F64) {
    ATC_CUDA_TRY(cudaMemcpyAsync(y, x, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    return ATC_OK;
  }
  to_f64<float><<<grid_for(n, 256), 256, 0, s>>>((const float*)x, n, y);
  ATC_LAUNCHED(1);
  return ATC_OK;
}

int launch_convert_f64_to(const double* x, int64_t n, void* y, int dtype, cudaStream_t s) {
  if (dtype == ATC_F64) {
    if ((const void*)x != y) ATC_CUDA_TRY(cudaMemcpyAsync(y, x, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    return ATC_OK;
  }
  f64_to_f32<<<grid_for(n, 256), 256, 0, s>>>(x, n, (float*)y);
  ATC_LAUNCHED(1);
  return ATC_OK;
}

// inverse == 0: y = transpose(x, perm) (y's axis i is x's axis perm[i]).
// inverse == 1: x is laid out in perm order (dims given in ORIGINAL order), undo it.
int launch_permute(const double* x, const int64_t* dims, const int* perm, int ndim, double* y, int inverse,
                   cudaStream_t s) {
  PermDesc pd;
  pd.ndim = ndim;
  int64_t total = 1;
  for (int i = 0; i < ndim; ++i) total *= dims[i];
  if (total == 0) return ATC_OK;
  bool ident = true;
  for (int i = 0; i < ndim; ++i) ident = ident && perm[i] == i;
  if (ident) {
    // the identity (equal ranks keep the mode order): a plain device copy
    ATC_CUDA_TRY(cudaMemcpyAsync(y, x, sizeof(double) * (size_t)total, cudaMemcpyDeviceToDevice, s));
    return ATC_OK;
  }
  // permuted dims: pdims[i] = dims[perm[i]]
  int64_t pdims[8], pstride[8], ostride[8];
  for (int i = 0; i < ndim; ++i) pdims[i] = dims[perm[i]];
  int64_t acc = 1;
  for (int i = ndim - 1; i >= 0; --i) { pstride[i] = acc; acc *= pdims[i]; }
  acc = 1;
  for (int i = ndim - 1; i >= 0; --i) { ostride[i] = acc; acc *= dims[i]; }
  if (!inverse) {
    // source = original layout; original axis perm[i] goes to permuted position i
    for (int a = 0; a < ndim; ++a) pd.dims[a] = dims[a];
    for (int i = 0; i < ndim; ++i) pd.dstride[perm[i]] = pstride[i];
  } else {
    // source = permuted layout; permuted axis i is original axis perm[i]
    for (int i = 0; i < ndim; ++i) { pd.dims[i] = pdims[i]; pd.dstride[i] = ostride[perm[i]]; }
  }
  permute_kernel<<<grid_for(total, 256), 256, 0, s>>>(x, total, pd, y);
  ATC_LAUNCHED(1);
  return ATC_OK;
}

}  // namespace atc
