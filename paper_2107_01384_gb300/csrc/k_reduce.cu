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

template <typename T>
__global__ void __launch_bounds__(kNormThreads) norm2_partial(const T* __restrict__ x, int64_t n,
                                                               double* __restrict__ part) {
  __shared__ double sh[32];
  double acc = 0.0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  if (sizeof(T) == 4 && ((uintptr_t)x & 15) == 0) {
    // FP32 input: every square is exact as a float pair (v*v, fma(v, v, -v*v));
    // four of them are summed as a double-float on the FP32 pipes and each
    // group of four is added into the FP64 accumulator (GB300 issues FP64 at
    // 1/64 of the FP32 rate, which would otherwise bound this HBM pass).
    const int64_t n4 = n / 4;
    const float4* x4 = reinterpret_cast<const float4*>(x);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n4; i += stride) {
      const float4 v = __ldg(x4 + i);
      const float q[4] = {v.x, v.y, v.z, v.w};
      float hi = 0.f, lo = 0.f;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float p = q[k] * q[k];
        const float e = fmaf(q[k], q[k], -p);
        const float s = hi + p;
        const float bp = s - hi;
        lo += ((hi - (s - bp)) + (p - bp)) + e;
        hi = s;
      }
      acc += (double)hi + (double)lo;
    }
    for (int64_t i = n4 * 4 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) {
      double v = (double)x[i];
      acc = fma(v, v, acc);
    }
  } else {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) {
      double v = (double)x[i];
      acc = fma(v, v, acc);
    }
  }
  double t = block_sum(acc, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// sum_i (x_i - z_i)^2 for the tensor x (FP32 or FP64) and its reproduction z
// (FP32): each difference is taken in the precision of x and rounded to FP32,
// its square is an exact float pair, four squares are summed as a double-float
// and added into the FP64 accumulator (the FP32 pipes carry the work; GB300
// issues FP64 at 1/64 of their rate).  Fixed grid and reduction tree.
__device__ __forceinline__ void dd_acc_sq(float d, float& hi, float& lo) {
  const float p = d * d;
  const float e = fmaf(d, d, -p);
  const float s = hi + p;
  const float bp = s - hi;
  lo += ((hi - (s - bp)) + (p - bp)) + e;
  hi = s;
}
template <typename T>
__global__ void __launch_bounds__(kNormThreads) diff2_partial(const T* __restrict__ x, const float* __restrict__ z,
                                                               int64_t n, double* __restrict__ part) {
  __shared__ double sh[32];
  double acc = 0.0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t done = 0;
  if (sizeof(T) == 4 && ((uintptr_t)x & 15) == 0 && ((uintptr_t)z & 15) == 0) {
    const int64_t n4 = n / 4;
    const float4* x4 = reinterpret_cast<const float4*>(x);
    const float4* z4 = reinterpret_cast<const float4*>(z);
    for (int64_t i = t0; i < n4; i += stride) {
      const float4 a = __ldg(x4 + i), b = __ldg(z4 + i);
      float hi = 0.f, lo = 0.f;
      dd_acc_sq(a.x - b.x, hi, lo);
      dd_acc_sq(a.y - b.y, hi, lo);
      dd_acc_sq(a.z - b.z, hi, lo);
      dd_acc_sq(a.w - b.w, hi, lo);
      acc += (double)hi + (double)lo;
    }
    done = n4 * 4;
  }
  for (int64_t i = done + t0; i < n; i += stride) {
    float hi = 0.f, lo = 0.f;
    dd_acc_sq((float)((double)x[i] - (double)z[i]), hi, lo);
    acc += (double)hi + (double)lo;
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

// e[j] partials: block (ch, j) sums y[(l r + j) R + c]^2 over its share of
// the (l, c) fibers; the partials are then summed in chunk order.
constexpr int kEnChunks = 64;
__global__ void __launch_bounds__(kNormThreads) row_energy_partial(const float* __restrict__ y, int64_t LR, int64_t r,
                                                                   int64_t R, double* __restrict__ part) {
  __shared__ double sh[32];
  const int64_t j = blockIdx.y;
  const int64_t per = (LR + gridDim.x - 1) / gridDim.x;
  const int64_t g0 = (int64_t)blockIdx.x * per, g1 = min(LR, g0 + per);
  double v = 0.0;
  for (int64_t g = g0 + threadIdx.x; g < g1; g += blockDim.x) {
    const int64_t l = g / R, c = g - l * R;
    const double t = (double)y[(l * r + j) * R + c];
    v = fma(t, t, v);
  }
  v = block_sum(v, sh);
  if (threadIdx.x == 0) part[j * gridDim.x + blockIdx.x] = v;
}
__global__ void row_energy_finish(const double* __restrict__ part, int nch, int64_t r, double* __restrict__ e) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < r; j += (int64_t)gridDim.x * blockDim.x) {
    double v = 0.0;
    for (int c = 0; c < nch; ++c) v += part[j * nch + c];
    e[j] = v;
  }
}
// (L, rh, R) -> (L, r, R), r <= rh: keep the leading r rows of every slab
__global__ void compact_kernel(const float* __restrict__ y, int64_t L, int64_t rh, int64_t R, int64_t r,
                               float* __restrict__ out) {
  const int64_t total = L * r * R;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = i % R, t = i / R, j = t % r, l = t / r;
    out[i] = y[(l * rh + j) * R + c];
  }
}

}  // namespace

int launch_row_energy(const float* y, int64_t L, int64_t r, int64_t R, double* e, cudaStream_t s) {
  if (r <= 0) return ATC_OK;
  if (r > 65535) return fail(ATC_EUNSUP, "row energy: too many rows");
  double* part = nullptr;
  ATC_TRY(Scratch::get(SLOT_ENERGY, sizeof(double) * (size_t)r * kEnChunks + 256, (void**)&part));
  {
    KTimed kt_(s, "row_energy_partial", (double)L * (double)R * (double)r * 4.0);
    row_energy_partial<<<dim3(kEnChunks, (unsigned)r), kNormThreads, 0, s>>>(y, L * R, r, R, part);
  }
  row_energy_finish<<<(unsigned)((r + 255) / 256), 256, 0, s>>>(part, kEnChunks, r, e);
  ATC_LAUNCHED(2);
  return ATC_OK;
}

int launch_compact(const float* y, int64_t L, int64_t rh, int64_t R, int64_t r, float* out, cudaStream_t s) {
  const int64_t total = L * r * R;
  if (total <= 0) return ATC_OK;
  const int blocks = (int)((total + 255) / 256 < 4096 ? (total + 255) / 256 : 4096);
  compact_kernel<<<blocks, 256, 0, s>>>(y, L, rh, R, r, out);
  ATC_LAUNCHED(1);
  return ATC_OK;
}

int launch_norm2(const void* x, int dtype, int64_t n, double* out, cudaStream_t s) {
  double* part = nullptr;
  ATC_TRY(Scratch::get(SLOT_SMALL, sizeof(double) * (kNormBlocks + 64), (void**)&part));
  if (dtype == ATC_F32)
    { KTimed kt_(s, "norm2_partial", (double)n * 4.0); norm2_partial<float><<<kNormBlocks, kNormThreads, 0, s>>>((const float*)x, n, part); }
  else
    { KTimed kt_(s, "norm2_partial", (double)n * 8.0); norm2_partial<double><<<kNormBlocks, kNormThreads, 0, s>>>((const double*)x, n, part); }
  ATC_LAUNCHED(1);
  sum_partials<<<1, kNormThreads, 0, s>>>(part, kNormBlocks, out);
  ATC_LAUNCHED(1);
  return ATC_OK;
}

int launch_diff_norm2(const void* x, int dtype, const float* z, int64_t n, double* out, cudaStream_t s) {
  double* part = nullptr;
  ATC_TRY(Scratch::get(SLOT_RES_PART, sizeof(double) * (kNormBlocks + 64), (void**)&part));
  if (dtype == ATC_F32)
    { KTimed kt_(s, "diff2_partial", (double)n * 8.0); diff2_partial<float><<<kNormBlocks, kNormThreads, 0, s>>>((const float*)x, z, n, part); }
  else
    { KTimed kt_(s, "diff2_partial", (double)n * 12.0); diff2_partial<double><<<kNormBlocks, kNormThreads, 0, s>>>((const double*)x, z, n, part); }
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
