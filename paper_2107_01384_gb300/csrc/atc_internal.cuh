// Internal declarations shared by the translation units of libatc.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/atc.h"

namespace atc {

// Thread-local error message, set by fail().
void set_error(const char* fmt, ...);
int fail(int code, const char* fmt, ...);

#define ATC_CUDA_TRY(expr)                                                              \
  do {                                                                                  \
    cudaError_t _e = (expr);                                                            \
    if (_e != cudaSuccess)                                                              \
      return ::atc::fail(ATC_ECUDA, "%s failed at %s:%d: %s", #expr, __FILE__, __LINE__, \
                         cudaGetErrorString(_e));                                       \
  } while (0)

// Every kernel launch of the library is followed by ATC_LAUNCHED(k): it
// counts the k kernels just launched and checks the launch error.
extern long long g_kernel_launches;
int trace_enabled();
int trace_point(const char* file, int line);
#define ATC_LAUNCHED(k)                                   \
  do {                                                    \
    __atomic_add_fetch(&::atc::g_kernel_launches, (k), __ATOMIC_RELAXED); \
    ATC_CUDA_TRY(cudaGetLastError());                     \
    if (::atc::trace_enabled()) ATC_TRY(::atc::trace_point(__FILE__, __LINE__)); \
  } while (0)

#define ATC_TRY(expr)          \
  do {                         \
    int _rc = (expr);          \
    if (_rc != ATC_OK) return _rc; \
  } while (0)

// Device scratch: a grow-only cached arena per device (cudaMalloc).
extern long long g_scratch_serial;  // changes whenever scratch memory is allocated or freed
struct Scratch {
  // Returns a device pointer to at least `bytes` bytes of slot `slot`, 256-B aligned.
  static int get(int slot, size_t bytes, void** ptr);
  static int release_all();
};

enum ScratchSlot {
  SLOT_GRAM_PART = 0,  // split-K Gram partials
  SLOT_EIG_A,          // eigen working matrix
  SLOT_EIG_V,          // Householder vectors
  SLOT_EIG_VEC,        // small vectors (d, e, tau, p, w, flags)
  SLOT_EIG_Z,          // tridiagonal eigenvectors
  SLOT_TEN_A,          // ping-pong tensor A
  SLOT_TEN_B,          // ping-pong tensor B
  SLOT_SMALL,          // small device scalars
  SLOT_Q,              // quantized magnitudes
  SLOT_QS,             // signs
  SLOT_QPART,          // tracker partials
  SLOT_ENC,            // encoder sizes / offsets
  SLOT_OUT,            // device stream staging
  SLOT_CORE,           // permuted core
  SLOT_LAM,            // eigenvalues
  SLOT_TTM_U,          // packed split factor
  SLOT_SPILL,          // encoder run spill (block sizes > 4096)
  SLOT_DEC,            // decompression ping-pong
  SLOT_DEC2,
  SLOT_FAC,            // uploaded factors
  SLOT_TC_ERR,         // tensor-core kernels' error word + pre-scales
  SLOT_CAND,           // candidate factor of the certified rank choice + its Rayleigh quotients
  SLOT_DEC_RUNS,       // decoded run lengths per (block, plane)
  SLOT_SLICES,         // integer slice planes of the Gram input
  SLOT_ADJ_A,          // adjoint / expansion chains
  SLOT_ADJ_B,
  SLOT_BATCH_TUNE,     // batched-path tile probe input
  SLOT_COLSHIFT,       // per-column scale exponents of the split expansions
  SLOT_SUBSPACE,       // subspace-iteration blocks
  SLOT_SUB_U,          // subspace-iteration Ritz vectors
  SLOT_SUB_V0,         // subspace-iteration start frame (kept while n and K stay the same)
  SLOT_TTM_AIMG,       // pre-sliced data operand of products with several output chunks
  SLOT_KEPT,           // per-slice significance flags of the quantized core
  SLOT_SCAN,           // range sums of the multi-CTA offset scans
  SLOT_COUNT
};

// ---------------------------------------------------------------- kernels
// norm / reductions (k_reduce.cu)
// ||x||^2 in FP64 into *out; mx_bits != nullptr: max |x| (float bits) is
// atomicMax-ed into it in the same pass (a slice scale's maxbits).
int launch_norm2(const void* x, int dtype, int64_t n, double* out, cudaStream_t s, unsigned* mx_bits = nullptr);
// *out = sum (x - z)^2 over n elements, x FP32/FP64 (dtype), z FP32; FP64 result
int launch_convert_to_f64(const void* x, int dtype, int64_t n, double* y, cudaStream_t s);
int launch_convert_f64_to(const double* x, int64_t n, void* y, int dtype, cudaStream_t s);
// e[j] = sum over (l, c) of y[(l r + j) R + c]^2 in FP64 (fixed order)
// out[j] = u_j^T G u_j for the rh columns of U (n x rh row-major, FP64), out[rh] = trace(G); n <= 1024
// u_j^T G u_j (j < rh, U n x rh row-major) and trace(G) in FP64, each as
// rayleigh_splits(n, rh) parts over row chunks of G: out[j * ns + c], the
// trace at j = rh; out holds (rh + 1) * kRaySplitMax doubles.
constexpr int kRaySplitMax = 16;
int rayleigh_splits(int64_t n, int rh);
int launch_rayleigh(const double* G, int64_t n, const double* U, int rh, double* out, cudaStream_t s);
// (L, rh, R) -> (L, r, R): the leading r of every rh rows
int launch_permute(const double* x, const int64_t* dims, const int* perm, int ndim, double* y, int inverse,
                   cudaStream_t s);

// FP64 contractions (k_fp64.cu)
int launch_gram_fp64(const void* x, int dtype, int64_t L, int64_t n, int64_t R, double* g, cudaStream_t s);
int launch_ttm_fp64(const void* x, int xdtype, int64_t L, int64_t n, int64_t R, const double* u, int64_t r,
                    int expand, void* y, int ydtype, cudaStream_t s);
// C[i][j] = sum_{l,c} A[l][i][c] B[l][j][c] for A (L, n, R) and B (L, m, R), FP64 accumulation
int launch_cross_gram_fp64(const void* a, int adt, const void* b, int bdt, int64_t L, int64_t n, int64_t m,
                           int64_t R, double* c, cudaStream_t s);

// split-precision tensor-core contractions (k_gram_tc.cu, k_ttm_tc.cu)
// Common power-of-two scale of a tensor's fixed-point slices: the kernels read
// v = x * 2^shift with |v| < 256 (shift = 8 - E, max|x| < 2^E).
struct SliceScale {
  unsigned maxbits;  // max |x| as float bits
  int shift;
};
int slice_scale(const void* x, int dtype, int64_t N, cudaStream_t s, const SliceScale** out);
// The two halves of slice_scale() around a pass that fills the record's
// maxbits itself (launch_norm2 with mx_bits): a zeroed record, then the
// kernel that turns maxbits into the scale.
int slice_scale_begin(cudaStream_t s, SliceScale** out);
int slice_scale_end(SliceScale* sc, cudaStream_t s);
// xs: the input's slice scale from slice_scale(), or nullptr to compute it here;
// nslice: 3 (24-bit fixed point) or 4 (32-bit)
int launch_gram_split(const void* x, int dtype, int64_t L, int64_t n, int64_t R, int precision, double* g,
                      cudaStream_t s, const SliceScale* xs = nullptr, int nslice = 3);
int launch_ttm_split(const void* x, int xdtype, int64_t L, int64_t n, int64_t R, const double* u, int64_t r,
                     int expand, int precision, void* y, int ydtype, cudaStream_t s,
                     const SliceScale* xs = nullptr);

// eigensolver (k_eig.cu)
int launch_eig_sym(const double* g, int n, double* lam, double* v, int nvec, cudaStream_t s);
// eigenvalues only, then eigenvectors of the top nvec (split so rank selection can run between)
int launch_eig_values(const double* g, int n, double* lam, cudaStream_t s);
int launch_eig_vectors(int n, int nvec, double* v, cudaStream_t s);
// tridiagonalise only (+ FP64 trace of G into *trace_dev); then the K largest eigenvalues
// use_dd: double-float (FP32-pair) solver for n <= 512 (the split paths); the
// following eig_more / eig_vectors calls use the same arithmetic
int launch_eig_tridiag(const double* g, int n, double* trace_dev, cudaStream_t s, bool use_dd = false);
int launch_eig_more(int n, int K, double* lam, cudaStream_t s);
int launch_rank_select(const double* lam, int n, double budget, int* r_dev, double* disc_dev, cudaStream_t s);
int eig_read_error(int* err);
int* eig_error_flag_dev();  // device word of the grid-barrier time-out flag, or nullptr
// Leading eigenpairs of a symmetric PSD n x n FP64 matrix by subspace iteration
// (T iterations of a K-column block, K <= min(64, n), n K double-floats in
// shared memory) and Rayleigh-Ritz (k_subspace.cu, k_rr.cu).  Enqueues the
// copy of decision_host[0..4) = {rp, nv, passed, *tc_err} (pinned host memory;
// valid once the stream is synchronised): rp the smallest rank whose tail
// trace(G) - sum_{j<rp} theta_j is <= budget, passed = 1 when rp >= 1, rp < n,
// nv = rp + extra <= nmax and (|theta_K| / theta_rp)^T <= conv; then the
// leading nv columns of U_dev (n x nmax row-major) are the Ritz vectors.
bool subspace_supported(int n, int K);
int subspace_solve(const double* G, int n, int K, int T, double budget, int extra, int nmax, double conv,
                   const int* tc_err, double* U_dev, int* decision_host, cudaStream_t s);
// the Rayleigh-Ritz kernel alone (k_rr.cu): B K x K FP64, trace_dev a device
// scalar; theta_dev (K), decision_dev (4 ints) and Y_dev (K x nv) on the device
size_t rr_smem_bytes(int K, int nmax);  // dynamic shared memory of the Rayleigh-Ritz kernel
int launch_rr_small(const double* B, int K, int n, const double* trace_dev, double budget, int extra, int nmax,
                    double conv, int T, const int* tc_err, double* theta_dev, int* decision_dev, double* Y_dev,
                    cudaStream_t s);
int tc_error_flag(int** flag);  // device error word of the tensor-core kernels (zeroed by the caller)

// quantizer / encoder (k_quant.cu)
struct QuantResult {
  int k;
  int p_star;
  int prio;        // split truncation of plane p_star: 0 leading bits first, 1 trailing first
  int64_t i_lead;  // last leading bit of plane p_star encoded (-1: none)
  int64_t i_trail; // last trailing bit of plane p_star encoded (-1: none)
  double sse_pred;
};
// The encoded "ATCQ" section: its fixed header and frequency tables on the
// host, the rest (size table + chunk bytes) left on the device for the caller
// to copy straight into its own buffer (valid until the next call on this device).
struct QuantSection {
  std::vector<uint8_t> head;
  const uint8_t* payload = nullptr;
  size_t payload_bytes = 0;
  size_t size() const { return head.size() + payload_bytes; }
};
int quantize_encode(const double* core, int64_t n, double target, int block_size, cudaStream_t s,
                    QuantSection* out, QuantResult* res, float* ms_quant, float* ms_encode);
int decode_dequantize(const uint8_t* bytes, size_t nbytes, double* core, int64_t n, cudaStream_t s);
// slices of the last quantized core holding a significant coefficient (k_quant.cu)
int core_kept_slices(int64_t n, const int64_t* ranks, const int* perm, int d, int p_star, int64_t i_lead,
                     uint8_t* kept_host, cudaStream_t s);

// Kernel timer (atc_kernel_timing): when enabled, the launch sites of the main
// kernels bracket their launch with CUDA events recorded on the launching
// stream; atc_kernel_times() reports launches and total device time per kernel.
// Off by default (one relaxed load per launch site).
// Each timed launch also records its algorithmic work: bytes the operation must
// move (inputs read once, outputs written once) and FLOPs of the operation it
// computes, plus the FLOPs the tensor cores issue for it (slice products and
// tile padding), 0 where not applicable.
int ktimer_begin(cudaStream_t s, const char* name, double bytes, double flops, double issued);  // token or -1
void ktimer_end(cudaStream_t s, int token);
struct KTimed {
  cudaStream_t s;
  int tok;
  KTimed(cudaStream_t st, const char* name, double bytes = 0.0, double flops = 0.0, double issued = 0.0)
      : s(st), tok(ktimer_begin(st, name, bytes, flops, issued)) {}
  ~KTimed() { ktimer_end(s, tok); }
};

// drop the cached device address of the no-allocation Gram array of `dev`
void noalloc_forget(int dev);

}  // namespace atc
