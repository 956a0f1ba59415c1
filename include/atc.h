/*
 * atc.h -- C ABI of the GB300 ST-HOSVD + bit-plane core compressor.
 *
 * The library computes the hot path of the ATC Tucker compressor (arXiv
 * 2107.01384) on one NVIDIA GB300 (sm_103a):
 *   ||X||^2 -> per mode: Gram SYRK -> eigensolve -> rank choice ->
 *   projection TTM (Algorithm 1, Section 4.1) -> core storage order ->
 *   scaling / rounding -> exact bit-plane tracking and breakpoint ->
 *   run-length + rANS block encoding (Sections 3.3, 4.2, 4.3, supplement S.6),
 * and the reverse for decompression.
 *
 * Conventions shared by every entry point
 *  - Tensors are row-major with the LAST index fastest (lexicographic order,
 *    supplement S.2).  For a mode k the tensor is viewed as (L, n_k, R) with
 *    L = prod(dims[:k]) and R = prod(dims[k+1:]); no transpose is ever made.
 *  - "_dev" pointers are CUDA device pointers of the current device, owned by
 *    the caller unless stated otherwise; they are read or written, never freed.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    All device work of a call is enqueued on it.  Calls that return host
 *    values (ranks, streams, stats) synchronise that stream before returning.
 *  - Return value: ATC_OK (0) or a negative ATC_E* code; nothing throws and
 *    nothing aborts.  atc_last_error() gives a thread-local message for the
 *    last failing call of the calling thread.
 *  - Scratch device memory is allocated by the library with cudaMalloc and
 *    cached per device (released by atc_release_workspace()); small per-mode
 *    readbacks go through one pinned host buffer of the process.
 *  - The library is meant for one host thread per device at a time (its
 *    scratch, pinned readback buffer and cached start frame are shared).
 *
 * Environment switches (read by the library; the defaults need none):
 *   ATC_TRACE=1 / 2        synchronise after every launch site and report its
 *                          status (2: also the host time since the previous one)
 *   ATC_SUBSPACE=0         split paths: full eigensolver instead of subspace iteration
 *   ATC_GRAM_CONVERT=1     split paths: converter-warp Gram (global loads) instead of
 *                          the TMA-fed ones
 *   ATC_BATCH_TUNE=0       batched ST-HOSVD: built-in Gram tile table, no probe
 */
#ifndef ATC_H
#define ATC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ATC_OK 0
#define ATC_EINVAL (-1)   /* bad argument: null pointer, ndim not in [1,8], dim <= 0, rel_eps not in (0,1], rtmss not in [0,1], ... */
#define ATC_ENOMEM (-2)   /* device or host allocation failed */
#define ATC_ECUDA (-3)    /* a CUDA runtime call or kernel launch failed */
#define ATC_ECORRUPT (-4) /* a compressed stream failed a magic / version / size / bounds check */
#define ATC_EUNSUP (-5)   /* unsupported combination (e.g. tensor too large for a kernel) */
#define ATC_ETIMEOUT (-6) /* a bounded device-side wait gave up; the results of the call are invalid */
#define ATC_ENUMERIC (-7) /* NaN / Inf in the input or a non-converged eigensolve */

typedef enum { ATC_F32 = 1, ATC_F64 = 2 } atc_dtype;

/* Arithmetic of the contractions and of the eigensolver.  In every mode the
 * discarded-energy sums that choose ranks are FP64.
 *  FP64:  FP64 SIMT contractions and intermediates, FP64 eigensolver, ranks from
 *         the eigenvalue tails.
 *  SPLIT: tcgen05 contractions on three integer slices per value (each exact in
 *         bf16 / fp16), all nine slice products accumulated in FP32 without
 *         rounding, FP64 split-K sums; FP32 intermediates; leading eigenvectors
 *         by double-float subspace iteration + Rayleigh-Ritz for mode lengths
 *         64..768 (else a double-float tridiagonal solver); ranks certified from
 *         the measured tails ||X - U ._k Y||^2 + sum_{j>=r} ||Y_j||^2. */
typedef enum {
  ATC_PREC_FP64 = 0,       /* plain FP64 */
  ATC_PREC_SPLIT_BF16 = 1, /* split, bf16 slices */
  ATC_PREC_SPLIT_FP16 = 2  /* split, fp16 slices */
} atc_precision;
/* Flag OR-ed into a split precision (atc_gram, atc_options.precision): the
 * Gram matrices use FOUR 8-bit slices (32-bit fixed point below max |x|, the
 * thirteen slice products of order <= 4, still exact in FP32) instead of three.
 * Without the flag a split compression starts every mode with three slices and
 * recomputes a mode's Gram matrix with four when the estimated shift of its kept
 * subspace from the 24-bit rounding, D = q/sqrt(12) sqrt(sum_{j<=r<k}
 * ((l_j + l_k)/(l_j - l_k))^2) for the eigenvalues l and grid q, exceeds
 * 1e-6 ||X|| (cuts inside dense spectra, e.g. noise floors); the count is
 * atc_stats.escalated_modes. */
#define ATC_PREC_WIDE 16

typedef enum {
  ATC_RANK_STATIC = 0,   /* budget_k = rtmss * TargetSSE_total / d for every mode */
  ATC_RANK_ADAPTIVE = 1  /* budget_k = (rtmss * TargetSSE_total - used) / (modes left) */
} atc_rank_rule;

typedef struct {
  double rtmss;          /* Section 4.1.3 share of the error given to rank truncation; default 0.5 */
  int precision;         /* atc_precision; default ATC_PREC_FP64 */
  int rank_rule;         /* atc_rank_rule; default ATC_RANK_STATIC */
  const int* mode_order; /* processing order (permutation of 0..ndim-1) or NULL = increasing length (Section 4.1.1) */
  int block_size;        /* coefficients per encoder block (Section 4.2); multiple of 32 in [32, 65535], or 0 = automatic
                            (a multiple of 32 giving >= 16 blocks, within [512, 4096]); default 4096 */
  void* stream;          /* cudaStream_t or NULL */
} atc_options;

/* Fill *opt with the defaults listed above. */
void atc_default_options(atc_options* opt);

/* Per-call statistics (host values). */
typedef struct {
  double norm2;           /* ||X||^2 (FP64) */
  double target_sse;      /* rel_eps^2 ||X||^2 */
  double sse_trunc;       /* sum of discarded eigenvalues over the modes (Theorem 6.4 of the cited ST-HOSVD paper) */
  double sse_quant_pred;  /* tracked core quantization error at the breakpoint (Section 4.3 reconstruction) */
  int order[8];           /* processing order used */
  int storage_order[8];   /* core mode storage order before vectorisation (supplement S.2) */
  int k;                  /* quantization scale exponent: 2^63 <= 2^k max|b| < 2^64 */
  int p_star;             /* last encoded plane (64 = nothing encoded) */
  int64_t i_lead;         /* plane p_star: leading bits (not yet significant) encoded for 0..i_lead (-1: none) */
  int64_t i_trail;        /* plane p_star: trailing bits (significant above) encoded for 0..i_trail (-1: none) */
  int prio;               /* split truncation (supplement S.3): 0 leading bits first, 1 trailing first */
  int escalated_modes;    /* split paths: modes whose Gram was recomputed with four slices (ATC_PREC_WIDE) */
  double ms_norm, ms_gram, ms_eig, ms_ttm, ms_quant, ms_encode, ms_total; /* device time per phase (CUDA events) */
  int subspace_modes;     /* split paths: modes whose eigenvectors came from subspace iteration + Rayleigh-Ritz */
  int block_size;         /* encoder block size used */
} atc_stats;

typedef struct atc_compressed atc_compressed; /* opaque, library-owned until atc_free() */

/*
 * Compress a tensor resident in device memory (Figure 1 pipeline restricted to
 * the core; factors are stored as raw float64).
 *   x_dev   : device pointer to prod(dims) elements of `dtype`, row-major; read only.
 *   dims    : host array of ndim positive sizes, 1 <= ndim <= 8.
 *   rel_eps : target relative error ||X - X_hat|| / ||X|| in (0, 1].
 *   opt     : NULL for defaults.
 *   out     : receives a handle (core, factors, ranks, stream, stats).
 * Errors: ATC_EINVAL, ATC_ENOMEM, ATC_ECUDA, ATC_ETIMEOUT, ATC_ENUMERIC.
 */
int atc_compress(const void* x_dev, const int64_t* dims, int ndim, int dtype, double rel_eps,
                 const atc_options* opt, atc_compressed** out);

/* ranks[ndim] (host) <- the multilinear rank chosen per mode (original mode index). */
int atc_get_ranks(const atc_compressed* c, int64_t* ranks);
/* *core_dev <- borrowed device pointer to the FP64 core, modes in their original
 * positions, shape (r_1..r_d), row-major.  Valid until atc_free(c). */
int atc_get_core(const atc_compressed* c, const double** core_dev);
/* *u_dev <- borrowed device pointer to factor U_mode, FP64 (n_mode x r_mode) row-major. */
int atc_get_factor(const atc_compressed* c, int mode, const double** u_dev);
/* *bytes <- borrowed HOST pointer to the compressed stream ("ATC1"), *nbytes its size. */
int atc_get_stream(const atc_compressed* c, const uint8_t** bytes, size_t* nbytes);
int atc_get_stats(const atc_compressed* c, atc_stats* stats);
/* Release a handle.  Its core and factors live in the device's stream-ordered
 * memory pool and go back to it in order on the legacy default stream: work of
 * the caller that still reads them (through atc_get_core / atc_get_factor)
 * must be finished, or ordered before that stream, when atc_free is called. */
void atc_free(atc_compressed* c);

/* Read ndim, dims (<= 8 entries) and dtype from a stream header (host only). */
int atc_peek_dims(const uint8_t* stream, size_t nbytes, int* ndim, int64_t* dims, int* dtype);

/*
 * Decompress a host stream into out_dev (device, prod(dims) elements of
 * out_dtype): decode + dequantize the core (Section 4.3 reconstruction), then
 * X_hat = B~ x_1 U_1 ... x_d U_d in the order minimising the operation count
 * (Section 4.1.1).  The expansion runs in FP64.
 * Errors: ATC_EINVAL, ATC_ECORRUPT, ATC_ENOMEM, ATC_ECUDA.
 */
int atc_decompress(const uint8_t* stream, size_t nbytes, void* out_dev, int out_dtype, void* cuda_stream);

/*
 * atc_decompress with options: opt->stream is the CUDA stream; with
 * opt->precision = ATC_PREC_SPLIT_BF16 / _FP16 the expansion runs on the
 * tensor cores (the same exact fixed-point slice products as the projection,
 * FP32 intermediates, one rounding per output), with ATC_PREC_FP64 (or
 * opt == NULL) exactly as atc_decompress.  Other option fields are ignored.
 * Errors: as atc_decompress; ATC_EUNSUP for a rank above 1024 on the split paths.
 */
int atc_decompress_ex(const uint8_t* stream, size_t nbytes, void* out_dev, int out_dtype, const atc_options* opt);

/*
 * Tucker expansion X_hat = G x_1 U_1 ... x_d U_d (the reconstruction of
 * Section 4.1.1 / 4.3, Algorithm 1's model) from DEVICE data, and its adjoint.
 *   core_dev   G, row-major (r_1..r_d), ATC_F32 or ATC_F64
 *   factors_dev[k]  U_k, n_k x r_k row-major FP64 (any matrices; orthonormality not assumed)
 *   dims       n_1..n_d (1 <= d <= 8, r_k <= n_k)
 *   out_dev    X_hat, row-major (n_1..n_d), out_dtype
 * opt->precision: ATC_PREC_FP64 (FP64 SIMT products) or a split precision
 * (tensor-core products with the exact slices, FP32 intermediates); opt->stream.
 * Errors: ATC_EINVAL, ATC_ENOMEM, ATC_ECUDA.
 */
int atc_tucker_expand(const void* core_dev, int core_dtype, const int64_t* ranks, int ndim,
                      const double* const* factors_dev, const int64_t* dims, void* out_dev, int out_dtype,
                      const atc_options* opt);

/*
 * Adjoint of atc_tucker_expand for a cotangent dY = dL/dX_hat (device, (n_1..n_d), F32/F64):
 *   dcore_dev     dL/dG = dY x_1 U_1^T ... x_d U_d^T          (r_1..r_d, FP64; may be NULL)
 *   dfactors_dev[k]  dL/dU_k = dY_(k) (G x_{j!=k} U_j)_(k)^T   (n_k x r_k, FP64; array or entries may be NULL)
 * The per-mode intermediates G x_{j!=k} U_j are recomputed for every k, never
 * stored together.  The paper has no adjoint; this extends its reconstruction.
 * Errors: as atc_tucker_expand.
 */
int atc_tucker_expand_adjoint(const void* dy_dev, int dy_dtype, const void* core_dev, int core_dtype,
                              const int64_t* ranks, int ndim, const double* const* factors_dev, const int64_t* dims,
                              double* dcore_dev, double* const* dfactors_dev, const atc_options* opt);

/* ------------------------------------------------------------------------
 * Batched ST-HOSVD.  `count` float32 tensors of one order d (1..8), each with
 * its own shape (every mode length <= 112) and rel_eps, go through Algorithm 1
 * (Section 4.1.3 error budget and rank rule, Section 4.1.1 mode order) in ONE
 * persistent kernel launch that is captured once in a CUDA graph and replayed
 * by atc_batch_run.  Arithmetic: exact float products summed in double-float
 * with FP64 flushes (Gram), double-float Jacobi eigensolve, FP64 tails for the
 * rank choice, double-float projection (FP32 intermediates, FP64 core).
 * opt->precision is ignored; opt->rtmss, rank_rule and mode_order apply to
 * every tensor.  Quantization and encoding of the cores are not part of it.
 * ------------------------------------------------------------------------ */
typedef struct atc_batch atc_batch; /* opaque, library-owned until atc_batch_free() */

/*
 * Plan a batch: dims is a host array of count * ndim sizes (tensor t's modes
 * at dims[t * ndim ...]), rel_eps a host array of count values in (0, 1],
 * dtype must be ATC_F32.  Allocates the outputs (cores, factors), the per-CTA
 * scratch and the graph.  The first plan of a process also measures the Gram
 * register tile per mode length on the device (atc_batch_tune; set the
 * environment variable ATC_BATCH_TUNE=0 to use the built-in table instead).
 * Errors: ATC_EINVAL, ATC_EUNSUP (dtype, a mode longer than 112), ATC_ENOMEM, ATC_ECUDA.
 */
int atc_batch_create(int count, int ndim, const int64_t* dims, int dtype, const double* rel_eps,
                     const atc_options* opt, atc_batch** out);
/*
 * Run the planned batch on `count` device tensors (host array of device
 * pointers, tensor t row-major with the planned shape; read only) on `stream`,
 * then wait for it.  Results stay valid until the next run or atc_batch_free.
 * Errors: ATC_EINVAL, ATC_ECUDA, ATC_ENUMERIC (NaN / Inf in an input).
 */
int atc_batch_run(atc_batch* b, const void* const* tensors_dev, void* stream);
/* ranks[ndim] (host) of tensor `index`, original mode order. */
int atc_batch_get_ranks(const atc_batch* b, int index, int64_t* ranks);
/* Borrowed device pointer to tensor index's FP64 core, shape (r_1..r_d) row-major. */
int atc_batch_get_core(const atc_batch* b, int index, const double** core_dev);
/* Borrowed device pointer to factor U_mode of tensor index, FP64 (n_mode x r_mode) row-major. */
int atc_batch_get_factor(const atc_batch* b, int index, int mode, const double** u_dev);
/* Host statistics of tensor index: ||X||^2, the discarded energy, the Jacobi
 * sweeps per mode (negative: the sweep limit was hit) and a status word
 * (0 ok, 2 a Jacobi solve hit its sweep limit).  Any pointer may be NULL. */
int atc_batch_get_stats(const atc_batch* b, int index, double* norm2, double* sse_trunc, int* sweeps,
                        int* status);
/* SM clock cycles the CTA that took tensor index spent in its phases
 * (cycles[4]: power-of-two scale + Gram, Jacobi, rank choice + factor output,
 * projection) and rounds[ndim]: the Jacobi rounds that rotated, per mode.  Either pointer may be NULL. */
int atc_batch_get_profile(const atc_batch* b, int index, int64_t* cycles, int* rounds);
/* Device time of the last atc_batch_run, graph launch to completion, in ms. */
float atc_batch_last_ms(const atc_batch* b);
/* Measure the Gram tile table now (table_out: NULL or 113 ints, the tile edge per mode length). */
int atc_batch_tune(void* stream, int* table_out);
void atc_batch_free(atc_batch* b);

/* ------------------------------------------------------------------------
 * Step entry points: one per stage of the hot path, for parity tests and
 * for callers that drive the loop themselves.  All sizes are element counts.
 * ------------------------------------------------------------------------ */

/* *out_dev (device, 1 double) <- sum x_i^2 in FP64 over n elements (Section 3.1 norm). */
int atc_norm2(const void* x_dev, int64_t n, int dtype, double* out_dev, void* stream);

/*
 * Mode Gram matrix G = X_(k) X_(k)^T of the (L, n, R) view (Section 3.1
 * unfolding, Algorithm 1 SVD step via Gram): G[i][j] = sum_{l,c} X[l][i][c] X[l][j][c].
 *   x_dev : L*n*R elements of dtype (device).   g_dev : n*n doubles (device), full symmetric output.
 *   precision : atc_precision.  n <= 1024 for the split paths.
 */
int atc_gram(const void* x_dev, int dtype, int64_t L, int64_t n, int64_t R, int precision,
             double* g_dev, void* stream);

/*
 * Symmetric eigensolve in FP64 (Algorithm 1 SVD step; lambda = sigma^2):
 *   g_dev   : n*n doubles (device, symmetric, read only).
 *   lam_dev : n doubles (device) <- eigenvalues in descending order (not clamped).
 *   v_dev   : n*nvec doubles (device, row-major n x nvec) <- eigenvectors of the
 *             nvec largest eigenvalues, the entry of largest magnitude of each
 *             column made positive; may be NULL when nvec == 0.
 *   1 <= n <= 1024, 0 <= nvec <= n.
 */
int atc_eig_sym(const double* g_dev, int n, double* lam_dev, double* v_dev, int nvec, void* stream);

/*
 * Rank choice (Section 4.1.3 error budget): clamp lambda at 0, tail sums
 * t[r] = sum_{j>=r} lambda_j accumulated from the smallest value, and
 * r = min{r >= 1 : t[r] <= budget}.
 *   lam_dev : n doubles (device, descending).  r_out / disc_out: host outputs
 *   (r and t[r]).  Synchronises the stream.
 */
int atc_rank_select(const double* lam_dev, int n, double budget, int* r_out, double* disc_out, void* stream);

/*
 * Mode-k product on the (L, n, R) view.
 *   project (expand == 0): y[l][j][c] = sum_i U[i][j] x[l][i][c],  y is (L, r, R)   (Algorithm 1 projection)
 *   expand  (expand == 1): y[l][i][c] = sum_j U[i][j] x[l][j][c],  x is (L, r, R), y is (L, n, R)
 *   u_dev : FP64 n x r row-major (device).
 *   x dtype / y dtype: ATC_F32 or ATC_F64.  precision: atc_precision (the
 *   split paths need n <= 1024, r <= 256 and write FP32 y).
 */
int atc_ttm(const void* x_dev, int xdtype, int64_t L, int64_t n, int64_t R, const double* u_dev, int64_t r,
            int expand, int precision, void* y_dev, int ydtype, void* stream);

/*
 * Quantize and encode a vectorised FP64 core (Sections 3.3, 4.2, 4.3, S.6),
 * with split bit-plane truncation of the last plane (supplement S.3): the
 * breakpoint plane p_star comes from the walk in coefficient order; on it the
 * category (leading or trailing bits) with the higher efficiency on plane
 * p_star + 1 is walked first, then the other, up to the first bit whose
 * tracked error meets the target.
 *   core_dev   : n doubles (device), already in storage order.
 *   target_sse : quantization error budget in core units (may be <= 0: encode all).
 *   *bytes     : receives a library-allocated HOST buffer (free with
 *                atc_free_buffer) holding the "ATCQ" section, *nbytes its size.
 *   info       : optional host int64[5] <- {k, p_star, prio, i_lead, i_trail}.
 * The bytes are identical to the plain C reference for the same core and target.
 */
int atc_quantize_core(const double* core_dev, int64_t n, double target_sse, int block_size, void* stream,
                      uint8_t** bytes, size_t* nbytes, int64_t* info);

/*
 * atc_gram with precision ATC_PREC_FP64, for callers that cannot allocate
 * device memory: real-time paths that must not block on the device allocator
 * (cudaMalloc can synchronise the device), or a host that gives this library a
 * fixed memory budget and accounts for every byte it may take.
 * The paper has no counterpart: it is an integration variant of the Gram step.
 *   Same arguments, layout and result as atc_gram (g_dev: n*n doubles, full
 *   symmetric).  It calls no cudaMalloc, cudaFree or allocating library
 *   routine: the split-K partial sums live in a 4 MiB array in this library's
 *   device memory, held by every GPU that loads the library until exit.
 *   Limit: n <= 724 (n * n <= 524288); larger n, or L * n * R beyond int64,
 *   returns ATC_EINVAL before anything runs.
 *   The first call on a device looks up the array's device address
 *   (cudaGetSymbolAddress) and keeps it; make that first call before any
 *   stream capture.  After a device reset call atc_release_workspace() so that
 *   the next call looks the address up again.
 *   All calls share the one array and it keeps the last call's contents (every
 *   entry a call reads is written by that call first): calls that overlap on
 *   the GPU (different streams or threads at the same time) race and give
 *   wrong results.
 */
int atc_gram_fp64_noalloc(const void* x_dev, int dtype, int64_t L, int64_t n, int64_t R, double* g_dev,
                          void* stream);

/* Decode an "ATCQ" section (host bytes) into n dequantized doubles (device). */
int atc_dequantize_core(const uint8_t* bytes, size_t nbytes, double* core_dev, int64_t n, void* stream);

void atc_free_buffer(void* p);
/* Number of CUDA kernels this library has launched in this process (host counter). */
long long atc_kernel_launches(void);
/* Kernel timer (measurement aid, not part of the paper's method).  enable != 0
 * starts a new timing window (earlier records are dropped): from then on the
 * library brackets every launch of its main kernels with two CUDA events on
 * the launching stream (at most 65536 launches a window).  enable == 0 stops
 * recording and drops the records.  Adds two event records per timed launch. */
int atc_kernel_timing(int enable);
/* Per-kernel totals of the current window, one line per kernel name:
 * "<name>|<launches>|<total device ms>|<bytes>|<flops>|<issued flops>\n" into
 * buf (host, cap bytes, NUL terminated), where bytes / flops are the
 * algorithmic work of the timed launches (inputs read once, outputs written
 * once; FLOPs of the operation computed) and issued flops the tensor-core work
 * they issue (slice products, tile padding; 0 for other kernels); waits for the
 * recorded events.  ATC_EINVAL if buf is too small. */
int atc_kernel_times(char* buf, size_t cap);
/* Free the cached device scratch of the current device (and forget the looked-up
   address of the no-allocation Gram array there). */
int atc_release_workspace(void);
const char* atc_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* ATC_H */
