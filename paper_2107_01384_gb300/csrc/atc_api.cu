// Host orchestrator and C ABI (include/atc.h).
//
// Compression (Figure 1 pipeline restricted to the core):
//   ||X||^2 -> TargetSSE_total = rel_eps^2 ||X||^2, ST-HOSVD budget
//   RTMSS * TargetSSE_total (Section 4.1.3) -> for each mode in processing
//   order (Section 4.1.1): Gram, eigenvalues, rank choice, eigenvectors of the
//   kept columns, projection (Algorithm 1) -> core in storage order
//   (supplement S.2) -> quantization with target TargetSSE_total -
//   ActualSSE_ST-HOSVD (end of Section 4.1.3) -> stream.
// Projected modes keep their position in the row-major layout, so no tensor
// is ever transposed; the (L, n, R) view of the current tensor is all a kernel
// needs.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <string>
#include <functional>
#include <chrono>
#include <vector>

#include "atc_internal.cuh"

namespace atc {

static thread_local std::string g_err;
long long g_kernel_launches = 0;

// ATC_TRACE=1: synchronise and check after every launch, printing the site
// (debugging aid; off by default).
int trace_enabled() {
  static int v = -1;
  if (v < 0) {
    const char* e = getenv("ATC_TRACE");
    v = (e && (e[0] == '1' || e[0] == '2')) ? e[0] - '0' : 0;
  }
  return v;
}
// ATC_TRACE=1: synchronise and report the status after every launch site;
// ATC_TRACE=2: also the host time since the previous trace point (kernel time
// plus launch overhead, for locating slow launches)
int trace_point(const char* file, int line) {
  static auto last = std::chrono::steady_clock::now();
  cudaError_t e = cudaDeviceSynchronize();
  const auto now = std::chrono::steady_clock::now();
  if (trace_enabled() == 2)
    fprintf(stderr, "[atc trace] %s:%d -> %s %.1f us\n", file, line, cudaGetErrorString(e),
            std::chrono::duration<double, std::micro>(now - last).count());
  else
    fprintf(stderr, "[atc trace] %s:%d -> %s\n", file, line, cudaGetErrorString(e));
  last = std::chrono::steady_clock::now();
  fflush(stderr);
  if (e != cudaSuccess) return fail(ATC_ECUDA, "trace %s:%d: %s", file, line, cudaGetErrorString(e));
  return ATC_OK;
}

void set_error(const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
}

int fail(int code, const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

// ------------------------------------------------------------------ scratch
namespace {
struct DevArena {
  void* ptr[SLOT_COUNT] = {};
  size_t cap[SLOT_COUNT] = {};
};
std::mutex g_arena_mu;
std::vector<DevArena> g_arenas;
}  // namespace

long long g_scratch_serial = 0;  // bumped whenever any scratch slot is allocated or freed

// ------------------------------------------------------------- kernel timer
namespace {
struct KRecord {
  const char* name;
  cudaEvent_t a, b;
  double bytes, flops, issued;
};
std::mutex g_kt_mu;
int g_kt_on = 0;
std::vector<KRecord> g_kt_rec;   // records of the current timing window
std::vector<cudaEvent_t> g_kt_pool;
constexpr size_t kKtMax = 65536;  // records per window (later launches are not timed)
cudaEvent_t kt_event() {
  cudaEvent_t e = nullptr;
  if (!g_kt_pool.empty()) {
    e = g_kt_pool.back();
    g_kt_pool.pop_back();
  } else if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    e = nullptr;
  }
  return e;
}
}  // namespace

int ktimer_begin(cudaStream_t s, const char* name, double bytes, double flops, double issued) {
  if (!__atomic_load_n(&g_kt_on, __ATOMIC_RELAXED)) return -1;
  std::lock_guard<std::mutex> lk(g_kt_mu);
  if (g_kt_rec.size() >= kKtMax) return -1;
  KRecord r{name, kt_event(), kt_event(), bytes, flops, issued};
  if (!r.a || !r.b || cudaEventRecord(r.a, s) != cudaSuccess) {
    cudaGetLastError();
    if (r.a) g_kt_pool.push_back(r.a);
    if (r.b) g_kt_pool.push_back(r.b);
    return -1;
  }
  g_kt_rec.push_back(r);
  return (int)g_kt_rec.size() - 1;
}
void ktimer_end(cudaStream_t s, int token) {
  if (token < 0) return;
  std::lock_guard<std::mutex> lk(g_kt_mu);
  if (token < (int)g_kt_rec.size() && cudaEventRecord(g_kt_rec[token].b, s) != cudaSuccess) cudaGetLastError();
}

int Scratch::get(int slot, size_t bytes, void** out) {
  if (slot < 0 || slot >= SLOT_COUNT) return fail(ATC_EINVAL, "bad scratch slot");
  int dev = 0;
  ATC_CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_arena_mu);
  if ((int)g_arenas.size() <= dev) g_arenas.resize(dev + 1);
  DevArena& a = g_arenas[dev];
  if (bytes == 0) bytes = 256;
  if (a.cap[slot] < bytes) {
    if (a.ptr[slot]) {
      // a device-wide sync is needed before freeing memory queued work may use
      cudaError_t e = cudaDeviceSynchronize();
      if (e != cudaSuccess) return fail(ATC_ECUDA, "cudaDeviceSynchronize: %s", cudaGetErrorString(e));
      cudaFree(a.ptr[slot]);
      a.ptr[slot] = nullptr;
      a.cap[slot] = 0;
      ++g_scratch_serial;
    }
    size_t want = bytes + bytes / 8;
    want = (want + 255) & ~(size_t)255;
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, want);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(ATC_ENOMEM, "cudaMalloc(%zu) for scratch slot %d failed: %s", want, slot, cudaGetErrorString(e));
    }
    a.ptr[slot] = p;
    a.cap[slot] = want;
    ++g_scratch_serial;
  }
  *out = a.ptr[slot];
  return ATC_OK;
}

int Scratch::release_all() {
  int dev = 0;
  ATC_CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_arena_mu);
  if ((int)g_arenas.size() <= dev) return ATC_OK;
  ATC_CUDA_TRY(cudaDeviceSynchronize());
  DevArena& a = g_arenas[dev];
  for (int i = 0; i < SLOT_COUNT; ++i) {
    if (a.ptr[i]) cudaFree(a.ptr[i]);
    a.ptr[i] = nullptr;
    a.cap[i] = 0;
  }
  ++g_scratch_serial;
  return ATC_OK;
}

}  // namespace atc

using namespace atc;

struct atc_compressed {
  int ndim = 0;
  int dtype = 0;
  int64_t dims[8] = {};
  int64_t ranks[8] = {};
  double* core = nullptr;      // device, FP64, (r_1..r_d)
  double* factors[8] = {};     // device, FP64, n_i x r_i
  uint8_t* stream = nullptr;   // host (malloc), stream_n bytes
  size_t stream_n = 0;
  atc_stats stats = {};
};

namespace {

int dtype_size(int dt) { return dt == ATC_F32 ? 4 : (dt == ATC_F64 ? 8 : 0); }

void put32(std::string& s, uint32_t v) { for (int i = 0; i < 4; ++i) s.push_back((char)(v >> (8 * i))); }
void put64(std::string& s, uint64_t v) { for (int i = 0; i < 8; ++i) s.push_back((char)(v >> (8 * i))); }
void putf64(std::string& s, double v) { uint64_t u; memcpy(&u, &v, 8); put64(s, u); }
uint32_t get32(const uint8_t* p) { uint32_t v = 0; for (int i = 0; i < 4; ++i) v |= (uint32_t)p[i] << (8 * i); return v; }
uint64_t get64(const uint8_t* p) { uint64_t v = 0; for (int i = 0; i < 8; ++i) v |= (uint64_t)p[i] << (8 * i); return v; }

// Non-blocking phase clock: events are recorded on the stream at phase
// boundaries and only read after the call's final synchronisation.
struct PhaseClock {
  static constexpr int kMax = 96;
  cudaEvent_t ev[kMax];
  int tag[kMax];
  int n = 0;
  cudaStream_t s;
  explicit PhaseClock(cudaStream_t st) : s(st) {
    for (int i = 0; i < kMax; ++i) ev[i] = nullptr;
  }
  // close the interval since the previous mark and charge it to `phase`
  void mark(int phase) {
    if (n >= kMax) return;
    if (!ev[n]) cudaEventCreate(&ev[n]);
    cudaEventRecord(ev[n], s);
    tag[n] = phase;
    ++n;
  }
  // after synchronisation: per-phase milliseconds
  void sum(double* out, int nphase) {
    for (int p = 0; p < nphase; ++p) out[p] = 0.0;
    for (int i = 1; i < n; ++i) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, ev[i - 1], ev[i]) == cudaSuccess && tag[i] >= 0 && tag[i] < nphase) out[tag[i]] += ms;
    }
  }
  double total() {
    float ms = 0.f;
    if (n >= 2) cudaEventElapsedTime(&ms, ev[0], ev[n - 1]);
    return ms;
  }
  ~PhaseClock() {
    for (int i = 0; i < kMax; ++i)
      if (ev[i]) cudaEventDestroy(ev[i]);
  }
};
enum { PH_NORM = 0, PH_GRAM, PH_EIG, PH_TTM, PH_QUANT, PH_OTHER, PH_COUNT };

int check_dims(const int64_t* dims, int ndim, int64_t* total) {
  if (!dims || ndim < 1 || ndim > 8) return fail(ATC_EINVAL, "ndim must be in [1, 8]");
  int64_t t = 1;
  for (int i = 0; i < ndim; ++i) {
    if (dims[i] <= 0) return fail(ATC_EINVAL, "dims[%d] = %lld must be positive", i, (long long)dims[i]);
    if (dims[i] > ((int64_t)1 << 40) / t) return fail(ATC_EINVAL, "tensor too large");
    t *= dims[i];
  }
  *total = t;
  return ATC_OK;
}

// extra eigenvectors beyond the provisional rank of a split path, from which
// the certified rank is chosen
constexpr int kCertExtra = 4;
// subspace iteration for the leading eigenvectors on the split paths
constexpr int kSubK = 32;      // block columns
constexpr int kSubIters = 1;   // iterations before Rayleigh-Ritz
constexpr int kSubMargin = 4;  // columns kept beyond the largest certified candidate count
// Ritz-ratio test (|theta_K| / theta_rp)^T <= kSubConv: the smallest Ritz value
// sits near the double-float floor of the K x K problem (~1e-14 theta_1), so a
// tighter bound would reject converged subspaces whenever theta_rp < 1e-8
// theta_1; the ranks are certified from measured tails either way
constexpr double kSubConv = 1e-4;
// ATC_SUBSPACE=0 (read on every call): the full eigensolver on every mode
bool subspace_enabled() {
  const char* e = getenv("ATC_SUBSPACE");
  return !(e && e[0] == '0');
}

// precision: an atc_precision, on the split paths optionally with ATC_PREC_WIDE
// (four slices: 32-bit fixed point)
int gram_dispatch(const void* x, int dtype, int64_t L, int64_t n, int64_t R, int precision, double* g, cudaStream_t s,
                  const SliceScale* xs = nullptr) {
  const int base = precision & ~ATC_PREC_WIDE;
  if (base == ATC_PREC_FP64) return launch_gram_fp64(x, dtype, L, n, R, g, s);
  return launch_gram_split(x, dtype, L, n, R, base, g, s, xs, (precision & ATC_PREC_WIDE) ? 4 : 3);
}
bool valid_precision(int p, bool allow_wide) {
  const int base = p & ~ATC_PREC_WIDE;
  if (base < ATC_PREC_FP64 || base > ATC_PREC_SPLIT_FP16) return false;
  if (p & ATC_PREC_WIDE) return allow_wide && base != ATC_PREC_FP64;
  return true;
}

// Subspace perturbation check of the split paths.  The sliced Gram matrix is
// that of X rounded to a fixed-point grid q (24 bits below max |x|): with
// independent rounding errors of variance q^2 / 12 the coupling it adds between
// eigen-directions j <= r < k is about sqrt(lambda_j + lambda_k) q / sqrt(12),
// which turns the kept subspace by theta_jk ~ that / (lambda_j - lambda_k)
// (first-order perturbation theory) and moves the projection of X by
//   D^2 = sum_{j <= r < k} theta_jk^2 (lambda_j + lambda_k)
//       = q^2 / 12 sum_{j <= r < k} ((lambda_j + lambda_k) / (lambda_j - lambda_k))^2.
// Eigenvalues beyond the known ones add ~1 per pair.  When D exceeds
// kWideTol ||X||, the Gram matrix is recomputed with four slices (q / 256).
constexpr double kWideTol = 1e-6;
double subspace_shift_estimate(const std::vector<double>& lam, int known, int r, int64_t n, double q) {
  double sum = 0.0;
  for (int j = 0; j < r && j < known; ++j) {
    const double lj = std::max(lam[j], 0.0);
    for (int k = r; k < known; ++k) {
      const double lk = std::max(lam[k], 0.0);
      const double gap = lj - lk;
      const double t = (gap > 1e-300 * (lj + 1e-300)) ? (lj + lk) / gap : 1e150;
      sum += t * t;
    }
  }
  sum += (double)std::min<int64_t>(r, known) * (double)(n - std::max<int64_t>(r, known));
  return std::sqrt(sum * q * q / 12.0);
}

int ttm_dispatch(const void* x, int xdt, int64_t L, int64_t n, int64_t R, const double* u, int64_t r, int expand,
                 int precision, void* y, int ydt, cudaStream_t s, const SliceScale* xs = nullptr) {
  if (precision == ATC_PREC_FP64) return launch_ttm_fp64(x, xdt, L, n, R, u, r, expand, y, ydt, s);
  return launch_ttm_split(x, xdt, L, n, R, u, r, expand, precision, y, ydt, s, xs);
}

// Pinned host memory for the small per-mode readbacks (norm, decisions,
// residual tails, error words): copies into it are truly asynchronous, so a
// mode needs one stream synchronisation instead of one per pageable copy.
// Layout: ints [0, 16) (0: grid-barrier flag, 1: tensor-core flag, 2..5: the
// subspace decision), doubles from byte 64.
struct PinnedReadback {
  int* ints = nullptr;
  double* dbl = nullptr;
  size_t ndbl = 0;
};
int pinned_readback(size_t ndbl, PinnedReadback* out) {
  static std::mutex mu;
  static void* buf = nullptr;
  static size_t cap = 0;
  std::lock_guard<std::mutex> lk(mu);
  const size_t want = 64 + sizeof(double) * (ndbl < 64 ? 64 : ndbl);
  if (cap < want) {
    if (buf) {
      ATC_CUDA_TRY(cudaDeviceSynchronize());
      cudaFreeHost(buf);
      buf = nullptr;
      cap = 0;
    }
    ATC_CUDA_TRY(cudaHostAlloc(&buf, want, cudaHostAllocPortable));
    cap = want;
  }
  out->ints = static_cast<int*>(buf);
  out->dbl = reinterpret_cast<double*>(static_cast<char*>(buf) + 64);
  out->ndbl = (cap - 64) / sizeof(double);
  return ATC_OK;
}

// Synchronise the stream and check the grid-barrier flag of the FP64
// tridiagonalisation (copied asynchronously into the pinned buffer first).
int eig_check(cudaStream_t s) {
  PinnedReadback pb;
  ATC_TRY(pinned_readback(0, &pb));
  int* fl = eig_error_flag_dev();
  if (fl) ATC_CUDA_TRY(cudaMemcpyAsync(&pb.ints[0], fl, sizeof(int), cudaMemcpyDeviceToHost, s));
  ATC_CUDA_TRY(cudaStreamSynchronize(s));
  if (fl && pb.ints[0]) return fail(ATC_ETIMEOUT, "grid barrier of the tridiagonalisation timed out");
  return ATC_OK;
}

// Decompression order (Section 4.1.1): exhaustive search over d! orders for
// the smallest sum_i n_p1..n_pi r_pi..r_pd; first minimum in lexicographic
// permutation order.
std::vector<int> decompression_order(int d, const int64_t* dims, const int64_t* ranks) {
  std::vector<int> p(d), best;
  for (int i = 0; i < d; ++i) p[i] = i;
  double best_cost = -1.0;
  do {
    double cost = 0.0;
    for (int i = 0; i < d; ++i) {
      double c = 1.0;
      for (int j = 0; j <= i; ++j) c *= (double)dims[p[j]];
      for (int j = i; j < d; ++j) c *= (double)ranks[p[j]];
      cost += c;
    }
    if (best_cost < 0.0 || cost < best_cost) { best_cost = cost; best = p; }
  } while (std::next_permutation(p.begin(), p.end()));
  return best;
}

// The handle's core and factors come from the device's stream-ordered memory
// pool (kept by the pool between calls, so a compress costs no cudaMalloc and
// a free no device synchronisation).  The pool keeps what it holds: its
// release threshold is raised once per device.
int handle_alloc(void** p, size_t bytes, cudaStream_t s) {
  static bool pool_set[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < 64 && !pool_set[dev]) {
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
      uint64_t keep = UINT64_MAX;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    cudaGetLastError();
    pool_set[dev] = true;
  }
  return cudaMallocAsync(p, bytes, s) == cudaSuccess ? ATC_OK : ATC_ENOMEM;
}

void free_compressed(atc_compressed* c) {
  if (!c) return;
  free(c->stream);
  // the handle's work on its stream ended before it was returned: freeing on
  // the legacy stream is ordered after it
  if (c->core) cudaFreeAsync(c->core, 0);
  for (int i = 0; i < 8; ++i)
    if (c->factors[i]) cudaFreeAsync(c->factors[i], 0);
  delete c;
}

}  // namespace

// Expands the modes listed in `modes` (in that order) of the tensor `src`
// (current sizes cur[], dtype sdt) with the factors U (n_m x r_m, FP64):
// mode m goes from r_m to dims[m].  FP64 intermediates on the plain path, FP32
// (tensor cores) on the split paths; ping-pong in bufA / bufB.  On return
// *res / *rdt is the result (one of the buffers, or src if no mode was given).
int expand_modes(const void* src, int sdt, int64_t* cur, int d, const double* const* U, const int64_t* dims,
                 const std::vector<int>& modes, int precision, void* bufA, void* bufB, cudaStream_t s,
                 const void** res, int* rdt) {
  const bool split = precision != ATC_PREC_FP64;
  const int odt = split ? ATC_F32 : ATC_F64;
  void* dst = bufA;
  for (int m : modes) {
    int64_t L = 1, R = 1;
    for (int i = 0; i < m; ++i) L *= cur[i];
    for (int i = m + 1; i < d; ++i) R *= cur[i];
    ATC_TRY(ttm_dispatch(src, sdt, L, dims[m], R, U[m], cur[m], 1, precision, dst, odt, s));
    cur[m] = dims[m];
    src = dst;
    sdt = odt;
    dst = (dst == bufA) ? bufB : bufA;
  }
  *res = src;
  *rdt = sdt;
  return ATC_OK;
}

// expansion order for a subset of modes: smallest growth n_m / r_m first
std::vector<int> growth_order(const std::vector<int>& ms, const int64_t* dims, const int64_t* ranks) {
  std::vector<int> o = ms;
  std::stable_sort(o.begin(), o.end(), [&](int a, int b) {
    return (double)dims[a] / (double)ranks[a] < (double)dims[b] / (double)ranks[b];
  });
  return o;
}

int tucker_args(const void* core, int cdt, const int64_t* ranks, int d, const double* const* U, const int64_t* dims,
                int precision, int64_t* N) {
  if (!core || !ranks || !U || !dims || d < 1 || d > 8 || !dtype_size(cdt))
    return fail(ATC_EINVAL, "tucker expansion: bad arguments");
  if (precision < 0 || precision > 2) return fail(ATC_EINVAL, "tucker expansion: bad precision");
  ATC_TRY(check_dims(dims, d, N));
  for (int i = 0; i < d; ++i) {
    if (!U[i]) return fail(ATC_EINVAL, "tucker expansion: factor %d is NULL", i);
    if (ranks[i] < 1 || ranks[i] > dims[i]) return fail(ATC_EINVAL, "tucker expansion: rank %d out of range", i);
  }
  return ATC_OK;
}

extern "C" {

void atc_default_options(atc_options* opt) {
  if (!opt) return;
  opt->rtmss = 0.5;
  opt->precision = ATC_PREC_FP64;
  opt->rank_rule = ATC_RANK_STATIC;
  opt->mode_order = nullptr;
  opt->block_size = 4096;
  opt->stream = nullptr;
}

const char* atc_last_error(void) { return g_err.c_str(); }

void atc_free_buffer(void* p) { free(p); }

int atc_release_workspace(void) {
  int dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) noalloc_forget(dev);
  return Scratch::release_all();
}

long long atc_kernel_launches(void) { return __atomic_load_n(&g_kernel_launches, __ATOMIC_RELAXED); }

int atc_kernel_timing(int enable) {
  std::lock_guard<std::mutex> lk(g_kt_mu);
  for (auto& r : g_kt_rec) {
    g_kt_pool.push_back(r.a);
    g_kt_pool.push_back(r.b);
  }
  g_kt_rec.clear();
  __atomic_store_n(&g_kt_on, enable ? 1 : 0, __ATOMIC_RELAXED);
  return ATC_OK;
}

int atc_kernel_times(char* buf, size_t cap) {
  if (!buf || cap == 0) return fail(ATC_EINVAL, "atc_kernel_times: bad arguments");
  std::lock_guard<std::mutex> lk(g_kt_mu);
  std::vector<std::string> names;
  std::vector<double> tot, byt, flo, iss;
  std::vector<long long> cnt;
  for (auto& r : g_kt_rec) {
    if (cudaEventSynchronize(r.b) != cudaSuccess) return fail(ATC_ECUDA, "kernel timer: event synchronisation failed");
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) return fail(ATC_ECUDA, "kernel timer: elapsed time failed");
    size_t k = 0;
    while (k < names.size() && names[k] != r.name) ++k;
    if (k == names.size()) {
      names.push_back(r.name);
      tot.push_back(0.0);
      byt.push_back(0.0);
      flo.push_back(0.0);
      iss.push_back(0.0);
      cnt.push_back(0);
    }
    tot[k] += ms;
    byt[k] += r.bytes;
    flo[k] += r.flops;
    iss[k] += r.issued;
    cnt[k] += 1;
  }
  std::string out;
  char line[320];
  for (size_t k = 0; k < names.size(); ++k) {
    snprintf(line, sizeof(line), "%s|%lld|%.6f|%.6e|%.6e|%.6e\n", names[k].c_str(), cnt[k], tot[k], byt[k], flo[k], iss[k]);
    out += line;
  }
  if (out.size() + 1 > cap) return fail(ATC_EINVAL, "atc_kernel_times: buffer of %zu bytes too small (%zu needed)", cap,
                                        out.size() + 1);
  memcpy(buf, out.c_str(), out.size() + 1);
  return ATC_OK;
}

int atc_norm2(const void* x_dev, int64_t n, int dtype, double* out_dev, void* stream) {
  if (!x_dev || !out_dev || n < 0 || !dtype_size(dtype)) return fail(ATC_EINVAL, "atc_norm2: bad arguments");
  return launch_norm2(x_dev, dtype, n, out_dev, (cudaStream_t)stream);
}

int atc_gram(const void* x_dev, int dtype, int64_t L, int64_t n, int64_t R, int precision, double* g_dev,
             void* stream) {
  if (!x_dev || !g_dev || L < 1 || n < 1 || R < 1 || !dtype_size(dtype)) return fail(ATC_EINVAL, "atc_gram: bad arguments");
  if (!valid_precision(precision, true)) return fail(ATC_EINVAL, "atc_gram: bad precision");
  return gram_dispatch(x_dev, dtype, L, n, R, precision, g_dev, (cudaStream_t)stream);
}

int atc_eig_sym(const double* g_dev, int n, double* lam_dev, double* v_dev, int nvec, void* stream) {
  if (!g_dev || !lam_dev || n < 1 || n > 1024 || nvec < 0 || nvec > n || (nvec > 0 && !v_dev))
    return fail(ATC_EINVAL, "atc_eig_sym: bad arguments");
  cudaStream_t s = (cudaStream_t)stream;
  ATC_TRY(launch_eig_sym(g_dev, n, lam_dev, v_dev, nvec, s));
  return eig_check(s);
}

int atc_rank_select(const double* lam_dev, int n, double budget, int* r_out, double* disc_out, void* stream) {
  if (!lam_dev || n < 1 || !r_out || !disc_out) return fail(ATC_EINVAL, "atc_rank_select: bad arguments");
  cudaStream_t s = (cudaStream_t)stream;
  int* r_dev = nullptr;
  ATC_TRY(Scratch::get(SLOT_LAM, 64, (void**)&r_dev));
  double* d_dev = reinterpret_cast<double*>(r_dev + 8);
  ATC_TRY(launch_rank_select(lam_dev, n, budget, r_dev, d_dev, s));
  ATC_CUDA_TRY(cudaMemcpyAsync(r_out, r_dev, sizeof(int), cudaMemcpyDeviceToHost, s));
  ATC_CUDA_TRY(cudaMemcpyAsync(disc_out, d_dev, sizeof(double), cudaMemcpyDeviceToHost, s));
  ATC_CUDA_TRY(cudaStreamSynchronize(s));
  return ATC_OK;
}

int atc_ttm(const void* x_dev, int xdtype, int64_t L, int64_t n, int64_t R, const double* u_dev, int64_t r,
            int expand, int precision, void* y_dev, int ydtype, void* stream) {
  if (!x_dev || !u_dev || !y_dev || L < 1 || n < 1 || R < 1 || r < 1 || !dtype_size(xdtype) || !dtype_size(ydtype))
    return fail(ATC_EINVAL, "atc_ttm: bad arguments");
  if (precision < 0 || precision > 2) return fail(ATC_EINVAL, "atc_ttm: bad precision");
  return ttm_dispatch(x_dev, xdtype, L, n, R, u_dev, r, expand ? 1 : 0, precision, y_dev, ydtype, (cudaStream_t)stream);
}

int atc_quantize_core(const double* core_dev, int64_t n, double target_sse, int block_size, void* stream,
                      uint8_t** bytes, size_t* nbytes, int64_t* info) {
  if (!core_dev || n < 1 || !bytes || !nbytes) return fail(ATC_EINVAL, "atc_quantize_core: bad arguments");
  QuantSection out;
  QuantResult qr;
  ATC_TRY(quantize_encode(core_dev, n, target_sse, block_size, (cudaStream_t)stream, &out, &qr, nullptr, nullptr));
  uint8_t* buf = (uint8_t*)malloc(out.size() ? out.size() : 1);
  if (!buf) return fail(ATC_ENOMEM, "host allocation failed");
  memcpy(buf, out.head.data(), out.head.size());
  if (out.payload_bytes &&
      (cudaMemcpyAsync(buf + out.head.size(), out.payload, out.payload_bytes, cudaMemcpyDeviceToHost,
                       (cudaStream_t)stream) != cudaSuccess ||
       cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess)) {
    free(buf);
    return fail(ATC_ECUDA, "core section readback failed");
  }
  *bytes = buf;
  *nbytes = out.size();
  if (info) {
    info[0] = qr.k;
    info[1] = qr.p_star;
    info[2] = qr.prio;
    info[3] = qr.i_lead;
    info[4] = qr.i_trail;
  }
  return ATC_OK;
}

int atc_dequantize_core(const uint8_t* bytes, size_t nbytes, double* core_dev, int64_t n, void* stream) {
  if (!bytes || !core_dev || n < 1) return fail(ATC_EINVAL, "atc_dequantize_core: bad arguments");
  return decode_dequantize(bytes, nbytes, core_dev, n, (cudaStream_t)stream);
}

int atc_compress(const void* x_dev, const int64_t* dims, int ndim, int dtype, double rel_eps,
                 const atc_options* opt_in, atc_compressed** out) {
  if (!out) return fail(ATC_EINVAL, "atc_compress: out is NULL");
  *out = nullptr;
  if (!x_dev) return fail(ATC_EINVAL, "atc_compress: x_dev is NULL");
  if (!dtype_size(dtype)) return fail(ATC_EINVAL, "atc_compress: dtype must be ATC_F32 or ATC_F64");
  int64_t N = 0;
  ATC_TRY(check_dims(dims, ndim, &N));
  if (!(rel_eps > 0.0 && rel_eps <= 1.0)) return fail(ATC_EINVAL, "rel_eps must lie in (0, 1]");
  atc_options opt;
  atc_default_options(&opt);
  if (opt_in) opt = *opt_in;
  if (!(opt.rtmss >= 0.0 && opt.rtmss <= 1.0)) return fail(ATC_EINVAL, "rtmss must lie in [0, 1]");
  if (!valid_precision(opt.precision, true)) return fail(ATC_EINVAL, "bad precision");
  // every Gram with four slices (ATC_PREC_WIDE), else three with the perturbation check
  const bool wide_all = (opt.precision & ATC_PREC_WIDE) != 0;
  opt.precision &= ~ATC_PREC_WIDE;
  if (opt.rank_rule != ATC_RANK_STATIC && opt.rank_rule != ATC_RANK_ADAPTIVE) return fail(ATC_EINVAL, "bad rank rule");
  if (opt.block_size != 0 && (opt.block_size < 32 || opt.block_size > 65535 || (opt.block_size % 32)))
    return fail(ATC_EINVAL, "bad block_size");
  const int d = ndim;
  std::vector<int> order(d);
  if (opt.mode_order) {
    std::vector<int> seen(d, 0);
    for (int i = 0; i < d; ++i) {
      int m = opt.mode_order[i];
      if (m < 0 || m >= d || seen[m]) return fail(ATC_EINVAL, "mode_order must be a permutation of 0..ndim-1");
      seen[m] = 1;
      order[i] = m;
    }
  } else {
    for (int i = 0; i < d; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return dims[a] < dims[b]; });
  }
  cudaStream_t s = (cudaStream_t)opt.stream;
  atc_compressed* c = new (std::nothrow) atc_compressed();
  if (!c) return fail(ATC_ENOMEM, "host allocation failed");
  c->ndim = d;
  c->dtype = dtype;
  for (int i = 0; i < d; ++i) c->dims[i] = dims[i];
  atc_stats& st = c->stats;
  memset(&st, 0, sizeof(st));
  for (int i = 0; i < 8; ++i) st.order[i] = st.storage_order[i] = -1;
  for (int i = 0; i < d; ++i) st.order[i] = order[i];
  auto bail = [&](int rc) {
    cudaStreamSynchronize(s);  // nothing of this call may still run when its buffers go back to the pool
    cudaGetLastError();
    free_compressed(c);
    return rc;
  };
  PhaseClock clk(s);
  clk.mark(PH_OTHER);
  // ||X||^2 and the budgets (Section 4.1.3)
  double* small = nullptr;
  int rc = Scratch::get(SLOT_SMALL, sizeof(double) * 2048, (void**)&small);
  if (rc) return bail(rc);
  double* dnorm = small + 1600;
  // split paths: the input's slice scale (max |x|) comes out of the norm pass
  SliceScale* xs0 = nullptr;
  {
    if (opt.precision != ATC_PREC_FP64) {
      rc = slice_scale_begin(s, &xs0);
      if (rc) return bail(rc);
    }
    rc = launch_norm2(x_dev, dtype, N, dnorm, s, xs0 ? &xs0->maxbits : nullptr);
    if (!rc && xs0) rc = slice_scale_end(xs0, s);
    if (rc) return bail(rc);
    clk.mark(PH_NORM);
    PinnedReadback pb;
    rc = pinned_readback(1, &pb);
    if (rc) return bail(rc);
    if (cudaMemcpyAsync(pb.dbl, dnorm, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return bail(fail(ATC_ECUDA, "norm readback failed"));
    st.norm2 = pb.dbl[0];
    clk.mark(PH_OTHER);
  }
  if (!(st.norm2 == st.norm2) || st.norm2 > 1.7e308) return bail(fail(ATC_ENUMERIC, "input contains NaN or Inf"));
  st.target_sse = rel_eps * rel_eps * st.norm2;
  const double budget_total = opt.rtmss * st.target_sse;
  // intermediate precision: FP64 for the plain path, FP32 for the split paths
  const int idt = (opt.precision == ATC_PREC_FP64) ? ATC_F64 : ATC_F32;
  const size_t ibytes = (size_t)dtype_size(idt);
  int64_t cur[8];
  for (int i = 0; i < d; ++i) cur[i] = dims[i];
  // the largest projected tensor is after the first mode: N * r / n <= N
  void* bufA = nullptr;
  void* bufB = nullptr;
  int64_t maxn = 1;
  for (int i = 0; i < d; ++i) maxn = std::max(maxn, dims[i]);
  double *G = nullptr, *lam = nullptr;
  rc = Scratch::get(SLOT_TEN_A, ibytes * (size_t)N, &bufA);
  if (!rc) rc = Scratch::get(SLOT_TEN_B, ibytes * (size_t)N, &bufB);
  if (!rc) rc = Scratch::get(SLOT_LAM, sizeof(double) * (size_t)(maxn * maxn + maxn + 64), (void**)&lam);
  if (rc) return bail(rc);
  G = lam + maxn + 16;
  int* rdev = reinterpret_cast<int*>(lam + maxn);
  double* ddev = lam + maxn + 2;
  int* tc_err = nullptr;
  if (opt.precision != ATC_PREC_FP64) {
    rc = tc_error_flag(&tc_err);
    if (!rc && cudaMemsetAsync(tc_err, 0, sizeof(int), s) != cudaSuccess) rc = fail(ATC_ECUDA, "memset failed");
    if (rc) return bail(rc);
  }
  const void* curp = x_dev;
  int curdt = dtype;
  void* next = bufA;
  // a work buffer that is neither `a` nor `b`
  auto other = [&](const void* a, const void* b) -> void* {
    for (void* q : {bufA, bufB})
      if (q && q != a && q != b) return q;
    return nullptr;
  };
  double used = 0.0;
  for (int step = 0; step < d; ++step) {
    bool have_y = false;  // the projected tensor of this mode is already in `next`
    const int m = order[step];
    int64_t L = 1, R = 1;
    for (int i = 0; i < m; ++i) L *= cur[i];
    for (int i = m + 1; i < d; ++i) R *= cur[i];
    const int64_t n = cur[m];
    if (n > 1024) return bail(fail(ATC_EUNSUP, "mode length %lld > 1024 is not supported", (long long)n));
    // split paths: one slice scale of the current tensor serves its Gram and its projection
    const SliceScale* xs = nullptr;
    if (opt.precision != ATC_PREC_FP64) {
      if (curp == x_dev && xs0) xs = xs0;
      else rc = slice_scale(curp, curdt, L * n * R, s, &xs);
      if (rc) return bail(rc);
    }
    bool wide = wide_all;
    {
      rc = gram_dispatch(curp, curdt, L, n, R, opt.precision | (wide ? ATC_PREC_WIDE : 0), G, s, xs);
      if (rc) return bail(rc);
      clk.mark(PH_GRAM);
    }
    int r = 0;
    double disc = 0.0;
    {
      const double budget =
          (opt.rank_rule == ATC_RANK_STATIC) ? budget_total / d : (budget_total - used) / (double)(d - step);
      {
        // Split paths: the rank is certified from the candidate factor itself.
        // With U the leading rh eigenvector estimates (orthonormal to ~1e-15)
        // and G the tensor-core Gram matrix of X on its 24-bit grid X~,
        //   tail(r) = ||X~||^2 - ||U_r^T X~||^2 = trace(G) - sum_{j<r} u_j^T G u_j
        // (FP64), exact for whatever subspace U spans: no eigenvalue of G is
        // trusted, and the difference to the tail of X itself is second order in
        // the 24-bit rounding (its cross term with the residual scales with the
        // square root of the tail).  Then the factor is the leading r columns and
        // the projection runs once with exactly r outputs.
        // certify(): 1 = rank and factor set, 0 = it needs more than rh_cap
        // candidate vectors, < 0 = error.
        int he = 0;  // tensor-core wait flag, read with the host readbacks
        // The rank from the quotients' row-chunk parts eh[j * ns + c] (j < rh,
        // the trace at j = rh): the smallest r <= rh_used with tail(r) <=
        // budget; -1 when none is.
        auto select_rank = [&](const double* eh, int ns, int rh, int rh_used, double* tail_out) -> int {
          auto part_sum = [&](int j) {
            double v = 0.0;
            for (int c2 = 0; c2 < ns; ++c2) v += eh[(size_t)j * ns + c2];
            return v;
          };
          const double tr = part_sum(rh);
          double acc = 0.0;
          for (int rr = 1; rr <= rh_used; ++rr) {
            acc += part_sum(rr - 1);
            double t = tr - acc;
            if (t < 0.0) t = 0.0;
            if (t <= budget) { *tail_out = t; return rr; }
          }
          *tail_out = std::max(0.0, tr - acc);
          return -1;
        };
        // the factor = the leading r columns of cand (row stride ldc), then the projection with r outputs
        auto finish = [&](int rn, double tail, const double* cand, int ldc) -> int {
          r = rn;
          disc = tail;
          if (handle_alloc((void**)&c->factors[m], sizeof(double) * (size_t)n * r, s) != ATC_OK)
            return fail(ATC_ENOMEM, "factor allocation failed");
          if (cudaMemcpy2DAsync(c->factors[m], sizeof(double) * r, cand, sizeof(double) * ldc, sizeof(double) * r, n,
                                cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return fail(ATC_ECUDA, "factor copy failed");
          int rc2 = ttm_dispatch(curp, curdt, L, n, R, c->factors[m], r, 0, opt.precision, next, idt, s, xs);
          if (rc2) return rc2;
          have_y = true;
          return 1;
        };
        auto certify = [&](int rh, int rh_cap, const std::function<int(int, double*)>& get_cand) -> int {
          for (;;) {
            double* cand = nullptr;
            const size_t nparts = (size_t)(rh + 1) * kRaySplitMax;
            int rc2 = Scratch::get(SLOT_CAND, sizeof(double) * ((size_t)n * rh + nparts + 8), (void**)&cand);
            if (rc2) return rc2;
            double* edev = cand + (size_t)n * rh;  // parts of rho[0..rh), then of trace(G)
            const int ns = rayleigh_splits(n, rh);
            rc2 = get_cand(rh, cand);
            if (!rc2) rc2 = launch_rayleigh(G, n, cand, rh, edev, s);
            if (rc2) return rc2;
            PinnedReadback pb;
            rc2 = pinned_readback((size_t)(rh + 1) * ns, &pb);
            if (rc2) return rc2;
            if (cudaMemcpyAsync(pb.dbl, edev, sizeof(double) * (rh + 1) * ns, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                cudaMemcpyAsync(&pb.ints[1], tc_err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess)
              return fail(ATC_ECUDA, "Rayleigh quotient readback failed");
            rc2 = eig_check(s);
            if (rc2) return rc2;
            he = pb.ints[1];
            if (he) return fail(ATC_ETIMEOUT, "a tensor-core kernel gave up waiting (bounded wait expired)");
            double tail = 0.0;
            int rn = select_rank(pb.dbl, ns, rh, rh, &tail);
            if (rn < 0 && rh < n) {
              const int nrh = (int)std::min<int64_t>(n, 2 * (int64_t)rh);
              if (nrh > rh_cap) return 0;
              rh = nrh;
              continue;
            }
            if (rn < 0) rn = (int)n;
            return finish(rn, tail, cand, rh);
          }
        };
        bool done = false;
        // Split paths, n >= 64: the leading eigenvectors by subspace iteration
        // (32 columns, 1 iteration, Rayleigh-Ritz); the Rayleigh-Ritz kernel
        // takes the provisional rank and passes the subspace when the Ritz
        // values show convergence for it; else the full solver.
        if (opt.precision != ATC_PREC_FP64 && n >= 64 && subspace_enabled() &&
            subspace_supported((int)n, (int)std::min<int64_t>(n, kSubK))) {
          const int Ks = (int)std::min<int64_t>(n, kSubK), Ts = kSubIters;
          const int nmax = Ks - kSubMargin;
          double* Usub = nullptr;
          double* edev = nullptr;
          PinnedReadback pb;
          const int ns = rayleigh_splits(n, nmax);
          rc = Scratch::get(SLOT_SUB_U, sizeof(double) * (size_t)n * nmax, (void**)&Usub);
          if (!rc) rc = Scratch::get(SLOT_CAND, sizeof(double) * ((size_t)(nmax + 1) * kRaySplitMax + 8), (void**)&edev);
          // sized for the quotients before anything is copied into it
          if (!rc) rc = pinned_readback((size_t)(nmax + 1) * ns, &pb);
          // decision {rp, nv, passed, tensor-core error word} lands in pb.ints[2..5]
          if (!rc) rc = subspace_solve(G, (int)n, Ks, Ts, budget, kCertExtra, nmax, kSubConv, tc_err, Usub, &pb.ints[2], s);
          // the certification of all nmax columns without waiting for the
          // decision: the leading nv of them are the Ritz vectors when it passes
          if (!rc) rc = launch_rayleigh(G, n, Usub, nmax, edev, s);
          if (!rc && cudaMemcpyAsync(pb.dbl, edev, sizeof(double) * (nmax + 1) * ns, cudaMemcpyDeviceToHost, s) != cudaSuccess)
            rc = fail(ATC_ECUDA, "Rayleigh quotient readback failed");
          if (rc) return bail(rc);
          if (cudaStreamSynchronize(s) != cudaSuccess) return bail(fail(ATC_ECUDA, "stream synchronisation failed"));
          const int dec[4] = {pb.ints[2], pb.ints[3], pb.ints[4], pb.ints[5]};
          he = dec[3];
          if (he) return bail(fail(ATC_ETIMEOUT, "a tensor-core kernel gave up waiting (bounded wait expired)"));
          if (dec[2] && dec[1] >= 1 && dec[1] <= nmax) {
            const int nv = dec[1];
            clk.mark(PH_EIG);
            double tail = 0.0;
            int rn = select_rank(pb.dbl, ns, nmax, nv, &tail);
            if (rn < 0 && nv >= n) rn = (int)n;
            if (rn >= 1) {
              rc = finish(rn, tail, Usub, nmax);  // 1, or an error (< 0)
              if (rc < 0) return bail(rc);
              rc = 0;
              done = true;
              ++st.subspace_modes;
              clk.mark(PH_TTM);
            }
          }
        }
        if (!done) {
        // tridiagonalisation, then only the largest K eigenvalues (more if
        // the rank is not decided among them); tail(r) = trace(G) - sum_{j<r}
        // lambda_j in FP64.
        int K = 0;
        std::vector<double> lh;
        auto eig_rank = [&]() -> int {
          int rc3 = launch_eig_tridiag(G, (int)n, ddev + 2, s, opt.precision != ATC_PREC_FP64);
          if (rc3) return rc3;
          K = (int)std::min<int64_t>(n, 48);
          double tr = 0.0;
          for (;;) {
            rc3 = launch_eig_more((int)n, K, lam, s);
            if (rc3) return rc3;
            lh.resize(K);
            if (cudaMemcpyAsync(lh.data(), lam, sizeof(double) * K, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                cudaMemcpyAsync(&tr, ddev + 2, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                (tc_err && cudaMemcpyAsync(&he, tc_err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess))
              return fail(ATC_ECUDA, "eigenvalue readback failed");
            rc3 = eig_check(s);
            if (rc3) return rc3;
            r = -1;
            double acc = 0.0;
            for (int rr = 1; rr <= K; ++rr) {
              acc += lh[rr - 1];
              double t = tr - acc;
              if (t < 0.0) t = 0.0;
              if (t <= budget) { r = rr; disc = t; break; }
            }
            if (r >= 1) break;
            if (K == n) { r = (int)n; disc = 0.0; break; }
            K = (int)n;
          }
          return ATC_OK;
        };
        rc = eig_rank();
        if (rc) return bail(rc);
        if (opt.precision != ATC_PREC_FP64 && !wide && r >= 1 && r < n && !he) {
          // the subspace of a cut inside a dense part of the spectrum is sensitive to the
          // 24-bit slicing of the Gram input: estimate the shift of the projection and,
          // if it is not negligible, recompute this mode's Gram matrix with four slices
          const SliceScale* sc = xs;
          int shift = 0;
          if (cudaMemcpyAsync(&shift, &sc->shift, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
              cudaStreamSynchronize(s) != cudaSuccess)
            return bail(fail(ATC_ECUDA, "slice scale readback failed"));
          const double q = std::ldexp(1.0, -16 - shift);  // grid of three 8-bit slices
          const double D = subspace_shift_estimate(lh, K, r, n, q);
          if (D > kWideTol * std::sqrt(st.norm2)) {
            wide = true;
            ++st.escalated_modes;
            clk.mark(PH_EIG);
            rc = gram_dispatch(curp, curdt, L, n, R, opt.precision | ATC_PREC_WIDE, G, s, xs);
            if (rc) return bail(rc);
            clk.mark(PH_GRAM);
            rc = eig_rank();
            if (rc) return bail(rc);
          }
        }
        if (he) return bail(fail(ATC_ETIMEOUT, "a tensor-core kernel gave up waiting (bounded wait expired)"));
        if (r < 1 || r > n) return bail(fail(ATC_ENUMERIC, "rank selection failed (r = %d)", r));
        if (opt.precision != ATC_PREC_FP64 && r < n) {
          clk.mark(PH_EIG);
          auto from_eig = [&](int rh, double* cand) -> int {
            if (rh > K) {
              const int rc3 = launch_eig_more((int)n, rh, lam, s);
              if (rc3) return rc3;
              K = rh;
            }
            return launch_eig_vectors((int)n, rh, cand, s);
          };
          rc = certify((int)std::min<int64_t>(n, (int64_t)r + kCertExtra), (int)n, from_eig);
          if (rc < 0) return bail(rc);
          clk.mark(PH_TTM);
        } else {
          if (handle_alloc((void**)&c->factors[m], sizeof(double) * (size_t)n * r, s) != ATC_OK)
            return bail(fail(ATC_ENOMEM, "factor allocation failed"));
          rc = launch_eig_vectors((int)n, r, c->factors[m], s);
          if (rc) return bail(rc);
        }
        }
      }
      clk.mark(PH_EIG);
    }
    if (!have_y) {
      rc = ttm_dispatch(curp, curdt, L, n, R, c->factors[m], r, 0, opt.precision, next, idt, s, xs);
      if (rc) return bail(rc);
      clk.mark(PH_TTM);
    }
    c->ranks[m] = r;
    cur[m] = r;
    used += disc;
    curp = next;
    curdt = idt;
    next = other(curp, nullptr);
  }
  st.sse_trunc = used;
  int64_t ncore = 1;
  for (int i = 0; i < d; ++i) ncore *= c->ranks[i];
  if (handle_alloc((void**)&c->core, sizeof(double) * (size_t)ncore, s) != ATC_OK)
    return bail(fail(ATC_ENOMEM, "core allocation failed"));
  rc = launch_convert_to_f64(curp, curdt, ncore, c->core, s);
  if (rc) return bail(rc);
  // storage order: increasing rank, ties by index (supplement S.2)
  std::vector<int> perm(d);
  for (int i = 0; i < d; ++i) perm[i] = i;
  std::stable_sort(perm.begin(), perm.end(), [&](int a, int b) { return c->ranks[a] < c->ranks[b]; });
  for (int i = 0; i < d; ++i) st.storage_order[i] = perm[i];
  bool ident = true;
  for (int i = 0; i < d; ++i) ident = ident && perm[i] == i;
  // the vectorised core: the core itself when the storage order keeps the mode
  // order (the quantizer only reads it), else its permuted copy
  double* vec = c->core;
  if (!ident) {
    rc = Scratch::get(SLOT_CORE, sizeof(double) * (size_t)ncore, (void**)&vec);
    if (rc) return bail(rc);
    rc = launch_permute(c->core, c->ranks, perm.data(), d, vec, 0, s);
    if (rc) return bail(rc);
  }
  QuantSection section;
  QuantResult qr;
  float msq = 0.f, mse = 0.f;
  clk.mark(PH_OTHER);
  // Split paths: the discarded energy comes from eigenvalues of a Gram matrix
  // with FP32-accumulation and split-residual perturbations; half a percent of
  // the target is held back from the quantizer so the total stays <= rel_eps.
  const double margin = (opt.precision == ATC_PREC_FP64) ? 0.0 : 0.005 * st.target_sse;
  // block_size 0: enough blocks for the GPU's independent (block, plane) streams (Section 4.2 asks for
  // at least as many blocks as workers): a multiple of 32 giving >= 16 blocks, within [512, 4096]
  int bsz = opt.block_size;
  if (bsz == 0) {
    const int64_t want = ((ncore + 15) / 16 + 31) / 32 * 32;
    bsz = (int)std::min<int64_t>(4096, std::max<int64_t>(512, want));
  }
  st.block_size = bsz;
  rc = quantize_encode(vec, ncore, st.target_sse - used - margin, bsz, s, &section, &qr, &msq, &mse);
  if (rc) return bail(rc);
  clk.mark(PH_QUANT);
  st.ms_quant = msq;
  st.ms_encode = mse;
  st.k = qr.k;
  st.p_star = qr.p_star;
  st.prio = qr.prio;
  st.i_lead = qr.i_lead;
  st.i_trail = qr.i_trail;
  st.sse_quant_pred = qr.sse_pred;
  // core slices left without a significant coefficient: their factor columns
  // are not stored (Section 3.3, the paragraph after Table 2)
  int64_t rsum = 0;
  for (int i = 0; i < d; ++i) rsum += c->ranks[i];
  std::vector<uint8_t> kept((size_t)rsum, 0);
  rc = core_kept_slices(ncore, c->ranks, perm.data(), d, qr.p_star, qr.i_lead, kept.data(), s);
  if (rc) return bail(rc);
  // stream (version 2): header, kept-column maps, kept factor columns (raw FP64), core section
  std::vector<std::vector<double>> hfac(d);
  for (int i = 0; i < d; ++i) {
    hfac[i].resize((size_t)dims[i] * c->ranks[i]);
    if (cudaMemcpyAsync(hfac[i].data(), c->factors[i], hfac[i].size() * 8, cudaMemcpyDeviceToHost, s) != cudaSuccess)
      return bail(fail(ATC_ECUDA, "factor readback failed"));
  }
  if (cudaStreamSynchronize(s) != cudaSuccess) return bail(fail(ATC_ECUDA, "stream synchronisation failed"));
  std::string S;  // everything before the core section
  S.append("ATC1", 4);
  put32(S, 2);
  put32(S, (uint32_t)d);
  put32(S, (uint32_t)dtype);
  for (int i = 0; i < d; ++i) put64(S, (uint64_t)dims[i]);
  for (int i = 0; i < d; ++i) put64(S, (uint64_t)c->ranks[i]);
  for (int i = 0; i < d; ++i) put32(S, (uint32_t)perm[i]);
  while (S.size() % 8) S.push_back('\0');
  putf64(S, st.norm2);
  putf64(S, st.sse_trunc);
  {
    int64_t o = 0;
    for (int i = 0; i < d; ++i) {
      for (int64_t b = 0; b < (c->ranks[i] + 7) / 8; ++b) {
        uint8_t byte = 0;
        for (int t = 0; t < 8 && 8 * b + t < c->ranks[i]; ++t) byte |= (uint8_t)(kept[(size_t)(o + 8 * b + t)] << t);
        S.push_back((char)byte);
      }
      o += c->ranks[i];
    }
    while (S.size() % 8) S.push_back('\0');
    o = 0;
    for (int i = 0; i < d; ++i) {
      const int64_t r = c->ranks[i];
      for (int64_t row = 0; row < dims[i]; ++row)
        for (int64_t col = 0; col < r; ++col)
          if (kept[(size_t)(o + col)]) putf64(S, hfac[i][(size_t)(row * r + col)]);
      o += r;
    }
  }
  put64(S, (uint64_t)section.size());
  // one uninitialised host buffer; the core section's payload goes there
  // straight from the device
  c->stream_n = S.size() + section.size();
  c->stream = (uint8_t*)malloc(c->stream_n);
  if (!c->stream) return bail(fail(ATC_ENOMEM, "stream allocation failed"));
  memcpy(c->stream, S.data(), S.size());
  memcpy(c->stream + S.size(), section.head.data(), section.head.size());
  if (section.payload_bytes &&
      (cudaMemcpyAsync(c->stream + S.size() + section.head.size(), section.payload, section.payload_bytes,
                       cudaMemcpyDeviceToHost, s) != cudaSuccess ||
       cudaStreamSynchronize(s) != cudaSuccess))
    return bail(fail(ATC_ECUDA, "core section readback failed"));
  clk.mark(PH_OTHER);
  int he_end = 0;
  if (tc_err && cudaMemcpyAsync(&he_end, tc_err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return bail(fail(ATC_ECUDA, "error flag readback failed"));
  if (cudaStreamSynchronize(s) != cudaSuccess) return bail(fail(ATC_ECUDA, "stream synchronisation failed"));
  if (he_end) return bail(fail(ATC_ETIMEOUT, "a tensor-core kernel gave up waiting (bounded wait expired)"));
  {
    double ph[PH_COUNT];
    clk.sum(ph, PH_COUNT);
    st.ms_norm = ph[PH_NORM];
    st.ms_gram = ph[PH_GRAM];
    st.ms_eig = ph[PH_EIG];
    st.ms_ttm = ph[PH_TTM];
    st.ms_total = clk.total();
  }
  *out = c;
  return ATC_OK;
}

int atc_get_ranks(const atc_compressed* c, int64_t* ranks) {
  if (!c || !ranks) return fail(ATC_EINVAL, "atc_get_ranks: bad arguments");
  for (int i = 0; i < c->ndim; ++i) ranks[i] = c->ranks[i];
  return ATC_OK;
}

int atc_get_core(const atc_compressed* c, const double** core_dev) {
  if (!c || !core_dev) return fail(ATC_EINVAL, "atc_get_core: bad arguments");
  *core_dev = c->core;
  return ATC_OK;
}

int atc_get_factor(const atc_compressed* c, int mode, const double** u_dev) {
  if (!c || !u_dev || mode < 0 || mode >= c->ndim) return fail(ATC_EINVAL, "atc_get_factor: bad arguments");
  *u_dev = c->factors[mode];
  return ATC_OK;
}

int atc_get_stream(const atc_compressed* c, const uint8_t** bytes, size_t* nbytes) {
  if (!c || !bytes || !nbytes) return fail(ATC_EINVAL, "atc_get_stream: bad arguments");
  *bytes = c->stream;
  *nbytes = c->stream_n;
  return ATC_OK;
}

int atc_get_stats(const atc_compressed* c, atc_stats* stats) {
  if (!c || !stats) return fail(ATC_EINVAL, "atc_get_stats: bad arguments");
  *stats = c->stats;
  return ATC_OK;
}

void atc_free(atc_compressed* c) { free_compressed(c); }

int atc_peek_dims(const uint8_t* stream, size_t nbytes, int* ndim, int64_t* dims, int* dtype) {
  if (!stream || !ndim || !dims || !dtype) return fail(ATC_EINVAL, "atc_peek_dims: bad arguments");
  if (nbytes < 16 || memcmp(stream, "ATC1", 4) != 0 || get32(stream + 4) != 2) return fail(ATC_ECORRUPT, "bad stream magic/version");
  const int d = (int)get32(stream + 8);
  const int dt = (int)get32(stream + 12);
  if (d < 1 || d > 8 || !dtype_size(dt)) return fail(ATC_ECORRUPT, "bad stream header");
  if (nbytes < 16 + (size_t)d * 16) return fail(ATC_ECORRUPT, "truncated stream header");
  for (int i = 0; i < d; ++i) dims[i] = (int64_t)get64(stream + 16 + 8 * i);
  *ndim = d;
  *dtype = dt;
  return ATC_OK;
}

int atc_decompress(const uint8_t* stream, size_t nbytes, void* out_dev, int out_dtype, void* cuda_stream) {
  atc_options o;
  atc_default_options(&o);
  o.stream = cuda_stream;
  return atc_decompress_ex(stream, nbytes, out_dev, out_dtype, &o);
}

int atc_decompress_ex(const uint8_t* stream, size_t nbytes, void* out_dev, int out_dtype, const atc_options* opt) {
  if (!stream || !out_dev || !dtype_size(out_dtype)) return fail(ATC_EINVAL, "atc_decompress: bad arguments");
  atc_options o;
  atc_default_options(&o);
  if (opt) o = *opt;
  void* cuda_stream = o.stream;
  const bool split = (o.precision == ATC_PREC_SPLIT_BF16 || o.precision == ATC_PREC_SPLIT_FP16);
  if (!split && o.precision != ATC_PREC_FP64) return fail(ATC_EINVAL, "bad precision %d", (int)o.precision);
  int d = 0, dt = 0;
  int64_t dims[8];
  ATC_TRY(atc_peek_dims(stream, nbytes, &d, dims, &dt));
  cudaStream_t s = (cudaStream_t)cuda_stream;
  size_t off = 16;
  int64_t ranks[8];
  int perm[8];
  off += 8 * d;
  for (int i = 0; i < d; ++i) ranks[i] = (int64_t)get64(stream + off + 8 * i);
  off += 8 * d;
  if (nbytes < off + 4 * d + 16) return fail(ATC_ECORRUPT, "truncated stream header");
  std::vector<int> seen(d, 0);
  for (int i = 0; i < d; ++i) {
    perm[i] = (int)get32(stream + off + 4 * i);
    if (perm[i] < 0 || perm[i] >= d || seen[perm[i]]) return fail(ATC_ECORRUPT, "bad storage order");
    seen[perm[i]] = 1;
  }
  off += 4 * d;
  off = (off + 7) & ~(size_t)7;
  off += 16;  // norm2, sse_trunc
  int64_t ncore = 1, maxn = 0, N = 1;
  for (int i = 0; i < d; ++i) {
    if (ranks[i] < 1 || ranks[i] > dims[i] || dims[i] > 1024) return fail(ATC_ECORRUPT, "bad ranks");
    ncore *= ranks[i];
    N *= dims[i];
    maxn = std::max(maxn, dims[i]);
  }
  // kept-column maps, then the kept columns of every factor; the dropped
  // columns multiply all-zero core slices, so they are rebuilt as zeros
  size_t map_bytes = 0, fac_total = 0, kept_total = 0;
  for (int i = 0; i < d; ++i) map_bytes += (size_t)(ranks[i] + 7) / 8;
  if (nbytes < off + map_bytes + 8) return fail(ATC_ECORRUPT, "truncated column maps");
  std::vector<std::vector<uint8_t>> keep(d);
  {
    size_t mo = off;
    for (int i = 0; i < d; ++i) {
      keep[i].resize((size_t)ranks[i]);
      for (int64_t col = 0; col < ranks[i]; ++col) {
        keep[i][(size_t)col] = (stream[mo + col / 8] >> (col % 8)) & 1;
        kept_total += (size_t)dims[i] * keep[i][(size_t)col];
      }
      mo += (size_t)(ranks[i] + 7) / 8;
      fac_total += (size_t)dims[i] * ranks[i];
    }
  }
  off += (map_bytes + 7) & ~(size_t)7;
  if (nbytes < off + kept_total * 8 + 8) return fail(ATC_ECORRUPT, "truncated factors");
  std::vector<double> hfac(fac_total, 0.0);
  {
    size_t at = off, acc = 0;
    for (int i = 0; i < d; ++i) {
      for (int64_t row = 0; row < dims[i]; ++row)
        for (int64_t col = 0; col < ranks[i]; ++col)
          if (keep[i][(size_t)col]) {
            uint64_t u = get64(stream + at);
            memcpy(&hfac[acc + (size_t)(row * ranks[i] + col)], &u, 8);
            at += 8;
          }
      acc += (size_t)dims[i] * ranks[i];
    }
  }
  double* fac = nullptr;
  ATC_TRY(Scratch::get(SLOT_FAC, fac_total * 8 + 64, (void**)&fac));
  ATC_CUDA_TRY(cudaMemcpyAsync(fac, hfac.data(), fac_total * 8, cudaMemcpyHostToDevice, s));
  double* U[8];
  {
    size_t acc = 0;
    for (int i = 0; i < d; ++i) { U[i] = fac + acc; acc += (size_t)dims[i] * ranks[i]; }
  }
  off += kept_total * 8;
  const uint64_t cb = get64(stream + off);
  off += 8;
  if (cb > nbytes - off) return fail(ATC_ECORRUPT, "truncated core section");
  double* vec = nullptr;
  ATC_TRY(Scratch::get(SLOT_CORE, sizeof(double) * (size_t)ncore, (void**)&vec));
  ATC_TRY(decode_dequantize(stream + off, (size_t)cb, vec, ncore, s));
  // expansion chain in FP64, ping-pong; sizes grow as modes expand
  size_t maxsz = 0;
  {
    std::vector<int> ord = decompression_order(d, dims, ranks);
    int64_t cur[8];
    for (int i = 0; i < d; ++i) cur[i] = ranks[i];
    int64_t sz = ncore;
    maxsz = (size_t)sz;
    for (int m : ord) { sz = sz / cur[m] * dims[m]; cur[m] = dims[m]; maxsz = std::max(maxsz, (size_t)sz); }
  }
  double *A = nullptr, *B = nullptr;
  ATC_TRY(Scratch::get(SLOT_DEC, sizeof(double) * maxsz, (void**)&A));
  ATC_TRY(Scratch::get(SLOT_DEC2, sizeof(double) * maxsz, (void**)&B));
  ATC_TRY(launch_permute(vec, ranks, perm, d, A, 1, s));
  std::vector<int> ord = decompression_order(d, dims, ranks);
  if (split) {
    // tensor-core expansion: FP64 core in, FP32 intermediates (ping-pong in the
    // same scratch), the last step straight into out_dev when it is FP32
    float* fa = reinterpret_cast<float*>(B);
    float* fb = reinterpret_cast<float*>(A);
    const void* src = A;
    int sdt = ATC_F64;
    int64_t cur[8];
    for (int i = 0; i < d; ++i) cur[i] = ranks[i];
    for (size_t q = 0; q < ord.size(); ++q) {
      const int m = ord[q];
      int64_t L = 1, R = 1;
      for (int i = 0; i < m; ++i) L *= cur[i];
      for (int i = m + 1; i < d; ++i) R *= cur[i];
      const bool last = (q + 1 == ord.size());
      float* dst = (last && out_dtype == ATC_F32) ? reinterpret_cast<float*>(out_dev) : fa;
      ATC_TRY(launch_ttm_split(src, sdt, L, dims[m], R, U[m], ranks[m], 1, o.precision, dst, ATC_F32, s));
      cur[m] = dims[m];
      src = dst;
      sdt = ATC_F32;
      std::swap(fa, fb);
    }
    // FP64 output: widen the FP32 result
    if (out_dtype != ATC_F32) ATC_TRY(launch_convert_to_f64(src, ATC_F32, N, reinterpret_cast<double*>(out_dev), s));
    ATC_CUDA_TRY(cudaStreamSynchronize(s));
    return ATC_OK;
  }
  int64_t cur[8];
  for (int i = 0; i < d; ++i) cur[i] = ranks[i];
  double* src = A;
  double* dst = B;
  for (int m : ord) {
    int64_t L = 1, R = 1;
    for (int i = 0; i < m; ++i) L *= cur[i];
    for (int i = m + 1; i < d; ++i) R *= cur[i];
    ATC_TRY(launch_ttm_fp64(src, ATC_F64, L, dims[m], R, U[m], ranks[m], 1, dst, ATC_F64, s));
    cur[m] = dims[m];
    std::swap(src, dst);
  }
  ATC_TRY(launch_convert_f64_to(src, N, out_dev, out_dtype, s));
  ATC_CUDA_TRY(cudaStreamSynchronize(s));
  return ATC_OK;
}

int atc_tucker_expand(const void* core_dev, int core_dtype, const int64_t* ranks, int ndim,
                      const double* const* factors_dev, const int64_t* dims, void* out_dev, int out_dtype,
                      const atc_options* opt) {
  atc_options o;
  atc_default_options(&o);
  if (opt) o = *opt;
  int64_t N = 0;
  ATC_TRY(tucker_args(core_dev, core_dtype, ranks, ndim, factors_dev, dims, o.precision, &N));
  if (!out_dev || !dtype_size(out_dtype)) return fail(ATC_EINVAL, "atc_tucker_expand: bad output");
  cudaStream_t s = (cudaStream_t)o.stream;
  void *A = nullptr, *B = nullptr;
  ATC_TRY(Scratch::get(SLOT_ADJ_A, sizeof(double) * (size_t)N, &A));
  ATC_TRY(Scratch::get(SLOT_ADJ_B, sizeof(double) * (size_t)N, &B));
  int64_t cur[8];
  for (int i = 0; i < ndim; ++i) cur[i] = ranks[i];
  std::vector<int> all(ndim);
  for (int i = 0; i < ndim; ++i) all[i] = i;
  const void* res = nullptr;
  int rdt = 0;
  ATC_TRY(expand_modes(core_dev, core_dtype, cur, ndim, factors_dev, dims, growth_order(all, dims, ranks), o.precision,
                       A, B, s, &res, &rdt));
  if (rdt == out_dtype)
    ATC_CUDA_TRY(cudaMemcpyAsync(out_dev, res, (size_t)N * dtype_size(out_dtype), cudaMemcpyDeviceToDevice, s));
  else if (rdt == ATC_F64)
    ATC_TRY(launch_convert_f64_to((const double*)res, N, out_dev, out_dtype, s));
  else
    ATC_TRY(launch_convert_to_f64(res, rdt, N, (double*)out_dev, s));
  return ATC_OK;
}

int atc_tucker_expand_adjoint(const void* dy_dev, int dy_dtype, const void* core_dev, int core_dtype,
                              const int64_t* ranks, int ndim, const double* const* factors_dev, const int64_t* dims,
                              double* dcore_dev, double* const* dfactors_dev, const atc_options* opt) {
  atc_options o;
  atc_default_options(&o);
  if (opt) o = *opt;
  int64_t N = 0;
  ATC_TRY(tucker_args(core_dev, core_dtype, ranks, ndim, factors_dev, dims, o.precision, &N));
  if (!dy_dev || !dtype_size(dy_dtype)) return fail(ATC_EINVAL, "atc_tucker_expand_adjoint: bad dY");
  cudaStream_t s = (cudaStream_t)o.stream;
  void *A = nullptr, *B = nullptr;
  ATC_TRY(Scratch::get(SLOT_ADJ_A, sizeof(double) * (size_t)N, &A));
  ATC_TRY(Scratch::get(SLOT_ADJ_B, sizeof(double) * (size_t)N, &B));
  int64_t ncore = 1;
  for (int i = 0; i < ndim; ++i) ncore *= ranks[i];
  // dG = dY x_1 U_1^T ... x_d U_d^T: project every mode, largest shrink first
  if (dcore_dev) {
    std::vector<int> ord(ndim);
    for (int i = 0; i < ndim; ++i) ord[i] = i;
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) {
      return (double)dims[a] / (double)ranks[a] > (double)dims[b] / (double)ranks[b];
    });
    const bool split = o.precision != ATC_PREC_FP64;
    const int odt = split ? ATC_F32 : ATC_F64;
    int64_t cur[8];
    for (int i = 0; i < ndim; ++i) cur[i] = dims[i];
    const void* src = dy_dev;
    int sdt = dy_dtype;
    void* dst = A;
    for (int m : ord) {
      int64_t L = 1, R = 1;
      for (int i = 0; i < m; ++i) L *= cur[i];
      for (int i = m + 1; i < ndim; ++i) R *= cur[i];
      ATC_TRY(ttm_dispatch(src, sdt, L, dims[m], R, factors_dev[m], ranks[m], 0, o.precision, dst, odt, s));
      cur[m] = ranks[m];
      src = dst;
      sdt = odt;
      dst = (dst == A) ? B : A;
    }
    if (sdt == ATC_F64)
      ATC_CUDA_TRY(cudaMemcpyAsync(dcore_dev, src, sizeof(double) * (size_t)ncore, cudaMemcpyDeviceToDevice, s));
    else
      ATC_TRY(launch_convert_to_f64(src, sdt, ncore, dcore_dev, s));
  }
  // dU_i = unfold_i(dY) unfold_i(Z_i)^T with Z_i = G x_{j != i} U_j, recomputed per mode
  if (dfactors_dev) {
    for (int i = 0; i < ndim; ++i) {
      if (!dfactors_dev[i]) continue;
      int64_t cur[8];
      for (int q = 0; q < ndim; ++q) cur[q] = ranks[q];
      std::vector<int> others;
      for (int q = 0; q < ndim; ++q)
        if (q != i) others.push_back(q);
      const void* z = nullptr;
      int zdt = 0;
      ATC_TRY(expand_modes(core_dev, core_dtype, cur, ndim, factors_dev, dims, growth_order(others, dims, ranks),
                           o.precision, A, B, s, &z, &zdt));
      int64_t L = 1, R = 1;
      for (int q = 0; q < i; ++q) L *= dims[q];
      for (int q = i + 1; q < ndim; ++q) R *= dims[q];
      ATC_TRY(launch_cross_gram_fp64(dy_dev, dy_dtype, z, zdt, L, dims[i], ranks[i], R, dfactors_dev[i], s));
    }
  }
  return ATC_OK;
}

}  // extern "C"
