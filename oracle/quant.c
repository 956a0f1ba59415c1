/*
 * Plain C oracle of the core quantizer, bit-plane tracker and encoder
 * (TEST INFRASTRUCTURE ONLY: used by the tests, smoke() and the CPU baseline of
 * bench.py; the CUDA library never links it and shares no code with it).
 *
 * What it follows:
 *  - Section 3.3: scale by 2^k with 2^63 <= 2^k max|b| < 2^64, round to the
 *    nearest integer, sign + magnitude bit matrix, bit planes processed from
 *    the most significant one, bit by bit within a plane in vectorised order,
 *    tracking the error that encoding every bit up to that point would give;
 *    the breakpoint is the first bit at which the target is reached.
 *    Leading bits (up to and including a coefficient's first 1) are run-length
 *    coded per plane; sign bits of significant coefficients and trailing bits
 *    are stored raw; insignificant coefficients decode to 0.
 *  - Section 4.2: the vectorised core is cut into equal contiguous blocks that
 *    are encoded independently, with a size table so decoding is parallel.
 *  - Section 4.3: a coefficient decoded down to plane p is reconstructed as
 *    a~ + 2^(p-1), and the tracker uses that same reconstruction.
 *  - Supplement S.6: the run lengths are entropy coded with range ANS.
 *
 * Exact integer tracking: every per-coefficient error is an integer below
 * 2^128 in units of 2^-2k, sums are kept in 192-bit unsigned integers, so the
 * breakpoint does not depend on summation order (this replaces the floating
 * point tracking and recalibration of supplement S.4).
 *
 *  - Supplement S.3 (split bit plane truncation): on the last plane p_star
 *    the leading bits (of coefficients not yet significant) and the trailing
 *    bits (of significant ones) get separate breakpoints i_lead and i_trail.
 *    The category that was encoded more efficiently on plane p_star + 1 (exact
 *    SSE reduction per encoded bit: rANS bytes x 8 + sign bits for the leading
 *    bits, one raw bit per trailing bit) goes first: the plane is walked as its
 *    first category's bits in coefficient order, then the other's, and the
 *    first position whose tracked error reaches the target splits it.
 *
 * Stream layout of one encoded core ("ATCQ" section, little-endian):
 *   char[4] "ATCQ" | u32 version=2 | u64 n | i32 k | u32 block_size |
 *   i32 p_star | u32 priority (0 leading first, 1 trailing first) |
 *   u64 i_lead | u64 i_trail | u32 nplanes | u32 nsym=17 |
 *   u16 freq[nplanes][17] | u32 sizes[nblocks][nplanes][2] | payload
 * Planes are listed from 63 down to p_star.  Payload: for each block, for each
 * plane, the rANS bytes then the raw-bit bytes of that (block, plane) chunk.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_NSYM 17
#define ORC_SCALE_BITS 12
#define ORC_M (1u << ORC_SCALE_BITS)
#define ORC_RANS_L (1u << 23)

typedef unsigned __int128 u128;

/* ---------------------------------------------------------------- 192-bit */
typedef struct { uint64_t w[3]; } u192; /* w[0] least significant */

static u192 u192_from128(u128 v) {
  u192 r; r.w[0] = (uint64_t)v; r.w[1] = (uint64_t)(v >> 64); r.w[2] = 0; return r;
}
static u192 u192_add(u192 a, u192 b) {
  u192 r; u128 s = (u128)a.w[0] + b.w[0];
  r.w[0] = (uint64_t)s;
  s = (u128)a.w[1] + b.w[1] + (uint64_t)(s >> 64);
  r.w[1] = (uint64_t)s;
  r.w[2] = a.w[2] + b.w[2] + (uint64_t)(s >> 64);
  return r;
}
static u192 u192_sub(u192 a, u192 b) { /* a - b mod 2^192 (the borrow propagates) */
  u192 r; uint64_t br = 0;
  for (int i = 0; i < 3; ++i) {
    uint64_t t = a.w[i] - b.w[i];
    uint64_t b1 = a.w[i] < b.w[i];
    uint64_t t2 = t - br;
    uint64_t b2 = t < br;
    r.w[i] = t2; br = b1 | b2;
  }
  return r;
}
static int u192_le(u192 a, u192 b) {
  for (int i = 2; i >= 0; --i) { if (a.w[i] != b.w[i]) return a.w[i] < b.w[i]; }
  return 1;
}

/* ------------------------------------------------------------- quantizer */

/* k such that 2^63 <= 2^k * m < 2^64 for m = max|b| (Section 3.3); 0 if m == 0. */
int orc_scale_exponent(const double* b, int64_t n, int* k_out) {
  double m = 0.0;
  for (int64_t i = 0; i < n; ++i) { double a = fabs(b[i]); if (a > m) m = a; }
  if (!(m == m) || isinf(m)) return -1;
  if (m == 0.0) { *k_out = 0; return 0; }
  int e; frexp(m, &e);      /* m = f 2^e, f in [0.5, 1) */
  *k_out = 64 - e;          /* 2^k m = f 2^64 in [2^63, 2^64) */
  return 0;
}

/* q_i = round-to-nearest-even(|b_i| 2^k), s_i = sign bit of b_i. */
void orc_quantize(const double* b, int64_t n, int k, uint64_t* q, uint8_t* s) {
  for (int64_t i = 0; i < n; ++i) {
    double a = ldexp(fabs(b[i]), k);
    q[i] = (uint64_t)nearbyint(a);
    s[i] = signbit(b[i]) ? 1 : 0;
  }
}

/* Error of one coefficient once all planes >= p are encoded, p in [0, 64]
 * (Section 3.3 with the Section 4.3 reconstruction a~ + 2^(p-1)). */
static u128 coef_err(uint64_t q, int p) {
  if (p >= 64 || (q >> p) == 0) return (u128)q * q;          /* insignificant: decodes to 0 */
  if (p == 0) return 0;                                       /* every bit encoded */
  uint64_t rem = q & ((1ull << p) - 1);                       /* bits below plane p */
  uint64_t c = 1ull << (p - 1);                               /* reconstruction offset */
  uint64_t d = (rem >= c) ? rem - c : c - rem;
  return (u128)d * d;
}

/* floor(T * 2^(2k)) as a u192; returns 0 if T < 0 (unreachable target). */
static int target_scaled(double t, int k, u192* out) {
  memset(out, 0, sizeof(*out));
  if (!(t >= 0.0)) return 0;
  if (t == 0.0) return 1;
  if (isinf(t)) { out->w[0] = out->w[1] = out->w[2] = ~0ull; return 1; }
  int e; double f = frexp(t, &e);
  uint64_t mant = (uint64_t)ldexp(f, 53);        /* exact: t = mant 2^(e-53) */
  long sh = (long)e - 53 + 2L * k;
  if (sh >= 0) {
    if (sh + 53 > 192) { out->w[0] = out->w[1] = out->w[2] = ~0ull; return 1; }
    int limb = (int)(sh / 64), bit = (int)(sh % 64);
    out->w[limb] = mant << bit;
    if (bit && limb + 1 < 3) out->w[limb + 1] = mant >> (64 - bit);
  } else {
    long r = -sh;
    out->w[0] = (r >= 64) ? 0 : (mant >> r);
  }
  return 1;
}

/* Breakpoint (Section 3.3): walk planes 63..0 and, within a plane, the
 * coefficients in order; after each bit the tracked error is updated and the
 * first position whose error is <= target ends the walk.  Coefficients
 * 0..i_star then carry planes >= p_star, the others planes >= p_star + 1.
 * p_star = 64 means nothing is encoded (target met by the all-zero core).
 * err_out receives the tracked error at the breakpoint (3 limbs). */
int orc_breakpoint(const uint64_t* q, int64_t n, double target, int k,
                   int* p_star, int64_t* i_star, uint64_t* err_out) {
  u192 tint; int reachable = target_scaled(target, k, &tint);
  u192 run = {{0, 0, 0}};
  for (int64_t i = 0; i < n; ++i) run = u192_add(run, u192_from128(coef_err(q[i], 64)));
  if (reachable && u192_le(run, tint)) {
    *p_star = 64; *i_star = n - 1;
    memcpy(err_out, run.w, sizeof(run.w));
    return 0;
  }
  for (int p = 63; p >= 0; --p) {
    for (int64_t i = 0; i < n; ++i) {
      u128 before = coef_err(q[i], p + 1), after = coef_err(q[i], p);
      run = u192_sub(u192_add(run, u192_from128(after)), u192_from128(before));
      if (reachable && u192_le(run, tint)) {
        *p_star = p; *i_star = i;
        memcpy(err_out, run.w, sizeof(run.w));
        return 0;
      }
    }
  }
  *p_star = 0; *i_star = n - 1;   /* unreachable target: everything encoded */
  memcpy(err_out, run.w, sizeof(run.w));
  return 0;
}

/* ----------------------------------------------------------- bit writers */
typedef struct { uint8_t* buf; int64_t nbits; int64_t cap; } bitbuf;
static int bb_put(bitbuf* b, int bit) {
  int64_t byte = b->nbits >> 3;
  if (byte >= b->cap) return -1;
  if ((b->nbits & 7) == 0) b->buf[byte] = 0;
  if (bit) b->buf[byte] |= (uint8_t)(1u << (b->nbits & 7));
  b->nbits++;
  return 0;
}

static int run_bucket(uint32_t v) { /* floor(log2(v + 1)) */
  uint32_t x = v + 1; int s = 0;
  while (x >>= 1) ++s;
  return s;
}

/* Leading-bit walk of one (block, plane) chunk: calls back for each run,
 * raw bit and, if cat != NULL, records the category of each visited bit. */
typedef struct { uint32_t* runs; int64_t nruns; int64_t cap; } runlist;

/* hl / ht: end (exclusive) of the coefficients whose leading / trailing bit of
 * plane p is encoded (both the block end except on the last plane). */
static int chunk_walk(const uint64_t* q, const uint8_t* s, int64_t lo, int64_t hl, int64_t ht, int p,
                      runlist* rl, bitbuf* raw, char* cat) {
  uint32_t run = 0;
  rl->nruns = 0;
  int64_t hi = hl > ht ? hl : ht;
  for (int64_t j = lo; j < hi; ++j) {
    int bit = (int)((q[j] >> p) & 1u);
    int sig_before = (p == 63) ? 0 : ((q[j] >> (p + 1)) != 0);
    if (sig_before ? (j >= ht) : (j >= hl)) continue;   /* this category stops earlier here */
    if (sig_before) {                       /* trailing bit, raw */
      if (raw && bb_put(raw, bit)) return -1;
      if (cat) cat[j * 64 + (63 - p)] = 'T';
    } else {                                /* leading bit, run-length coded */
      if (cat) cat[j * 64 + (63 - p)] = 'L';
      if (!bit) { run++; }
      else {
        if (rl->nruns >= rl->cap) return -1;
        rl->runs[rl->nruns++] = run; run = 0;
        if (raw && bb_put(raw, s[j])) return -1;   /* sign of a new significant coefficient */
      }
    }
  }
  if (run > 0) {               /* final run of zeros up to the chunk end */
    if (rl->nruns >= rl->cap) return -1;
    rl->runs[rl->nruns++] = run;
  }
  return 0;
}

/* Deterministic normalisation of a histogram to ORC_M (12-bit) frequencies. */
static void normalize_freq(const uint64_t* cnt, uint16_t* f) {
  uint64_t tot = 0; int best = -1;
  for (int i = 0; i < ORC_NSYM; ++i) { tot += cnt[i]; if (best < 0 || cnt[i] > cnt[best]) best = i; }
  if (tot == 0) { for (int i = 0; i < ORC_NSYM; ++i) f[i] = 0; return; }
  int64_t sum = 0;
  for (int i = 0; i < ORC_NSYM; ++i) {
    uint64_t v = 0;
    if (cnt[i]) { v = (uint64_t)(((u128)cnt[i] * ORC_M) / tot); if (v == 0) v = 1; }
    f[i] = (uint16_t)v; sum += (int64_t)v;
  }
  f[best] = (uint16_t)((int64_t)f[best] + ((int64_t)ORC_M - sum));
}

/* rANS encode of a run list (reverse order); writes into [buf, buf+cap) from
 * the end and returns the number of bytes, which are moved to buf[0..]. */
static int64_t rans_encode(const uint32_t* runs, int64_t nruns, const uint16_t* f, const uint32_t* cum,
                           uint8_t* buf, int64_t cap) {
  if (nruns == 0) return 0;
  uint8_t* end = buf + cap; uint8_t* p = end;
  uint32_t x = ORC_RANS_L;
  for (int64_t r = nruns - 1; r >= 0; --r) {
    uint32_t v = runs[r]; int sb = run_bucket(v);
    uint32_t extra = v + 1 - (1u << sb);
    if (sb > 0) {                           /* uniform extra bits, encoded first (decoded last) */
      uint32_t xmax = (ORC_RANS_L >> sb) << 8;
      while (x >= xmax) { if (p == buf) return -1; *--p = (uint8_t)(x & 0xff); x >>= 8; }
      x = (x << sb) | extra;
    }
    uint32_t fr = f[sb], c = cum[sb];
    uint32_t xmax = ((ORC_RANS_L >> ORC_SCALE_BITS) << 8) * fr;
    while (x >= xmax) { if (p == buf) return -1; *--p = (uint8_t)(x & 0xff); x >>= 8; }
    x = ((x / fr) << ORC_SCALE_BITS) + (x % fr) + c;
  }
  if (p - buf < 4) return -1;
  p -= 4; p[0] = (uint8_t)x; p[1] = (uint8_t)(x >> 8); p[2] = (uint8_t)(x >> 16); p[3] = (uint8_t)(x >> 24);
  int64_t len = end - p;
  memmove(buf, p, (size_t)len);
  return len;
}

static void put_u32(uint8_t* p, uint32_t v) { for (int i = 0; i < 4; ++i) p[i] = (uint8_t)(v >> (8 * i)); }
static void put_u64(uint8_t* p, uint64_t v) { for (int i = 0; i < 8; ++i) p[i] = (uint8_t)(v >> (8 * i)); }
static uint32_t get_u32(const uint8_t* p) { uint32_t v = 0; for (int i = 0; i < 4; ++i) v |= (uint32_t)p[i] << (8 * i); return v; }
static uint64_t get_u64(const uint8_t* p) { uint64_t v = 0; for (int i = 0; i < 8; ++i) v |= (uint64_t)p[i] << (8 * i); return v; }

#define ORC_HDR 56

static int64_t chunk_hi(int64_t lo, int64_t hi, int p, int p_star, int64_t i_star) {
  if (p == p_star && hi > i_star + 1) hi = i_star + 1;
  return hi < lo ? lo : hi;
}

/* rANS bytes of the runs of one full plane p over every block (its own
 * normalised table): the leading-bit encoding cost of that plane. */
int64_t orc_plane_rans_bytes(const uint64_t* q, const uint8_t* s, int64_t n, int block_size, int p) {
  if (block_size < 32 || n < 0 || p < 0 || p > 63) return -1;
  int64_t nblocks = (n + block_size - 1) / block_size;
  uint64_t hist[ORC_NSYM] = {0};
  runlist rl; rl.cap = block_size + 1; rl.runs = malloc(sizeof(uint32_t) * (size_t)rl.cap);
  if (!rl.runs) return -1;
  for (int64_t b = 0; b < nblocks; ++b) {
    int64_t lo = b * block_size, hi = lo + block_size; if (hi > n) hi = n;
    chunk_walk(q, s, lo, hi, hi, p, &rl, NULL, NULL);
    for (int64_t r = 0; r < rl.nruns; ++r) hist[run_bucket(rl.runs[r])]++;
  }
  uint16_t f[ORC_NSYM]; uint32_t cum[ORC_NSYM];
  normalize_freq(hist, f);
  uint32_t c = 0;
  for (int i = 0; i < ORC_NSYM; ++i) { cum[i] = c; c += f[i]; }
  int64_t cap = (int64_t)block_size * 8 + 64, total = 0;
  uint8_t* buf = malloc((size_t)cap);
  if (!buf) { free(rl.runs); return -1; }
  for (int64_t b = 0; b < nblocks; ++b) {
    int64_t lo = b * block_size, hi = lo + block_size; if (hi > n) hi = n;
    chunk_walk(q, s, lo, hi, hi, p, &rl, NULL, NULL);
    int64_t len = rans_encode(rl.runs, rl.nruns, f, cum, buf, cap);
    if (len < 0) { total = -1; break; }
    total += len;
  }
  free(buf); free(rl.runs);
  return total;
}

/* Exact statistics of plane p as one would encode it whole: the SSE
 * reductions of its leading bits (dl) and trailing bits (dt) as signed 192-bit
 * two's-complement limbs, and the counts of leading ones (= signs) and of
 * trailing bits. */
void orc_plane_stats(const uint64_t* q, int64_t n, int p, uint64_t* dl, uint64_t* dt, int64_t* n_ones, int64_t* n_trail) {
  u192 l = {{0, 0, 0}}, t = {{0, 0, 0}};
  int64_t ones = 0, trail = 0;
  for (int64_t j = 0; j < n; ++j) {
    if ((q[j] >> p) == 0) continue;                 /* insignificant through plane p: D = 0 */
    u128 before = coef_err(q[j], p + 1), after = coef_err(q[j], p);
    int sig_before = (p == 63) ? 0 : ((q[j] >> (p + 1)) != 0);
    /* D = before - after, accumulated mod 2^192 (two's complement; u192_sub
     * propagates the borrow, so it is exact modular subtraction) */
    if (sig_before) { t = u192_sub(u192_add(t, u192_from128(before)), u192_from128(after)); ++trail; }
    else { l = u192_sub(u192_add(l, u192_from128(before)), u192_from128(after)); ++ones; }
  }
  memcpy(dl, l.w, sizeof(l.w)); memcpy(dt, t.w, sizeof(t.w));
  *n_ones = ones; *n_trail = trail;
}

/* The split walk of plane p (Supplement S.3): starting from the tracked error
 * after every plane above p, the bits of category `first` (0 leading, 1
 * trailing) in coefficient order, then those of the other category; the first
 * position whose error is <= the target gives (i_lead, i_trail): the first
 * category encoded up to that coefficient and the other not at all, or the
 * first whole and the second up to it.  Returns 1 if the target is reached on
 * the plane, 0 if not (err_out: tracked error at the split point). */
int orc_split_walk(const uint64_t* q, int64_t n, int p, int first, double target, int k,
                   int64_t* i_lead, int64_t* i_trail, uint64_t* err_out) {
  u192 tint; int reachable = target_scaled(target, k, &tint);
  u192 run = {{0, 0, 0}};
  for (int64_t j = 0; j < n; ++j) run = u192_add(run, u192_from128(coef_err(q[j], p + 1)));
  for (int pass = 0; pass < 2; ++pass) {
    int cat = pass == 0 ? first : 1 - first;          /* 0 leading, 1 trailing */
    for (int64_t j = 0; j < n; ++j) {
      int sig_before = (p == 63) ? 0 : ((q[j] >> (p + 1)) != 0);
      if (sig_before != cat) continue;
      u128 before = coef_err(q[j], p + 1), after = coef_err(q[j], p);
      run = u192_sub(u192_add(run, u192_from128(after)), u192_from128(before));
      if (reachable && u192_le(run, tint)) {
        int64_t* ifirst = (first == 0) ? i_lead : i_trail;
        int64_t* isecond = (first == 0) ? i_trail : i_lead;
        if (pass == 0) { *ifirst = j; *isecond = -1; }
        else { *ifirst = n - 1; *isecond = j; }
        memcpy(err_out, run.w, sizeof(run.w));
        return 1;
      }
    }
  }
  memcpy(err_out, run.w, sizeof(run.w));
  return 0;
}

/* Encode the quantized core (q, s) given k and the breakpoint.  Returns the
 * stream size, or -(needed) if cap is too small / -1 on bad arguments.
 * cat (optional, n*64 chars, plane 63 first) receives 'L' / 'T' per encoded bit. */
int64_t orc_encode(const uint64_t* q, const uint8_t* s, int64_t n, int k, int p_star, int prio, int64_t i_lead,
                   int64_t i_trail, int block_size, uint8_t* out, int64_t cap, char* cat) {
  if (block_size < 32 || block_size > 65535 || (block_size % 32) || n < 0) return -1;
  int nplanes = (p_star >= 64) ? 0 : 64 - p_star;
  int64_t nblocks = (n + block_size - 1) / block_size;
  int64_t hdr = ORC_HDR + (int64_t)nplanes * ORC_NSYM * 2;
  int64_t tab = hdr;
  int64_t payload = tab + nblocks * nplanes * 8;
  /* pass 1: per-plane histograms */
  uint64_t* hist = calloc((size_t)(nplanes ? nplanes : 1) * ORC_NSYM, sizeof(uint64_t));
  runlist rl; rl.cap = block_size + 1; rl.runs = malloc(sizeof(uint32_t) * (size_t)rl.cap);
  if (!hist || !rl.runs) { free(hist); free(rl.runs); return -1; }
  for (int pi = 0; pi < nplanes; ++pi) {
    int p = 63 - pi;
    for (int64_t b = 0; b < nblocks; ++b) {
      int64_t lo = b * block_size, hi = lo + block_size; if (hi > n) hi = n;
      chunk_walk(q, s, lo, chunk_hi(lo, hi, p, p_star, i_lead), chunk_hi(lo, hi, p, p_star, i_trail), p, &rl, NULL, cat);
      for (int64_t r = 0; r < rl.nruns; ++r) hist[pi * ORC_NSYM + run_bucket(rl.runs[r])]++;
    }
  }
  uint16_t* freq = calloc((size_t)(nplanes ? nplanes : 1) * ORC_NSYM, sizeof(uint16_t));
  uint32_t* cum = calloc((size_t)(nplanes ? nplanes : 1) * ORC_NSYM, sizeof(uint32_t));
  for (int pi = 0; pi < nplanes; ++pi) {
    normalize_freq(hist + pi * ORC_NSYM, freq + pi * ORC_NSYM);
    uint32_t c = 0;
    for (int i = 0; i < ORC_NSYM; ++i) { cum[pi * ORC_NSYM + i] = c; c += freq[pi * ORC_NSYM + i]; }
  }
  /* pass 2: chunks */
  int64_t scratch_cap = (int64_t)block_size * 8 + 64;
  uint8_t* rbuf = malloc((size_t)scratch_cap);
  uint8_t* wbuf = malloc((size_t)scratch_cap);
  int64_t pos = payload;
  int64_t ok = 1;
  for (int64_t b = 0; b < nblocks && ok; ++b) {
    for (int pi = 0; pi < nplanes; ++pi) {
      int p = 63 - pi;
      int64_t lo = b * block_size, hi = lo + block_size; if (hi > n) hi = n;
      bitbuf raw = {wbuf, 0, scratch_cap};
      if (chunk_walk(q, s, lo, chunk_hi(lo, hi, p, p_star, i_lead), chunk_hi(lo, hi, p, p_star, i_trail), p, &rl, &raw,
                     NULL)) { ok = 0; break; }
      int64_t rlen = rans_encode(rl.runs, rl.nruns, freq + pi * ORC_NSYM, cum + pi * ORC_NSYM, rbuf, scratch_cap);
      if (rlen < 0) { ok = 0; break; }
      int64_t wlen = (raw.nbits + 7) >> 3;
      if (pos + rlen + wlen <= cap) {
        memcpy(out + pos, rbuf, (size_t)rlen);
        memcpy(out + pos + rlen, wbuf, (size_t)wlen);
        put_u32(out + tab + (b * nplanes + pi) * 8, (uint32_t)rlen);
        put_u32(out + tab + (b * nplanes + pi) * 8 + 4, (uint32_t)wlen);
      }
      pos += rlen + wlen;
    }
  }
  free(hist); free(rl.runs); free(rbuf); free(wbuf);
  if (!ok) { free(freq); free(cum); return -1; }
  if (pos > cap) { free(freq); free(cum); return -pos; }
  memcpy(out, "ATCQ", 4);
  put_u32(out + 4, 2);
  put_u64(out + 8, (uint64_t)n);
  put_u32(out + 16, (uint32_t)k);
  put_u32(out + 20, (uint32_t)block_size);
  put_u32(out + 24, (uint32_t)p_star);
  put_u32(out + 28, (uint32_t)prio);
  put_u64(out + 32, (uint64_t)i_lead);
  put_u64(out + 40, (uint64_t)i_trail);
  put_u32(out + 48, (uint32_t)nplanes);
  put_u32(out + 52, ORC_NSYM);
  for (int i = 0; i < nplanes * ORC_NSYM; ++i) { out[ORC_HDR + 2 * i] = (uint8_t)freq[i]; out[ORC_HDR + 2 * i + 1] = (uint8_t)(freq[i] >> 8); }
  free(freq); free(cum);
  return pos;
}

/* ---------------------------------------------------------------- decoder */
typedef struct { const uint8_t* p; const uint8_t* end; uint32_t x; } rdec;
static int rd_byte(rdec* d, uint32_t* b) { if (d->p >= d->end) return -1; *b = *d->p++; return 0; }
static int rd_renorm(rdec* d) {
  while (d->x < ORC_RANS_L) { uint32_t b; if (rd_byte(d, &b)) return -1; d->x = (d->x << 8) | b; }
  return 0;
}
static int rd_run(rdec* d, const uint16_t* f, const uint32_t* cum, uint32_t* v) {
  uint32_t slot = d->x & (ORC_M - 1); int sb = -1;
  for (int i = 0; i < ORC_NSYM; ++i) if (f[i] && slot >= cum[i] && slot < cum[i] + f[i]) { sb = i; break; }
  if (sb < 0) return -1;
  d->x = f[sb] * (d->x >> ORC_SCALE_BITS) + slot - cum[sb];
  if (rd_renorm(d)) return -1;
  uint32_t extra = 0;
  if (sb > 0) { extra = d->x & ((1u << sb) - 1); d->x >>= sb; if (rd_renorm(d)) return -1; }
  *v = (1u << sb) - 1 + extra;
  return 0;
}

/* Parse an ATCQ section; returns 0 and fills the header fields. */
int orc_peek(const uint8_t* in, int64_t nbytes, int64_t* n, int* k, int* block_size, int* p_star, int* prio,
             int64_t* i_lead, int64_t* i_trail) {
  if (nbytes < ORC_HDR || memcmp(in, "ATCQ", 4) || get_u32(in + 4) != 2) return -1;
  *n = (int64_t)get_u64(in + 8); *k = (int)get_u32(in + 16); *block_size = (int)get_u32(in + 20);
  *p_star = (int)get_u32(in + 24); *prio = (int)get_u32(in + 28);
  *i_lead = (int64_t)get_u64(in + 32); *i_trail = (int64_t)get_u64(in + 40);
  return 0;
}

/* Decode to the integer magnitudes q~ (bits of the encoded planes only), the
 * signs and the dequantized doubles (Section 4.3 reconstruction). */
int orc_decode(const uint8_t* in, int64_t nbytes, uint64_t* qt, uint8_t* sg, double* b_out, int64_t n_expect) {
  int64_t n; int k, bs, p_star, prio; int64_t i_lead, i_trail;
  if (orc_peek(in, nbytes, &n, &k, &bs, &p_star, &prio, &i_lead, &i_trail)) return -1;
  if (n != n_expect || bs < 32 || bs > 65535) return -2;
  int nplanes = (int)get_u32(in + 48);
  if (get_u32(in + 52) != ORC_NSYM || nplanes != ((p_star >= 64) ? 0 : 64 - p_star) || nplanes < 0) return -3;
  int64_t nblocks = (n + bs - 1) / bs;
  int64_t tab = ORC_HDR + (int64_t)nplanes * ORC_NSYM * 2;
  int64_t pos = tab + nblocks * nplanes * 8;
  if (pos > nbytes) return -4;
  uint16_t f[64][ORC_NSYM]; uint32_t cum[64][ORC_NSYM];
  for (int pi = 0; pi < nplanes; ++pi) {
    uint32_t c = 0;
    for (int i = 0; i < ORC_NSYM; ++i) {
      const uint8_t* fp = in + ORC_HDR + 2 * (pi * ORC_NSYM + i);
      f[pi][i] = (uint16_t)(fp[0] | (fp[1] << 8)); cum[pi][i] = c; c += f[pi][i];
    }
    if (c != 0 && c != ORC_M) return -5;
  }
  for (int64_t j = 0; j < n; ++j) { qt[j] = 0; sg[j] = 0; }
  for (int64_t b = 0; b < nblocks; ++b) {
    for (int pi = 0; pi < nplanes; ++pi) {
      int p = 63 - pi;
      uint32_t rl = get_u32(in + tab + (b * nplanes + pi) * 8), wl = get_u32(in + tab + (b * nplanes + pi) * 8 + 4);
      if (pos + (int64_t)rl + (int64_t)wl > nbytes) return -6;
      rdec d = {in + pos, in + pos + rl, 0};
      if (rl) { if (rl < 4) return -7; d.x = get_u32(d.p); d.p += 4; }
      const uint8_t* raw = in + pos + rl; int64_t rbit = 0, rcap = (int64_t)wl * 8;
      int64_t lo = b * bs, hi = lo + bs; if (hi > n) hi = n;
      const int64_t hl = chunk_hi(lo, hi, p, p_star, i_lead), ht = chunk_hi(lo, hi, p, p_star, i_trail);
      hi = hl > ht ? hl : ht;
      int need = 1; uint32_t left = 0;
      for (int64_t j = lo; j < hi; ++j) {
        if (qt[j] != 0 ? (j >= ht) : (j >= hl)) continue;
        if (qt[j] != 0) {
          if (rbit >= rcap) return -8;
          uint64_t bit = (raw[rbit >> 3] >> (rbit & 7)) & 1u; rbit++;
          qt[j] |= bit << p;
        } else {
          if (need) { if (!rl) return -9; if (rd_run(&d, f[pi], cum[pi], &left)) return -10; need = 0; }
          if (left > 0) { left--; }
          else {
            qt[j] |= 1ull << p;
            if (rbit >= rcap) return -11;
            sg[j] = (raw[rbit >> 3] >> (rbit & 7)) & 1u; rbit++;
            need = 1;
          }
        }
      }
      pos += rl + wl;
    }
  }
  for (int64_t j = 0; j < n; ++j) {
    if (qt[j] == 0) { b_out[j] = 0.0; continue; }
    /* lowest encoded plane: p_star for a coefficient that became significant
     * on p_star (its leading 1 is there) or whose trailing bit of p_star is
     * encoded (j <= i_trail); p_star + 1 otherwise */
    int sig_above = (p_star >= 63) ? 0 : ((qt[j] >> (p_star + 1)) != 0);
    int pj = (!sig_above || j <= i_trail) ? p_star : p_star + 1;
    uint64_t v = qt[j] + ((pj >= 1) ? (1ull << (pj - 1)) : 0);
    double a = ldexp((double)v, -k);
    b_out[j] = sg[j] ? -a : a;
  }
  return 0;
}
