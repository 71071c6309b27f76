/*
 * lcp_oracle.c -- CPU oracle of the LCP hot path (arXiv 2411.00761).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by tests/, the smoke check and the
 * bench's CPU-baseline leg, never by the product path.  Single-threaded,
 * deliberately plain: every step follows the paper's order and the
 * container rules written out in the design notes, with no blocking, fusion
 * or reordering.
 *
 * Parity status of each part is stated at the function that implements it.
 */
#include "lcp_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ======================================================================== */
/* Exact dyadic arithmetic.                                                  */
/*                                                                           */
/* Every finite binary32 value, and every integer multiple of one, is an     */
/* integer multiple of 2^-149.  A 384-bit two's-complement integer in units  */
/* of 2^-149 holds all values this file needs (|x| < 2^128, (2q+1) e <       */
/* 2^160), so sums, differences and comparisons below are exact.             */
/* ======================================================================== */
#define WL 6
typedef struct {
  uint64_t w[WL];
} wide;

static wide w_zero(void) {
  wide r;
  memset(&r, 0, sizeof r);
  return r;
}
static int w_neg_p(wide a) { return (int)(a.w[WL - 1] >> 63); }
static int w_is_zero(wide a) {
  for (int i = 0; i < WL; i++)
    if (a.w[i]) return 0;
  return 1;
}
static wide w_add(wide a, wide b) {
  wide r;
  unsigned __int128 c = 0;
  for (int i = 0; i < WL; i++) {
    c += (unsigned __int128)a.w[i] + b.w[i];
    r.w[i] = (uint64_t)c;
    c >>= 64;
  }
  return r;
}
static wide w_neg(wide a) {
  wide one = w_zero();
  one.w[0] = 1;
  for (int i = 0; i < WL; i++) a.w[i] = ~a.w[i];
  return w_add(a, one);
}
static wide w_sub(wide a, wide b) { return w_add(a, w_neg(b)); }
static int w_sign(wide a) {
  if (w_neg_p(a)) return -1;
  return w_is_zero(a) ? 0 : 1;
}
static int w_cmp(wide a, wide b) { return w_sign(w_sub(a, b)); }
/* v * 2^sh, v >= 0, 0 <= sh <= 320 */
static wide w_u64_shl(uint64_t v, int sh) {
  wide r = w_zero();
  int limb = sh / 64, bit = sh % 64;
  r.w[limb] |= v << bit;
  if (bit && limb + 1 < WL) r.w[limb + 1] |= v >> (64 - bit);
  return r;
}
/* logical right shift of a non-negative value */
static wide w_shr(wide a, int s) {
  wide r = w_zero();
  for (int i = 0; i < WL; i++) {
    int src = i + s / 64;
    if (src >= WL) continue;
    uint64_t v = a.w[src] >> (s % 64);
    if (s % 64 && src + 1 < WL) v |= a.w[src + 1] << (64 - s % 64);
    r.w[i] = v;
  }
  return r;
}
static int w_msb(wide a) {
  for (int i = WL - 1; i >= 0; i--)
    if (a.w[i]) return i * 64 + 63 - __builtin_clzll(a.w[i]);
  return -1;
}

/* f = (-1)^neg * M * 2^E with integer M < 2^24 */
static void f_parts(float f, int *neg, uint64_t *M, int *E) {
  uint32_t b;
  memcpy(&b, &f, 4);
  *neg = (int)(b >> 31);
  uint32_t ex = (b >> 23) & 0xFFu, fr = b & 0x7FFFFFu;
  if (ex == 0) {
    *M = fr;
    *E = -149;
  } else {
    *M = fr | 0x800000u;
    *E = (int)ex - 150;
  }
}
/* exact value of f in units of 2^-149 */
static wide w_of_f(float f) {
  int neg, E;
  uint64_t M;
  f_parts(f, &neg, &M, &E);
  wide r = w_u64_shl(M, E + 149);
  return neg ? w_neg(r) : r;
}
/* exact value of k * f (k >= 0, k < 2^38) in units of 2^-149 */
static wide w_of_kf(uint64_t k, float f) {
  int neg, E;
  uint64_t M;
  f_parts(f, &neg, &M, &E);
  wide r = w_u64_shl(k * M, E + 149);
  return neg ? w_neg(r) : r;
}
/* nearest binary32 (ties to even) to the exact value a * 2^-149 */
static float w_to_f32_rn(wide a) {
  uint32_t bits;
  if (w_is_zero(a)) return 0.0f;
  int neg = w_neg_p(a);
  wide mag = neg ? w_neg(a) : a;
  int t = w_msb(mag);
  if (t < 23) {
    bits = (uint32_t)mag.w[0]; /* subnormal: exact */
  } else {
    int sh = t - 23;
    uint64_t mant = w_shr(mag, sh).w[0];
    if (sh > 0) {
      wide rem = w_sub(mag, w_u64_shl(mant, sh));
      int c = w_cmp(rem, w_u64_shl(1, sh - 1));
      if (c > 0 || (c == 0 && (mant & 1u))) mant++;
    }
    if (mant == (1ull << 24)) {
      mant >>= 1;
      sh++;
    }
    int bexp = sh + 1;
    if (bexp >= 255)
      bits = 0x7F800000u;
    else
      bits = ((uint32_t)bexp << 23) | (uint32_t)(mant & 0x7FFFFFu);
  }
  if (neg) bits |= 0x80000000u;
  float r;
  memcpy(&r, &bits, 4);
  return r;
}

/* ======================================================================== */
/* Element rules.  Parity pinned by tests/test_oracle_numerics.py against     */
/* Python fractions (exact rationals) on random and bin-edge values.          */
/* ======================================================================== */

/* m + k h <= x ? (exact) */
static int bin_start_le(uint64_t k, float h, float m, float x) {
  wide lhs = w_add(w_of_f(m), w_of_kf(k, h));
  return w_cmp(lhs, w_of_f(x)) <= 0;
}

/* Eq. quantization: q = floor((x - min) / (2 eb)).  The estimate only picks
 * the starting point; the exact predicate decides. */
int64_t orc_q1(float x, float m, float e) {
  float h = 2.0f * e;
  double est = floor(((double)x - (double)m) / (double)h);
  if (!(est >= 0)) est = 0;
  if (est > 1099511627776.0) est = 1099511627776.0; /* 2^40 */
  uint64_t q = (uint64_t)est;
  while (q > 0 && !bin_start_le(q, h, m, x)) q--;
  while (bin_start_le(q + 1, h, m, x)) q++;
  return (int64_t)q;
}

/* Eq. quantization (reverse): x' = (2q + 1) eb + min, rounded once to f32. */
float orc_q2(int64_t q, float m, float e) {
  wide c = w_add(w_of_f(m), w_of_kf((uint64_t)(2 * q + 1), e));
  return w_to_f32_rn(c);
}

/* Eq. abs: the bound is violated when |x - x'| > eb. */
int orc_q3_violates(float x, float xr, float e) {
  wide d = w_sub(w_of_f(x), w_of_f(xr));
  if (w_neg_p(d)) d = w_neg(d);
  return w_cmp(d, w_of_f(e)) > 0;
}

float orc_round_down_f32(double d) {
  float f = (float)d;
  if ((double)f > d) f = nextafterf(f, 0.0f);
  return f;
}

void orc_q1_many(const float *x, size_t n, float m, float e, int64_t *q) {
  for (size_t i = 0; i < n; i++) q[i] = orc_q1(x[i], m, e);
}
void orc_q2_many(const int64_t *q, size_t n, float m, float e, float *xr) {
  for (size_t i = 0; i < n; i++) xr[i] = orc_q2(q[i], m, e);
}
void orc_q3_many(const float *x, const float *xr, size_t n, float e, uint8_t *v) {
  for (size_t i = 0; i < n; i++) v[i] = (uint8_t)orc_q3_violates(x[i], xr[i], e);
}

/* ======================================================================== */
/* Plan: min/max, resolved bounds, qmax, domain rules.                       */
/* ======================================================================== */
static uint32_t f_bits(float f) {
  uint32_t b;
  memcpy(&b, &f, 4);
  return b;
}
/* IEEE totalOrder key for finite values (-0 sorts below +0) */
static uint32_t order_key(float f) {
  uint32_t b = f_bits(f);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

int orc_plan(const float *fields, uint64_t n, uint32_t d, double eb, int eb_mode,
             orc_field_plan *plan) {
  if (d < 1 || d > 8) return ORC_ERR_ARG;
  if (!(eb > 0) || !isfinite(eb)) return ORC_ERR_ARG;
  if (eb_mode != ORC_EB_ABS && eb_mode != ORC_EB_REL) return ORC_ERR_ARG;
  for (uint64_t i = 0; i < n * d; i++)
    if (!isfinite(fields[i])) return ORC_ERR_NONFINITE;
  for (uint32_t f = 0; f < d; f++) {
    float mn = 0.0f, mx = 0.0f;
    if (n > 0) {
      mn = mx = fields[(uint64_t)f * n];
      for (uint64_t i = 1; i < n; i++) {
        float v = fields[(uint64_t)f * n + i];
        if (order_key(v) < order_key(mn)) mn = v;
        if (order_key(v) > order_key(mx)) mx = v;
      }
    }
    double range = (double)mx - (double)mn;
    double ebf = eb;
    if (eb_mode == ORC_EB_REL && range > 0) ebf = eb * range;
    float e = orc_round_down_f32(ebf);
    if (!(e >= 0x1p-100f) || !(e <= 0x1p100f)) return ORC_ERR_ARG;
    plan[f].min_f = mn;
    plan[f].max_f = mx;
    plan[f].eb_f = ebf;
    plan[f].e = e;
    /* The bins of a field must number below 2^30 (the key space rule).  A
     * quotient estimate at or above 2^31 settles that without the exact
     * count: the double estimate is within a relative 2^-51 of the exact
     * quotient, whose floor is then at least 2^31 - 1 >= 2^30, so the frame
     * is refused exactly when the exact rule below would refuse it. */
    double qest = ((double)mx - (double)mn) / (2.0 * (double)e);
    if (!(qest < 2147483648.0)) return ORC_ERR_RANGE;
    int64_t qmax = orc_q1(mx, mn, e);
    if (qmax >= (1ll << 30)) return ORC_ERR_RANGE;
    /* No rule on |value| / eb: Eq. quantization is defined for every real
     * value, and the exact arithmetic above covers every finite binary32. */
    plan[f].qmax = (uint32_t)qmax;
  }
  return ORC_OK;
}

/* ======================================================================== */
/* Streams: Huffman / fixed-length choice (Sec. "Block coding").             */
/* ======================================================================== */
#define ALPHA 4096
#define ESC 4095
#define LMAX 24

static int bits_of(uint64_t v) { return v ? 64 - __builtin_clzll(v) : 0; }
static uint64_t pad16(uint64_t b) { return (b + 15) & ~(uint64_t)15; }
static uint64_t words_of_bits(uint64_t bits) { return (bits + 31) / 32; }

typedef struct {
  uint64_t f;
  uint32_t s;
} leaf;
static int leaf_cmp(const void *a, const void *b) {
  const leaf *x = a, *y = b;
  if (x->f != y->f) return x->f < y->f ? -1 : 1;
  return x->s < y->s ? -1 : (x->s > y->s);
}

/* Code lengths by the two-queue Huffman construction: leaves ordered by
 * (weight, symbol); when a leaf and an internal node weigh the same the leaf
 * is taken first; internal nodes leave their queue in creation order.  Lengths
 * above 24 halve every used weight (rounding up) and rebuild.  One used
 * symbol gets length 1.  Parity pinned by brute-force optimal prefix codes
 * and the Kraft equality in tests/test_oracle_huffman.py. */
int orc_huffman_lengths(const uint64_t *freq, uint8_t *len) {
  uint64_t w[ALPHA];
  uint32_t U = 0;
  for (int s = 0; s < ALPHA; s++) {
    w[s] = freq[s];
    len[s] = 0;
    if (freq[s]) U++;
  }
  if (U == 0) return 0;
  if (U == 1) {
    for (int s = 0; s < ALPHA; s++)
      if (w[s]) len[s] = 1;
    return 1;
  }
  leaf *lv = malloc(sizeof(leaf) * U);
  uint64_t *nw = malloc(sizeof(uint64_t) * 2 * U);
  uint32_t *parent = malloc(sizeof(uint32_t) * 2 * U);
  uint32_t *depth = malloc(sizeof(uint32_t) * 2 * U);
  int maxlen;
  for (;;) {
    uint32_t k = 0;
    for (int s = 0; s < ALPHA; s++)
      if (w[s]) {
        lv[k].f = w[s];
        lv[k].s = (uint32_t)s;
        k++;
      }
    qsort(lv, U, sizeof(leaf), leaf_cmp);
    for (uint32_t i = 0; i < U; i++) nw[i] = lv[i].f;
    uint32_t nl = 0, ni = U, nnew = U;
    while (nnew < 2 * U - 1) {
      uint32_t pick[2];
      for (int t = 0; t < 2; t++) {
        if (nl < U && (ni == nnew || nw[nl] <= nw[ni]))
          pick[t] = nl++;
        else
          pick[t] = ni++;
      }
      nw[nnew] = nw[pick[0]] + nw[pick[1]];
      parent[pick[0]] = nnew;
      parent[pick[1]] = nnew;
      nnew++;
    }
    depth[2 * U - 2] = 0;
    for (int64_t i = (int64_t)(2 * U) - 3; i >= 0; i--) depth[i] = depth[parent[i]] + 1;
    maxlen = 0;
    for (uint32_t i = 0; i < U; i++)
      if ((int)depth[i] > maxlen) maxlen = (int)depth[i];
    if (maxlen <= LMAX) {
      for (uint32_t i = 0; i < U; i++) len[lv[i].s] = (uint8_t)depth[i];
      break;
    }
    for (int s = 0; s < ALPHA; s++)
      if (w[s]) w[s] = (w[s] + 1) >> 1;
  }
  free(lv);
  free(nw);
  free(parent);
  free(depth);
  return maxlen;
}

typedef struct {
  int coder; /* 0 fixed, 1 huffman */
  int width; /* fixed: w; huffman: escape width */
  uint32_t U;
  uint64_t n, payload_bits, maxv, n_chunks;
  uint8_t len[ALPHA];
  uint32_t code[ALPHA];
  uint16_t cnt_len[LMAX + 1];
  uint16_t syms[ALPHA];
  uint64_t bytes;
} stream_plan;

static void plan_stream(const uint64_t *v, uint64_t n, uint32_t log2_chunk, stream_plan *sp) {
  memset(sp, 0, sizeof *sp);
  sp->n = n;
  uint64_t maxv = 0;
  for (uint64_t i = 0; i < n; i++)
    if (v[i] > maxv) maxv = v[i];
  sp->maxv = maxv;
  int w = bits_of(maxv);
  uint64_t fixed_bits = n * (uint64_t)w;
  uint64_t fixed_bytes = 32 + pad16(4 * words_of_bits(fixed_bits));
  sp->coder = 0;
  sp->width = w;
  sp->payload_bits = fixed_bits;
  sp->bytes = fixed_bytes;
  if (n == 0) return;

  uint64_t *hist = calloc(ALPHA, sizeof(uint64_t));
  for (uint64_t i = 0; i < n; i++) hist[v[i] < ESC ? v[i] : ESC]++;
  int wesc = hist[ESC] ? bits_of(maxv) : 0;
  uint8_t len[ALPHA];
  orc_huffman_lengths(hist, len);
  uint64_t bits = 0;
  uint32_t U = 0;
  for (int s = 0; s < ALPHA; s++) {
    bits += hist[s] * len[s];
    if (len[s]) U++;
  }
  bits += hist[ESC] * (uint64_t)wesc;
  uint64_t n_chunks = (n + (1ull << log2_chunk) - 1) >> log2_chunk;
  uint64_t huff_bytes =
      pad16(80 + 2ull * U) + pad16(8 * n_chunks) + pad16(4 * words_of_bits(bits));
  free(hist);
  if (huff_bytes < fixed_bytes) {
    sp->coder = 1;
    sp->width = wesc;
    sp->U = U;
    sp->payload_bits = bits;
    sp->n_chunks = n_chunks;
    sp->bytes = huff_bytes;
    memcpy(sp->len, len, ALPHA);
    /* canonical codes: symbols by (length, symbol), codes counted upward */
    uint32_t k = 0, code = 0;
    int prev = 0;
    for (int L = 1; L <= LMAX; L++)
      for (int s = 0; s < ALPHA; s++)
        if (len[s] == L) {
          if (k > 0) code = (code + 1) << (L - prev);
          sp->code[s] = code;
          sp->syms[k++] = (uint16_t)s;
          sp->cnt_len[L]++;
          prev = L;
        }
  }
}

/* little-endian stores into the byte buffer */
static void st8(uint8_t *p, uint8_t v) { p[0] = v; }
static void st16(uint8_t *p, uint16_t v) {
  for (int i = 0; i < 2; i++) p[i] = (uint8_t)(v >> (8 * i));
}
static void st32(uint8_t *p, uint32_t v) {
  for (int i = 0; i < 4; i++) p[i] = (uint8_t)(v >> (8 * i));
}
static void st64(uint8_t *p, uint64_t v) {
  for (int i = 0; i < 8; i++) p[i] = (uint8_t)(v >> (8 * i));
}
static uint16_t ld16(const uint8_t *p) { return (uint16_t)(p[0] | (p[1] << 8)); }
static uint32_t ld32(const uint8_t *p) {
  uint32_t v = 0;
  for (int i = 3; i >= 0; i--) v = (v << 8) | p[i];
  return v;
}
static uint64_t ld64(const uint8_t *p) {
  uint64_t v = 0;
  for (int i = 7; i >= 0; i--) v = (v << 8) | p[i];
  return v;
}
static float ldf(const uint8_t *p) {
  uint32_t b = ld32(p);
  float f;
  memcpy(&f, &b, 4);
  return f;
}

/* Bit order: bit b of a payload is bit (31 - b % 32) of little-endian u32
 * word b / 32; values are written most significant bit first. */
static void put_bits(uint8_t *payload, uint64_t *pos, uint64_t v, int nbits) {
  for (int i = nbits - 1; i >= 0; i--) {
    if ((v >> i) & 1u) {
      uint64_t b = *pos;
      uint8_t *wp = payload + 4 * (b / 32);
      uint32_t word = ld32(wp) | (1u << (31 - b % 32));
      st32(wp, word);
    }
    (*pos)++;
  }
}
static uint64_t get_bits(const uint8_t *payload, uint64_t *pos, int nbits) {
  uint64_t v = 0;
  for (int i = 0; i < nbits; i++) {
    uint64_t b = *pos;
    uint32_t word = ld32(payload + 4 * (b / 32));
    v = (v << 1) | ((word >> (31 - b % 32)) & 1u);
    (*pos)++;
  }
  return v;
}

/* writes the section planned in sp for values v at dst (zeroed, sp->bytes) */
static void write_stream(uint8_t *dst, const stream_plan *sp, const uint64_t *v,
                         uint32_t log2_chunk) {
  st8(dst + 0, (uint8_t)sp->coder);
  st8(dst + 1, (uint8_t)sp->width);
  st16(dst + 2, (uint16_t)sp->U);
  st32(dst + 4, 0);
  st64(dst + 8, sp->n);
  st64(dst + 16, sp->payload_bits);
  st64(dst + 24, sp->maxv);
  if (sp->coder == 0) {
    uint8_t *pl = dst + 32;
    uint64_t pos = 0;
    for (uint64_t i = 0; i < sp->n; i++) put_bits(pl, &pos, v[i], sp->width);
    return;
  }
  for (int L = 1; L <= LMAX; L++) st16(dst + 32 + 2 * (L - 1), sp->cnt_len[L]);
  for (uint32_t k = 0; k < sp->U; k++) st16(dst + 80 + 2 * k, sp->syms[k]);
  uint8_t *ct = dst + pad16(80 + 2ull * sp->U);
  uint8_t *pl = ct + pad16(8 * sp->n_chunks);
  uint64_t pos = 0;
  for (uint64_t i = 0; i < sp->n; i++) {
    if ((i & ((1ull << log2_chunk) - 1)) == 0) st64(ct + 8 * (i >> log2_chunk), pos);
    uint32_t s = v[i] < ESC ? (uint32_t)v[i] : ESC;
    put_bits(pl, &pos, sp->code[s], sp->len[s]);
    if (s == ESC) put_bits(pl, &pos, v[i], sp->width);
  }
}

/* decodes a section of `bytes` at src into v[n]; returns status */
static int read_stream(const uint8_t *src, uint64_t bytes, uint64_t n_expect,
                       uint32_t log2_chunk, uint64_t *v) {
  if (bytes < 32) return ORC_ERR_FORMAT;
  int coder = src[0], width = src[1];
  uint32_t U = ld16(src + 2);
  uint64_t n = ld64(src + 8), pbits = ld64(src + 16);
  if (n != n_expect || width > 64) return ORC_ERR_FORMAT;
  if (coder == 0) {
    if (pbits != n * (uint64_t)width) return ORC_ERR_FORMAT;
    if (bytes != 32 + pad16(4 * words_of_bits(pbits))) return ORC_ERR_FORMAT;
    uint64_t pos = 0;
    for (uint64_t i = 0; i < n; i++) v[i] = get_bits(src + 32, &pos, width);
    return ORC_OK;
  }
  if (coder != 1 || U == 0 || U > ALPHA) return ORC_ERR_FORMAT;
  uint64_t n_chunks = (n + (1ull << log2_chunk) - 1) >> log2_chunk;
  uint64_t hdr = pad16(80 + 2ull * U);
  if (bytes != hdr + pad16(8 * n_chunks) + pad16(4 * words_of_bits(pbits)))
    return ORC_ERR_FORMAT;
  uint32_t count[LMAX + 1], first[LMAX + 2], index[LMAX + 2];
  uint32_t total = 0;
  for (int L = 1; L <= LMAX; L++) {
    count[L] = ld16(src + 32 + 2 * (L - 1));
    total += count[L];
  }
  if (total != U) return ORC_ERR_FORMAT;
  /* canonical decode tables: first code and first symbol index per length */
  uint32_t code = 0, idx = 0;
  for (int L = 1; L <= LMAX; L++) {
    code <<= 1;
    first[L] = code;
    index[L] = idx;
    code += count[L];
    idx += count[L];
  }
  const uint8_t *ct = src + hdr;
  const uint8_t *pl = ct + pad16(8 * n_chunks);
  uint64_t pos = 0;
  for (uint64_t i = 0; i < n; i++) {
    if ((i & ((1ull << log2_chunk) - 1)) == 0 && ld64(ct + 8 * (i >> log2_chunk)) != pos)
      return ORC_ERR_FORMAT;
    uint32_t c = 0;
    int L = 0, found = 0;
    uint32_t sym = 0;
    while (L < LMAX) {
      c = (c << 1) | (uint32_t)get_bits(pl, &pos, 1);
      L++;
      if (c - first[L] < count[L]) {
        sym = ld16(src + 80 + 2 * (index[L] + (c - first[L])));
        found = 1;
        break;
      }
    }
    if (!found || pos > pbits) return ORC_ERR_FORMAT;
    v[i] = sym;
    if (sym == ESC) v[i] = get_bits(pl, &pos, width);
  }
  if (pos != pbits) return ORC_ERR_FORMAT;
  return ORC_OK;
}

/* ======================================================================== */
/* Container                                                                  */
/* ======================================================================== */
#define HDR_FIXED 48

static uint64_t header_bytes(uint32_t d, uint32_t ns) { return HDR_FIXED + 16ull * d + 16ull * ns + 16; }

size_t orc_max_compressed_size(uint64_t n, uint32_t d, uint32_t log2_chunk) {
  (void)log2_chunk;
  return (size_t)(HDR_FIXED + 16ull * d + 64 + 256 + (24 + 16ull * d) * n);
}

static uint64_t zz(int64_t v) { return v >= 0 ? (uint64_t)v << 1 : ((uint64_t)(-(v + 1)) << 1) | 1u; }
static int64_t unzz(uint64_t u) { return (u & 1u) ? -(int64_t)(u >> 1) - 1 : (int64_t)(u >> 1); }

static void write_header(uint8_t *out, int method, uint32_t d, uint32_t log2_chunk, uint32_t flags,
                         uint32_t p, uint64_t n, uint64_t k, uint64_t m, uint64_t total,
                         const orc_field_plan *plan, uint32_t ns, const uint64_t *sec_off,
                         const uint64_t *sec_bytes) {
  out[0] = 'L';
  out[1] = 'C';
  out[2] = 'P';
  out[3] = '1';
  out[4] = 1;
  out[5] = (uint8_t)method;
  out[6] = (uint8_t)d;
  out[7] = (uint8_t)log2_chunk;
  st32(out + 8, flags);
  st32(out + 12, p);
  st64(out + 16, n);
  st64(out + 24, k);
  st64(out + 32, m);
  st64(out + 40, total);
  for (uint32_t f = 0; f < d; f++) {
    uint8_t *fp = out + HDR_FIXED + 16 * f;
    st32(fp, f_bits(plan[f].min_f));
    st32(fp + 4, f_bits(plan[f].e));
    st32(fp + 8, plan[f].qmax);
    st32(fp + 12, 0);
  }
  uint8_t *sd = out + HDR_FIXED + 16 * d;
  for (uint32_t s = 0; s <= ns; s++) {
    st64(sd + 16 * s, sec_off[s]);
    st64(sd + 16 * s + 8, sec_bytes[s]);
  }
}

/* ======================================================================== */
/* LCP-S (Sec. "LCP-S"): quantize, block, sort, delta, code.                 */
/* ======================================================================== */
typedef struct {
  uint64_t key;
  uint64_t idx;
} keyed;
static int keyed_cmp(const void *a, const void *b) {
  const keyed *x = a, *y = b;
  if (x->key != y->key) return x->key < y->key ? -1 : 1;
  return x->idx < y->idx ? -1 : (x->idx > y->idx);
}

static int log2_exact(uint32_t p) {
  int l = 0;
  while ((1u << l) < p) l++;
  return (1u << l) == p ? l : -1;
}

int orc_compress_s(const float *fields, uint64_t n, uint32_t d, double eb, int eb_mode,
                   uint32_t p, uint32_t log2_chunk, uint32_t flags, uint8_t *out,
                   size_t out_cap, size_t *out_size, uint32_t *pi_out, int32_t *q_out,
                   uint64_t *ids, uint64_t *cnts, uint64_t *rels, uint64_t *m_out,
                   uint64_t *k_out) {
  if (d < 1 || d > 8) return ORC_ERR_ARG;
  int lp = log2_exact(p);
  if (p < 1 || p > 65536 || lp < 0 || (uint32_t)lp * d > 32) return ORC_ERR_ARG;
  if (log2_chunk < 5 || log2_chunk > 16) return ORC_ERR_ARG;
  orc_field_plan plan[8];
  int st = orc_plan(fields, n, d, eb, eb_mode, plan);
  if (st) return st;

  /* Eq. block size and id: bn_f blocks per dimension, field 0 fastest */
  uint64_t bn[8], stride[8];
  unsigned __int128 blocks = 1;
  for (uint32_t f = 0; f < d; f++) {
    bn[f] = (uint64_t)(plan[f].qmax >> lp) + 1;
    stride[f] = (uint64_t)blocks;
    blocks *= bn[f];
    if (blocks > ((unsigned __int128)1 << 64)) return ORC_ERR_RANGE;
  }
  if ((blocks << (lp * d)) > ((unsigned __int128)1 << 63)) return ORC_ERR_RANGE;

  int64_t *q = malloc(sizeof(int64_t) * (n * d + 1));
  uint8_t *outl = calloc(n + 1, 1);
  keyed *arr = malloc(sizeof(keyed) * (n + 1));
  if (!q || !outl || !arr) {
    free(q);
    free(outl);
    free(arr);
    return ORC_ERR_NOMEM;
  }
  /* Eq. quantization per field; a particle whose reconstruction misses the
   * bound in any field is kept raw (an outlier) */
  uint64_t K = 0;
  for (uint64_t i = 0; i < n; i++) {
    for (uint32_t f = 0; f < d; f++) {
      float x = fields[(uint64_t)f * n + i];
      int64_t qq = orc_q1(x, plan[f].min_f, plan[f].e);
      q[(uint64_t)f * n + i] = qq;
      float xr = orc_q2(qq, plan[f].min_f, plan[f].e);
      if (orc_q3_violates(x, xr, plan[f].e)) outl[i] = 1;
    }
    K += outl[i];
  }
  /* key = block_id * p^D + rel, rel_f = q_f mod p placed at bits f*lp */
  uint64_t nb = 0;
  for (uint64_t i = 0; i < n; i++) {
    if (outl[i]) continue;
    uint64_t bid = 0, rel = 0;
    for (uint32_t f = 0; f < d; f++) {
      uint64_t qq = (uint64_t)q[(uint64_t)f * n + i];
      bid += (qq >> lp) * stride[f];
      rel |= (qq & ((1ull << lp) - 1)) << (f * lp);
    }
    arr[nb].key = (bid << (lp * d)) | rel;
    arr[nb].idx = i;
    nb++;
  }
  /* blocks in increasing id, particles of a block by relative code; equal
   * keys by original index (this only fixes the slot permutation) */
  qsort(arr, nb, sizeof(keyed), keyed_cmp);

  uint64_t M = 0;
  for (uint64_t k = 0; k < nb; k++)
    if (k == 0 || (arr[k].key >> (lp * d)) != (arr[k - 1].key >> (lp * d))) M++;
  uint64_t *s_id = malloc(sizeof(uint64_t) * (M + 1));
  uint64_t *s_cnt = malloc(sizeof(uint64_t) * (M + 1));
  uint64_t *s_rel = malloc(sizeof(uint64_t) * (nb + 1));
  /* delta coding of the three arrays (Sec. "Block coding") */
  uint64_t prev_bid = 0;
  int64_t prev_cnt = 0;
  uint64_t bi = 0, cur = 0, chunk_mask = (1ull << log2_chunk) - 1;
  for (uint64_t k = 0; k < nb; k++) {
    uint64_t bid = arr[k].key >> (lp * d);
    uint64_t rel = arr[k].key & ((lp * d) == 64 ? ~0ull : ((1ull << (lp * d)) - 1));
    int start = (k == 0) || bid != (arr[k - 1].key >> (lp * d));
    if (start) {
      if (k > 0) {
        s_cnt[bi - 1] = zz((int64_t)cur - prev_cnt);
        prev_cnt = (int64_t)cur;
      }
      s_id[bi] = bid - prev_bid;
      prev_bid = bid;
      bi++;
      cur = 0;
    }
    cur++;
    if (start || (k & chunk_mask) == 0)
      s_rel[k] = rel;
    else
      s_rel[k] = rel - (arr[k - 1].key & ((1ull << (lp * d)) - 1));
  }
  if (nb > 0) s_cnt[bi - 1] = zz((int64_t)cur - prev_cnt);

  stream_plan *sp = malloc(sizeof(stream_plan) * 3);
  plan_stream(s_id, M, log2_chunk, &sp[0]);
  plan_stream(s_cnt, M, log2_chunk, &sp[1]);
  plan_stream(s_rel, nb, log2_chunk, &sp[2]);
  uint64_t sec_off[4], sec_bytes[4];
  uint64_t off = header_bytes(d, 3);
  for (int s = 0; s < 3; s++) {
    sec_off[s] = off;
    sec_bytes[s] = sp[s].bytes;
    off += sp[s].bytes;
  }
  sec_off[3] = off;
  sec_bytes[3] = pad16(4ull * d * K);
  off += sec_bytes[3];
  uint64_t total = off;
  *out_size = (size_t)total;
  if (m_out) *m_out = M;
  if (k_out) *k_out = K;
  if (ids) memcpy(ids, s_id, sizeof(uint64_t) * M);
  if (cnts) memcpy(cnts, s_cnt, sizeof(uint64_t) * M);
  if (rels) memcpy(rels, s_rel, sizeof(uint64_t) * nb);
  if (pi_out || q_out) {
    uint64_t j = 0;
    for (uint64_t k = 0; k < nb; k++, j++) {
      if (pi_out) pi_out[j] = (uint32_t)arr[k].idx;
      if (q_out)
        for (uint32_t f = 0; f < d; f++)
          q_out[(uint64_t)f * n + j] = (int32_t)q[(uint64_t)f * n + arr[k].idx];
    }
    for (uint64_t i = 0; i < n; i++)
      if (outl[i]) {
        if (pi_out) pi_out[j] = (uint32_t)i;
        if (q_out)
          for (uint32_t f = 0; f < d; f++) q_out[(uint64_t)f * n + j] = (int32_t)q[(uint64_t)f * n + i];
        j++;
      }
  }
  if (total > out_cap || !out) {
    st = ORC_ERR_CAPACITY;
  } else {
    memset(out, 0, (size_t)total);
    write_header(out, 0, d, log2_chunk, flags, p, n, K, M, total, plan, 3, sec_off, sec_bytes);
    write_stream(out + sec_off[0], &sp[0], s_id, log2_chunk);
    write_stream(out + sec_off[1], &sp[1], s_cnt, log2_chunk);
    write_stream(out + sec_off[2], &sp[2], s_rel, log2_chunk);
    /* outliers: raw values, field-major, in increasing original index */
    uint64_t j = 0;
    for (uint64_t i = 0; i < n; i++)
      if (outl[i]) {
        for (uint32_t f = 0; f < d; f++)
          st32(out + sec_off[3] + 4 * ((uint64_t)f * K + j), f_bits(fields[(uint64_t)f * n + i]));
        j++;
      }
    st = ORC_OK;
  }
  free(sp);
  free(s_id);
  free(s_cnt);
  free(s_rel);
  free(q);
  free(outl);
  free(arr);
  return st;
}

/* ======================================================================== */
/* LCP-T (Sec. "LCP-T"): quantize, predict from the reference, code the      */
/* difference.  The reference is held as its codes in decoded-slot order and  */
/* the slot -> original-index map of the chain.                               */
/* ======================================================================== */
int orc_compress_t(const float *fields, uint64_t n, uint32_t d, double eb, int eb_mode,
                   const int32_t *ref_q, const uint32_t *ref_pi, uint32_t log2_chunk,
                   uint32_t flags, uint8_t *out, size_t out_cap, size_t *out_size,
                   int32_t *q_out, uint64_t *syms, uint64_t *k_out) {
  if (log2_chunk < 5 || log2_chunk > 16) return ORC_ERR_ARG;
  if (!ref_q || !ref_pi) return ORC_ERR_STATE;
  orc_field_plan plan[8];
  int st = orc_plan(fields, n, d, eb, eb_mode, plan);
  if (st) return st;
  uint64_t nd = n * d;
  uint64_t *sym = malloc(sizeof(uint64_t) * (nd + 1));
  uint64_t *pidx = malloc(sizeof(uint64_t) * (nd + 1));
  float *praw = malloc(sizeof(float) * (nd + 1));
  int32_t *qt = malloc(sizeof(int32_t) * (nd + 1));
  uint64_t K = 0;
  /* symbol s = f * n + j: zigzag of this frame's code of the particle in slot
   * j minus the reference code of slot j */
  for (uint32_t f = 0; f < d; f++)
    for (uint64_t j = 0; j < n; j++) {
      uint64_t i = ref_pi[j];
      float x = fields[(uint64_t)f * n + i];
      int64_t qq = orc_q1(x, plan[f].min_f, plan[f].e);
      uint64_t s = (uint64_t)f * n + j;
      qt[s] = (int32_t)qq;
      sym[s] = zz(qq - (int64_t)ref_q[s]);
      float xr = orc_q2(qq, plan[f].min_f, plan[f].e);
      if (orc_q3_violates(x, xr, plan[f].e)) {
        pidx[K] = s;
        praw[K] = x;
        K++;
      }
    }
  stream_plan *sp = malloc(sizeof(stream_plan));
  plan_stream(sym, nd, log2_chunk, sp);
  uint64_t sec_off[2], sec_bytes[2];
  uint64_t off = header_bytes(d, 1);
  sec_off[0] = off;
  sec_bytes[0] = sp->bytes;
  off += sp->bytes;
  sec_off[1] = off;
  sec_bytes[1] = pad16(8 * K) + pad16(4 * K);
  off += sec_bytes[1];
  *out_size = (size_t)off;
  if (k_out) *k_out = K;
  if (q_out) memcpy(q_out, qt, sizeof(int32_t) * nd);
  if (syms) memcpy(syms, sym, sizeof(uint64_t) * nd);
  if (off > out_cap || !out) {
    st = ORC_ERR_CAPACITY;
  } else {
    memset(out, 0, (size_t)off);
    write_header(out, 1, d, log2_chunk, flags, 0, n, K, 0, off, plan, 1, sec_off, sec_bytes);
    write_stream(out + sec_off[0], sp, sym, log2_chunk);
    for (uint64_t k = 0; k < K; k++) {
      st64(out + sec_off[1] + 8 * k, pidx[k]);
      st32(out + sec_off[1] + pad16(8 * K) + 4 * k, f_bits(praw[k]));
    }
    st = ORC_OK;
  }
  free(sp);
  free(sym);
  free(pidx);
  free(praw);
  free(qt);
  return st;
}

/* ======================================================================== */
/* Decode                                                                     */
/* ======================================================================== */
int orc_peek(const uint8_t *in, size_t in_size, uint64_t *n, uint32_t *d, uint32_t *flags,
             uint32_t *p) {
  if (in_size < HDR_FIXED) return ORC_ERR_FORMAT;
  if (in[0] != 'L' || in[1] != 'C' || in[2] != 'P' || in[3] != '1' || in[4] != 1)
    return ORC_ERR_FORMAT;
  if (in[5] > 1 || in[6] < 1 || in[6] > 8) return ORC_ERR_FORMAT;
  if (n) *n = ld64(in + 16);
  if (d) *d = in[6];
  if (flags) *flags = ld32(in + 8);
  if (p) *p = ld32(in + 12);
  return in[5];
}

int orc_decompress(const uint8_t *in, size_t in_size, const int32_t *ref_q, float *out,
                   uint64_t n_cap, int32_t *q_out) {
  int method = orc_peek(in, in_size, NULL, NULL, NULL, NULL);
  if (method < 0) return method;
  uint32_t d = in[6], log2_chunk = in[7], p = ld32(in + 12);
  uint64_t n = ld64(in + 16), K = ld64(in + 24), M = ld64(in + 32), total = ld64(in + 40);
  uint32_t ns = method == 0 ? 3 : 1;
  if (log2_chunk < 5 || log2_chunk > 16) return ORC_ERR_FORMAT;
  if (in_size < header_bytes(d, ns) || total > in_size) return ORC_ERR_FORMAT;
  if (n > n_cap) return ORC_ERR_CAPACITY;
  if (method == 1 && !ref_q) return ORC_ERR_STATE;
  float mn[8], e[8];
  uint32_t qmax[8];
  for (uint32_t f = 0; f < d; f++) {
    mn[f] = ldf(in + HDR_FIXED + 16 * f);
    e[f] = ldf(in + HDR_FIXED + 16 * f + 4);
    qmax[f] = ld32(in + HDR_FIXED + 16 * f + 8);
  }
  uint64_t sec_off[4], sec_bytes[4];
  for (uint32_t s = 0; s <= ns; s++) {
    sec_off[s] = ld64(in + HDR_FIXED + 16 * d + 16 * s);
    sec_bytes[s] = ld64(in + HDR_FIXED + 16 * d + 16 * s + 8);
    if (sec_off[s] + sec_bytes[s] > total) return ORC_ERR_FORMAT;
  }
  int st = ORC_OK;
  if (method == 0) {
    int lp = log2_exact(p);
    if (lp < 0 || (uint32_t)lp * d > 32 || K > n || M > n - K) return ORC_ERR_FORMAT;
    uint64_t nb = n - K;
    uint64_t *s_id = malloc(sizeof(uint64_t) * (M + 1));
    uint64_t *s_cnt = malloc(sizeof(uint64_t) * (M + 1));
    uint64_t *s_rel = malloc(sizeof(uint64_t) * (nb + 1));
    if (!st) st = read_stream(in + sec_off[0], sec_bytes[0], M, log2_chunk, s_id);
    if (!st) st = read_stream(in + sec_off[1], sec_bytes[1], M, log2_chunk, s_cnt);
    if (!st) st = read_stream(in + sec_off[2], sec_bytes[2], nb, log2_chunk, s_rel);
    if (!st && sec_bytes[3] != pad16(4ull * d * K)) st = ORC_ERR_FORMAT;
    uint64_t bn[8], stride[8], blocks = 1;
    for (uint32_t f = 0; f < d; f++) {
      bn[f] = (uint64_t)(qmax[f] >> lp) + 1;
      stride[f] = blocks;
      blocks *= bn[f];
    }
    uint64_t k = 0, bid = 0;
    int64_t cnt = 0;
    uint64_t rel_prev = 0, chunk_mask = (1ull << log2_chunk) - 1;
    for (uint64_t b = 0; !st && b < M; b++) {
      bid += s_id[b];
      cnt += unzz(s_cnt[b]);
      if (cnt < 1 || (uint64_t)cnt > nb - k) {
        st = ORC_ERR_FORMAT;
        break;
      }
      for (int64_t c = 0; c < cnt; c++, k++) {
        uint64_t rel = (c == 0 || (k & chunk_mask) == 0) ? s_rel[k] : rel_prev + s_rel[k];
        rel_prev = rel;
        for (uint32_t f = 0; f < d; f++) {
          uint64_t bf = (bid / stride[f]) % bn[f];
          uint64_t rf = (rel >> (f * lp)) & ((1ull << lp) - 1);
          uint64_t qq = (bf << lp) + rf;
          if (qq > qmax[f]) {
            st = ORC_ERR_FORMAT;
            break;
          }
          out[(uint64_t)f * n + k] = orc_q2((int64_t)qq, mn[f], e[f]);
          if (q_out) q_out[(uint64_t)f * n + k] = (int32_t)qq;
        }
      }
    }
    if (!st && k != nb) st = ORC_ERR_FORMAT;
    for (uint64_t j = 0; !st && j < K; j++)
      for (uint32_t f = 0; f < d; f++) {
        float x = ldf(in + sec_off[3] + 4 * ((uint64_t)f * K + j));
        out[(uint64_t)f * n + nb + j] = x;
        if (q_out) q_out[(uint64_t)f * n + nb + j] = (int32_t)orc_q1(x, mn[f], e[f]);
      }
    free(s_id);
    free(s_cnt);
    free(s_rel);
    return st;
  }
  /* LCP-T: code = reference code + difference; patches restore raw values */
  uint64_t nd = n * d;
  uint64_t *sym = malloc(sizeof(uint64_t) * (nd + 1));
  st = read_stream(in + sec_off[0], sec_bytes[0], nd, log2_chunk, sym);
  if (!st && sec_bytes[1] != pad16(8 * K) + pad16(4 * K)) st = ORC_ERR_FORMAT;
  for (uint64_t s = 0; !st && s < nd; s++) {
    uint32_t f = (uint32_t)(s / (n ? n : 1));
    int64_t qq = (int64_t)ref_q[s] + unzz(sym[s]);
    if (qq < 0 || qq > (int64_t)qmax[f]) {
      st = ORC_ERR_FORMAT;
      break;
    }
    out[s] = orc_q2(qq, mn[f], e[f]);
    if (q_out) q_out[s] = (int32_t)qq;
  }
  for (uint64_t k = 0; !st && k < K; k++) {
    uint64_t s = ld64(in + sec_off[1] + 8 * k);
    if (s >= nd) {
      st = ORC_ERR_FORMAT;
      break;
    }
    out[s] = ldf(in + sec_off[1] + pad16(8 * K) + 4 * k);
  }
  free(sym);
  return st;
}

/* ======================================================================== */
/* Dictionary stage (Sec. "Block coding": dictionary coding is the last     */
/* step of the encoding stage).  The paper uses Zstd; this is an LZ77-style */
/* coder with the LCPZ layout:                                              */
/*   0  "LCPZ", u8 version 1, u8 log2 chunk (16), u16 0                     */
/*   8  u64 raw bytes S, 16 u64 chunks C = ceil(S / 2^16), 24 u64 total T   */
/*   32 the first min(S, 48) raw bytes, zero padded to 48 (a preview of the */
/*      container header)                                                   */
/*   80 u32 per chunk: its coded bytes, bit 31 set when stored raw          */
/*   pad16, then the chunks back to back, pad16 to T.                       */
/* A coded chunk is a list of sequences: a token byte (literal count in the */
/* high nibble, copy length - 4 in the low one, 15 meaning "add the         */
/* extension": bytes 255 ... 255 r summed), the extension of the literal    */
/* count, the literals, then, unless the chunk is complete after the        */
/* literals, a u16 copy offset and the extension of the copy length.        */
/* Parity status: pinned by hand-worked byte strings and closed forms.      */
/* ======================================================================== */
#define DICT_CHUNK (1u << ORC_DICT_LOG2_CHUNK)
#define DICT_NONE 0xffffffffu

size_t orc_dict_max_size(uint64_t raw_bytes) {
  uint64_t c = (raw_bytes + DICT_CHUNK - 1) >> ORC_DICT_LOG2_CHUNK;
  return (size_t)pad16(pad16(ORC_DICT_HEAD + 4 * c) + raw_bytes);
}

/* the four bytes at x as a little-endian word, multiplied by 2654435761
 * (Knuth's multiplicative hash) modulo 2^32, top 12 bits */
static uint32_t dict_hash(const uint8_t *x) {
  uint32_t w = (uint32_t)x[0] | ((uint32_t)x[1] << 8) | ((uint32_t)x[2] << 16) |
               ((uint32_t)x[3] << 24);
  return (uint32_t)(w * 2654435761u) >> 20;
}

static uint64_t dict_ext_bytes(uint64_t v) { return v >= 15 ? (v - 15) / 255 + 1 : 0; }

static uint64_t dict_put_ext(uint8_t *o, uint64_t v) {
  uint64_t k = 0;
  v -= 15;
  while (v >= 255) {
    o[k++] = 255;
    v -= 255;
  }
  o[k++] = (uint8_t)v;
  return k;
}

/* one sequence; ml = 0 for the literal-only last one.  Returns its size and
 * writes it when o is non-null. */
static uint64_t dict_sequence(uint8_t *o, const uint8_t *lit, uint64_t ll, uint64_t off,
                              uint64_t ml) {
  uint64_t sz = 1 + dict_ext_bytes(ll) + ll + (ml ? 2 + dict_ext_bytes(ml - 4) : 0);
  if (!o) return sz;
  uint64_t k = 0;
  o[k++] = (uint8_t)(((ll < 15 ? ll : 15) << 4) | (ml ? (ml - 4 < 15 ? ml - 4 : 15) : 0));
  if (ll >= 15) k += dict_put_ext(o + k, ll);
  memcpy(o + k, lit, ll);
  k += ll;
  if (ml) {
    o[k++] = (uint8_t)(off & 0xff);
    o[k++] = (uint8_t)(off >> 8);
    if (ml - 4 >= 15) k += dict_put_ext(o + k, ml - 4);
  }
  return k;
}

/* codes x[0..m) into o (room for m bytes); returns the coded size, or m
 * when the coding is not strictly shorter (the chunk is then stored) */
static uint64_t dict_chunk(const uint8_t *x, uint64_t m, uint8_t *o) {
  uint32_t *cand = (uint32_t *)malloc(sizeof(uint32_t) * (m ? m : 1));
  uint32_t table[4096];
  for (int h = 0; h < 4096; h++) table[h] = DICT_NONE;
  /* every position with four bytes left enters the table in order; its
   * candidate is the table entry just before it enters */
  for (uint64_t i = 0; i < m; i++) {
    cand[i] = DICT_NONE;
    if (i + 4 <= m) {
      uint32_t h = dict_hash(x + i);
      cand[i] = table[h];
      table[h] = (uint32_t)i;
    }
  }
  /* greedy parse: a copy wherever the candidate agrees on >= 4 bytes */
  uint64_t size = 0, p = 0, lit = 0;
  int stored = 0;
  while (p < m && !stored) {
    uint64_t len = 0;
    if (cand[p] != DICT_NONE) {
      uint64_t j = cand[p];
      while (p + len < m && x[j + len] == x[p + len]) len++;
    }
    if (len < 4) {
      p++;
      continue;
    }
    uint64_t sz = dict_sequence(NULL, x + lit, p - lit, p - cand[p], len);
    if (size + sz >= m) {
      stored = 1;
      break;
    }
    dict_sequence(o + size, x + lit, p - lit, p - cand[p], len);
    size += sz;
    p += len;
    lit = p;
  }
  if (!stored && lit < m) {
    uint64_t sz = dict_sequence(NULL, x + lit, m - lit, 0, 0);
    if (size + sz >= m)
      stored = 1;
    else {
      dict_sequence(o + size, x + lit, m - lit, 0, 0);
      size += sz;
    }
  }
  free(cand);
  return stored ? m : size;
}

int orc_dict_compress(const uint8_t *in, uint64_t in_size, uint8_t *out, size_t out_cap,
                      size_t *out_size) {
  if ((!in && in_size) || !out_size) return ORC_ERR_ARG;
  const uint64_t C = (in_size + DICT_CHUNK - 1) >> ORC_DICT_LOG2_CHUNK;
  const uint64_t p0 = pad16(ORC_DICT_HEAD + 4 * C);
  uint8_t *tmp = (uint8_t *)malloc(DICT_CHUNK);
  uint32_t *sz = (uint32_t *)malloc(sizeof(uint32_t) * (C ? C : 1));
  uint8_t *body = (uint8_t *)malloc(in_size ? in_size : 1);
  if (!tmp || !sz || !body) {
    free(tmp);
    free(sz);
    free(body);
    return ORC_ERR_NOMEM;
  }
  uint64_t at = 0;
  for (uint64_t k = 0; k < C; k++) {
    const uint8_t *x = in + (k << ORC_DICT_LOG2_CHUNK);
    uint64_t m = in_size - (k << ORC_DICT_LOG2_CHUNK);
    if (m > DICT_CHUNK) m = DICT_CHUNK;
    uint64_t c = dict_chunk(x, m, tmp);
    if (c == m) {
      memcpy(body + at, x, m);
      sz[k] = (uint32_t)m | 0x80000000u;
    } else {
      memcpy(body + at, tmp, c);
      sz[k] = (uint32_t)c;
    }
    at += c;
  }
  const uint64_t total = pad16(p0 + at);
  *out_size = (size_t)total;
  int st = ORC_OK;
  if (total > out_cap) {
    st = ORC_ERR_CAPACITY;
  } else {
    memset(out, 0, total);
    out[0] = 'L';
    out[1] = 'C';
    out[2] = 'P';
    out[3] = 'Z';
    out[4] = 1;
    out[5] = ORC_DICT_LOG2_CHUNK;
    st64(out + 8, in_size);
    st64(out + 16, C);
    st64(out + 24, total);
    memcpy(out + 32, in, in_size < 48 ? in_size : 48);
    for (uint64_t k = 0; k < C; k++) st32(out + ORC_DICT_HEAD + 4 * k, sz[k]);
    memcpy(out + p0, body, at);
  }
  free(tmp);
  free(sz);
  free(body);
  return st;
}

/* reads an extension (255 ... 255 r) at in[*q], below end */
static int dict_get_ext(const uint8_t *in, uint64_t *q, uint64_t end, uint64_t *v) {
  for (;;) {
    if (*q >= end) return ORC_ERR_FORMAT;
    uint8_t b = in[(*q)++];
    *v += b;
    if (b != 255) return ORC_OK;
  }
}

int orc_dict_decompress(const uint8_t *in, size_t in_size, uint8_t *out, size_t out_cap,
                        size_t *out_size) {
  if (!in || !out_size || in_size < ORC_DICT_HEAD) return ORC_ERR_FORMAT;
  if (in[0] != 'L' || in[1] != 'C' || in[2] != 'P' || in[3] != 'Z' || in[4] != 1 ||
      in[5] != ORC_DICT_LOG2_CHUNK)
    return ORC_ERR_FORMAT;
  const uint64_t S = ld64(in + 8), C = ld64(in + 16), T = ld64(in + 24);
  if (C != (S + DICT_CHUNK - 1) >> ORC_DICT_LOG2_CHUNK || T > in_size) return ORC_ERR_FORMAT;
  const uint64_t p0 = pad16(ORC_DICT_HEAD + 4 * C);
  if (p0 > T) return ORC_ERR_FORMAT;
  *out_size = (size_t)S;
  if (S > out_cap) return ORC_ERR_CAPACITY;
  uint64_t at = p0;
  for (uint64_t k = 0; k < C; k++) {
    uint32_t e = ld32(in + ORC_DICT_HEAD + 4 * k);
    uint64_t c = e & 0x7fffffffu;
    uint64_t m = S - (k << ORC_DICT_LOG2_CHUNK);
    if (m > DICT_CHUNK) m = DICT_CHUNK;
    if (c > T - at) return ORC_ERR_FORMAT;
    uint8_t *y = out + (k << ORC_DICT_LOG2_CHUNK);
    const uint64_t end = at + c;
    if (e & 0x80000000u) {
      if (c != m) return ORC_ERR_FORMAT;
      memcpy(y, in + at, m);
    } else {
      if (c >= m) return ORC_ERR_FORMAT; /* a coded chunk is shorter than its bytes */
      uint64_t q = at, w = 0;
      while (w < m) {
        if (q >= end) return ORC_ERR_FORMAT;
        uint8_t tok = in[q++];
        uint64_t ll = tok >> 4, ml = tok & 15;
        if (ll == 15 && dict_get_ext(in, &q, end, &ll)) return ORC_ERR_FORMAT;
        if (ll > m - w || ll > end - q) return ORC_ERR_FORMAT;
        memcpy(y + w, in + q, ll);
        w += ll;
        q += ll;
        if (w == m) break;
        if (end - q < 2) return ORC_ERR_FORMAT;
        uint64_t off = (uint64_t)in[q] | ((uint64_t)in[q + 1] << 8);
        q += 2;
        if (ml == 15 && dict_get_ext(in, &q, end, &ml)) return ORC_ERR_FORMAT;
        ml += 4;
        if (off == 0 || off > w || ml > m - w) return ORC_ERR_FORMAT;
        for (uint64_t t = 0; t < ml; t++) y[w + t] = y[w - off + t];  /* may overlap */
        w += ml;
      }
      if (q != end) return ORC_ERR_FORMAT;
    }
    at = end;
  }
  if (pad16(at) != T) return ORC_ERR_FORMAT;
  return ORC_OK;
}
