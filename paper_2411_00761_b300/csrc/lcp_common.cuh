// lcp_common.cuh -- shared definitions of the B300 LCP kernels.
//
// Plans, stream descriptors and the element rules of LCP (arXiv 2411.00761):
//   Q1  q  = floor((x - min) / (2 eb))          Eq. quantization
//   Q2  x' = RN32(min + (2q + 1) eb)             Eq. quantization (reverse)
//   Q3  |x - x'| > eb                            Eq. abs (a violation)
// all evaluated over the reals, bit-exact.  The common case runs in a few
// float/int instructions whose error is bounded and certified; the rare
// uncertain cases fall through to exact expansion arithmetic (TwoSum /
// FMA products) or, beyond that, to a 320-bit integer path.  FP64 appears
// only on paths that run for a vanishing fraction of elements (B300's FP64
// rate is far below its FP32 rate).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace lcp {

constexpr int kMaxD = 8;
constexpr int kAlpha = 4096;  // Huffman alphabet; the last symbol escapes
constexpr int kEsc = 4095;
constexpr int kLmax = 24;      // longest Huffman code
constexpr int kFastBits = 12;  // first-level decode table index bits
constexpr unsigned long long kOutlierBit = 1ull << 63;

enum Status : int {
  OK = 0,
  ERR_ARG = -1,
  ERR_NONFINITE = -2,
  ERR_RANGE = -3,
  ERR_CAPACITY = -4,
  ERR_FORMAT = -5,
  ERR_STATE = -6,
  ERR_NOMEM = -7,
  ERR_TIMEOUT = -8,
  ERR_CUDA = -9
};

// Per-field parameters, resolved on the device from the frame's min/max.
struct FieldPlan {
  float m;      // field minimum (IEEE totalOrder, so -0 < +0)
  float e;      // bound used: largest f32 <= eb_f
  float h;      // bin width 2e (exact)
  float inv_h;  // RN32(1/h)
  float win;    // bin fraction within which a rounded centre may miss e
  uint32_t qmax;
  int32_t g1;           // x' = RN32(W) * 2^g1, W = 2 (A c8 + mb) + sticky
  uint32_t c8;          // mantissa of e, times 8
  long long mb;         // floor(m / 2^(g1 + 1))
  uint32_t sticky;      // m has bits below 2^(g1 + 1)
  uint32_t wide;        // |value| can reach 2^32 * 2e: c8, mb and sticky are
                        // unused and Q2 takes the 320-bit path
  unsigned long long bn;      // blocks along this axis
  unsigned long long stride;  // block-id stride of this axis
  unsigned long long bmagic;  // r / bn = umulhi(r, bmagic) >> bshift (r < 2^63, bn >= 2)
  uint32_t bshift;            // 255 when bn == 1
  uint32_t pad1;
};

// Decoder-side block grid of a field from its qmax: bn = (qmax >> lp) + 1
// blocks along the axis and the constants of floor(r / bn) for r < 2^63:
// m = ceil(2^(63+l) / bn), l = ceil(log2 bn), then floor(r m / 2^(63+l)) =
// floor(r / bn) (Granlund-Montgomery, division by invariant integers using
// multiplication, Thm. 4.2).  The stride is the caller's (it depends on the
// fields before this one).
__device__ inline void field_block_grid(FieldPlan &F, uint32_t lp) {
  const unsigned long long bn = ((unsigned long long)F.qmax >> lp) + 1ull;
  F.bn = bn;
  if (bn <= 1) {
    F.bmagic = 0;
    F.bshift = 255;
    return;
  }
  uint32_t l = 0;
  while ((1ull << l) < bn) ++l;
  // binary long division of 2^(63+l) by bn; the quotient fits 64 bits
  unsigned long long q = 0, rem = 0;
  for (int bit = 63 + (int)l; bit >= 0; --bit) {
    rem = (rem << 1) | (bit == 63 + (int)l ? 1ull : 0ull);
    q <<= 1;
    if (rem >= bn) {
      rem -= bn;
      q |= 1ull;
    }
  }
  F.bmagic = q + (rem != 0 ? 1ull : 0ull);
  F.bshift = l - 1;
}

struct MinMax {
  uint32_t lo[kMaxD];  // totalOrder keys
  uint32_t hi[kMaxD];
  uint32_t nonfinite;
  uint32_t pad[3];
};

struct Plan {
  int status;
  uint32_t d, lp;       // fields, log2 p (S frames)
  uint32_t nbits;       // bucket bits used by the partition pass
  uint32_t key_bits;    // bits of the largest key
  uint32_t part_shift;  // bucket = key >> part_shift
  uint32_t rel_bits;    // d * lp
  uint32_t method;      // 0 S, 1 T
  unsigned long long n;
  FieldPlan f[kMaxD];
};

// Coder plan of one stream.
struct StreamDesc {
  unsigned long long n;            // values
  unsigned long long maxv;         // largest value
  unsigned long long payload_bits;
  unsigned long long bytes;        // section bytes
  unsigned long long offset;       // section offset in the container
  unsigned long long n_chunks;
  uint32_t coder;                  // 0 fixed, 1 huffman
  uint32_t width;                  // fixed width, or escape width
  uint32_t used;                   // huffman: used symbols
  uint32_t pad;
};

// Host-visible summary written at the end of a compression.
struct Summary {
  int status;
  uint32_t pad;
  unsigned long long total;  // container bytes
  unsigned long long M, K;
};

__host__ __device__ inline unsigned long long pad16(unsigned long long b) {
  return (b + 15ull) & ~15ull;
}
__host__ __device__ inline unsigned long long words_of(unsigned long long bits) {
  return (bits + 31ull) >> 5;
}
__host__ __device__ inline unsigned long long zigzag(long long v) {
  return v >= 0 ? (unsigned long long)v << 1 : (((unsigned long long)(-(v + 1))) << 1) | 1ull;
}
__host__ __device__ inline long long unzigzag(unsigned long long u) {
  return (u & 1ull) ? -(long long)(u >> 1) - 1 : (long long)(u >> 1);
}
__host__ __device__ inline uint32_t bitlen64(unsigned long long v) {
#ifdef __CUDA_ARCH__
  return v ? 64u - (uint32_t)__clzll((long long)v) : 0u;
#else
  return v ? 64u - (uint32_t)__builtin_clzll(v) : 0u;
#endif
}

// ---------------------------------------------------------------------------
// asynchronous 4-byte copies global -> shared (cp.async, zero fill when not
// valid), per-thread commit groups
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cp_async4(uint32_t *dst, const uint32_t *src, bool valid) {
  const unsigned sdst = (unsigned)__cvta_generic_to_shared(dst);
  const int n = valid ? 4 : 0;
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(sdst), "l"(src), "r"(n)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait1() {
  asm volatile("cp.async.wait_group 1;\n" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait0() {
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// ---------------------------------------------------------------------------
// float helpers
// ---------------------------------------------------------------------------
// Runs of equal values held by consecutive lanes of a warp (a lane that is
// not valid forms a run of its own): the run's first lane, this lane's rank
// in the run and the run's length.  One shared-memory atomic per run then
// serves clustered inputs, whose neighbouring lanes often hit one counter.
// All 32 lanes must call it.
__device__ __forceinline__ void lane_runs(uint32_t v, bool valid, int &leader, uint32_t &rank,
                                          uint32_t &len) {
  const int lane = threadIdx.x & 31;
  const uint32_t up = __shfl_up_sync(0xffffffffu, v, 1);
  const uint32_t vmask = __ballot_sync(0xffffffffu, valid);
  const bool prev_valid = lane > 0 && ((vmask >> (lane - 1)) & 1u);
  const bool head = !valid || !prev_valid || up != v;
  const uint32_t heads = __ballot_sync(0xffffffffu, head);
  const uint32_t le = 0xffffffffu >> (31 - lane);  // lanes 0..lane
  leader = 31 - __clz(heads & le);
  const uint32_t above = heads & ~le;
  const int next = above ? __ffs(above) - 1 : 32;
  rank = (uint32_t)(lane - leader);
  len = (uint32_t)(next - leader);
}

__device__ __forceinline__ uint32_t order_key(float f) {
  uint32_t b = __float_as_uint(f);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float order_key_inv(uint32_t k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}
// Knuth's branch-free exact sum: a + b = s + err, exactly (round to nearest)
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &err) {
  s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float aa = __fsub_rn(s, bb);
  err = __fadd_rn(__fsub_rn(a, aa), __fsub_rn(b, bb));
}

// ---------------------------------------------------------------------------
// 320-bit sign-magnitude integers in units of 2^-149 (slow paths only)
// ---------------------------------------------------------------------------
struct Big {
  unsigned long long w[5];
  int neg;
};
__device__ inline Big big_shl(unsigned long long v, int sh, int neg) {
  Big r;
  for (int i = 0; i < 5; ++i) r.w[i] = 0;
  int limb = sh >> 6, off = sh & 63;
  r.w[limb] = v << off;
  if (off && limb + 1 < 5) r.w[limb + 1] = v >> (64 - off);
  r.neg = neg && v != 0;
  return r;
}
__device__ inline void float_parts(float f, int &neg, uint32_t &M, int &E) {
  uint32_t b = __float_as_uint(f);
  neg = (int)(b >> 31);
  uint32_t ex = (b >> 23) & 0xffu;
  M = ex ? ((b & 0x7fffffu) | 0x800000u) : (b & 0x7fffffu);
  E = ex ? (int)ex - 150 : -149;
}
__device__ inline Big big_of(float f) {
  int neg, E;
  uint32_t M;
  float_parts(f, neg, M, E);
  return big_shl(M, E + 149, neg);
}
__device__ inline Big big_of_mul(unsigned long long k, float f) {  // k * f, k < 2^38
  int neg, E;
  uint32_t M;
  float_parts(f, neg, M, E);
  return big_shl(k * (unsigned long long)M, E + 149, neg);
}
__device__ inline bool big_is_zero(const Big &a) {
  return (a.w[0] | a.w[1] | a.w[2] | a.w[3] | a.w[4]) == 0;
}
__device__ inline int mag_cmp(const Big &a, const Big &b) {
  for (int i = 4; i >= 0; --i)
    if (a.w[i] != b.w[i]) return a.w[i] < b.w[i] ? -1 : 1;
  return 0;
}
__device__ inline Big big_add(const Big &a, const Big &b) {
  Big r;
  if (a.neg == b.neg) {
    unsigned long long c = 0;
    for (int i = 0; i < 5; ++i) {
      unsigned long long s = a.w[i] + b.w[i];
      unsigned long long c1 = s < a.w[i];
      unsigned long long s2 = s + c;
      c = c1 | (s2 < s);
      r.w[i] = s2;
    }
    r.neg = a.neg;
  } else {
    const Big *x = &a, *y = &b;
    if (mag_cmp(a, b) < 0) {
      x = &b;
      y = &a;
    }
    unsigned long long br = 0;
    for (int i = 0; i < 5; ++i) {
      unsigned long long d = x->w[i] - y->w[i];
      unsigned long long b1 = x->w[i] < y->w[i];
      unsigned long long d2 = d - br;
      br = b1 | (d < br);
      r.w[i] = d2;
    }
    r.neg = x->neg;
  }
  if (big_is_zero(r)) r.neg = 0;
  return r;
}
__device__ inline Big big_negate(Big a) {
  if (!big_is_zero(a)) a.neg ^= 1;
  return a;
}
__device__ inline int big_sign(const Big &a) { return big_is_zero(a) ? 0 : (a.neg ? -1 : 1); }
__device__ inline int big_msb(const Big &a) {
  for (int i = 4; i >= 0; --i)
    if (a.w[i]) return i * 64 + 63 - __clzll((long long)a.w[i]);
  return -1;
}
__device__ inline unsigned long long big_bits(const Big &a, int pos, int n) {  // n <= 32
  int limb = pos >> 6, off = pos & 63;
  unsigned long long v = a.w[limb] >> off;
  if (off && limb + 1 < 5) v |= a.w[limb + 1] << (64 - off);
  return v & ((1ull << n) - 1ull);
}
__device__ inline bool big_any_below(const Big &a, int pos) {  // a bit < pos set
  for (int i = 0; i < 5 && pos > 0; ++i, pos -= 64) {
    unsigned long long mask = pos >= 64 ? ~0ull : ((1ull << pos) - 1ull);
    if (a.w[i] & mask) return true;
  }
  return false;
}
// nearest f32 to a * 2^-149, ties to even
__device__ inline float big_to_f32(const Big &a) {
  int t = big_msb(a);
  if (t < 0) return 0.0f;
  uint32_t bits;
  if (t < 23) {
    bits = (uint32_t)a.w[0];
  } else {
    int sh = t - 23;
    unsigned long long mant = big_bits(a, sh, 24);
    if (sh > 0) {
      bool half = big_bits(a, sh - 1, 1) != 0;
      bool rest = big_any_below(a, sh - 1);
      if (half && (rest || (mant & 1ull))) ++mant;
    }
    if (mant == (1ull << 24)) {
      mant >>= 1;
      ++sh;
    }
    int bexp = sh + 1;
    bits = bexp >= 255 ? 0x7f800000u : (((uint32_t)bexp << 23) | (uint32_t)(mant & 0x7fffffu));
  }
  if (a.neg) bits |= 0x80000000u;
  return __uint_as_float(bits);
}

// ---------------------------------------------------------------------------
// Q1
// ---------------------------------------------------------------------------
// exact sign of (x - m) - k h, 0 <= k < 2^24, via Shewchuk's expansion growth
__device__ inline int sign_rem(float x, float m, float h, int k) {
  float t, te;
  two_sum(x, -m, t, te);
  float kf = (float)k;
  float P = __fmul_rn(kf, h);
  float p = __fmaf_rn(kf, h, -P);
  float e[4];
  int n = 0;
  float in[4] = {te, t, -p, -P};
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    float Q = in[j];
    for (int i = 0; i < n; ++i) {
      float s, err;
      two_sum(Q, e[i], s, err);
      e[i] = err;
      Q = s;
    }
    e[n++] = Q;
  }
  for (int i = n - 1; i >= 0; --i)
    if (e[i] != 0.0f) return e[i] > 0.0f ? 1 : -1;
  return 0;
}

// fully general exact floor (large quotients): estimate in FP64, settle
// against the exact remainder
static __device__ __noinline__ int32_t q1_wide(float x, const FieldPlan &F) {
  double est = floor(((double)x - (double)F.m) / (double)F.h);
  if (!(est >= 0.0)) est = 0.0;
  if (est > 2147483647.0) est = 2147483647.0;
  long long q = (long long)est;
  Big D = big_add(big_of(x), big_negate(big_of(F.m)));
  Big H = big_of(F.h);
  Big R = big_add(D, big_negate(big_of_mul((unsigned long long)q, F.h)));
  // the FP64 estimate is within a few units in the codec's domain; the caps
  // only bound the loops for inputs outside it
  for (int it = 0; it < 64 && big_sign(R) < 0 && q > 0; ++it) {
    --q;
    R = big_add(R, H);
  }
  for (int it = 0; it < 64 && mag_cmp(R, H) >= 0 && big_sign(R) >= 0; ++it) {
    ++q;
    R = big_add(R, big_negate(H));
  }
  return (int32_t)q;
}

// exact floor when the float estimate y sits close to an integer
static __device__ __noinline__ int32_t q1_settle(float x, const FieldPlan &F, float y) {
  if (!(y < 4194304.0f)) return q1_wide(x, F);  // y >= 2^22
  float B = __fmul_rn(y, 0x1p-20f);
  int lo = (int)floorf(__fsub_rn(y, B)) - 1;
  int hi = (int)floorf(__fadd_rn(y, B)) + 1;
  if (lo < 0) lo = 0;
  // largest k in [lo, hi] with (x - m) - k h >= 0
  int q = lo;
  for (int k = hi; k > lo; --k)
    if (sign_rem(x, F.m, F.h, k) >= 0) {
      q = k;
      break;
    }
  return q;
}

// Q1 with the certified fast path.  chk is set when x may sit close enough to
// a bin edge that the rounded centre could miss the bound (Q3 must be checked
// exactly); otherwise Q3 is certainly false.
__device__ __forceinline__ int32_t quantize(float x, const FieldPlan &F, bool &chk) {
  float t = __fsub_rn(x, F.m);
  float y = __fmul_rn(t, F.inv_h);
  float k = floorf(y);
  float fr = __fsub_rn(y, k);
  float om = __fsub_rn(1.0f, fr);
  float B = __fmul_rn(y, 0x1p-20f);  // > 4x the error bound of y
  if (t != 0.0f && fr > B && om > B) {
    float lo = __fadd_rn(B, F.win);
    chk = !(fr > lo && om > lo);
    return (int32_t)k;
  }
  chk = true;
  if (t == 0.0f) return 0;
  return q1_settle(x, F, y);
}

// ---------------------------------------------------------------------------
// Q2
// ---------------------------------------------------------------------------
static __device__ __noinline__ float recon_wide(long long q, const FieldPlan &F) {
  Big c = big_add(big_of(F.m), big_of_mul((unsigned long long)(2 * q + 1), F.e));
  return big_to_f32(c);
}
// x' = RN32(m + (2q+1) e): the exact centre is (2V + sticky) 2^g1 with the
// low bits of m folded into one sticky bit, which cannot change the rounding
// because |2V| >= 2^26 whenever m has bits below the grid.  Falls back when
// the result is subnormal (a second rounding would be needed).
__device__ __forceinline__ float reconstruct(long long q, const FieldPlan &F) {
  if (F.wide) return recon_wide(q, F);
  long long V = (2 * q + 1) * (long long)F.c8 + F.mb;
  long long W = 2 * V + (long long)F.sticky;
  float r = __ll2float_rn(W);
  uint32_t b = __float_as_uint(r);
  if ((b & 0x7fffffffu) == 0) return r;
  int ne = (int)((b >> 23) & 0xffu) + F.g1;
  if (ne >= 1 && ne <= 254) return __uint_as_float((uint32_t)((int)b + F.g1 * (1 << 23)));
  return recon_wide(q, F);
}

// Q2 in binary32 arithmetic alone, for 0 <= q < 2^23 (so that 2q+1 is
// exact): the product (2q+1) e is split exactly into ph + pl (FMA), m + ph
// into th + tl (TwoSum), and RN(m + ph + pl) = RN(th + RO(tl + pl)) with RO
// rounding to odd (round toward zero, lowest bit set when inexact) -- the
// correctly rounded sum of three terms by rounding to odd of Boldo and
// Melquiond ("Emulation of FMA and correctly rounded sums: proved algorithms
// using rounding to odd", IEEE Trans. Computers 57(4), 2008).  Returns false
// (the caller falls back) outside that range or when the result is
// subnormal.  These are FMA-pipe operations; the 64-bit integer conversion
// of reconstruct() issues on the FP64 pipe.
__device__ __forceinline__ bool recon_rn_f32(long long q, float m, float e, float &z) {
  if ((unsigned long long)q >= (1ull << 23)) return false;
  const float qf = __int2float_rn((int)(2 * q + 1));
  const float ph = __fmul_rn(qf, e);
  const float pl = __fmaf_rn(qf, e, -ph);
  const float th = __fadd_rn(m, ph);
  const float bb = __fsub_rn(th, m);
  const float aa = __fsub_rn(th, bb);
  const float tl = __fadd_rn(__fsub_rn(m, aa), __fsub_rn(ph, bb));
  const float rz = __fadd_rz(tl, pl);
  const bool inexact = __fadd_ru(tl, pl) != __fadd_rd(tl, pl);
  const float v = __uint_as_float(__float_as_uint(rz) | (inexact ? 1u : 0u));
  z = __fadd_rn(th, v);
  if (z == 0.0f) {
    z = 0.0f;
    return true;
  }
  return fabsf(z) >= 0x1p-126f;
}

// out-of-line Q2 for the rare values the binary32 path declines
static __device__ __noinline__ float recon_slow(long long q, const FieldPlan &F) {
  return reconstruct(q, F);
}

// reconstruct() with the plan's constants already in registers; Fs (the
// plan, e.g. in shared memory) serves the rare wide fallback
__device__ __forceinline__ float reconstruct_c(long long q, uint32_t c8, long long mb,
                                               uint32_t sticky, int32_t g1,
                                               const FieldPlan &Fs) {
  if (Fs.wide) return recon_wide(q, Fs);
  long long V = (2 * q + 1) * (long long)c8 + mb;
  long long W = 2 * V + (long long)sticky;
  float r = __ll2float_rn(W);
  uint32_t b = __float_as_uint(r);
  if ((b & 0x7fffffffu) == 0) return r;
  int ne = (int)((b >> 23) & 0xffu) + g1;
  if (ne >= 1 && ne <= 254) return __uint_as_float((uint32_t)((int)b + g1 * (1 << 23)));
  return recon_wide(q, Fs);
}

// ---------------------------------------------------------------------------
// Q3: |x - xr| > e exactly
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool violates(float x, float xr, float e) {
  float d, err;
  two_sum(x, -xr, d, err);
  float ad = fabsf(d);
  if (ad > e) return true;
  if (ad < e) return false;
  return err != 0.0f && (signbit(err) == signbit(d));
}

// ---------------------------------------------------------------------------
// field plan from min, max and the requested bound (domain rules in order:
// bound outside [2^-100, 2^100] -> ERR_ARG; 2^30 bins or more -> ERR_RANGE).
// A field whose minimum reaches 2^32 * 2e in magnitude is marked wide: its
// centre no longer fits the 64-bit form of reconstruct(), so Q2 runs on the
// exact 320-bit path there (Q1 and Q3 need no change).  W = 2 ((2q + 1) c8
// + mb) + sticky stays below 2^62 when |m| < 2^33 e: (2q + 1) c8 < 2^58 and
// |mb| <= |m| 2^27 / e < 2^60.
// ---------------------------------------------------------------------------
__device__ inline int plan_field(float mn, float mx, double eb, int mode, uint32_t lp, FieldPlan &F) {
  double range = (double)mx - (double)mn;
  double ebf = (mode == 1 && range > 0.0) ? eb * range : eb;
  float e = __double2float_rd(ebf);
  if (!(e >= 0x1p-100f) || !(e <= 0x1p100f)) return ERR_ARG;
  F.m = mn;
  F.e = e;
  F.h = 2.0f * e;
  F.inv_h = __double2float_rn(1.0 / (double)F.h);
  double qest = range / (2.0 * (double)e);
  if (!(qest < 2147483648.0)) return ERR_RANGE;
  // guard window first (quantize() reads it)
  double amax = fmax(fabs((double)mn), fabs((double)mx));
  {
    double A = amax + 2.0 * (double)e;
    int ex;
    frexp(A, &ex);
    double ulp = A < 0x1p-126 ? 0x1p-149 : ldexp(1.0, ex - 24);
    F.win = __double2float_ru(ulp / (2.0 * (double)F.h) * 1.001);
  }
  bool chk;
  int32_t qmax = quantize(mx, F, chk);
  if (qmax >= (1 << 30) || qmax < 0) return ERR_RANGE;
  F.qmax = (uint32_t)qmax;
  F.wide = (fabs((double)mn) < ldexp(2.0 * (double)e, 32)) ? 0u : 1u;
  // reconstruction constants: grid 2^G, G = (lsb exponent of e) - 3
  int eneg, Ee, mneg, Em;
  uint32_t Me, Mm;
  float_parts(e, eneg, Me, Ee);
  float_parts(mn, mneg, Mm, Em);
  const int G = Ee - 3;
  F.g1 = G - 1;
  F.c8 = Me << 3;
  long long mb = 0;
  uint32_t st = 0;
  if (Mm != 0 && !F.wide) {
    if (Em >= G) {
      mb = (long long)((unsigned long long)Mm << (Em - G));
      if (mneg) mb = -mb;
    } else {
      int k = G - Em;
      unsigned long long hi = k >= 40 ? 0ull : ((unsigned long long)Mm >> k);
      unsigned long long low = k >= 40 ? Mm : ((unsigned long long)Mm & ((1ull << k) - 1ull));
      st = low != 0;
      mb = mneg ? -(long long)(hi + (low != 0)) : (long long)hi;
    }
  }
  F.mb = mb;
  F.sticky = st;
  F.bn = ((unsigned long long)F.qmax >> lp) + 1ull;
  F.stride = 0;
  F.bmagic = 0;  // every byte defined: plans are compared and checkpointed
  F.bshift = 0;
  F.pad1 = 0;
  return OK;
}

}  // namespace lcp

#define LCP_CUDA_TRY(expr)                     \
  do {                                         \
    cudaError_t _e = (expr);                   \
    if (_e != cudaSuccess) return lcp::ERR_CUDA; \
  } while (0)
