// k_decode.cu -- decompression kernels.
//
// Decoding follows the coding chain backwards (Sec. "Block coding"): decode
// each stream (chunks in parallel), undo the delta coding with scans, place
// particles block by block and reconstruct every field with Eq. quantization
// (reverse): x' = (2q + 1) eb + min, rounded once to f32.
#include <algorithm>

#include "lcp_kernels.h"

namespace lcp {

// ---------------------------------------------------------------------------
// field plans for decoding (reconstruction and, for raw outliers, Q1)
// ---------------------------------------------------------------------------
__global__ void k_decode_plan(const DecodeFields *df, uint32_t d, Plan *plan) {
  int f = threadIdx.x;
  if (f < (int)d) {
    FieldPlan F;
    int st = plan_field(df->m[f], df->m[f], (double)df->e[f], 0, df->lp, F);
    F.qmax = df->qmax[f];
    F.bn = ((unsigned long long)df->qmax[f] >> df->lp) + 1ull;
    plan->f[f] = F;
    if (st != OK) atomicCAS(&plan->status, OK, ERR_FORMAT);
  }
  if (f == 0) {
    plan->d = d;
    plan->lp = df->lp;
    plan->rel_bits = df->lp * d;
  }
  __syncthreads();
  if (f == 0) {
    unsigned long long stride = 1ull;
    for (uint32_t k = 0; k < d; ++k) {
      plan->f[k].stride = stride;
      stride *= plan->f[k].bn;
    }
  }
  if (f < (int)d) {
    // floor(r / bn) for r < 2^63: m = ceil(2^(63+l) / bn), l = ceil(log2 bn), then
    // floor(r m / 2^(63+l)) = floor(r / bn) (Granlund-Montgomery, division by
    // invariant integers using multiplication, Thm. 4.2)
    const unsigned long long bn = plan->f[f].bn;
    if (bn <= 1) {
      plan->f[f].bmagic = 0;
      plan->f[f].bshift = 255;
    } else {
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
      plan->f[f].bmagic = q + (rem != 0 ? 1ull : 0ull);
      plan->f[f].bshift = l - 1;
    }
  }
}

void launch_decode_plan(const DecodeFields *df, uint32_t d, Plan *plan, cudaStream_t s) {
  note_launch();
  k_decode_plan<<<1, 32, 0, s>>>(df, d, plan);
}

// ---------------------------------------------------------------------------
// Huffman decode tables from the section's (count per length, symbols)
// ---------------------------------------------------------------------------
__global__ void k_huff_table(const uint8_t *__restrict__ sec, HuffTable *__restrict__ T) {
  __shared__ uint32_t cnt[kLmax + 1], first[kLmax + 2], index[kLmax + 2];
  const uint32_t U = (uint32_t)sec[2] | ((uint32_t)sec[3] << 8);
  if (threadIdx.x == 0) {
    uint32_t code = 0, idx = 0, total = 0;
    for (int L = 1; L <= kLmax; ++L) {
      cnt[L] = (uint32_t)sec[32 + 2 * (L - 1)] | ((uint32_t)sec[33 + 2 * (L - 1)] << 8);
      total += cnt[L];
    }
    for (int L = 1; L <= kLmax; ++L) {
      code = (L == 1) ? 0u : (code + cnt[L - 1]) << 1;
      first[L] = code;
      index[L] = idx;
      idx += cnt[L];
      T->first[L] = code;
      T->index[L] = index[L];
      T->count[L] = cnt[L];
    }
    T->used = U;
    T->ok = (total == U && U > 0 && U <= (uint32_t)kAlpha) ? 1u : 0u;
  }
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < U && i < (uint32_t)kAlpha; i += blockDim.x)
    T->syms[i] = (uint16_t)((uint32_t)sec[80 + 2 * i] | ((uint32_t)sec[81 + 2 * i] << 8));
  // first-level table: codes of up to kFastBits bits, entry = sym << 5 | len
  for (uint32_t e = threadIdx.x; e < (1u << kFastBits); e += blockDim.x) T->fast[e] = 0u;
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < U && i < (uint32_t)kAlpha; i += blockDim.x) {
    // length of the i-th symbol in canonical order
    int L = 1;
    while (L < kLmax && i >= index[L] + cnt[L]) ++L;
    if (L > kFastBits) continue;
    uint32_t code = first[L] + (i - index[L]);
    uint32_t sym = (uint32_t)sec[80 + 2 * i] | ((uint32_t)sec[81 + 2 * i] << 8);
    uint32_t lo = code << (kFastBits - L), hi = (code + 1) << (kFastBits - L);
    for (uint32_t e = lo; e < hi && e < (1u << kFastBits); ++e) T->fast[e] = (sym << 5) | (uint32_t)L;
  }
}

void launch_huff_table(const uint8_t *sec, HuffTable *T, cudaStream_t s) {
  note_launch();
  k_huff_table<<<1, 256, 0, s>>>(sec, T);
}

// ---------------------------------------------------------------------------
// bit reader over a u32 payload (MSB first); loads past the end read zero
// ---------------------------------------------------------------------------
struct BitReader {
  const uint32_t *pl;
  unsigned long long nwords, next;
  unsigned long long win;
  int nb;  // valid bits in win (left aligned), kept > 32
  __device__ __forceinline__ uint32_t word(unsigned long long i) const {
    return i < nwords ? __ldg(pl + i) : 0u;
  }
  __device__ __forceinline__ void init(const uint32_t *p, unsigned long long nw,
                                       unsigned long long pos) {
    pl = p;
    nwords = nw;
    unsigned long long wi = pos >> 5;
    int off = (int)(pos & 31);
    win = ((unsigned long long)word(wi) << 32) | word(wi + 1);
    win <<= off;
    nb = 64 - off;
    next = wi + 2;
    if (nb <= 32) {
      win |= (unsigned long long)word(next++) << (32 - nb);
      nb += 32;
    }
  }
  __device__ __forceinline__ uint32_t peek(int n) const {  // 1 <= n <= 32
    return (uint32_t)(win >> (64 - n));
  }
  __device__ __forceinline__ void skip(int n) {  // n <= 32
    win <<= n;
    nb -= n;
    if (nb <= 32) {
      win |= (unsigned long long)word(next++) << (32 - nb);
      nb += 32;
    }
  }
  __device__ __forceinline__ unsigned long long read(int n) {  // n <= 64
    unsigned long long v = 0;
    if (n > 32) {
      v = (unsigned long long)peek(n - 32) << 32;
      skip(n - 32);
      n = 32;
    }
    if (n > 0) {
      v |= peek(n);
      skip(n);
    }
    return v;
  }
};

// Bit reader over a 16-byte aligned u32 payload that keeps one 16-byte load
// in flight ahead of the window (loads past the end read zero).
struct BitReader4 {
  const uint4 *p4;
  unsigned long long n4, next4;
  uint4 b0, b1;
  int bi;
  unsigned long long win;
  int nb;
  __device__ __forceinline__ uint4 load(unsigned long long i) const {
    return i < n4 ? __ldg(p4 + i) : make_uint4(0, 0, 0, 0);
  }
  __device__ __forceinline__ uint32_t take() {
    if (bi == 4) {
      b0 = b1;
      b1 = load(next4++);
      bi = 0;
    }
    const int i = bi++;
    return i == 0 ? b0.x : i == 1 ? b0.y : i == 2 ? b0.z : b0.w;
  }
  __device__ __forceinline__ void init(const uint32_t *pl, unsigned long long nwords,
                                       unsigned long long pos) {
    p4 = reinterpret_cast<const uint4 *>(pl);
    n4 = (nwords + 3) >> 2;
    const unsigned long long w = pos >> 5;
    b0 = load(w >> 2);
    b1 = load((w >> 2) + 1);
    next4 = (w >> 2) + 2;
    bi = (int)(w & 3);
    win = ((unsigned long long)take() << 32);
    win |= take();
    const int off = (int)(pos & 31);
    win <<= off;
    nb = 64 - off;
    if (nb <= 32) {
      win |= (unsigned long long)take() << (32 - nb);
      nb += 32;
    }
  }
  __device__ __forceinline__ uint32_t peek(int n) const { return (uint32_t)(win >> (64 - n)); }
  __device__ __forceinline__ void skip(int n) {
    win <<= n;
    nb -= n;
    if (nb <= 32) {
      win |= (unsigned long long)take() << (32 - nb);
      nb += 32;
    }
  }
  __device__ __forceinline__ unsigned long long read(int n) {
    unsigned long long v = 0;
    if (n > 32) {
      v = (unsigned long long)peek(n - 32) << 32;
      skip(n - 32);
      n = 32;
    }
    if (n > 0) {
      v |= peek(n);
      skip(n);
    }
    return v;
  }
};

// All Huffman streams of a container in one launch.  CTA b serves stream s
// with cta_base[s] <= b < cta_base[s+1]; inside it, a warp decodes 32
// consecutive chunks, lane l the chunk c0 + l, kDecR symbols per round into
// a shared-memory stage; each store instruction then writes kDecR
// consecutive values of 32 / kDecR chunks.
constexpr int kDecWarps = 8;
constexpr int kDecR = 16;
constexpr size_t kDecStage = sizeof(unsigned long long) * kDecWarps * 32 * (kDecR + 1);

struct HuffJob {
  const uint8_t *sec;
  StreamInfo info;
  const HuffTable *ht;
  void *out;
  int wide;  // 8-byte outputs
  unsigned cta_base;
};
struct HuffJobs {
  HuffJob j[3];
  int n;
};

// MSB-first bit window over one lane's payload words: w holds nb valid bits
// (left aligned), kept above 32 after every refill; nx is the next word,
// loaded one refill ahead.  Words past the payload read as zero.
struct LaneBits {
  unsigned long long w;
  int nb;
  uint32_t nx;
  const uint32_t *p, *end;
  __device__ __forceinline__ uint32_t ld(const uint32_t *q) const { return q < end ? __ldg(q) : 0u; }
  __device__ __forceinline__ void init(const uint32_t *pl, unsigned long long nwords,
                                       unsigned long long pos) {
    end = pl + nwords;
    const uint32_t *q = pl + (pos >> 5);
    w = ((unsigned long long)ld(q) << 32) | ld(q + 1);
    const int off = (int)(pos & 31);
    w <<= off;
    nb = 64 - off;
    p = q + 2;
    nx = ld(p);
    refill();
  }
  __device__ __forceinline__ void refill() {
    if (nb <= 32) {
      w |= (unsigned long long)nx << (32 - nb);
      nb += 32;
      ++p;
      nx = ld(p);
    }
  }
  __device__ __forceinline__ void drop(int n) {  // n <= 32
    w <<= n;
    nb -= n;
    refill();
  }
  __device__ __forceinline__ unsigned long long raw(int width) {  // 1 <= width <= 64
    if (width <= 32) {
      const unsigned long long v = w >> (64 - width);
      drop(width);
      return v;
    }
    const int h = width - 32;
    const unsigned long long hi = w >> (64 - h);
    drop(h);
    const unsigned long long lo = w >> 32;
    drop(32);
    return (hi << 32) | lo;
  }
};

__global__ void __launch_bounds__(32 * kDecWarps) k_huff_decode(HuffJobs jobs,
                                                                int *__restrict__ err) {
  __shared__ uint32_t fast[1 << kFastBits];
  __shared__ uint32_t first[kLmax + 1], index[kLmax + 1], count[kLmax + 1];
  __shared__ uint16_t syms[kAlpha];
  extern __shared__ unsigned long long dec_stage[];  // [warp][lane][kDecR + 1]
  int js = 0;
  while (js + 1 < jobs.n && blockIdx.x >= jobs.j[js + 1].cta_base) ++js;
  const HuffJob &J = jobs.j[js];
  const HuffTable *HT = J.ht;
  const StreamInfo info = J.info;
  for (int i = threadIdx.x; i < (1 << kFastBits); i += blockDim.x) fast[i] = HT->fast[i];
  for (int i = threadIdx.x; i < (int)HT->used && i < kAlpha; i += blockDim.x) syms[i] = HT->syms[i];
  if (threadIdx.x <= kLmax) {
    first[threadIdx.x] = HT->first[threadIdx.x];
    index[threadIdx.x] = HT->index[threadIdx.x];
    count[threadIdx.x] = HT->count[threadIdx.x];
  }
  __syncthreads();
  if (!HT->ok) {
    if (threadIdx.x == 0) atomicExch(err, 1);
    return;
  }
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  unsigned long long(*stage)[kDecR + 1] =
      reinterpret_cast<unsigned long long(*)[kDecR + 1]>(dec_stage + (size_t)wl * 32 * (kDecR + 1));
  const unsigned long long cs = 1ull << info.log2_chunk;
  const uint8_t *ct = J.sec + pad16(80ull + 2ull * info.used);
  const uint32_t *pl = reinterpret_cast<const uint32_t *>(ct + pad16(8ull * info.n_chunks));
  const unsigned long long nwords = words_of(info.payload_bits);
  const unsigned long long g = (unsigned long long)(blockIdx.x - J.cta_base) * kDecWarps + wl;
  const unsigned long long groups = (info.n_chunks + 31) / 32;
  if (g >= groups) return;
  const unsigned long long c = g * 32 + lane;
  const bool act = c < info.n_chunks;
  const unsigned long long lo = c * cs;
  const unsigned long long hi = act ? min(info.n, lo + cs) : lo;
  LaneBits br;
  bool ok = true;
  if (act) {
    const unsigned long long pos = (unsigned long long)reinterpret_cast<const uint32_t *>(ct)[2 * c] |
                                   ((unsigned long long)reinterpret_cast<const uint32_t *>(ct)[2 * c + 1] << 32);
    if (pos > info.payload_bits) ok = false;
    br.init(pl, nwords, ok ? pos : 0ull);
  }
  const uint32_t mine = (act && ok) ? (uint32_t)(hi - lo) : 0u;
  const int width = (int)info.width;
  bool bad = act && !ok;
  unsigned long long *o64 = reinterpret_cast<unsigned long long *>(J.out);
  uint32_t *o32 = reinterpret_cast<uint32_t *>(J.out);
  constexpr int kChunksPerStore = 32 / kDecR;
  const int wsub = lane % kDecR, wch = lane / kDecR;
  for (uint32_t r0 = 0; r0 < (uint32_t)cs; r0 += kDecR) {
    const uint32_t todo = mine > r0 ? min(mine - r0, (uint32_t)kDecR) : 0u;
    for (uint32_t k = 0; k < todo; ++k) {
      const uint32_t e = fast[(uint32_t)(br.w >> (64 - kFastBits))];
      uint32_t sym;
      int len;
      if (e) {
        sym = e >> 5;
        len = (int)(e & 31u);
      } else {
        int L = kFastBits + 1;
        uint32_t code = 0;
        for (; L <= kLmax; ++L) {
          code = (uint32_t)(br.w >> (64 - L));
          if (code - first[L] < count[L]) break;
        }
        if (L > kLmax) {
          bad = true;
          sym = 0;
          len = 1;
        } else {
          sym = syms[index[L] + (code - first[L])];
          len = L;
        }
      }
      br.drop(len);
      unsigned long long v = sym;
      if (sym == (uint32_t)kEsc && width > 0) v = br.raw(width);
      stage[lane][k] = v;
    }
    __syncwarp();
#pragma unroll 4
    for (int it = 0; it < 32 / kChunksPerStore; ++it) {
      const int l = it * kChunksPerStore + wch;
      const unsigned long long cl = g * 32 + l;
      const unsigned long long base = cl * cs + r0 + wsub;
      if (cl < info.n_chunks && base < min(info.n, cl * cs + cs)) {
        if (J.wide) o64[base] = stage[l][wsub];
        else o32[base] = (uint32_t)stage[l][wsub];
      }
    }
    __syncwarp();
    if (__all_sync(0xffffffffu, r0 + kDecR >= mine)) break;
  }
  if (bad) atomicExch(err, 1);
}

template <typename T>
__global__ void k_fixed_decode(const uint8_t *__restrict__ sec, StreamInfo info,
                               T *__restrict__ out) {
  const uint32_t *pl = reinterpret_cast<const uint32_t *>(sec + 32);
  const uint32_t w = info.width;
  const unsigned long long nwords = words_of(info.payload_bits);
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < info.n;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    if (w == 0) {
      out[i] = (T)0;
      continue;
    }
    const unsigned long long pos = i * w;
    const unsigned long long wi = pos >> 5;
    const int off = (int)(pos & 31);
    // up to 64 + 31 bits: three words
    unsigned long long a = __ldg(pl + wi);
    unsigned long long b = wi + 1 < nwords ? __ldg(pl + wi + 1) : 0u;
    unsigned long long c = wi + 2 < nwords ? __ldg(pl + wi + 2) : 0u;
    unsigned long long hi64 = (a << 32) | b;  // bits [wi*32, wi*32+64)
    unsigned long long v;
    if (off + (int)w <= 64) {
      v = (hi64 << off) >> (64 - w);
    } else {
      // value spills into the third word
      unsigned long long top = (hi64 << off);  // 64 - off valid bits at the top
      int rest = off + (int)w - 64;
      v = (top >> (64 - w)) | (c >> (32 - rest));
    }
    out[i] = (T)v;
  }
}

void launch_decode_streams(int ns, const uint8_t *const *secs, const StreamInfo *infos,
                           HuffTable *ht, void *const *outs, const int *wide, int *err, int sms,
                           cudaStream_t s) {
  HuffJobs jobs;
  jobs.n = 0;
  unsigned ctas = 0;
  for (int k = 0; k < ns; ++k) {
    const StreamInfo &I = infos[k];
    if (I.n == 0) continue;
    if (I.coder == 0) {
      unsigned g = (unsigned)std::min<unsigned long long>((I.n + 255) / 256, 8ull * sms);
      note_launch();
      if (wide[k])
        k_fixed_decode<unsigned long long><<<g, 256, 0, s>>>(secs[k], I,
                                                            (unsigned long long *)outs[k]);
      else
        k_fixed_decode<uint32_t><<<g, 256, 0, s>>>(secs[k], I, (uint32_t *)outs[k]);
      continue;
    }
    launch_huff_table(secs[k], ht + k, s);
    HuffJob &J = jobs.j[jobs.n++];
    J.sec = secs[k];
    J.info = I;
    J.ht = ht + k;
    J.out = outs[k];
    J.wide = wide[k];
    J.cta_base = ctas;
    const unsigned long long groups = (I.n_chunks + 31) / 32;
    ctas += (unsigned)((groups + kDecWarps - 1) / kDecWarps);
  }
  (void)sms;
  if (jobs.n) {
    static const bool attr =  // once per process, thread-safe
        cudaFuncSetAttribute(k_huff_decode, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kDecStage) == cudaSuccess;
    (void)attr;
    note_launch();
    k_huff_decode<<<ctas, 32 * kDecWarps, kDecStage, s>>>(jobs, err);
  }
}

// ---------------------------------------------------------------------------
// scans over blocks (reduce, scan of tile sums, rescan)
// ---------------------------------------------------------------------------
constexpr int kScanTile = 4096;

// mode 0: plain values; mode 1: unzigzag of the values
template <int MODE>
__global__ void __launch_bounds__(1024) k_tile_sum(const unsigned long long *__restrict__ in,
                                                   uint64_t n,
                                                   unsigned long long *__restrict__ sums) {
  __shared__ unsigned long long s[32];
  const uint64_t lo = (uint64_t)blockIdx.x * kScanTile;
  unsigned long long acc = 0;
  for (uint64_t i = lo + threadIdx.x; i < min(n, lo + kScanTile); i += blockDim.x) {
    unsigned long long v = in[i];
    acc += MODE ? (unsigned long long)unzigzag(v) : v;
  }
  for (int o = 16; o; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    acc = s[threadIdx.x];
    for (int o = 16; o; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (threadIdx.x == 0) sums[blockIdx.x] = acc;
  }
}

// out[i] = base + (inclusive or exclusive) prefix of f(in)
template <int MODE, bool INCL>
__global__ void __launch_bounds__(1024) k_tile_scan(const unsigned long long *__restrict__ in,
                                                    uint64_t n,
                                                    const unsigned long long *__restrict__ bases,
                                                    unsigned long long *__restrict__ out) {
  __shared__ unsigned long long s_warp[32];
  const uint64_t lo = (uint64_t)blockIdx.x * kScanTile;
  constexpr int per = kScanTile / 1024;
  unsigned long long v[per];
  unsigned long long sum = 0;
  const uint64_t my = lo + (uint64_t)threadIdx.x * per;
#pragma unroll
  for (int k = 0; k < per; ++k) {
    uint64_t i = my + k;
    unsigned long long x = i < n ? in[i] : 0ull;
    v[k] = MODE ? (unsigned long long)unzigzag(x) : x;
    if (i >= n) v[k] = 0ull;
    sum += v[k];
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  unsigned long long x = sum;
  for (int o = 1; o < 32; o <<= 1) {
    unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[w] = x;
  __syncthreads();
  if (w == 0) {
    unsigned long long t = s_warp[lane];
    for (int o = 1; o < 32; o <<= 1) {
      unsigned long long y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    s_warp[lane] = t;
  }
  __syncthreads();
  unsigned long long run = bases[blockIdx.x] + (w ? s_warp[w - 1] : 0ull) + x - sum;
#pragma unroll
  for (int k = 0; k < per; ++k) {
    uint64_t i = my + k;
    if (INCL) run += v[k];
    if (i < n) out[i] = run;
    if (!INCL) run += v[k];
  }
}

void launch_scan_u64(const unsigned long long *in, uint64_t n, int mode, bool inclusive,
                     unsigned long long *out, unsigned long long *tile_tmp,
                     unsigned long long *tile_base, cudaStream_t s) {
  if (n == 0) return;
  const uint64_t tiles = (n + kScanTile - 1) / kScanTile;
  note_launch();
  if (mode) k_tile_sum<1><<<(unsigned)tiles, 1024, 0, s>>>(in, n, tile_tmp);
  else k_tile_sum<0><<<(unsigned)tiles, 1024, 0, s>>>(in, n, tile_tmp);
  launch_scan_small(tile_tmp, (uint32_t)tiles, tile_base, s);
  note_launch();
  if (mode) {
    if (inclusive) k_tile_scan<1, true><<<(unsigned)tiles, 1024, 0, s>>>(in, n, tile_base, out);
    else k_tile_scan<1, false><<<(unsigned)tiles, 1024, 0, s>>>(in, n, tile_base, out);
  } else {
    if (inclusive) k_tile_scan<0, true><<<(unsigned)tiles, 1024, 0, s>>>(in, n, tile_base, out);
    else k_tile_scan<0, false><<<(unsigned)tiles, 1024, 0, s>>>(in, n, tile_base, out);
  }
}

// ---------------------------------------------------------------------------
// block scans of an LCP-S frame: block ids (inclusive scan of the id deltas),
// counts (inclusive scan of the count deltas) and block starts (exclusive
// scan of the counts).  Here only the bases of each tile of kBsTile blocks
// are formed; k_expand_blocks applies them.  Tile aggregates: id sum A, count
// delta sum B, and P = sum of the local inclusive count prefixes, so that the
// counts of a tile with carry-in C sum to len * C + P.
// ---------------------------------------------------------------------------
constexpr int kBsTile = 1024;   // blocks per aggregate tile = blocks per expand CTA
constexpr int kBsThreads = 256;
constexpr int kExpTile = 1024;

struct BsAgg {
  unsigned long long a, b, p, len;
};

template <int THREADS>
__device__ __forceinline__ unsigned long long blk_exscan(unsigned long long v,
                                                         unsigned long long *s_warp,
                                                         unsigned long long &total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  unsigned long long x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[w] = x;
  __syncthreads();
  if (w == 0) {
    unsigned long long t = lane < THREADS / 32 ? s_warp[lane] : 0ull;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      unsigned long long y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    s_warp[lane] = t;
  }
  __syncthreads();
  unsigned long long base = w > 0 ? s_warp[w - 1] : 0ull;
  total = s_warp[THREADS / 32 - 1];
  __syncthreads();
  return base + x - v;
}

__global__ void __launch_bounds__(kBsThreads) k_bscan_sum(const unsigned long long *__restrict__ sid,
                                                          const unsigned long long *__restrict__ scnt,
                                                          uint64_t M, BsAgg *__restrict__ agg) {
  __shared__ unsigned long long s_warp[32];
  constexpr int per = kBsTile / kBsThreads;
  const uint64_t lo = (uint64_t)blockIdx.x * kBsTile + (uint64_t)threadIdx.x * per;
  unsigned long long a = 0, b = 0, d[per];
#pragma unroll
  for (int k = 0; k < per; ++k) {
    const uint64_t i = lo + k;
    d[k] = 0;
    if (i < M) {
      a += sid[i];
      d[k] = (unsigned long long)unzigzag(scnt[i]);
    }
    b += d[k];
  }
  unsigned long long ta, tb;
  blk_exscan<kBsThreads>(a, s_warp, ta);
  unsigned long long run = blk_exscan<kBsThreads>(b, s_warp, tb);  // prefix of deltas before me
  unsigned long long p = 0;
#pragma unroll
  for (int k = 0; k < per; ++k) {
    run += d[k];
    if (lo + k < M) p += run;
  }
  unsigned long long tp;
  blk_exscan<kBsThreads>(p, s_warp, tp);
  if (threadIdx.x == 0) {
    const uint64_t t0 = (uint64_t)blockIdx.x * kBsTile;
    agg[blockIdx.x] = BsAgg{ta, tb, tp, (M - t0) < (uint64_t)kBsTile ? M - t0 : (uint64_t)kBsTile};
  }
}

// Two-level tile bases.  Level 1: CTA c scans the aggregates of tiles
// [1024 c, 1024 c + 1024), one per thread, coalesced; each tile's aggregate
// is replaced by its bases within the chunk (id base, count carry-in, start
// base, and the chunk's blocks before it), and the chunk's own aggregate goes
// to cagg[c].  Level 2 (k_bscan_top) scans the chunk aggregates.  A tile's
// start base is then the chunk's start base + the chunk's count carry-in x
// the chunk's blocks before the tile + the tile's start base in the chunk.
constexpr int kBsChunk = 1024;
__global__ void __launch_bounds__(kBsChunk) k_bscan_chunk(BsAgg *__restrict__ agg, uint32_t tiles,
                                                          BsAgg *__restrict__ cagg) {
  __shared__ unsigned long long s_warp[32];
  const uint32_t t = blockIdx.x * kBsChunk + threadIdx.x;
  const BsAgg g = t < tiles ? agg[t] : BsAgg{0, 0, 0, 0};
  unsigned long long ta, tb, tl, ts;
  const unsigned long long ra = blk_exscan<kBsChunk>(g.a, s_warp, ta);
  const unsigned long long rb = blk_exscan<kBsChunk>(g.b, s_warp, tb);
  const unsigned long long rl = blk_exscan<kBsChunk>(g.len, s_warp, tl);
  const unsigned long long rs = blk_exscan<kBsChunk>(g.len * rb + g.p, s_warp, ts);
  if (t < tiles) agg[t] = BsAgg{ra, rb, rs, rl};
  if (threadIdx.x == 0) cagg[blockIdx.x] = BsAgg{ta, tb, ts, tl};
}

// chunk bases: id base, count carry-in, start base (one CTA).  Rounds of
// 1024 chunks, one per thread (coalesced; the next round's aggregates loaded
// before the current one is scanned), with the three running carries.
__global__ void __launch_bounds__(1024) k_bscan_top(BsAgg *__restrict__ agg, uint32_t tiles) {
  __shared__ unsigned long long s_warp[32];
  unsigned long long ca = 0, cb = 0, cs = 0;  // carries into the round
  BsAgg cur = threadIdx.x < tiles ? agg[threadIdx.x] : BsAgg{0, 0, 0, 0};
  for (uint32_t r0 = 0; r0 < tiles; r0 += 1024) {
    const uint32_t t = r0 + threadIdx.x;
    const uint32_t tn = t + 1024;
    const BsAgg nxt = tn < tiles ? agg[tn] : BsAgg{0, 0, 0, 0};
    unsigned long long ta, tb, ts;
    const unsigned long long ra = ca + blk_exscan<1024>(cur.a, s_warp, ta);
    const unsigned long long rb = cb + blk_exscan<1024>(cur.b, s_warp, tb);
    // the counts of this tile sum to len * (its count carry-in) + p
    const unsigned long long mine = cur.len * rb + cur.p;
    const unsigned long long rs = cs + blk_exscan<1024>(mine, s_warp, ts);
    if (t < tiles) agg[t] = BsAgg{ra, rb, rs, cur.len};
    ca += ta;
    cb += tb;
    cs += ts;
    cur = nxt;
  }
}


// counts (inclusive scan of count deltas) must be >= 1 and sum to nb
__global__ void k_check_counts(const unsigned long long *__restrict__ counts, uint64_t m,
                               const unsigned long long *__restrict__ starts_total, uint64_t nb,
                               int *__restrict__ err) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
       i += (uint64_t)gridDim.x * blockDim.x) {
    long long c = (long long)counts[i];
    if (c < 1 || (unsigned long long)c > nb) atomicExch(err, 1);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && *starts_total != nb) atomicExch(err, 1);
}

void launch_check_counts(const unsigned long long *counts, uint64_t m,
                         const unsigned long long *starts_total, uint64_t nb, int *err, int sms,
                         cudaStream_t s) {
  note_launch();
  k_check_counts<<<2 * sms, 256, 0, s>>>(counts, m, starts_total, nb, err);
}

// ---------------------------------------------------------------------------
// LCP-S expand by block tiles (the block scans' last pass fused in): CTA t
// takes blocks [1024 t, 1024 t + 1024) and the particles they hold, a
// contiguous slot range [P0, P1).  From the decoded id and count deltas and
// the tile bases it forms the blocks' ids, counts and starts in shared memory
// (per-axis block corners by multiply-shift division), then expands the
// particles in windows of 1024 slots, four consecutive slots per thread:
// block ordinal by counting start flags, relative codes by a segmented scan
// (segments at block and chunk starts) carried across windows, values by Q2.
// ---------------------------------------------------------------------------
constexpr int kXThreads = 256;
constexpr int kXPer = kBsTile / kXThreads;  // blocks, then slots, per thread
static_assert(kXPer == 4 && kExpTile == kXThreads * 4, "four blocks / slots per thread");

template <int D>
__global__ void __launch_bounds__(kXThreads, 3) k_expand_blocks(
    const Plan *__restrict__ plan, const unsigned long long *__restrict__ sid,
    const unsigned long long *__restrict__ scnt, uint64_t M, const BsAgg *__restrict__ agg,
    const BsAgg *__restrict__ cagg, const uint32_t *__restrict__ s_rel, uint64_t nb, uint64_t n,
    uint32_t log2_chunk, float *__restrict__ out, int32_t *__restrict__ qout,
    int *__restrict__ err) {
  __shared__ FieldPlan sF[D];
  __shared__ uint32_t sb_f[kBsTile][D];  // per-axis block corners
  __shared__ unsigned long long s_st[kBsTile];  // absolute block starts
  __shared__ __align__(16) uint8_t s_flag[kExpTile];
  __shared__ unsigned long long s_warp[32];
  __shared__ uint32_t s_wv[kXThreads / 32], s_wf[kXThreads / 32], s_wb[kXThreads / 32];
  __shared__ uint32_t s_lp, s_cv, s_cb;
  if (threadIdx.x < D) sF[threadIdx.x] = plan->f[threadIdx.x];
  if (threadIdx.x == 0) s_lp = plan->lp;
  BsAgg base;  // a: id base, b: count carry-in, p: first start
  {
    const BsAgg lb = agg[blockIdx.x], cb = cagg[blockIdx.x / kBsChunk];
    base.a = cb.a + lb.a;
    base.b = cb.b + lb.b;
    base.p = cb.p + cb.b * lb.len + lb.p;
  }
  const uint64_t b0 = (uint64_t)blockIdx.x * kBsTile + (uint64_t)threadIdx.x * kXPer;
  // ---- blocks: ids, counts, starts ----
  unsigned long long a[kXPer], dl[kXPer];
  unsigned long long sa = 0, sd = 0;
#pragma unroll
  for (int j = 0; j < kXPer; ++j) {
    a[j] = 0ull;
    dl[j] = 0ull;
    if (b0 + j < M) {
      a[j] = sid[b0 + j];
      dl[j] = (unsigned long long)unzigzag(scnt[b0 + j]);
    }
    sa += a[j];
    sd += dl[j];
  }
  unsigned long long tot;
  unsigned long long ra = base.a + blk_exscan<kXThreads>(sa, s_warp, tot);
  unsigned long long rd = blk_exscan<kXThreads>(sd, s_warp, tot);
  unsigned long long cnt[kXPer], cs = 0;
  {
    unsigned long long lp = rd;
#pragma unroll
    for (int j = 0; j < kXPer; ++j) {
      lp += dl[j];
      cnt[j] = base.b + lp;  // the count: carry-in plus the deltas so far
      if (b0 + j < M) cs += cnt[j];
    }
  }
  unsigned long long L;
  unsigned long long rs = base.p + blk_exscan<kXThreads>(cs, s_warp, L);
  const uint32_t lp = s_lp;
  bool bad = false;
#pragma unroll
  for (int j = 0; j < kXPer; ++j) {
    const uint64_t i = b0 + j;
    if (i >= M) continue;
    ra += a[j];
    const long long c = (long long)cnt[j];
    if (c < 1 || (unsigned long long)c > nb || rs + (unsigned long long)c > nb) bad = true;
    if (i == M - 1 && rs + (unsigned long long)(c > 0 ? c : 0) != nb) bad = true;
    s_st[threadIdx.x * kXPer + j] = rs;
    unsigned long long r = ra;
#pragma unroll
    for (int f = 0; f < D; ++f) {
      const FieldPlan &F = sF[f];
      const unsigned long long qd = F.bshift == 255u ? r : (__umul64hi(r, F.bmagic) >> F.bshift);
      const unsigned long long bf = r - qd * F.bn;
      sb_f[threadIdx.x * kXPer + j][f] = (uint32_t)(bf << lp);
      r = qd;
    }
    rs += (unsigned long long)(c > 0 ? c : 0);
  }
  if (bad) atomicExch(err, 1);
  if (threadIdx.x == 0) {
    s_cv = 0u;
    s_cb = 0u;
  }
  // ---- particles of the tile's blocks: slots [P0, P1) ----
  const uint64_t P0 = base.p < nb ? base.p : nb;
  const uint64_t P1 = base.p + L < nb ? base.p + L : nb;
  const uint64_t cmask = (1ull << log2_chunk) - 1ull;
  const uint32_t pm = (1u << lp) - 1u;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const bool aligned = (n & 3ull) == 0 && ((((uintptr_t)out) | (uintptr_t)qout) & 15u) == 0;
  for (uint64_t R0 = P0 & ~3ull; R0 < P1; R0 += kExpTile) {
    reinterpret_cast<uint32_t *>(s_flag)[threadIdx.x] = 0u;
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kXPer; ++j) {
      if (b0 + j >= M) continue;
      const unsigned long long st = s_st[threadIdx.x * kXPer + j];
      if (st >= R0 && st < R0 + kExpTile) s_flag[st - R0] = 1;
    }
    __syncthreads();
    const uint32_t cv_in = s_cv, cb_in = s_cb;
    const uint64_t k0 = R0 + (uint64_t)threadIdx.x * 4;
    const uint32_t flags4 = reinterpret_cast<const uint32_t *>(s_flag)[threadIdx.x];
    uint32_t x[4], fl[4];
    const bool full = k0 >= P0 && k0 + 4 <= P1;
    if (full) {
      const uint4 v = *reinterpret_cast<const uint4 *>(s_rel + k0);
      x[0] = v.x;
      x[1] = v.y;
      x[2] = v.z;
      x[3] = v.w;
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j) x[j] = (k0 + j >= P0 && k0 + j < P1) ? s_rel[k0 + j] : 0u;
    }
    uint32_t tv = 0u, tf = 0u, tb = 0u;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const uint64_t k = k0 + j;
      const uint32_t f = (flags4 >> (8 * j)) & 1u;
      fl[j] = f;
      const bool seg = f || ((k & cmask) == 0);
      if (seg) {
        tv = x[j];
        tf = 1u;
      } else {
        tv += x[j];
      }
      x[j] = tv;
      tb += f;
    }
    uint32_t cvv = tv, cff = tf, ccc = tb;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, cvv, o);
      const uint32_t g = __shfl_up_sync(0xffffffffu, cff, o);
      const uint32_t c = __shfl_up_sync(0xffffffffu, ccc, o);
      if (lane >= o) {
        if (!cff) cvv += y;
        cff |= g;
        ccc += c;
      }
    }
    if (lane == 31) {
      s_wv[w] = cvv;
      s_wf[w] = cff;
      s_wb[w] = ccc;
    }
    __syncthreads();
    // carry into this warp: the previous window, then warps 0..w-1
    uint32_t wv = cv_in, wb = cb_in;
    for (int u = 0; u < w; ++u) {
      if (s_wf[u]) wv = s_wv[u];
      else wv += s_wv[u];
      wb += s_wb[u];
    }
    uint32_t ev = __shfl_up_sync(0xffffffffu, cvv, 1);
    uint32_t ef = __shfl_up_sync(0xffffffffu, cff, 1);
    uint32_t ec = __shfl_up_sync(0xffffffffu, ccc, 1);
    if (lane == 0) {
      ev = 0u;
      ef = 0u;
      ec = 0u;
    }
    const uint32_t inv = ef ? ev : ev + wv;
    uint32_t blk[4], rel[4];
    {
      bool seen = false;
      uint32_t bc = ec + wb;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const uint64_t k = k0 + j;
        seen |= fl[j] || ((k & cmask) == 0);
        rel[j] = seen ? x[j] : x[j] + inv;
        bc += fl[j];
        blk[j] = bc - 1u;  // ordinal of the block holding slot k within the tile
      }
    }
#pragma unroll
    for (int f = 0; f < D; ++f) {
      const uint32_t qmax = sF[f].qmax;
      float r[4];
      int32_t q4[4];
      bool over = false;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const bool valid = k0 + j >= P0 && k0 + j < P1;
        const uint32_t bj = valid ? blk[j] : 0u;
        const uint32_t q = sb_f[bj < (uint32_t)kBsTile ? bj : 0u][f] + ((rel[j] >> (f * lp)) & pm);
        over |= valid && (bj >= (uint32_t)kBsTile || q > qmax);
        q4[j] = (int32_t)q;
      }
      if (qmax < (1u << 23)) {  // every code of the field takes the binary32 path
        const float fm = sF[f].m, fe = sF[f].e;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          float z;
          r[j] = recon_rn_f32((long long)(uint32_t)q4[j], fm, fe, z)
                     ? z
                     : recon_slow((long long)(uint32_t)q4[j], sF[f]);
        }
      } else {
        const uint32_t c8 = sF[f].c8, sticky = sF[f].sticky;
        const long long mb = sF[f].mb;
        const int32_t g1 = sF[f].g1;
#pragma unroll
        for (int j = 0; j < 4; ++j)
          r[j] = reconstruct_c((long long)(uint32_t)q4[j], c8, mb, sticky, g1, sF[f]);
      }
      if (over) atomicExch(err, 1);
      float *o = out + (uint64_t)f * n + k0;
      if (full && aligned) {
        *reinterpret_cast<float4 *>(o) = make_float4(r[0], r[1], r[2], r[3]);
        if (qout)
          *reinterpret_cast<int4 *>(qout + (uint64_t)f * n + k0) =
              make_int4(q4[0], q4[1], q4[2], q4[3]);
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (k0 + j >= P0 && k0 + j < P1) {
            o[j] = r[j];
            if (qout) qout[(uint64_t)f * n + k0 + j] = q4[j];
          }
      }
    }
    // carries for the next window: the last slot's segmented value and
    // the start flags seen so far
    __syncthreads();
    if (threadIdx.x == kXThreads - 1) {
      s_cv = rel[3];
      s_cb = blk[3] + 1u;
    }
    __syncthreads();
  }
}

template <int D>
static void expand_blocks_t(const Plan *plan, const unsigned long long *sid,
                            const unsigned long long *scnt, uint64_t M, const BsAgg *agg,
                            const uint32_t *s_rel, uint64_t nb, uint64_t n, uint32_t log2_chunk,
                            float *out, int32_t *qout, int *err, cudaStream_t s) {
  const uint64_t tiles = (M + kBsTile - 1) / kBsTile;
  if (tiles == 0) return;
  note_launch();
  k_expand_blocks<D><<<(unsigned)tiles, kXThreads, 0, s>>>(plan, sid, scnt, M, agg, agg + tiles,
                                                          s_rel, nb, n, log2_chunk, out, qout,
                                                          err);
}

void launch_expand_blocks(uint32_t d, const Plan *plan, const unsigned long long *sid,
                          const unsigned long long *scnt, uint64_t M, const void *agg,
                          const uint32_t *s_rel, uint64_t nb, uint64_t n, uint32_t log2_chunk,
                          float *out, int32_t *qout, int *err, cudaStream_t s) {
  const BsAgg *g = reinterpret_cast<const BsAgg *>(agg);
  switch (d) {
    case 1: expand_blocks_t<1>(plan, sid, scnt, M, g, s_rel, nb, n, log2_chunk, out, qout, err, s); break;
    case 2: expand_blocks_t<2>(plan, sid, scnt, M, g, s_rel, nb, n, log2_chunk, out, qout, err, s); break;
    case 3: expand_blocks_t<3>(plan, sid, scnt, M, g, s_rel, nb, n, log2_chunk, out, qout, err, s); break;
    case 4: expand_blocks_t<4>(plan, sid, scnt, M, g, s_rel, nb, n, log2_chunk, out, qout, err, s); break;
    case 5: expand_blocks_t<5>(plan, sid, scnt, M, g, s_rel, nb, n, log2_chunk, out, qout, err, s); break;
    case 6: expand_blocks_t<6>(plan, sid, scnt, M, g, s_rel, nb, n, log2_chunk, out, qout, err, s); break;
    case 7: expand_blocks_t<7>(plan, sid, scnt, M, g, s_rel, nb, n, log2_chunk, out, qout, err, s); break;
    default: expand_blocks_t<8>(plan, sid, scnt, M, g, s_rel, nb, n, log2_chunk, out, qout, err, s); break;
  }
}

// block-tile aggregates and their bases only (the expand applies them):
// agg holds the tiles' entries, then the chunks'
uint64_t block_bases_bytes(uint64_t M) {
  const uint64_t tiles = (M + kBsTile - 1) / kBsTile;
  return (tiles + (tiles + kBsChunk - 1) / kBsChunk + 1) * sizeof(BsAgg);
}

void launch_block_bases(const unsigned long long *sid, const unsigned long long *scnt, uint64_t M,
                        void *agg, cudaStream_t s) {
  if (M == 0) return;
  const uint64_t tiles = (M + kBsTile - 1) / kBsTile;
  const uint64_t chunks = (tiles + kBsChunk - 1) / kBsChunk;
  BsAgg *g = reinterpret_cast<BsAgg *>(agg);
  note_launch();
  k_bscan_sum<<<(unsigned)tiles, kBsThreads, 0, s>>>(sid, scnt, M, g);
  note_launch();
  k_bscan_chunk<<<(unsigned)chunks, kBsChunk, 0, s>>>(g, (uint32_t)tiles, g + tiles);
  note_launch();
  k_bscan_top<<<1, 1024, 0, s>>>(g + tiles, (uint32_t)chunks);
}

// raw outliers of an LCP-S frame go to the last K slots; their codes (for a
// trajectory reference) are Q1 of the raw values
__global__ void k_outliers_decode(const Plan *__restrict__ plan, const float *__restrict__ raw,
                                  uint64_t K, uint64_t n, uint32_t d, float *__restrict__ out,
                                  int32_t *__restrict__ qout) {
  const uint64_t nb = n - K;
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < K * d;
       t += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t f = t / K, j = t % K;
    float x = raw[f * K + j];
    out[f * n + nb + j] = x;
    if (qout) {
      bool chk;
      qout[f * n + nb + j] = quantize(x, plan->f[f], chk);
    }
  }
}

void launch_outliers_decode(const Plan *plan, const float *raw, uint64_t K, uint64_t n, uint32_t d,
                            float *out, int32_t *qout, int sms, cudaStream_t s) {
  if (K == 0) return;
  note_launch();
  k_outliers_decode<<<2 * sms, 256, 0, s>>>(plan, raw, K, n, d, out, qout);
}

}  // namespace lcp
