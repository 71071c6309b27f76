// k_decode.cu -- decompression kernels.
//
// Decoding follows the coding chain backwards (Sec. "Block coding"): decode
// each stream (chunks in parallel), undo the delta coding with scans, place
// particles block by block and reconstruct every field with Eq. quantization
// (reverse): x' = (2q + 1) eb + min, rounded once to f32.
#include <algorithm>
#include <type_traits>

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
    field_block_grid(F, df->lp);
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
}

// The bytes the host reads before decoding, gathered into one small buffer
// so that a single copy (and synchronization) brings them over: the fixed
// header with its field table and section directory (kHeadBytes, or the
// container if shorter) and the 32-byte header of each stream section the
// directory names (zeros where a section lies outside the container).
__global__ void k_head_gather(const uint8_t *__restrict__ in, uint64_t in_size,
                              uint8_t *__restrict__ stage) {
  const uint32_t t = threadIdx.x;
  const uint64_t head = in_size < (uint64_t)kHeadBytes ? in_size : (uint64_t)kHeadBytes;
  for (uint32_t i = t; i < (uint32_t)kHeadBytes; i += blockDim.x) stage[i] = i < head ? in[i] : 0;
  if (head < 48) return;
  const uint32_t method = in[5], d = in[6];
  if (d < 1 || d > kMaxD || method > 1) return;
  const uint32_t ns = method == 0 ? 3u : 1u;
  for (uint32_t k = 0; k < ns; ++k) {
    const uint64_t at = 48ull + 16ull * d + 16ull * k;
    uint64_t off = 0;
    for (int b = 7; b >= 0; --b) off = (off << 8) | in[at + b];
    const bool ok = (off & 15) == 0 && off + 32 <= in_size;
    for (uint32_t i = t; i < 32; i += blockDim.x)
      stage[kHeadBytes + 32 * k + i] = ok ? in[off + i] : 0;
  }
}

void launch_head_gather(const uint8_t *in, uint64_t in_size, uint8_t *stage, cudaStream_t s) {
  note_launch();
  k_head_gather<<<1, 64, 0, s>>>(in, in_size, stage);
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
  __syncthreads();
  // first-level table: codes of up to kFastBits bits, entry = sym << 5 | len
  huff_fill_fast(first, cnt, index, T->syms, min(U, (uint32_t)kAlpha), T->fast);
}

void launch_huff_table(const uint8_t *sec, HuffTable *T, cudaStream_t s) {
  note_launch();
  k_huff_table<<<1, 256, 0, s>>>(sec, T);
}

// ---------------------------------------------------------------------------
// stream decoding
// ---------------------------------------------------------------------------
// All Huffman streams of a container in one launch.  CTA b serves stream s
// with cta_base[s] <= b < cta_base[s+1]; inside it, a warp decodes 32
// consecutive chunks, lane l the chunk c0 + l, kDecR symbols per round into
// a shared-memory stage; each store instruction then writes kDecR
// consecutive values of 32 / kDecR chunks.  Outputs are 4-byte values, or
// 8-byte ones for streams whose largest value needs them.
constexpr int kDecWarps = 8;
constexpr int kDecR = 8;
constexpr int kRingWords = 64;  // payload ring per lane (see k_huff_decode)
// per warp: the payload ring
template <bool WIDE>
constexpr size_t kDecSmem() {
  return sizeof(uint32_t) * kRingWords * 32 * kDecWarps;
}

// block-tile aggregates of the LCP-S block scans: id delta sum a, count
// delta sum b, and p = the sum of the local inclusive count-delta prefixes,
// so that the counts of an aggregate of len blocks with count carry-in C sum
// to len C + p
struct BsAgg {
  unsigned long long a, b, p, len;
};

struct HuffJob {
  const uint8_t *sec;
  StreamInfo info;
  const HuffTable *ht;
  void *out;
  int wide;      // 8-byte outputs
  int agg_mode;  // 0 none; 1 block-id deltas (a, len); 2 count deltas (b, p)
  BsAgg *agg;    // one aggregate per chunk
  unsigned cta_base;
};
struct HuffJobs {
  HuffJob j[3];
  int n;
};

// Each lane decodes one chunk through a ring of kRing payload words in
// shared memory (word i of the lane's chunk at ring[i % kRing][lane], so
// that the 32 lanes of a warp always read 32 different banks).  Rounds of
// kDecR symbols: at the start of a round the lane refills the words it
// consumed in the previous round with asynchronous copies (cp.async, zero
// fill past the payload) and waits only for the copies issued one round
// earlier; a round reads at most kDecR (24 + 64) bits, and the ring keeps
// the words of the next two rounds, so no symbol waits on memory.
constexpr int kRing = kRingWords;
static_assert(kDecR * (kLmax + 64) <= 32 * (kRing / 2 - 2), "ring covers two rounds");


// WIDE: 8-byte values (streams whose largest value needs them); otherwise
// 4-byte values, and escapes are at most 32 bits wide.  A round's kDecR
// values stay in registers and are written with 16-byte stores straight to
// the lane's own chunk (whole 32-byte sectors).
template <bool WIDE>
__global__ void __launch_bounds__(32 * kDecWarps) k_huff_decode(HuffJobs jobs,
                                                                int *__restrict__ err) {
  using V = typename std::conditional<WIDE, unsigned long long, uint32_t>::type;
  __shared__ uint16_t fast[1 << kFastBits];  // sym << 4 | len (len <= 12), 0: longer code
  __shared__ unsigned long long lim[kLmax + 2];  // left-aligned end of the codes of each length
  __shared__ uint32_t first[kLmax + 1], index[kLmax + 1];
  __shared__ uint16_t syms[kAlpha];
  extern __shared__ __align__(16) uint32_t dec_smem[];
  int js = 0;
  while (js + 1 < jobs.n && blockIdx.x >= jobs.j[js + 1].cta_base) ++js;
  const HuffJob &J = jobs.j[js];
  const HuffTable *HT = J.ht;
  const StreamInfo info = J.info;
  for (int i = threadIdx.x; i < (1 << kFastBits); i += blockDim.x) {
    const uint32_t e = HT->fast[i];
    fast[i] = (uint16_t)(((e >> 5) << 4) | (e & 15u));
  }
  for (int i = threadIdx.x; i < (int)HT->used && i < kAlpha; i += blockDim.x) syms[i] = HT->syms[i];
  if (threadIdx.x <= kLmax) {
    const int L = threadIdx.x;
    first[L] = HT->first[L];
    index[L] = HT->index[L];
    // codes of length L are first[L] .. first[L] + count[L] - 1; in
    // canonical order a 32-bit window below (first[L] + count[L]) 2^(32 - L)
    // starts with a code of length <= L
    lim[L] = L == 0 ? 0ull : ((unsigned long long)HT->first[L] + HT->count[L]) << (32 - L);
  }
  __syncthreads();
  if (!HT->ok || (!WIDE && info.width > 32)) {
    if (threadIdx.x == 0) atomicExch(err, 1);
    return;
  }
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  uint32_t *myring = dec_smem + (size_t)wl * (kRing * 32) + lane;
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
  unsigned long long pos0 = 0;
  bool ok = true;
  if (act) {
    pos0 = (unsigned long long)reinterpret_cast<const uint32_t *>(ct)[2 * c] |
           ((unsigned long long)reinterpret_cast<const uint32_t *>(ct)[2 * c + 1] << 32);
    if (pos0 > info.payload_bits) ok = false;
  }
  if (!ok) pos0 = 0;
  // the lane's words: src + i for i < avail, zeros beyond
  const uint32_t *src = pl + (pos0 >> 5);
  const unsigned long long left = nwords - (pos0 >> 5);
  const uint32_t avail = left < 0xffffffffull ? (uint32_t)left : 0xffffffffu;
  uint32_t bp = (uint32_t)(pos0 & 31);  // bit position relative to word 0 of src
  uint32_t issued = 0;                  // words requested so far
  const uint32_t mine = (act && ok) ? (uint32_t)(hi - lo) : 0u;
  if (mine) {
    for (; issued < (uint32_t)kRing; ++issued)
      cp_async4(myring + issued * 32, issued < avail ? src + issued : pl, issued < avail);
  }
  cp_async_commit();
  cp_async_wait0();
  auto peek32 = [&](uint32_t b) {
    const uint32_t wi = b >> 5;
    const uint32_t x = myring[(wi & (kRing - 1)) * 32];
    const uint32_t y = myring[((wi + 1) & (kRing - 1)) * 32];
    return __funnelshift_l(y, x, b & 31);
  };
  const uint32_t width = info.width;
  const uint32_t esc_shift = (width && width <= 32u) ? 32u - width : 0u;
  const int amode = J.agg_mode;
  bool bad = act && !ok;
  unsigned long long s1 = 0ull, s2 = 0ull;  // aggregate sums (a; or b and p)
  V *out = reinterpret_cast<V *>(J.out) + lo;
  for (uint32_t r0 = 0; r0 < mine; r0 += kDecR) {
    if (r0) {  // refill what the last round consumed; wait for the round before
      const uint32_t need = (bp >> 5) + (uint32_t)kRing;
      for (; issued < need; ++issued)
        cp_async4(myring + (issued & (kRing - 1)) * 32, issued < avail ? src + issued : pl,
                  issued < avail);
    }
    cp_async_commit();
    cp_async_wait1();
    const uint32_t todo = min(mine - r0, (uint32_t)kDecR);
    V v[kDecR];
    if (!WIDE && todo == (uint32_t)kDecR) {
      // a full round of 4-byte values: one 64-bit window per symbol (three
      // ring words) gives the code and the escape bits after it
#pragma unroll
      for (int k = 0; k < kDecR; ++k) {
        const uint32_t wi = bp >> 5, sh = bp & 31u;
        const uint32_t a0 = myring[(wi & (kRing - 1)) * 32];
        const uint32_t a1 = myring[((wi + 1) & (kRing - 1)) * 32];
        const uint32_t a2 = myring[((wi + 2) & (kRing - 1)) * 32];
        const uint32_t hi = __funnelshift_l(a1, a0, sh);  // bits [bp, bp + 32)
        const uint32_t lo = __funnelshift_l(a2, a1, sh);  // bits [bp + 32, bp + 64)
        const uint32_t e = fast[hi >> (32 - kFastBits)];
        uint32_t sym = e >> 4;
        uint32_t len = e & 15u;
        if (__any_sync(__activemask(), e == 0u)) {
          if (e == 0u) {  // a code longer than the first-level table
            int L = kFastBits + 1;
            while (L <= kLmax && (unsigned long long)hi >= lim[L]) ++L;
            if (L > kLmax) {
              bad = true;
              sym = 0;
              len = 1;
            } else {
              sym = syms[index[L] + ((hi >> (32 - L)) - first[L])];
              len = (uint32_t)L;
            }
          }
        }
        const uint32_t after = __funnelshift_l(lo, hi, len);  // bits [bp + len, +32)
        const bool esc = sym == (uint32_t)kEsc && width > 0;
        v[k] = esc ? (V)(after >> esc_shift) : (V)sym;
        bp += len + (esc ? width : 0u);
      }
    } else {
#pragma unroll
      for (uint32_t k = 0; k < (uint32_t)kDecR; ++k) {
        const bool on = k < todo;
        const uint32_t win = peek32(bp);
        const uint32_t e = fast[win >> (32 - kFastBits)];
        uint32_t sym = e >> 4;
        uint32_t len = e & 15u;
        const bool longc = on && e == 0u;
        if (__any_sync(__activemask(), longc)) {
          if (longc) {  // a code longer than the first-level table
            int L = kFastBits + 1;
            while (L <= kLmax && (unsigned long long)win >= lim[L]) ++L;
            if (L > kLmax) {
              bad = true;
              sym = 0;
              len = 1;
            } else {
              sym = syms[index[L] + ((win >> (32 - L)) - first[L])];
              len = (uint32_t)L;
            }
          }
        }
        // the raw bits after an escape code, read by every lane (off the
        // dependency chain of the bit position: no branch on the escape)
        const bool esc = on && sym == (uint32_t)kEsc && width > 0;
        const uint32_t hw = peek32(bp + len);
        V x;
        if (!WIDE) {
          x = esc ? (hw >> (32u - width)) : sym;
        } else {
          x = sym;
          if (__any_sync(__activemask(), esc)) {
            if (esc) {
              if (width <= 32) {
                x = hw >> (32 - width);
              } else {
                const uint32_t lw = peek32(bp + len + 32);
                x = (V)((((unsigned long long)hw << 32) | lw) >> (64 - width));
              }
            }
          }
        }
        bp += on ? len + (esc ? width : 0u) : 0u;
        v[k] = on ? x : (V)0;
      }
    }
    if (amode == 1) {
#pragma unroll
      for (int k = 0; k < kDecR; ++k) s1 += (unsigned long long)v[k];
    } else if (amode == 2) {
#pragma unroll
      for (int k = 0; k < kDecR; ++k) {
        s1 += (unsigned long long)unzigzag((unsigned long long)v[k]);
        s2 += (uint32_t)k < todo ? s1 : 0ull;
      }
    }
    V *o = out + r0;
    if (todo == (uint32_t)kDecR) {
      if (WIDE) {
#pragma unroll
        for (int k = 0; k < kDecR; k += 2)
          *reinterpret_cast<ulonglong2 *>(o + k) =
              make_ulonglong2((unsigned long long)v[k], (unsigned long long)v[k + 1]);
      } else {
#pragma unroll
        for (int k = 0; k < kDecR; k += 4)
          *reinterpret_cast<uint4 *>(o + k) = make_uint4((uint32_t)v[k], (uint32_t)v[k + 1],
                                                         (uint32_t)v[k + 2], (uint32_t)v[k + 3]);
      }
    } else {
#pragma unroll
      for (int k = 0; k < kDecR; ++k)
        if ((uint32_t)k < todo) o[k] = v[k];
    }
  }
  cp_async_wait0();
  if (act && (pos0 & ~31ull) + bp > info.payload_bits) bad = true;
  if (act && amode == 1) {
    J.agg[c].a = s1;
    J.agg[c].len = hi - lo;
  } else if (act && amode == 2) {
    J.agg[c].b = s1;
    J.agg[c].p = s2;
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
                           HuffTable *ht, void *const *outs, const int *wide, const int *agg_mode,
                           void *agg, int *err, int sms, cudaStream_t s) {
  HuffJobs jobs[2];  // 4-byte and 8-byte values
  jobs[0].n = jobs[1].n = 0;
  unsigned ctas[2] = {0u, 0u};
  for (int k = 0; k < ns; ++k) {
    const StreamInfo &I = infos[k];
    if (I.n == 0 || !outs[k]) continue;
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
    const int wi = wide[k] ? 1 : 0;
    HuffJob &J = jobs[wi].j[jobs[wi].n++];
    J.sec = secs[k];
    J.info = I;
    J.ht = ht + k;
    J.out = outs[k];
    J.wide = wide[k];
    J.agg_mode = agg_mode ? agg_mode[k] : 0;
    J.agg = reinterpret_cast<BsAgg *>(agg);
    J.cta_base = ctas[wi];
    const unsigned long long groups = (I.n_chunks + 31) / 32;
    ctas[wi] += (unsigned)((groups + kDecWarps - 1) / kDecWarps);
  }
  // once per process, thread-safe
  static const bool attr =
      cudaFuncSetAttribute(k_huff_decode<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)kDecSmem<false>()) == cudaSuccess &&
      cudaFuncSetAttribute(k_huff_decode<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)kDecSmem<true>()) == cudaSuccess;
  (void)attr;
  if (jobs[0].n) {
    note_launch();
    k_huff_decode<false><<<ctas[0], 32 * kDecWarps, kDecSmem<false>(), s>>>(jobs[0], err);
  }
  if (jobs[1].n) {
    note_launch();
    k_huff_decode<true><<<ctas[1], 32 * kDecWarps, kDecSmem<true>(), s>>>(jobs[1], err);
  }
}

// ---------------------------------------------------------------------------
// block scans of an LCP-S frame: block ids (inclusive scan of the id deltas),
// counts (inclusive scan of the count deltas) and block starts (exclusive
// scan of the counts).  Only the bases of each aggregate (a run of 2^agg_log2
// blocks) are formed; the expand applies them.  The aggregates come from the
// Huffman decode (one per chunk) or from k_bscan_sum (one per 1024 blocks).
// ---------------------------------------------------------------------------
constexpr int kBsTile = 1024;   // blocks per expand tile
constexpr int kBsThreads = 256;
constexpr int kExpTile = 1024;  // slots per expand window

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

template <typename IdT>
__global__ void __launch_bounds__(kBsThreads) k_bscan_sum(const IdT *__restrict__ sid,
                                                          const IdT *__restrict__ scnt,
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
      a += (unsigned long long)sid[i];
      d[k] = (unsigned long long)unzigzag((unsigned long long)scnt[i]);
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

// Two-level aggregate bases.  Level 1: CTA c scans the aggregates
// [1024 c, 1024 c + 1024), one per thread, coalesced; each aggregate is
// replaced by its bases within the chunk (id base, count carry-in, start
// base, and the chunk's blocks before it), and the chunk's own aggregate
// goes to cagg[c].  Level 2 (k_bscan_top) scans the chunk aggregates.  An
// aggregate's start base is then the chunk's start base + the chunk's count
// carry-in x the chunk's blocks before it + its start base in the chunk.
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
    // the counts of this aggregate sum to len * (its count carry-in) + p
    const unsigned long long mine = cur.len * rb + cur.p;
    const unsigned long long rs = cs + blk_exscan<1024>(mine, s_warp, ts);
    if (t < tiles) agg[t] = BsAgg{ra, rb, rs, cur.len};
    ca += ta;
    cb += tb;
    cs += ts;
    cur = nxt;
  }
}

// ---------------------------------------------------------------------------
// reconstruction table: lut[off_f + q] = Q2 of code q of field f, for every
// q in [0, qmax_f] (Eq. quantization, reverse; exact)
// ---------------------------------------------------------------------------
__global__ void k_recon_lut(const Plan *__restrict__ plan, uint32_t d, LutOffsets lo,
                            float *__restrict__ lut) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < lo.off[d];
       i += gridDim.x * blockDim.x) {
    uint32_t f = 0;
    while (f + 1 < d && i >= lo.off[f + 1]) ++f;
    const FieldPlan &F = plan->f[f];
    const long long q = (long long)(i - lo.off[f]);
    float z;
    lut[i] = recon_rn_f32(q, F.m, F.e, z) ? z : reconstruct(q, F);
  }
}

void launch_recon_lut(const Plan *plan, uint32_t d, const LutOffsets &lo, float *lut, int sms,
                      cudaStream_t s) {
  if (lo.off[d] == 0) return;
  const unsigned g = (unsigned)std::min<uint64_t>((lo.off[d] + 255) / 256, (uint64_t)sms * 4);
  note_launch();
  k_recon_lut<<<g, 256, 0, s>>>(plan, d, lo, lut);
}

// ---------------------------------------------------------------------------
// LCP-S expand (Sec. "Block coding" backwards, Eq. quantization reversed).
// Persistent CTAs take block tiles t = blockIdx.x, blockIdx.x + gridDim.x,
// ...: tile t holds blocks [1024 t, 1024 t + 1024) and the particles they
// hold, a contiguous slot range [P0, P1).  From the decoded id and count
// deltas (4 or 8 bytes each) and the aggregate bases the CTA forms the
// blocks' ids, counts and starts (per-axis block corners by multiply-shift
// division, starts relative to the tile's first window) in shared memory,
// then expands the particles in windows of 1024 slots, four consecutive
// slots per thread: block ordinal by counting start flags, relative codes
// by a segmented scan (segments at block and chunk starts) carried across
// windows, codes q = corner + digit.  The relative-location deltas come from
// a decoded array, or straight from a fixed-width stream (the window's words
// staged in shared memory).  Values: with LUT, one shared-memory read of the
// reconstruction table per code; otherwise Q2 in arithmetic.  With out null
// only codes are written (a reference frame for LCP-T).
// ---------------------------------------------------------------------------
constexpr int kXThreads = 256;
constexpr int kXPer = kBsTile / kXThreads;  // blocks, then slots, per thread
static_assert(kXPer == 4 && kExpTile == kXThreads * 4, "four blocks / slots per thread");
constexpr int kRelStage = kExpTile + 4;     // staged words of a fixed-width window (w <= 32)


template <int THREADS>
__device__ __forceinline__ uint32_t blk_exscan32(uint32_t v, uint32_t *s_warp, uint32_t &total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[w] = x;
  __syncthreads();
  if (w == 0) {
    uint32_t t = lane < THREADS / 32 ? s_warp[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    s_warp[lane] = t;
  }
  __syncthreads();
  const uint32_t base = w > 0 ? s_warp[w - 1] : 0u;
  total = s_warp[THREADS / 32 - 1];
  __syncthreads();
  return base + x - v;
}

template <int D, bool LUT, bool C16>
__global__ void __launch_bounds__(kXThreads, 4) k_expand(const ExpandArgs a) {
  extern __shared__ __align__(16) float s_lut[];
  __shared__ FieldPlan sF[D];
  __shared__ uint4 s_c16[C16 ? kBsTile : 1];           // corners, 16 bits each
  __shared__ uint32_t s_c32[C16 ? 1 : kBsTile * D];    // corners, 32 bits each
  __shared__ uint32_t s_st[kBsTile];  // block starts, relative to the first window
  __shared__ __align__(16) uint8_t s_flag[kExpTile];
  __shared__ uint32_t s_rw[kRelStage];
  __shared__ unsigned long long s_w64[32];
  __shared__ uint32_t s_w32[32];
  __shared__ uint32_t s_wv[kXThreads / 32], s_wf[kXThreads / 32], s_wb[kXThreads / 32];
  __shared__ uint32_t s_cv, s_cb;
  if (threadIdx.x < D) sF[threadIdx.x] = a.plan->f[threadIdx.x];
  if (LUT) {
    const uint32_t tot = a.lut_off.off[D];
    for (uint32_t i = threadIdx.x; i < tot; i += kXThreads) s_lut[i] = a.lut[i];
  }
  const uint32_t lp = a.plan->lp;
  const uint64_t M = a.M, nb = a.nb, n = a.n;
  const uint64_t cmask = (1ull << a.log2_chunk) - 1ull;
  const uint32_t pm = (1u << lp) - 1u;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const bool aligned = (n & 3ull) == 0 && ((((uintptr_t)a.out) | (uintptr_t)a.qout) & 15u) == 0;
  const unsigned long long *sid64 = reinterpret_cast<const unsigned long long *>(a.sid);
  const unsigned long long *scnt64 = reinterpret_cast<const unsigned long long *>(a.scnt);
  const uint32_t *sid32 = reinterpret_cast<const uint32_t *>(a.sid);
  const uint32_t *scnt32 = reinterpret_cast<const uint32_t *>(a.scnt);
  const BsAgg *agg = reinterpret_cast<const BsAgg *>(a.agg);
  const BsAgg *cagg = agg + ((M + (1ull << a.agg_log2) - 1) >> a.agg_log2);
  bool bad = false;
  __syncthreads();
  for (uint64_t t = blockIdx.x; t < a.tiles; t += gridDim.x) {
    BsAgg base;  // a: id base, b: count carry-in, p: first start
    {
      const uint64_t e0 = t << (10 - a.agg_log2);
      const BsAgg lb = agg[e0], cb = cagg[e0 / kBsChunk];
      base.a = cb.a + lb.a;
      base.b = cb.b + lb.b;
      base.p = cb.p + cb.b * lb.len + lb.p;
    }
    const uint64_t b0 = t * kBsTile + (uint64_t)threadIdx.x * kXPer;
    // ---- blocks: ids (64-bit), counts and starts (32-bit, modulo 2^32:
    // exact, since every count and every tile's total is below 2^32) ----
    unsigned long long id[kXPer];
    uint32_t dl[kXPer];
    unsigned long long sa = 0;
    uint32_t sd = 0;
#pragma unroll
    for (int j = 0; j < kXPer; ++j) {
      id[j] = 0ull;
      dl[j] = 0u;
      if (b0 + j < M) {
        id[j] = a.wide ? sid64[b0 + j] : (unsigned long long)sid32[b0 + j];
        dl[j] = (uint32_t)unzigzag(a.wide ? scnt64[b0 + j] : (unsigned long long)scnt32[b0 + j]);
      }
      sa += id[j];
      sd += dl[j];
    }
    unsigned long long tot;
    unsigned long long ra = base.a + blk_exscan<kXThreads>(sa, s_w64, tot);
    uint32_t t32;
    uint32_t run = (uint32_t)base.b + blk_exscan32<kXThreads>(sd, s_w32, t32);
    uint32_t cnt[kXPer], cs = 0;
#pragma unroll
    for (int j = 0; j < kXPer; ++j) {
      run += dl[j];
      cnt[j] = run;
      if (b0 + j < M) cs += run;
    }
    uint32_t L;
    uint32_t rs = blk_exscan32<kXThreads>(cs, s_w32, L);
    const uint64_t P0 = base.p < nb ? base.p : nb;
    const uint64_t P1 = base.p + L < nb ? base.p + L : nb;
    const uint64_t W0 = P0 & ~3ull;  // first window start (16-byte stores)
    const uint32_t off0 = (uint32_t)(base.p - W0);
#pragma unroll
    for (int j = 0; j < kXPer; ++j) {
      const uint64_t i = b0 + j;
      if (i >= M) continue;
      ra += id[j];
      const uint32_t c = cnt[j];
      const uint64_t st = base.p + rs;
      if (c == 0u || (uint64_t)c > nb || st + c > nb) bad = true;
      if (i == M - 1 && st + c != nb) bad = true;
      s_st[threadIdx.x * kXPer + j] = off0 + rs;
      unsigned long long r = ra;
      uint32_t cor[D];
#pragma unroll
      for (int f = 0; f < D; ++f) {
        const FieldPlan &F = sF[f];
        unsigned long long qd;
        if (F.bshift == 255u) {
          qd = r;
        } else if ((r >> 32) == 0ull) {  // 32-bit dividend: two 32 x 32 products
          const uint32_t r32 = (uint32_t)r;
          const unsigned long long x = (unsigned long long)r32 * (uint32_t)F.bmagic;
          const unsigned long long y =
              (unsigned long long)r32 * (uint32_t)(F.bmagic >> 32) + (x >> 32);
          qd = (y >> 32) >> F.bshift;
        } else {
          qd = __umul64hi(r, F.bmagic) >> F.bshift;
        }
        cor[f] = (uint32_t)(r - qd * F.bn) << lp;
        r = qd;
      }
      if (C16) {
        uint32_t pk[4] = {0u, 0u, 0u, 0u};
#pragma unroll
        for (int f = 0; f < D; ++f) pk[f >> 1] |= cor[f] << (16 * (f & 1));
        s_c16[threadIdx.x * kXPer + j] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
      } else {
#pragma unroll
        for (int f = 0; f < D; ++f) s_c32[(threadIdx.x * kXPer + j) * D + f] = cor[f];
      }
      rs += c;
    }
    if (threadIdx.x == 0) {
      s_cv = 0u;
      s_cb = 0u;
    }
    // ---- particles of the tile's blocks: slots [P0, P1) ----
    for (uint64_t R0 = W0; R0 < P1; R0 += kExpTile) {
      const uint32_t wr = (uint32_t)(R0 - W0);  // window start, relative
      reinterpret_cast<uint32_t *>(s_flag)[threadIdx.x] = 0u;
      unsigned long long wlo = 0;
      if (!a.rel) {  // stage the window's fixed-width words
        const uint32_t rw = a.rel_w;
        wlo = (R0 * rw) >> 5;
        const uint32_t nw = (uint32_t)((((R0 + kExpTile) * rw + 31) >> 5) - wlo) + 1;
        for (uint32_t i = threadIdx.x; i < nw && i < (uint32_t)kRelStage; i += kXThreads)
          s_rw[i] = wlo + i < a.rel_words ? __ldg(a.rel_pl + wlo + i) : 0u;
      }
      __syncthreads();
#pragma unroll
      for (int j = 0; j < kXPer; ++j) {
        if (b0 + j >= M) continue;
        const uint32_t st = s_st[threadIdx.x * kXPer + j] - wr;
        if (st < (uint32_t)kExpTile) s_flag[st] = 1;
      }
      __syncthreads();
      const uint32_t cv_in = s_cv, cb_in = s_cb;
      const uint64_t k0 = R0 + (uint64_t)threadIdx.x * 4;
      uint32_t vm = 0u;  // valid slots of this thread
#pragma unroll
      for (int j = 0; j < 4; ++j) vm |= (k0 + j >= P0 && k0 + j < P1) ? (1u << j) : 0u;
      const bool full = vm == 0xfu;
      const uint32_t flags4 = reinterpret_cast<const uint32_t *>(s_flag)[threadIdx.x];
      uint32_t x[4], fl[4];
      if (a.rel) {
        if (full) {
          const uint4 v = *reinterpret_cast<const uint4 *>(a.rel + k0);
          x[0] = v.x;
          x[1] = v.y;
          x[2] = v.z;
          x[3] = v.w;
        } else {
#pragma unroll
          for (int j = 0; j < 4; ++j) x[j] = ((vm >> j) & 1u) ? a.rel[k0 + j] : 0u;
        }
      } else {
        const uint32_t rw = a.rel_w;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const unsigned long long bit = (k0 + j) * rw - (wlo << 5);
          const uint32_t wi = (uint32_t)(bit >> 5), off = (uint32_t)(bit & 31);
          const uint32_t v = __funnelshift_l(s_rw[wi + 1], s_rw[wi], off);
          x[j] = (rw && ((vm >> j) & 1u)) ? (v >> (32 - rw)) : 0u;
        }
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
      bool over = false;
      {
        bool seen = false;
        uint32_t bc = ec + wb;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const uint64_t k = k0 + j;
          seen |= fl[j] || ((k & cmask) == 0);
          const uint32_t rv = seen ? x[j] : x[j] + inv;
          bc += fl[j];
          const bool valid = (vm >> j) & 1u;
          over |= valid && (bc - 1u) >= (uint32_t)kBsTile;
          // slots outside [P0, P1) take block 0 and digits 0 (never stored)
          blk[j] = valid && (bc - 1u) < (uint32_t)kBsTile ? bc - 1u : 0u;
          rel[j] = valid ? rv : 0u;
        }
      }
      uint4 c16[C16 ? 4 : 1];
      if (C16) {
#pragma unroll
        for (int j = 0; j < 4; ++j) c16[j] = s_c16[blk[j]];
      }
#pragma unroll
      for (int f = 0; f < D; ++f) {
        const uint32_t qmax = sF[f].qmax;
        float r[4];
        int32_t q4[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          uint32_t cf;
          if (C16) {
            const uint32_t wd = (f >> 1) == 0 ? c16[j].x : (f >> 1) == 1 ? c16[j].y
                                : (f >> 1) == 2 ? c16[j].z : c16[j].w;
            cf = (f & 1) ? (wd >> 16) : (wd & 0xffffu);
          } else {
            cf = s_c32[blk[j] * D + f];
          }
          const uint32_t q = cf + ((rel[j] >> (f * lp)) & pm);
          over |= q > qmax;
          q4[j] = (int32_t)min(q, qmax);
        }
        if (a.out) {
          if (LUT) {
            const uint32_t o = a.lut_off.off[f];
#pragma unroll
            for (int j = 0; j < 4; ++j) r[j] = s_lut[o + (uint32_t)q4[j]];
          } else if (qmax < (1u << 23)) {  // every code of the field takes the binary32 path
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
          float *o = a.out + (uint64_t)f * n + k0;
          if (full && aligned) {
            *reinterpret_cast<float4 *>(o) = make_float4(r[0], r[1], r[2], r[3]);
          } else {
#pragma unroll
            for (int j = 0; j < 4; ++j)
              if ((vm >> j) & 1u) o[j] = r[j];
          }
        }
        if (a.qout) {
          int32_t *qo = a.qout + (uint64_t)f * n + k0;
          if (full && aligned) {
            *reinterpret_cast<int4 *>(qo) = make_int4(q4[0], q4[1], q4[2], q4[3]);
          } else {
#pragma unroll
            for (int j = 0; j < 4; ++j)
              if ((vm >> j) & 1u) qo[j] = q4[j];
          }
        }
      }
      if (over) bad = true;
      // carries for the next window: the last slot's segmented value and
      // the start flags seen so far
      __syncthreads();
      if (threadIdx.x == kXThreads - 1) {  // slot 3 is valid whenever a window follows
        s_cv = rel[3];
        s_cb = blk[3] + 1u;
      }
      __syncthreads();
    }
  }
  if (bad) atomicExch(a.err, 1);
}

// Fast path of the LCP-S expand: every field's codes fit 16 bits (block
// corners packed two per word), the reconstruction table fits shared memory,
// and below the first field the block space fits 32 bits.  Per-field
// constants come in the launch parameters.  Windows of kFwin slots, eight
// consecutive slots per thread.  Codes of a pair of fields are formed,
// clamped and checked with 16 x 2 SIMD operations.  Same outputs as
// k_expand.
constexpr int kFper = 8;                      // slots per thread
constexpr int kFwin = kXThreads * kFper;      // slots per window
constexpr int kFrel = kFwin + 4;              // staged words of a window (w <= 32)

template <int D, bool DIV32>
__global__ void __launch_bounds__(kXThreads, 4) k_expand_fast(const ExpandArgs a) {
  constexpr int NP = (D + 1) / 2;  // field pairs
  extern __shared__ __align__(16) float s_lut[];
  __shared__ uint32_t s_c16[kBsTile][4];  // corners, 16 bits each, two per word
  __shared__ uint32_t s_st[kBsTile];      // block starts, relative to the first window
  __shared__ __align__(16) uint8_t s_flag[kFwin];
  __shared__ uint32_t s_rw[kFrel];
  __shared__ unsigned long long s_w64[32];
  __shared__ uint32_t s_w32[32];
  __shared__ uint32_t s_wv[kXThreads / 32], s_wf[kXThreads / 32], s_wb[kXThreads / 32];
  __shared__ uint32_t s_cv, s_cb;
  {
    const uint32_t tot = a.lut_off.off[D];
    for (uint32_t i = threadIdx.x; i < tot; i += kXThreads) s_lut[i] = a.lut[i];
  }
  const uint32_t lp = a.lp;
  const uint32_t pm = (1u << lp) - 1u;
  const uint64_t M = a.M, nb = a.nb, n = a.n;
  const uint32_t cmask = (1u << a.log2_chunk) - 1u;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const bool aligned = (n & 3ull) == 0 && (((uintptr_t)a.out) & 15u) == 0 &&
                       (((uintptr_t)a.qout) & 15u) == 0;
  const unsigned long long *sid64 = reinterpret_cast<const unsigned long long *>(a.sid);
  const unsigned long long *scnt64 = reinterpret_cast<const unsigned long long *>(a.scnt);
  const uint32_t *sid32 = reinterpret_cast<const uint32_t *>(a.sid);
  const uint32_t *scnt32 = reinterpret_cast<const uint32_t *>(a.scnt);
  const BsAgg *agg = reinterpret_cast<const BsAgg *>(a.agg);
  const BsAgg *cagg = agg + ((M + (1ull << a.agg_log2) - 1) >> a.agg_log2);
  bool bad = false;
  __syncthreads();
  for (uint64_t t = blockIdx.x; t < a.tiles; t += gridDim.x) {
    BsAgg base;  // a: id base, b: count carry-in, p: first start
    {
      const uint64_t e0 = t << (10 - a.agg_log2);
      const BsAgg lb = agg[e0], cb = cagg[e0 / kBsChunk];
      base.a = cb.a + lb.a;
      base.b = cb.b + lb.b;
      base.p = cb.p + cb.b * lb.len + lb.p;
    }
    const uint64_t b0 = t * kBsTile + (uint64_t)threadIdx.x * kXPer;
    const int nv = b0 < M ? (int)min((uint64_t)kXPer, M - b0) : 0;  // valid blocks here
    // ---- blocks: ids (64-bit), counts and starts (32-bit, modulo 2^32:
    // exact, since every count and every tile's total is below 2^32) ----
    unsigned long long id[kXPer];
    uint32_t dl[kXPer];
    unsigned long long sa = 0;
    uint32_t sd = 0;
#pragma unroll
    for (int j = 0; j < kXPer; ++j) {
      id[j] = 0ull;
      dl[j] = 0u;
      if (j < nv) {
        id[j] = a.wide ? sid64[b0 + j] : (unsigned long long)sid32[b0 + j];
        const unsigned long long z = a.wide ? scnt64[b0 + j] : (unsigned long long)scnt32[b0 + j];
        dl[j] = (uint32_t)(z >> 1) ^ (0u - (uint32_t)(z & 1u));  // unzigzag, modulo 2^32
      }
      sa += id[j];
      sd += dl[j];
    }
    unsigned long long tot;
    unsigned long long ra = base.a + blk_exscan<kXThreads>(sa, s_w64, tot);
    uint32_t t32;
    uint32_t run = (uint32_t)base.b + blk_exscan32<kXThreads>(sd, s_w32, t32);
    uint32_t cnt[kXPer], cs = 0;
#pragma unroll
    for (int j = 0; j < kXPer; ++j) {
      run += dl[j];
      cnt[j] = run;
      cs += j < nv ? run : 0u;
    }
    uint32_t L;
    uint32_t rs = blk_exscan32<kXThreads>(cs, s_w32, L);
    const uint64_t P0 = base.p < nb ? base.p : nb;
    const uint64_t P1 = base.p + L < nb ? base.p + L : nb;
    const uint64_t W0 = P0 & ~3ull;  // first window start (16-byte stores)
    const uint32_t off0 = (uint32_t)(base.p - W0);
    const uint64_t room64 = nb - P0;  // slots left from the tile's start
    const uint32_t room = room64 < 0xffffffffull ? (uint32_t)room64 : 0xffffffffu;
    const bool last_tile = b0 + kXPer >= M && b0 < M;
#pragma unroll
    for (int j = 0; j < kXPer; ++j) {
      if (j >= nv) continue;
      ra += id[j];
      const uint32_t c = cnt[j];
      if (c == 0u || rs + c < rs || rs + c > room) bad = true;
      if (last_tile && j == nv - 1 && rs + c != room) bad = true;
      s_st[threadIdx.x * kXPer + j] = off0 + rs;
      // per-axis corners: mixed-radix digits of the block id
      uint32_t cor[D];
      uint32_t r32;
      {
        unsigned long long q0;
        if (a.div0_64) {
          q0 = a.bshift[0] == 255u ? ra : (__umul64hi(ra, a.bmagic[0]) >> a.bshift[0]);
        } else {
          const uint32_t r = (uint32_t)ra;
          const unsigned long long x = (unsigned long long)r * (uint32_t)a.bmagic[0];
          const unsigned long long y =
              (unsigned long long)r * (uint32_t)(a.bmagic[0] >> 32) + (x >> 32);
          q0 = a.bshift[0] == 255u ? ra : ((y >> 32) >> a.bshift[0]);
        }
        cor[0] = ((uint32_t)ra - (uint32_t)q0 * a.bn[0]) << lp;
        r32 = (uint32_t)q0;
      }
#pragma unroll
      for (int f = 1; f < D; ++f) {
        uint32_t q;
        if (a.bshift[f] == 255u) {
          q = r32;
        } else if (DIV32) {  // below the first axis the block space is < 2^31
          q = __umulhi(r32, a.bmagic32[f]) >> a.bshift[f];
        } else {
          const unsigned long long x = (unsigned long long)r32 * (uint32_t)a.bmagic[f];
          const unsigned long long y =
              (unsigned long long)r32 * (uint32_t)(a.bmagic[f] >> 32) + (x >> 32);
          q = (uint32_t)((y >> 32) >> a.bshift[f]);
        }
        cor[f] = (r32 - q * a.bn[f]) << lp;
        r32 = q;
      }
      uint32_t pk[4] = {0u, 0u, 0u, 0u};
#pragma unroll
      for (int f = 0; f < D; ++f) pk[f >> 1] |= cor[f] << (16 * (f & 1));
      *reinterpret_cast<uint4 *>(s_c16[threadIdx.x * kXPer + j]) =
          make_uint4(pk[0], pk[1], pk[2], pk[3]);
      rs += c;
    }
    if (threadIdx.x == 0) {
      s_cv = 0u;
      s_cb = 0u;
    }
    // ---- particles of the tile's blocks: slots [P0, P1), relative to W0 ----
    const uint32_t p0r = (uint32_t)(P0 - W0);
    const uint64_t span64 = P1 - W0;
    const uint32_t p1r = span64 < 0xffffffffull ? (uint32_t)span64 : 0xffffffffu;
    const uint32_t w0lo = (uint32_t)W0;
    for (uint32_t wr = 0; wr < p1r; wr += kFwin) {
      reinterpret_cast<uint2 *>(s_flag)[threadIdx.x] = make_uint2(0u, 0u);
      uint32_t rb0 = 0;  // bit offset of the window's first slot in the staged words
      if (!a.rel) {  // stage the window's fixed-width words
        const uint32_t rw = a.rel_w;
        const unsigned long long bit0 = (W0 + wr) * (unsigned long long)rw;
        const unsigned long long wlo = bit0 >> 5;
        rb0 = (uint32_t)(bit0 & 31);
        const uint32_t nw = ((rb0 + (uint32_t)kFwin * rw + 31) >> 5) + 1;
        for (uint32_t i = threadIdx.x; i < nw; i += kXThreads)
          s_rw[i] = wlo + i < a.rel_words ? __ldg(a.rel_pl + wlo + i) : 0u;
      }
      __syncthreads();
#pragma unroll
      for (int j = 0; j < kXPer; ++j) {
        if (j >= nv) continue;
        const uint32_t st = s_st[threadIdx.x * kXPer + j] - wr;
        if (st < (uint32_t)kFwin) s_flag[st] = 1;
      }
      __syncthreads();
      const uint32_t cv_in = s_cv, cb_in = s_cb;
      const uint32_t k0 = wr + (uint32_t)threadIdx.x * kFper;  // relative to W0
      uint32_t vm = 0u;  // valid slots of this thread
#pragma unroll
      for (int j = 0; j < kFper; ++j) vm |= (k0 + j >= p0r && k0 + j < p1r) ? (1u << j) : 0u;
      const bool full = vm == 0xffu;
      const uint2 fl2 = reinterpret_cast<const uint2 *>(s_flag)[threadIdx.x];
      // start flags as bits
      uint32_t fb = 0u;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        fb |= ((fl2.x >> (8 * j)) & 1u) << j;
        fb |= ((fl2.y >> (8 * j)) & 1u) << (j + 4);
      }
      uint32_t x[kFper];
      if (a.rel) {
        const uint32_t *rp = a.rel + W0 + k0;
        if (full) {
          const uint4 v0 = *reinterpret_cast<const uint4 *>(rp);
          const uint4 v1 = *reinterpret_cast<const uint4 *>(rp + 4);
          x[0] = v0.x;
          x[1] = v0.y;
          x[2] = v0.z;
          x[3] = v0.w;
          x[4] = v1.x;
          x[5] = v1.y;
          x[6] = v1.z;
          x[7] = v1.w;
        } else {
#pragma unroll
          for (int j = 0; j < kFper; ++j) x[j] = ((vm >> j) & 1u) ? rp[j] : 0u;
        }
      } else {
        const uint32_t rw = a.rel_w;
        const uint32_t sh = 32u - rw;
        const uint32_t bb = rb0 + (uint32_t)threadIdx.x * kFper * rw;
#pragma unroll
        for (int j = 0; j < kFper; ++j) {
          const uint32_t bit = bb + (uint32_t)j * rw;
          const uint32_t wi = bit >> 5;
          const uint32_t v = __funnelshift_l(s_rw[wi + 1], s_rw[wi], bit & 31);
          x[j] = (rw != 0u && ((vm >> j) & 1u)) ? (v >> sh) : 0u;
        }
      }
      // segment starts: block starts and chunk starts of the relative stream
      uint32_t segs = fb;
#pragma unroll
      for (int j = 0; j < kFper; ++j) segs |= (((w0lo + k0 + j) & cmask) == 0u) ? (1u << j) : 0u;
      // segmented scan of the deltas
      uint32_t tv = 0u;
#pragma unroll
      for (int j = 0; j < kFper; ++j) {
        tv = ((segs >> j) & 1u) ? x[j] : tv + x[j];
        x[j] = tv;
      }
      const uint32_t tf = segs != 0u ? 1u : 0u, tb = __popc(fb);
      uint32_t cvv = tv, cff = tf, ccc = tb;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, cvv, o);
        const uint32_t g = __shfl_up_sync(0xffffffffu, cff, o);
        const uint32_t c = __shfl_up_sync(0xffffffffu, ccc, o);
        if (lane >= o) {
          cvv = cff ? cvv : cvv + y;
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
        const uint32_t sv = s_wv[u];
        wv = s_wf[u] ? sv : wv + sv;
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
      const uint32_t bc0 = ec + wb;  // blocks started before this thread's slots
      // per slot: the block's ordinal within the tile, the relative code
      uint32_t bk[kFper];
      bool over = false;
      {
        const uint32_t first_seg = segs ? (uint32_t)(__ffs(segs) - 1) : 32u;
#pragma unroll
        for (int j = 0; j < kFper; ++j) {
          const uint32_t bj = bc0 + __popc(fb & ((2u << j) - 1u)) - 1u;
          const bool valid = (vm >> j) & 1u;
          over |= valid && bj >= (uint32_t)kBsTile;
          bk[j] = valid && bj < (uint32_t)kBsTile ? bj : 0u;
          x[j] = valid ? ((uint32_t)j < first_seg ? x[j] + inv : x[j]) : 0u;
        }
      }
      float *ob = a.out ? a.out + W0 + k0 : nullptr;
      int32_t *qb = a.qout ? a.qout + W0 + k0 : nullptr;
#pragma unroll
      for (int pr = 0; pr < NP; ++pr) {
        const int f0 = 2 * pr, f1 = 2 * pr + 1;
        const uint32_t qm2 = a.qmax2[pr];  // qmax of both fields, 16 bits each
        uint32_t qc[kFper];
#pragma unroll
        for (int j = 0; j < kFper; ++j) {
          const uint32_t cw = s_c16[bk[j]][pr];
          const uint32_t dg = x[j] >> (f0 * lp);
          uint32_t dd = dg & pm;
          if (f1 < D) dd |= ((dg >> lp) & pm) << 16;
          const uint32_t q2 = cw + dd;  // no carry between halves: each half is below 2^16
          qc[j] = __vminu2(q2, qm2);
          over |= qc[j] != q2;
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int f = f0 + h;
          if (f >= D) continue;
          uint32_t q[kFper];
#pragma unroll
          for (int j = 0; j < kFper; ++j) q[j] = h ? (qc[j] >> 16) : (qc[j] & 0xffffu);
          if (a.out) {
            const uint32_t o0 = a.lut_off.off[f];
            float r[kFper];
#pragma unroll
            for (int j = 0; j < kFper; ++j) r[j] = s_lut[o0 + q[j]];
            float *o = ob + (uint64_t)f * n;
            if (full && aligned) {
              *reinterpret_cast<float4 *>(o) = make_float4(r[0], r[1], r[2], r[3]);
              *reinterpret_cast<float4 *>(o + 4) = make_float4(r[4], r[5], r[6], r[7]);
            } else {
#pragma unroll
              for (int j = 0; j < kFper; ++j)
                if ((vm >> j) & 1u) o[j] = r[j];
            }
          }
          if (a.qout) {
            int32_t *qo = qb + (uint64_t)f * n;
            if (full && aligned) {
              *reinterpret_cast<int4 *>(qo) =
                  make_int4((int32_t)q[0], (int32_t)q[1], (int32_t)q[2], (int32_t)q[3]);
              *reinterpret_cast<int4 *>(qo + 4) =
                  make_int4((int32_t)q[4], (int32_t)q[5], (int32_t)q[6], (int32_t)q[7]);
            } else {
#pragma unroll
              for (int j = 0; j < kFper; ++j)
                if ((vm >> j) & 1u) qo[j] = (int32_t)q[j];
            }
          }
        }
      }
      if (over) bad = true;
      // carries for the next window: the last slot's segmented value and
      // the start flags seen so far
      __syncthreads();
      if (threadIdx.x == kXThreads - 1) {  // its slots are valid whenever a window follows
        s_cv = x[kFper - 1];
        s_cb = bc0 + tb;
      }
      __syncthreads();
    }
  }
  if (bad) atomicExch(a.err, 1);
}

template <int D, bool C16>
static void expand_t(const ExpandArgs &a, bool lut, int sms, cudaStream_t s) {
  const size_t dyn = lut ? sizeof(float) * (size_t)a.lut_off.off[D] : 0;
  auto kern = lut ? k_expand<D, true, C16> : k_expand<D, false, C16>;
  // the largest table, opted in once per process (thread-safe static init)
  static const bool attr =
      cudaFuncSetAttribute(k_expand<D, true, C16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(sizeof(float) * kLutMax)) == cudaSuccess;
  (void)attr;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kXThreads, dyn) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  const uint64_t grid = std::min<uint64_t>(a.tiles, (uint64_t)sms * per_sm);
  note_launch();
  kern<<<(unsigned)grid, kXThreads, dyn, s>>>(a);
}

template <int D, bool DIV32>
static void expand_fast_t(const ExpandArgs &a, int sms, cudaStream_t s) {
  const size_t dyn = sizeof(float) * (size_t)a.lut_off.off[D];
  static const bool attr =
      cudaFuncSetAttribute(k_expand_fast<D, DIV32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(sizeof(float) * kLutMax)) == cudaSuccess;
  (void)attr;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_expand_fast<D, DIV32>, kXThreads,
                                                    dyn) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  const uint64_t grid = std::min<uint64_t>(a.tiles, (uint64_t)sms * per_sm);
  note_launch();
  k_expand_fast<D, DIV32><<<(unsigned)grid, kXThreads, dyn, s>>>(a);
}

// floor(r / bn) for r < 2^63: m = ceil(2^(63+l) / bn), l = ceil(log2 bn), then
// floor(r m / 2^(63+l)) = floor(r / bn) (Granlund-Montgomery, division by
// invariant integers using multiplication, Thm. 4.2); the same constants as
// the decode plan's
static void block_magic(unsigned long long bn, unsigned long long &m, uint32_t &sh) {
  if (bn <= 1) {
    m = 0;
    sh = 255;
    return;
  }
  uint32_t l = 0;
  while ((1ull << l) < bn) ++l;
  const unsigned __int128 num = (unsigned __int128)1 << (63 + l);
  m = (unsigned long long)(num / bn) + ((num % bn) != 0 ? 1ull : 0ull);
  sh = l - 1;
}

template <int D>
static void expand_d(ExpandArgs a, bool lut, int sms, cudaStream_t s) {
  // block corners in 16 bits when every field's codes fit
  bool c16 = true, fast = lut;
  unsigned __int128 space = 1, rest = 1;  // blocks in all, and below the first axis
  for (int f = 0; f < D; ++f) {
    const unsigned long long bn = ((unsigned long long)a.qmax[f] >> a.lp) + 1ull;
    c16 = c16 && a.qmax[f] < 65536u;
    fast = fast && (bn << a.lp) <= 65536ull;  // corner + digit never carries past 16 bits
    a.bn[f] = (uint32_t)bn;
    block_magic(bn, a.bmagic[f], a.bshift[f]);
    a.bmagic32[f] = 0u;
    if (bn > 1 && bn <= 65536ull) {  // ceil(2^(31 + l) / bn) < 2^32
      const unsigned long long num = 1ull << (a.bshift[f] + 32u);  // l = bshift + 1
      a.bmagic32[f] = (uint32_t)(num / bn + ((num % bn) != 0 ? 1ull : 0ull));
    }
    space *= bn;
    if (f > 0) rest *= bn;
  }
  for (int k = 0; k < kMaxD / 2; ++k) {
    const uint32_t lo = 2 * k < D ? a.qmax[2 * k] : 0u, hi = 2 * k + 1 < D ? a.qmax[2 * k + 1] : 0u;
    a.qmax2[k] = (lo & 0xffffu) | (hi << 16);
  }
  a.div0_64 = space > ((unsigned __int128)1 << 32) ? 1 : 0;
  fast = fast && rest <= ((unsigned __int128)1 << 32);
  const bool div32 = rest <= ((unsigned __int128)1 << 31);
  if (fast && div32) expand_fast_t<D, true>(a, sms, s);
  else if (fast) expand_fast_t<D, false>(a, sms, s);
  else if (c16) expand_t<D, true>(a, lut, sms, s);
  else expand_t<D, false>(a, lut, sms, s);
}

void launch_expand(uint32_t d, const ExpandArgs &a, bool lut, int sms, cudaStream_t s) {
  if (a.tiles == 0) return;
  switch (d) {
    case 1: expand_d<1>(a, lut, sms, s); break;
    case 2: expand_d<2>(a, lut, sms, s); break;
    case 3: expand_d<3>(a, lut, sms, s); break;
    case 4: expand_d<4>(a, lut, sms, s); break;
    case 5: expand_d<5>(a, lut, sms, s); break;
    case 6: expand_d<6>(a, lut, sms, s); break;
    case 7: expand_d<7>(a, lut, sms, s); break;
    default: expand_d<8>(a, lut, sms, s); break;
  }
}

// aggregate bases: agg holds one entry per 2^agg_log2 blocks, then one per
// 1024 entries, then one spare
uint64_t block_bases_bytes(uint64_t M, uint32_t agg_log2) {
  const uint64_t ents = (M + (1ull << agg_log2) - 1) >> agg_log2;
  return (ents + (ents + kBsChunk - 1) / kBsChunk + 1) * sizeof(BsAgg);
}

// sums per 1024-block aggregate, when the decode did not produce them
void launch_block_sums(const void *sid, const void *scnt, int wide, uint64_t M, void *agg,
                       cudaStream_t s) {
  if (M == 0) return;
  const uint64_t ents = (M + kBsTile - 1) / kBsTile;
  BsAgg *g = reinterpret_cast<BsAgg *>(agg);
  note_launch();
  if (wide)
    k_bscan_sum<unsigned long long><<<(unsigned)ents, kBsThreads, 0, s>>>(
        reinterpret_cast<const unsigned long long *>(sid),
        reinterpret_cast<const unsigned long long *>(scnt), M, g);
  else
    k_bscan_sum<uint32_t><<<(unsigned)ents, kBsThreads, 0, s>>>(
        reinterpret_cast<const uint32_t *>(sid), reinterpret_cast<const uint32_t *>(scnt), M, g);
}

void launch_block_bases(uint64_t M, uint32_t agg_log2, void *agg, cudaStream_t s) {
  if (M == 0) return;
  const uint64_t ents = (M + (1ull << agg_log2) - 1) >> agg_log2;
  const uint64_t chunks = (ents + kBsChunk - 1) / kBsChunk;
  BsAgg *g = reinterpret_cast<BsAgg *>(agg);
  note_launch();
  k_bscan_chunk<<<(unsigned)chunks, kBsChunk, 0, s>>>(g, (uint32_t)ents, g + ents);
  note_launch();
  k_bscan_top<<<1, 1024, 0, s>>>(g + ents, (uint32_t)chunks);
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
    if (out) out[f * n + nb + j] = x;
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
