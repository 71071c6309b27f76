// k_code.cu -- stream coding and the container.
//
// Sec. "Block coding": every delta-coded array is written with Huffman or
// fixed-length bits, whichever is shorter once the Huffman table is counted
// (Table 3 shows either can win).  Code lengths come from the two-queue
// Huffman construction (leaves ordered by weight then symbol, a leaf taken
// before an internal node of equal weight, internal nodes first-in
// first-out), limited to 24 bits by halving weights; codes are canonical.
// Streams are cut into chunks of 2^log2_chunk symbols whose starting bit
// offsets are stored, so the decoder can work on chunks in parallel.
#include <algorithm>
#include <type_traits>

#include "lcp_kernels.h"

namespace lcp {

// ---------------------------------------------------------------------------
// codebook: one CTA per stream
// ---------------------------------------------------------------------------
constexpr int kCbThreads = 1024;

__device__ void bitonic_sort_u64(unsigned long long *a, int n /*power of two*/) {
  for (int k = 2; k <= n; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        int p = i ^ j;
        if (p > i) {
          bool up = (i & k) == 0;
          unsigned long long x = a[i], y = a[p];
          if ((x > y) == up) {
            a[i] = y;
            a[p] = x;
          }
        }
      }
      __syncthreads();
    }
  }
}

// Code lengths of one stream for one number of halvings k (blockIdx.x):
// weights ceil(count / 2^k) -- k halvings (w + 1) >> 1 -- then the
// two-queue construction and the leaf depths.  All k in [0, kHalvings) are
// built at once; the codebook takes the smallest k whose longest code fits
// kLmax bits, which is where halving one step at a time stops (k = 32 leaves
// all weights equal: depth <= 12).
constexpr int kHalvings = 33;

__global__ void __launch_bounds__(kCbThreads) k_cb_build(const uint32_t *__restrict__ hist,
                                                         const unsigned long long *__restrict__ nv,
                                                         uint8_t *__restrict__ lens_k,
                                                         uint32_t *__restrict__ maxlen_k) {
  const int k = blockIdx.x, s = blockIdx.y;
  extern __shared__ __align__(16) unsigned char cb_smem[];
  unsigned long long *sk = reinterpret_cast<unsigned long long *>(cb_smem);  // weight<<12|sym
  uint32_t *nodew = reinterpret_cast<uint32_t *>(sk + kAlpha);              // leaves, internal
  uint32_t *dist = nodew + 2 * kAlpha;
  uint16_t *parent = reinterpret_cast<uint16_t *>(dist + 2 * kAlpha);
  __shared__ int s_U, s_maxlen;
  uint8_t *lens = lens_k + ((uint64_t)s * kHalvings + k) * kAlpha;
  const unsigned long long n = nv[s];
  const uint32_t *h = hist + (uint64_t)s * kAlpha;
  if (threadIdx.x == 0) {
    s_U = 0;
    s_maxlen = 0;
  }
  __syncthreads();
  // the used symbols' (weight, symbol) keys, gathered in any order (the sort
  // below orders them; the keys are distinct)
  for (int i = threadIdx.x; i < kAlpha; i += blockDim.x) {
    const unsigned long long c = n ? h[i] : 0u;
    const unsigned long long wk = (c + (1ull << k) - 1ull) >> k;
    if (c) sk[atomicAdd(&s_U, 1)] = (wk << 12) | (unsigned long long)i;
  }
  __syncthreads();
  const int U = s_U;
  if (U <= 1) {
    for (int i = threadIdx.x; i < kAlpha; i += blockDim.x) lens[i] = 0;
    __syncthreads();
    if (threadIdx.x == 0) {
      if (U == 1) lens[sk[0] & 4095ull] = 1;
      maxlen_k[s * kHalvings + k] = (uint32_t)U;
    }
    return;
  }
  // k > 0 matters only when some code exceeds kLmax bits, impossible with at
  // most kLmax + 1 symbols (depth <= U - 1)
  if (k > 0 && U <= kLmax + 1) {
    if (threadIdx.x == 0) maxlen_k[s * kHalvings + k] = 0xffffffffu;
    return;
  }
  // sort the next power of two at or above U (padding sorts last)
  int P2 = 2;
  while (P2 < U) P2 <<= 1;
  for (int i = U + threadIdx.x; i < P2; i += blockDim.x) sk[i] = ~0ull;
  __syncthreads();
  bitonic_sort_u64(sk, P2);
  constexpr uint32_t kInf = 0xffffffffu;  // above every weight (U >= 2: each < n < 2^32)
  for (int i = threadIdx.x; i < 2 * U - 1; i += blockDim.x)
    nodew[i] = i < U ? (uint32_t)(sk[i] >> 12) : kInf;  // internal nodes not made yet
  __syncthreads();
  if (threadIdx.x == 0) {
    // leaves nodew[0..U) ascending; internal node j (id U + j) has weight
    // nodew[U + j], created in non-decreasing order.  The heads of both
    // queues and the entries behind them are kept in registers, an empty
    // queue's head reading as kInf, so a pick is one comparison (a leaf on
    // ties); the entry after them is loaded right after a pick and used at
    // the next one, so its latency overlaps that pick.  An internal entry
    // loaded before it is made (kInf) is filled in when its node is made.
    const uint32_t *lw = nodew;
    uint32_t *iw = nodew + U;
    int nl = 0, ni = 0;
    uint32_t L0 = lw[0], L1 = lw[1], pL = U > 2 ? lw[2] : kInf;
    uint32_t I0 = kInf, I1 = kInf, pI = kInf;
    for (int nn = 0; nn < U - 1; ++nn) {
      uint32_t sum = 0u;
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        const bool leaf = L0 <= I0;
        sum += leaf ? L0 : I0;
        parent[leaf ? nl : U + ni] = (uint16_t)(U + nn);
        L0 = leaf ? L1 : L0;
        L1 = leaf ? pL : L1;
        I0 = leaf ? I0 : I1;
        I1 = leaf ? I1 : pI;
        nl += leaf ? 1 : 0;
        ni += leaf ? 0 : 1;
        pL = nl + 2 < U ? lw[nl + 2] : kInf;
        pI = ni + 2 <= U - 2 ? iw[ni + 2] : kInf;
      }
      iw[nn] = sum;
      const int q = nn - ni;  // queue length before this node joins
      I0 = q == 0 ? sum : I0;
      I1 = q == 1 ? sum : I1;
      pI = q == 2 ? sum : pI;  // loaded before this store
    }
    parent[2 * U - 2] = (uint16_t)(2 * U - 2);
  }
  __syncthreads();
  // depths by pointer jumping: distance to the root
  constexpr int kPer = (2 * kAlpha + kCbThreads - 1) / kCbThreads;
  const int nodes = 2 * U - 1;
  uint32_t anc[kPer];
#pragma unroll
  for (int q = 0; q < kPer; ++q) {
    const int i = threadIdx.x + q * kCbThreads;
    if (i < nodes) {
      anc[q] = parent[i];
      dist[i] = (i == nodes - 1) ? 0u : 1u;
    }
  }
  __syncthreads();
  for (int round = 0; round < 14; ++round) {
    uint32_t nd[kPer], na[kPer];
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      const int i = threadIdx.x + q * kCbThreads;
      if (i < nodes) {
        nd[q] = dist[i] + dist[anc[q]];
        na[q] = parent[anc[q]];
      }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      const int i = threadIdx.x + q * kCbThreads;
      if (i < nodes) {
        dist[i] = nd[q];
        anc[q] = na[q];
        parent[i] = (uint16_t)na[q];
      }
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < kAlpha; i += blockDim.x) lens[i] = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < U; i += blockDim.x) {
    const uint32_t sym = (uint32_t)(sk[i] & 4095ull);
    const uint32_t L = dist[i];
    lens[sym] = (uint8_t)(L > 255 ? 255 : L);
    atomicMax(&s_maxlen, (int)L);
  }
  __syncthreads();
  if (threadIdx.x == 0) maxlen_k[s * kHalvings + k] = (uint32_t)s_maxlen;
}

__global__ void __launch_bounds__(kCbThreads) k_codebook(const uint32_t *__restrict__ hist,
                                                         const unsigned long long *__restrict__ maxv,
                                                         const unsigned long long *__restrict__ nv,
                                                         uint32_t log2_chunk,
                                                         const uint8_t *__restrict__ lens_k,
                                                         const uint32_t *__restrict__ maxlen_k,
                                                         StreamDesc *__restrict__ desc,
                                                         uint32_t *__restrict__ codes,
                                                         uint8_t *__restrict__ lens,
                                                         uint16_t *__restrict__ tables) {
  const int s = blockIdx.x;
  __shared__ uint8_t depth8[kAlpha];
  __shared__ uint32_t s_lc[kLmax + 2];
  __shared__ uint32_t s_first[kLmax + 2], s_index[kLmax + 2];
  __shared__ int s_U, s_k;
  __shared__ unsigned long long s_bits;
  const unsigned long long n = nv[s];
  const unsigned long long mx = n ? maxv[s] : 0ull;
  const uint32_t wfix = bitlen64(mx);
  const unsigned long long fixed_bytes = 32ull + pad16(4ull * words_of(n * (unsigned long long)wfix));
  StreamDesc D;
  D.n = n;
  D.maxv = mx;
  D.payload_bits = n * (unsigned long long)wfix;
  D.bytes = fixed_bytes;
  D.offset = 0;
  D.n_chunks = 0;
  D.coder = 0;
  D.width = wfix;
  D.used = 0;
  D.pad = 0;
  const uint32_t *h = hist + (uint64_t)s * kAlpha;
  if (threadIdx.x == 0) {
    s_U = 0;
    s_bits = 0ull;
    int kk = kHalvings - 1;
    for (int q = 0; q < kHalvings; ++q)
      if (maxlen_k[s * kHalvings + q] <= (uint32_t)kLmax) {
        kk = q;
        break;
      }
    s_k = kk;
  }
  __syncthreads();
  const uint8_t *lk = lens_k + ((uint64_t)s * kHalvings + s_k) * kAlpha;
  for (int i = threadIdx.x; i < kAlpha; i += blockDim.x) {
    const bool used = n && h[i];
    depth8[i] = used ? lk[i] : 0;
    if (used) atomicAdd(&s_U, 1);
  }
  __syncthreads();
  const int U = s_U;
  if (U == 0) {
    if (threadIdx.x == 0) desc[s] = D;
    return;
  }
  const uint32_t wesc = (n && h[kEsc]) ? wfix : 0u;
  __syncthreads();
  // canonical codes: per length, symbols in increasing order
  if (threadIdx.x < kLmax + 2) s_lc[threadIdx.x] = 0u;
  __syncthreads();
  for (int i = threadIdx.x; i < kAlpha; i += blockDim.x)
    if (depth8[i]) atomicAdd(&s_lc[depth8[i]], 1u);
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t code = 0, idx = 0;
    for (int L = 1; L <= kLmax; ++L) {
      code = (code + (L > 1 ? s_lc[L - 1] : 0u)) << 1;
      if (L == 1) code = 0;
      s_first[L] = code;
      s_index[L] = idx;
      idx += s_lc[L];
    }
  }
  __syncthreads();
  {
    // ranks among the codes of one length in symbol order: warp w owns
    // symbols 128 w + 32 k + lane (k = 0..3, in that order); lanes of equal
    // length are grouped by __match_any_sync, a warp's running count per
    // length is kept in shared memory, and the warps' counts per length are
    // turned into bases by one thread per length
    constexpr int kW = kCbThreads / 32;
    __shared__ uint32_t s_wl[kW][kLmax + 1];  // per warp, per length: count, then base
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    for (int L = lane; L <= kLmax; L += 32) s_wl[wp][L] = 0u;
    __syncwarp();
    const uint32_t lt = (1u << lane) - 1u;
    uint32_t lrank[kAlpha / kCbThreads];
#pragma unroll
    for (int k = 0; k < kAlpha / kCbThreads; ++k) {
      const int sym = wp * 128 + k * 32 + lane;
      const uint32_t L = depth8[sym];
      const uint32_t m = __match_any_sync(0xffffffffu, L);
      lrank[k] = L ? s_wl[wp][L] + __popc(m & lt) : 0u;
      __syncwarp();
      if (L && (m & lt) == 0u) s_wl[wp][L] += __popc(m);  // the group's first lane
      __syncwarp();
    }
    __syncthreads();
    if (threadIdx.x >= 1 && threadIdx.x <= kLmax) {
      const int L = threadIdx.x;
      uint32_t run = 0u;
      for (int w = 0; w < kW; ++w) {
        const uint32_t c = s_wl[w][L];
        s_wl[w][L] = run;
        run += c;
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kAlpha / kCbThreads; ++k) {
      const int sym = wp * 128 + k * 32 + lane;
      const uint32_t L = depth8[sym];
      if (L) {
        const uint32_t rank = s_wl[wp][L] + lrank[k];
        codes[(uint64_t)s * kAlpha + sym] = s_first[L] + rank;
        tables[(uint64_t)s * (kAlpha + 32) + 32 + s_index[L] + rank] = (uint16_t)sym;
      }
    }
  }
  for (int i = threadIdx.x; i < kAlpha; i += blockDim.x) {
    lens[(uint64_t)s * kAlpha + i] = depth8[i];
    if (!depth8[i]) codes[(uint64_t)s * kAlpha + i] = 0u;
  }
  // payload bits with the original histogram
  {
    unsigned long long local = 0;
    for (int i = threadIdx.x; i < kAlpha; i += blockDim.x)
      local += (unsigned long long)h[i] * depth8[i];
    atomicAdd(&s_bits, local);
  }
  if (threadIdx.x < kLmax) tables[(uint64_t)s * (kAlpha + 32) + threadIdx.x] =
      (uint16_t)s_lc[threadIdx.x + 1];
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long bits = s_bits + (unsigned long long)h[kEsc] * wesc;
    unsigned long long chunks = (n + (1ull << log2_chunk) - 1ull) >> log2_chunk;
    unsigned long long hb =
        pad16(80ull + 2ull * (unsigned long long)U) + pad16(8ull * chunks) + pad16(4ull * words_of(bits));
    if (hb < fixed_bytes) {
      D.coder = 1;
      D.width = wesc;
      D.used = (uint32_t)U;
      D.payload_bits = bits;
      D.n_chunks = chunks;
      D.bytes = hb;
    }
    desc[s] = D;
  }
}

size_t codebook_work_size(int ns) { return (size_t)ns * kHalvings * (kAlpha + 4); }

void launch_codebook(int ns, const uint32_t *hist, const unsigned long long *maxv,
                     const unsigned long long *n_vals, uint32_t log2_chunk, uint8_t *work,
                     StreamDesc *desc, uint32_t *codes, uint8_t *lens, uint16_t *tables,
                     cudaStream_t s) {
  // sort keys, node weights, distances, parents
  const size_t smem = 8ull * kAlpha + 4ull * 2 * kAlpha + 4ull * 2 * kAlpha + 2ull * 2 * kAlpha;
  // once per process; thread-safe (function-local static initialization)
  static const bool attr =
      cudaFuncSetAttribute(k_cb_build, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) ==
      cudaSuccess;
  (void)attr;
  uint8_t *lens_k = work;
  uint32_t *maxlen_k = reinterpret_cast<uint32_t *>(work + (size_t)ns * kHalvings * kAlpha);
  note_launch();
  k_cb_build<<<dim3(kHalvings, ns), kCbThreads, smem, s>>>(hist, n_vals, lens_k, maxlen_k);
  note_launch();
  k_codebook<<<ns, kCbThreads, 0, s>>>(hist, maxv, n_vals, log2_chunk, lens_k, maxlen_k, desc,
                                       codes, lens, tables);
}

// ---------------------------------------------------------------------------
// layout: offsets, total size, header, stream headers and tables
// ---------------------------------------------------------------------------
__device__ __forceinline__ void st_u8(uint8_t *p, uint32_t v) { p[0] = (uint8_t)v; }
__device__ __forceinline__ void st_u16(uint8_t *p, uint32_t v) {
  p[0] = (uint8_t)v;
  p[1] = (uint8_t)(v >> 8);
}
__device__ __forceinline__ void st_u32(uint8_t *p, uint32_t v) {
  *reinterpret_cast<uint32_t *>(p) = v;  // 4-aligned by construction
}
__device__ __forceinline__ void st_u64(uint8_t *p, unsigned long long v) {
  *reinterpret_cast<uint32_t *>(p) = (uint32_t)v;
  *reinterpret_cast<uint32_t *>(p + 4) = (uint32_t)(v >> 32);
}

__global__ void k_layout_size(LayoutArgs a) {
  if (threadIdx.x != 0) return;
  Summary S;
  S.pad = 0;
  S.status = a.plan->status;
  S.M = a.method == 0 ? *a.mcount : 0ull;
  S.K = *a.kcount;
  S.total = 0;
  if (S.status == OK) {
    const int ns = a.method == 0 ? 3 : 1;
    unsigned long long off = 48ull + 16ull * a.d + 16ull * ns + 16ull;
    for (int k = 0; k < ns; ++k) {
      a.desc[k].offset = off;
      off += a.desc[k].bytes;
    }
    unsigned long long ob = a.method == 0 ? pad16(4ull * a.d * S.K) : pad16(8ull * S.K) + pad16(4ull * S.K);
    a.desc[ns].offset = off;  // outlier section
    a.desc[ns].bytes = ob;
    off += ob;
    S.total = off;
    if (off > a.cap) S.status = ERR_CAPACITY;
  }
  *a.summary = S;
}

__global__ void k_zero(uint8_t *out, const Summary *summary) {
  if (summary->status != OK) return;
  const unsigned long long total = summary->total;  // multiple of 16
  uint4 *o = reinterpret_cast<uint4 *>(out);
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
       i < total / 16; i += (unsigned long long)gridDim.x * blockDim.x)
    o[i] = make_uint4(0, 0, 0, 0);
}

__global__ void k_layout_write(LayoutArgs a) {
  const Summary S = *a.summary;
  if (S.status != OK) return;
  const int ns = a.method == 0 ? 3 : 1;
  uint8_t *o = a.out;
  if (threadIdx.x == 0) {
    o[0] = 'L';
    o[1] = 'C';
    o[2] = 'P';
    o[3] = '1';
    o[4] = 1;
    o[5] = (uint8_t)a.method;
    o[6] = (uint8_t)a.d;
    o[7] = (uint8_t)a.log2_chunk;
    st_u32(o + 8, a.flags);
    st_u32(o + 12, a.method == 0 ? a.p : 0u);
    st_u64(o + 16, a.n);
    st_u64(o + 24, S.K);
    st_u64(o + 32, S.M);
    st_u64(o + 40, S.total);
    for (uint32_t f = 0; f < a.d; ++f) {
      uint8_t *fp = o + 48 + 16 * f;
      st_u32(fp, __float_as_uint(a.plan->f[f].m));
      st_u32(fp + 4, __float_as_uint(a.plan->f[f].e));
      st_u32(fp + 8, a.plan->f[f].qmax);
      st_u32(fp + 12, 0u);
    }
    uint8_t *sd = o + 48 + 16 * a.d;
    for (int k = 0; k <= ns; ++k) {
      st_u64(sd + 16 * k, a.desc[k].offset);
      st_u64(sd + 16 * k + 8, a.desc[k].bytes);
    }
    for (int k = 0; k < ns; ++k) {
      const StreamDesc &D = a.desc[k];
      uint8_t *sp = o + D.offset;
      st_u8(sp, D.coder);
      st_u8(sp + 1, D.width);
      st_u16(sp + 2, D.used);
      st_u32(sp + 4, 0u);
      st_u64(sp + 8, D.n);
      st_u64(sp + 16, D.payload_bits);
      st_u64(sp + 24, D.maxv);
    }
  }
  // Huffman tables: counts per length then symbols by (length, symbol)
  for (int k = 0; k < ns; ++k) {
    const StreamDesc &D = a.desc[k];
    if (D.coder != 1) continue;
    uint8_t *sp = o + D.offset;
    const uint16_t *t = a.tables + (uint64_t)k * (kAlpha + 32);
    for (int i = threadIdx.x; i < kLmax; i += blockDim.x) st_u16(sp + 32 + 2 * i, t[i]);
    for (uint32_t i = threadIdx.x; i < D.used; i += blockDim.x) st_u16(sp + 80 + 2 * i, t[32 + i]);
  }
}

void launch_layout(const LayoutArgs &a, int sms, bool size_only, cudaStream_t s) {
  note_launch();
  k_layout_size<<<1, 32, 0, s>>>(a);
  if (size_only) return;
  note_launch();
  k_zero<<<2 * sms, 512, 0, s>>>(a.out, a.summary);
  note_launch();
  k_layout_write<<<1, 256, 0, s>>>(a);
}

// ---------------------------------------------------------------------------
// fixed-length payload, groups of 32 consecutive values (32 * w bits, w whole
// words).  Widths up to 32: lane k assembles word k of the group from the
// values it overlaps, fetched by shuffles, and the w words go out in one
// coalesced store.  Wider values (8-byte streams): the lanes OR their bits
// into a shared-memory stage.
// ---------------------------------------------------------------------------
constexpr int kFixWarps = 8;
constexpr int kFixGroups = 8;  // groups per warp iteration (their loads issued together)

template <typename T>
__global__ void __launch_bounds__(32 * kFixWarps) k_encode_fixed(
    const T *__restrict__ vals, const StreamDesc *__restrict__ dp, uint8_t *__restrict__ out,
    const Summary *__restrict__ summary) {
  __shared__ uint32_t stage[kFixWarps][64];
  if (summary->status != OK) return;
  const StreamDesc D = *dp;
  if (D.coder != 0 || D.width == 0 || D.n == 0) return;
  const uint32_t w = D.width;
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  uint32_t *buf = stage[wl];
  uint32_t *pl = reinterpret_cast<uint32_t *>(out + D.offset + 32);
  const unsigned long long words = words_of(D.payload_bits);
  const unsigned long long groups = (D.n + 31) >> 5;
  const unsigned long long nw = (unsigned long long)gridDim.x * kFixWarps;
  // word `lane` of a group spans bits [32 lane, 32 lane + 32): values
  // i_lo = floor(32 lane / w) onwards, value i shifted left by
  // sh = 32 lane + 64 - (i + 1) w within a 64-bit accumulator whose high word
  // is the output (bits of neighbouring words fall off either end)
  const uint32_t i_lo = w <= 32u ? (32u * (uint32_t)lane) / w : 0u;
  const int nj = w <= 32u ? (int)((32u + w - 1u) / w) + 1 : 0;  // values a word can touch
  // for w >= 8 (at most kFixJ values per word) the high word of each shifted
  // value is (x << L) >> R with (L, R) = (sh - 32, 0) or (0, 32 - sh); the
  // sources, shifts and validity depend only on the lane and are set once
  constexpr int kFixJ = 5;
  uint32_t src[kFixJ], shl[kFixJ], shr[kFixJ], jm = 0u;
#pragma unroll
  for (int j = 0; j < kFixJ; ++j) {
    const uint32_t i = i_lo + (uint32_t)j;
    const int sh = 32 * lane + 64 - (int)((i + 1u) * w);
    const bool ok = w >= 8u && j < nj && i < 32u && (int)(i * w) < 32 * lane + 32 && sh < 64;
    src[j] = i & 31u;
    shl[j] = ok && sh >= 32 ? (uint32_t)(sh - 32) : 0u;
    shr[j] = ok && sh < 32 ? (uint32_t)(32 - sh) : 0u;
    jm |= ok ? (1u << j) : 0u;
  }
  if constexpr (std::is_same<T, uint32_t>::value) {
    if (w >= 8u && w <= 32u) {
      // 4-byte values: a warp stages 1024 of them (32 groups) with 16-byte
      // loads, all in flight together, then assembles each group's words from
      // the staged values (the sources and shifts above, read from shared
      // memory instead of shuffled)
      __shared__ __align__(16) uint32_t st32[kFixWarps][1024];
      uint32_t *sv = st32[wl];
      const unsigned long long supers = (D.n + 1023) >> 10;
      const unsigned long long nsw = (unsigned long long)gridDim.x * kFixWarps;
      const bool vec = (((uintptr_t)vals) & 15u) == 0;
      for (unsigned long long sg = (unsigned long long)blockIdx.x * kFixWarps + wl; sg < supers;
           sg += nsw) {
        const unsigned long long base = sg << 10;
        uint4 r[8];
#pragma unroll
        for (int a = 0; a < 8; ++a) {
          const unsigned long long i = base + (unsigned long long)a * 128 + 4ull * lane;
          if (vec && i + 4 <= D.n) {
            r[a] = *reinterpret_cast<const uint4 *>(vals + i);
          } else {
            r[a].x = i < D.n ? (uint32_t)vals[i] : 0u;
            r[a].y = i + 1 < D.n ? (uint32_t)vals[i + 1] : 0u;
            r[a].z = i + 2 < D.n ? (uint32_t)vals[i + 2] : 0u;
            r[a].w = i + 3 < D.n ? (uint32_t)vals[i + 3] : 0u;
          }
        }
#pragma unroll
        for (int a = 0; a < 8; ++a) reinterpret_cast<uint4 *>(sv)[a * 32 + lane] = r[a];
        __syncwarp();
        const unsigned long long g_first = base >> 5;
        const uint32_t ng = (uint32_t)min(32ull, groups - g_first);
        for (uint32_t gq = 0; gq < ng; ++gq) {
          const uint32_t *gv = sv + gq * 32;
          uint32_t word = 0u;
#pragma unroll
          for (int j = 0; j < kFixJ; ++j)
            if ((jm >> j) & 1u) word |= (gv[src[j]] << shl[j]) >> shr[j];
          const unsigned long long wb = (g_first + gq) * (unsigned long long)w;
          if ((uint32_t)lane < w && wb + lane < words) pl[wb + lane] = word;
        }
        __syncwarp();
      }
      return;
    }
  }
  for (unsigned long long g0 = ((unsigned long long)blockIdx.x * kFixWarps + wl) * kFixGroups;
       g0 < groups; g0 += nw * kFixGroups) {
    unsigned long long v[kFixGroups];
#pragma unroll
    for (int q = 0; q < kFixGroups; ++q) {
      const unsigned long long i = (g0 + q) * 32ull + lane;
      v[q] = i < D.n ? (unsigned long long)vals[i] : 0ull;
    }
#pragma unroll
    for (int q = 0; q < kFixGroups; ++q) {
      const unsigned long long g = g0 + q;
      if (g >= groups) break;
      const unsigned long long wbase = g * (unsigned long long)w;
      if (w >= 8u && w <= 32u) {
        const uint32_t x32 = (uint32_t)v[q];
        uint32_t word = 0u;
#pragma unroll
        for (int j = 0; j < kFixJ; ++j) {
          const uint32_t x = __shfl_sync(0xffffffffu, x32, (int)src[j]);
          word |= ((jm >> j) & 1u) ? ((x << shl[j]) >> shr[j]) : 0u;
        }
        if ((uint32_t)lane < w && wbase + lane < words) pl[wbase + lane] = word;
      } else if (w <= 32u) {
        const uint32_t x32 = (uint32_t)v[q];
        unsigned long long acc = 0ull;
        for (int j = 0; j < nj; ++j) {
          const uint32_t i = i_lo + (uint32_t)j;
          const uint32_t x = __shfl_sync(0xffffffffu, x32, (int)(i & 31u));
          const int sh = 32 * lane + 64 - (int)((i + 1u) * w);
          if (i < 32u && (int)(i * w) < 32 * lane + 32 && sh < 64)
            acc |= (unsigned long long)x << sh;
        }
        if ((uint32_t)lane < w && wbase + lane < words) pl[wbase + lane] = (uint32_t)(acc >> 32);
      } else {
        buf[lane] = 0u;
        buf[lane + 32] = 0u;
        __syncwarp();
        const unsigned long long i = g * 32ull + lane;
        if (i < D.n) {
          // bits [lane*w, lane*w + w) of the group, MSB first
          uint32_t left = w, pos = (uint32_t)lane * w;
          while (left) {
            const uint32_t wi = pos >> 5, off = pos & 31u;
            const uint32_t take = min(left, 32u - off);
            const unsigned long long part = (v[q] >> (left - take)) & ((1ull << take) - 1ull);
            atomicOr(&buf[wi], (uint32_t)part << (32u - off - take));
            pos += take;
            left -= take;
          }
        }
        __syncwarp();
        for (uint32_t k = lane; k < w; k += 32)
          if (wbase + k < words) pl[wbase + k] = buf[k];
        __syncwarp();
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Huffman payload: per-chunk bit counts, their scan (the chunk table), then
// one warp per chunk, each lane a run of consecutive symbols, the chunk's
// words assembled in a shared-memory stage
// ---------------------------------------------------------------------------
constexpr int kEncWarps = 8;
constexpr int kStageWords = 2848;  // >= (1024 * (24 + 64)) / 32 + 2
constexpr size_t kEncSmem = sizeof(uint32_t) * ((size_t)kEncWarps * kStageWords + kAlpha);
// a warp's stage for chunks of 2^log2_chunk symbols (at most 24 + 64 bits each)
__host__ __device__ constexpr uint32_t enc_stage_words(uint32_t log2_chunk) {
  return (uint32_t)((((1ull << log2_chunk) * (kLmax + 64)) + 31) / 32 + 2);
}
static_assert(enc_stage_words(10) <= (uint32_t)kStageWords, "stage of the largest chunks");

// code table of the stream in shared memory: (code << 5) | length
__device__ __forceinline__ void load_code_table(uint32_t *t, const uint32_t *codes,
                                                const uint8_t *lens) {
  for (int k = threadIdx.x; k < kAlpha; k += blockDim.x)
    t[k] = (codes[k] << 5) | (uint32_t)lens[k];
}

template <typename T>
__global__ void __launch_bounds__(256) k_chunk_bits(const T *__restrict__ vals,
                                                    const StreamDesc *__restrict__ dp,
                                                    const uint32_t *__restrict__ codes,
                                                    const uint8_t *__restrict__ lens,
                                                    uint32_t log2_chunk,
                                                    unsigned long long *__restrict__ chunk_bits,
                                                    const Summary *__restrict__ summary) {
  __shared__ uint32_t tab[kAlpha];
  if (summary->status != OK) return;
  const StreamDesc D = *dp;
  if (D.coder != 1) return;
  load_code_table(tab, codes, lens);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const unsigned long long warp = ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const unsigned long long nw = ((unsigned long long)gridDim.x * blockDim.x) >> 5;
  const unsigned long long cs = 1ull << log2_chunk;
  for (unsigned long long c = warp; c < D.n_chunks; c += nw) {
    const unsigned long long lo = c * cs, hi = min(D.n, lo + cs);
    unsigned long long bits = 0;
    for (unsigned long long i0 = lo + lane; i0 < hi; i0 += 32 * 8) {
      unsigned long long v[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const unsigned long long i = i0 + 32ull * q;
        v[q] = i < hi ? (unsigned long long)vals[i] : 0ull;
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        if (i0 + 32ull * q >= hi) continue;
        const uint32_t sym = v[q] < (unsigned long long)kEsc ? (uint32_t)v[q] : (uint32_t)kEsc;
        bits += (tab[sym] & 31u) + (sym == kEsc ? D.width : 0u);
      }
    }
    for (int o = 16; o; o >>= 1) bits += __shfl_down_sync(0xffffffffu, bits, o);
    if (lane == 0) chunk_bits[c] = bits;
  }
}

__global__ void k_chunk_table(const unsigned long long *__restrict__ chunk_off,
                              const StreamDesc *__restrict__ dp, uint8_t *__restrict__ out,
                              const Summary *__restrict__ summary) {
  if (summary->status != OK) return;
  const StreamDesc D = *dp;
  if (D.coder != 1) return;
  uint8_t *ct = out + D.offset + pad16(80ull + 2ull * D.used);
  for (unsigned long long c = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
       c < D.n_chunks; c += (unsigned long long)gridDim.x * blockDim.x)
    st_u64(ct + 8 * c, chunk_off[c]);
}

// Rounds of 128 consecutive symbols of the chunk, four per lane (loaded
// together, so a warp's loads stay contiguous): the lane's bit count, a warp
// scan for its start, then its codes shifted through a 64-bit accumulator
// whose full words go to the warp's stage.  A lane's first and last words
// may be shared with its neighbours and are ORed in; the words between are
// the lane's alone.
constexpr int kEncPer = 4;

template <typename T>
__device__ __forceinline__ void enc_load4(const T *vals, unsigned long long i,
                                          unsigned long long hi, unsigned long long (&v)[kEncPer]);
template <>
__device__ __forceinline__ void enc_load4<unsigned long long>(const unsigned long long *vals,
                                                              unsigned long long i,
                                                              unsigned long long hi,
                                                              unsigned long long (&v)[kEncPer]) {
  if (i + kEncPer <= hi) {
    const ulonglong2 a = *reinterpret_cast<const ulonglong2 *>(vals + i);
    const ulonglong2 b = *reinterpret_cast<const ulonglong2 *>(vals + i + 2);
    v[0] = a.x;
    v[1] = a.y;
    v[2] = b.x;
    v[3] = b.y;
  } else {
#pragma unroll
    for (int j = 0; j < kEncPer; ++j) v[j] = i + j < hi ? vals[i + j] : 0ull;
  }
}
template <>
__device__ __forceinline__ void enc_load4<uint32_t>(const uint32_t *vals, unsigned long long i,
                                                    unsigned long long hi,
                                                    unsigned long long (&v)[kEncPer]) {
  if (i + kEncPer <= hi) {
    const uint4 a = *reinterpret_cast<const uint4 *>(vals + i);
    v[0] = a.x;
    v[1] = a.y;
    v[2] = a.z;
    v[3] = a.w;
  } else {
#pragma unroll
    for (int j = 0; j < kEncPer; ++j) v[j] = i + j < hi ? vals[i + j] : 0ull;
  }
}

template <typename T>
__global__ void __launch_bounds__(32 * kEncWarps) k_huff_encode(
    const T *__restrict__ vals, const StreamDesc *__restrict__ dp,
    const uint32_t *__restrict__ codes, const uint8_t *__restrict__ lens, uint32_t log2_chunk,
    const unsigned long long *__restrict__ chunk_off, uint8_t *__restrict__ out,
    const Summary *__restrict__ summary) {
  extern __shared__ uint32_t enc_smem[];  // per-warp stages, then the code table
  const uint32_t stage_words = enc_stage_words(log2_chunk);
  uint32_t *tab = enc_smem + (size_t)kEncWarps * stage_words;
  if (summary->status != OK) return;
  const StreamDesc D = *dp;
  if (D.coder != 1) return;
  load_code_table(tab, codes, lens);
  __syncthreads();
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  const unsigned long long cs = 1ull << log2_chunk;
  const uint32_t width = D.width;
  uint32_t *buf = enc_smem + (size_t)wl * stage_words;
  uint32_t *pl = reinterpret_cast<uint32_t *>(out + D.offset + pad16(80ull + 2ull * D.used) +
                                              pad16(8ull * D.n_chunks));
  const unsigned long long total_words = words_of(D.payload_bits);
  const unsigned long long warp = (unsigned long long)blockIdx.x * kEncWarps + wl;
  const unsigned long long nw = (unsigned long long)gridDim.x * kEncWarps;
  for (unsigned long long c = warp; c < D.n_chunks; c += nw) {
    const unsigned long long lo = c * cs, hi = min(D.n, lo + cs);
    const unsigned long long start = chunk_off[c];
    const unsigned long long end = (c + 1 < D.n_chunks) ? chunk_off[c + 1] : D.payload_bits;
    const unsigned long long w0 = start >> 5, w1 = (end + 31) >> 5;  // [w0, w1)
    const uint32_t nwords = (uint32_t)(w1 - w0);
    if (nwords > stage_words || w1 > total_words) continue;  // cannot happen
    for (uint32_t i = lane; i < nwords; i += 32) buf[i] = 0u;
    __syncwarp();
    uint32_t base = (uint32_t)(start & 31ull);  // bit position relative to word w0
    unsigned long long vn[kEncPer];  // the next round's values, loaded a round ahead
    enc_load4<T>(vals, lo + (unsigned long long)lane * kEncPer, hi, vn);
    for (unsigned long long b0 = lo; b0 < hi; b0 += 32 * kEncPer) {
      const unsigned long long i0 = b0 + (unsigned long long)lane * kEncPer;
      unsigned long long v[kEncPer];
#pragma unroll
      for (int j = 0; j < kEncPer; ++j) v[j] = vn[j];
      if (b0 + 32 * kEncPer < hi) enc_load4<T>(vals, i0 + 32 * kEncPer, hi, vn);
      uint32_t e[kEncPer], bits = 0u, em = 0u;  // em: escapes with raw bits
#pragma unroll
      for (int j = 0; j < kEncPer; ++j) {
        const bool on = i0 + j < hi;
        const uint32_t sym = v[j] < (unsigned long long)kEsc ? (uint32_t)v[j] : (uint32_t)kEsc;
        e[j] = on ? tab[sym] : 0u;
        const bool esc = on && sym == (uint32_t)kEsc && width;
        em |= esc ? (1u << j) : 0u;
        bits += (e[j] & 31u) + (esc ? width : 0u);
      }
      uint32_t x = bits;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      const uint32_t pos0 = base + x - bits;
      base += __shfl_sync(0xffffffffu, x, 31);
      if (bits == 0u) continue;
      uint32_t wp = pos0 >> 5, nacc = pos0 & 31u;  // next word; bits held (the
      unsigned long long acc = 0ull;                 // first nacc are a neighbour's)
      bool first = true;
      auto emit = [&](uint32_t word) {
        if (first) {
          if (word) atomicOr(&buf[wp], word);
          first = false;
        } else {
          buf[wp] = word;
        }
        ++wp;
      };
#pragma unroll
      for (int j = 0; j < kEncPer; ++j) {
        const uint32_t L = e[j] & 31u;
        acc = (acc << L) | (unsigned long long)(e[j] >> 5);
        nacc += L;  // < 56
        if (nacc >= 32u) {
          nacc -= 32u;
          emit((uint32_t)(acc >> nacc));
        }
        if ((em >> j) & 1u) {
          const unsigned long long w = v[j];  // the raw value, MSB first
          if (width > 32u) {
            const uint32_t hw = width - 32u;
            acc = (acc << hw) | ((w >> 32) & ((1ull << hw) - 1ull));
            nacc += hw;
            if (nacc >= 32u) {
              nacc -= 32u;
              emit((uint32_t)(acc >> nacc));
            }
            acc = (acc << 32) | (w & 0xffffffffull);
            nacc += 32u;
          } else {
            acc = (acc << width) | (w & ((1ull << width) - 1ull));
            nacc += width;
          }
          if (nacc >= 32u) {
            nacc -= 32u;
            emit((uint32_t)(acc >> nacc));
          }
        }
      }
      if (nacc) {  // the last partial word, shared with the next lane
        const uint32_t word = (uint32_t)(acc << (32u - nacc));
        if (word) atomicOr(&buf[wp], word);
      }
    }
    __syncwarp();
    for (uint32_t i = lane; i < nwords; i += 32) {
      const uint32_t word = buf[i];
      if (i == 0 || i + 1 == nwords) {
        if (word) atomicOr(&pl[w0 + i], word);
      } else {
        pl[w0 + i] = word;
      }
    }
    __syncwarp();
  }
}

template <typename T>
static void encode_stream(const T *vals, uint64_t n, const StreamDesc *desc, const uint32_t *codes,
                          const uint8_t *lens, uint32_t log2_chunk, uint8_t *out,
                          const Summary *summary, unsigned long long *chunk_bits,
                          unsigned long long *chunk_off, int sms, cudaStream_t s) {
  // fixed-length (no-op unless chosen)
  const unsigned long long groups = (n + 31ull) / 32ull;
  const unsigned long long units = (groups + kFixGroups - 1) / kFixGroups;
  unsigned g = (unsigned)std::min<unsigned long long>((units + kFixWarps - 1) / kFixWarps,
                                                      8ull * sms);
  if (g == 0) g = 1;
  note_launch();
  k_encode_fixed<T><<<g, 32 * kFixWarps, 0, s>>>(vals, desc, out, summary);
  // Huffman (no-op unless chosen)
  unsigned long long chunks = (n + (1ull << log2_chunk) - 1ull) >> log2_chunk;
  if (chunks == 0) return;
  unsigned gc = (unsigned)std::min<unsigned long long>((chunks * 32 + 255) / 256, 16ull * sms);
  note_launch();
  k_chunk_bits<T><<<gc, 256, 0, s>>>(vals, desc, codes, lens, log2_chunk, chunk_bits, summary);
  // chunk_bits holds scan_tmp_len(chunks) spare entries after the counts
  launch_scan_small(chunk_bits, (uint32_t)chunks, chunk_off, s, &desc->coder,
                    chunk_bits + chunks);
  unsigned gt = (unsigned)std::min<unsigned long long>((chunks + 255) / 256, 4ull * sms);
  note_launch();
  k_chunk_table<<<gt, 256, 0, s>>>(chunk_off, desc, out, summary);
  static const bool attr =  // once per instantiation, thread-safe
      cudaFuncSetAttribute(k_huff_encode<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)kEncSmem) == cudaSuccess;
  (void)attr;
  // stages sized for this chunk size: more CTAs fit an SM for small chunks
  const size_t esmem =
      sizeof(uint32_t) * ((size_t)kEncWarps * enc_stage_words(log2_chunk) + kAlpha);
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_huff_encode<T>, 32 * kEncWarps,
                                                    esmem) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  unsigned ge = (unsigned)std::min<unsigned long long>((chunks + kEncWarps - 1) / kEncWarps,
                                                       (unsigned long long)per_sm * sms);
  note_launch();
  k_huff_encode<T><<<ge, 32 * kEncWarps, esmem, s>>>(vals, desc, codes, lens, log2_chunk,
                                                     chunk_off, out, summary);
}

void launch_encode_u64(const unsigned long long *vals, uint64_t n, const StreamDesc *desc,
                       const uint32_t *codes, const uint8_t *lens, uint32_t log2_chunk,
                       uint8_t *out, const Summary *summary, unsigned long long *chunk_bits,
                       unsigned long long *chunk_off, int sms, cudaStream_t s) {
  encode_stream<unsigned long long>(vals, n, desc, codes, lens, log2_chunk, out, summary,
                                    chunk_bits, chunk_off, sms, s);
}
void launch_encode_u32(const uint32_t *vals, uint64_t n, const StreamDesc *desc,
                       const uint32_t *codes, const uint8_t *lens, uint32_t log2_chunk,
                       uint8_t *out, const Summary *summary, unsigned long long *chunk_bits,
                       unsigned long long *chunk_off, int sms, cudaStream_t s) {
  encode_stream<uint32_t>(vals, n, desc, codes, lens, log2_chunk, out, summary, chunk_bits,
                          chunk_off, sms, s);
}

// ---------------------------------------------------------------------------
// outliers of an LCP-S frame: raw values, field-major, ascending input index
// ---------------------------------------------------------------------------
__global__ void k_outliers_s(const float *__restrict__ fields, uint64_t n, uint32_t d,
                             const uint32_t *__restrict__ outl_idx,
                             const StreamDesc *__restrict__ od, uint8_t *__restrict__ out,
                             const Summary *__restrict__ summary) {
  const Summary S = *summary;
  if (S.status != OK || S.K == 0) return;
  float *o = reinterpret_cast<float *>(out + od->offset);
  for (unsigned long long t = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
       t < S.K * d; t += (unsigned long long)gridDim.x * blockDim.x) {
    unsigned long long f = t / S.K, j = t % S.K;
    o[f * S.K + j] = fields[f * n + outl_idx[j]];
  }
}

void launch_outliers_s(const float *fields, uint64_t n, uint32_t d, const uint32_t *outl_idx,
                       const StreamDesc *desc_outl, uint8_t *out, const Summary *summary,
                       int sms, cudaStream_t s) {
  note_launch();
  k_outliers_s<<<2 * sms, 256, 0, s>>>(fields, n, d, outl_idx, desc_outl, out, summary);
}

}  // namespace lcp
