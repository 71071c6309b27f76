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

__global__ void __launch_bounds__(kCbThreads) k_codebook(const uint32_t *__restrict__ hist,
                                                         const unsigned long long *__restrict__ maxv,
                                                         const unsigned long long *__restrict__ nv,
                                                         uint32_t log2_chunk,
                                                         StreamDesc *__restrict__ desc,
                                                         uint32_t *__restrict__ codes,
                                                         uint8_t *__restrict__ lens,
                                                         uint16_t *__restrict__ tables) {
  const int s = blockIdx.x;
  extern __shared__ __align__(16) unsigned char cb_smem[];
  unsigned long long *sk = reinterpret_cast<unsigned long long *>(cb_smem);  // weight<<12|sym
  uint32_t *w = reinterpret_cast<uint32_t *>(sk + kAlpha);         // weights per symbol
  uint32_t *nodew = w + kAlpha;                                    // leaves then internal
  uint16_t *parent = reinterpret_cast<uint16_t *>(nodew + 2 * kAlpha);
  uint8_t *depth8 = reinterpret_cast<uint8_t *>(parent + 2 * kAlpha);  // code lengths
  __shared__ uint32_t s_lc[kLmax + 2];
  __shared__ uint32_t s_first[kLmax + 2], s_index[kLmax + 2];
  __shared__ int s_U, s_maxlen;
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
  }
  for (int i = threadIdx.x; i < kAlpha; i += blockDim.x) {
    w[i] = n ? h[i] : 0u;
    depth8[i] = 0;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kAlpha; i += blockDim.x)
    if (w[i]) atomicAdd(&s_U, 1);
  __syncthreads();
  const int U = s_U;
  if (U == 0) {
    if (threadIdx.x == 0) desc[s] = D;
    return;
  }
  const uint32_t wesc = w[kEsc] ? wfix : 0u;
  if (U == 1) {
    for (int i = threadIdx.x; i < kAlpha; i += blockDim.x)
      if (w[i]) depth8[i] = 1;
  } else {
    for (;;) {
      for (int i = threadIdx.x; i < kAlpha; i += blockDim.x)
        sk[i] = w[i] ? (((unsigned long long)w[i] << 12) | (unsigned long long)i) : ~0ull;
      __syncthreads();
      bitonic_sort_u64(sk, kAlpha);
      for (int i = threadIdx.x; i < U; i += blockDim.x) nodew[i] = (uint32_t)(sk[i] >> 12);
      __syncthreads();
      if (threadIdx.x == 0) {
        // two-queue merge: leaves nodew[0..U), internal nodes nodew[U..2U-1)
        int nl = 0, ni = U, nn = U;
        while (nn < 2 * U - 1) {
          int pick[2];
#pragma unroll
          for (int t = 0; t < 2; ++t) {
            if (nl < U && (ni == nn || nodew[nl] <= nodew[ni])) pick[t] = nl++;
            else pick[t] = ni++;
          }
          nodew[nn] = nodew[pick[0]] + nodew[pick[1]];
          parent[pick[0]] = (uint16_t)nn;
          parent[pick[1]] = (uint16_t)nn;
          ++nn;
        }
        parent[2 * U - 2] = (uint16_t)(2 * U - 2);
      }
      __syncthreads();
      // depths by pointer jumping: dist to the root
      constexpr int kPer = (2 * kAlpha + kCbThreads - 1) / kCbThreads;
      uint32_t dist[kPer], anc[kPer];
      const int nodes = 2 * U - 1;
#pragma unroll
      for (int k = 0; k < kPer; ++k) {
        int i = threadIdx.x + k * kCbThreads;
        if (i < nodes) {
          anc[k] = parent[i];
          dist[k] = (i == nodes - 1) ? 0u : 1u;
        }
      }
      // store dist in nodew (weights are no longer needed)
      __syncthreads();
#pragma unroll
      for (int k = 0; k < kPer; ++k) {
        int i = threadIdx.x + k * kCbThreads;
        if (i < nodes) nodew[i] = dist[k];
      }
      __syncthreads();
      for (int round = 0; round < 14; ++round) {
        uint32_t nd[kPer], na[kPer];
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
          int i = threadIdx.x + k * kCbThreads;
          if (i < nodes) {
            nd[k] = nodew[i] + nodew[anc[k]];
            na[k] = parent[anc[k]];
          }
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
          int i = threadIdx.x + k * kCbThreads;
          if (i < nodes) {
            nodew[i] = nd[k];
            anc[k] = na[k];
            parent[i] = (uint16_t)na[k];
          }
        }
        __syncthreads();
      }
      if (threadIdx.x == 0) s_maxlen = 0;
      __syncthreads();
      for (int i = threadIdx.x; i < U; i += blockDim.x) {
        uint32_t sym = (uint32_t)(sk[i] & 4095ull);
        uint32_t L = nodew[i];
        depth8[sym] = (uint8_t)(L > 255 ? 255 : L);
        atomicMax(&s_maxlen, (int)L);
      }
      __syncthreads();
      if (s_maxlen <= kLmax) break;
      for (int i = threadIdx.x; i < kAlpha; i += blockDim.x)
        if (w[i]) w[i] = (w[i] + 1u) >> 1;
      __syncthreads();
    }
  }
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
    __shared__ uint32_t s_wsum[32];
    const int per = kAlpha / kCbThreads;  // 4
    for (int L = 1; L <= kLmax; ++L) {
      if (s_lc[L] == 0) continue;  // uniform across the block
      uint32_t c = 0;
      for (int k = 0; k < per; ++k) c += depth8[threadIdx.x * per + k] == L;
      // block exclusive scan of c
      uint32_t x = c;
      const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
      for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      if (lane == 31) s_wsum[wp] = x;
      __syncthreads();
      if (wp == 0) {
        uint32_t t = s_wsum[lane];
        for (int o = 1; o < 32; o <<= 1) {
          uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
          if (lane >= o) t += y;
        }
        s_wsum[lane] = t;
      }
      __syncthreads();
      uint32_t rank = (wp ? s_wsum[wp - 1] : 0u) + x - c;
      for (int k = 0; k < per; ++k) {
        int sym = threadIdx.x * per + k;
        if (depth8[sym] == L) {
          codes[(uint64_t)s * kAlpha + sym] = s_first[L] + rank;
          tables[(uint64_t)s * (kAlpha + 32) + 32 + s_index[L] + rank] = (uint16_t)sym;
          ++rank;
        }
      }
      __syncthreads();
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

void launch_codebook(int ns, const uint32_t *hist, const unsigned long long *maxv,
                     const unsigned long long *n_vals, uint32_t log2_chunk, StreamDesc *desc,
                     uint32_t *codes, uint8_t *lens, uint16_t *tables, cudaStream_t s) {
  const size_t smem = 8ull * kAlpha + 4ull * kAlpha + 8ull * kAlpha + 4ull * kAlpha + kAlpha;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_codebook, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr = true;
  }
  note_launch();
  k_codebook<<<ns, kCbThreads, smem, s>>>(hist, maxv, n_vals, log2_chunk, desc, codes, lens,
                                          tables);
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
// fixed-length payload: one thread per output word
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_encode_fixed(const T *__restrict__ vals, const StreamDesc *__restrict__ dp,
                               uint8_t *__restrict__ out, const Summary *__restrict__ summary) {
  if (summary->status != OK) return;
  const StreamDesc D = *dp;
  if (D.coder != 0 || D.width == 0 || D.n == 0) return;
  const uint32_t w = D.width;
  const unsigned long long words = words_of(D.payload_bits);
  uint32_t *pl = reinterpret_cast<uint32_t *>(out + D.offset + 32);
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < words;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const unsigned long long b0 = i * 32ull;
    unsigned long long v0 = b0 / w, v1 = (b0 + 31ull) / w;
    if (v1 >= D.n) v1 = D.n - 1;
    uint32_t word = 0;
    for (unsigned long long v = v0; v <= v1; ++v) {
      unsigned long long val = (unsigned long long)vals[v];
      long long sh = (long long)(b0 + 32ull) - (long long)(v * w + w);
      word |= sh >= 0 ? (uint32_t)(val << sh) : (uint32_t)(val >> (-sh));
    }
    pl[i] = word;
  }
}

// ---------------------------------------------------------------------------
// Huffman payload: per-chunk bit counts, their scan (the chunk table), then
// one warp per chunk assembling words in shared memory
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_chunk_bits(const T *__restrict__ vals, const StreamDesc *__restrict__ dp,
                             const uint8_t *__restrict__ lens, uint32_t log2_chunk,
                             unsigned long long *__restrict__ chunk_bits,
                             const Summary *__restrict__ summary) {
  if (summary->status != OK) return;
  const StreamDesc D = *dp;
  if (D.coder != 1) return;
  const int lane = threadIdx.x & 31;
  const unsigned long long warp = ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const unsigned long long nw = ((unsigned long long)gridDim.x * blockDim.x) >> 5;
  const unsigned long long cs = 1ull << log2_chunk;
  for (unsigned long long c = warp; c < D.n_chunks; c += nw) {
    const unsigned long long lo = c * cs, hi = min(D.n, lo + cs);
    unsigned long long bits = 0;
    for (unsigned long long i = lo + lane; i < hi; i += 32) {
      unsigned long long v = (unsigned long long)vals[i];
      uint32_t sym = v < (unsigned long long)kEsc ? (uint32_t)v : (uint32_t)kEsc;
      bits += lens[sym] + (sym == kEsc ? D.width : 0u);
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

// writes nbits of v (MSB first) at bit position pos of a u32 word array
__device__ __forceinline__ void put_bits_smem(uint32_t *buf, unsigned long long pos,
                                              unsigned long long v, uint32_t nbits) {
  while (nbits) {
    uint32_t wi = (uint32_t)(pos >> 5), off = (uint32_t)(pos & 31);
    uint32_t take = min(nbits, 32u - off);
    uint32_t part = (uint32_t)((v >> (nbits - take)) & ((take == 32) ? 0xffffffffull : ((1ull << take) - 1ull)));
    atomicOr(&buf[wi], part << (32 - off - take));
    pos += take;
    nbits -= take;
  }
}

constexpr int kEncWarps = 4;
constexpr int kStageWords = 2848;  // >= (1024 * (24 + 64)) / 32 + 2

template <typename T>
__global__ void __launch_bounds__(32 * kEncWarps) k_huff_encode(
    const T *__restrict__ vals, const StreamDesc *__restrict__ dp,
    const uint32_t *__restrict__ codes, const uint8_t *__restrict__ lens, uint32_t log2_chunk,
    const unsigned long long *__restrict__ chunk_off, uint8_t *__restrict__ out,
    const Summary *__restrict__ summary) {
  __shared__ uint32_t stage[kEncWarps][kStageWords];
  if (summary->status != OK) return;
  const StreamDesc D = *dp;
  if (D.coder != 1) return;
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  const unsigned long long cs = 1ull << log2_chunk;
  const uint32_t per = (uint32_t)(cs >> 5);  // symbols per lane
  uint32_t *buf = stage[wl];
  uint32_t *pl = reinterpret_cast<uint32_t *>(out + D.offset + pad16(80ull + 2ull * D.used) +
                                              pad16(8ull * D.n_chunks));
  const unsigned long long warp = (unsigned long long)blockIdx.x * kEncWarps + wl;
  const unsigned long long nw = (unsigned long long)gridDim.x * kEncWarps;
  for (unsigned long long c = warp; c < D.n_chunks; c += nw) {
    const unsigned long long lo = c * cs, hi = min(D.n, lo + cs);
    const unsigned long long start = chunk_off[c];
    const unsigned long long end = (c + 1 < D.n_chunks) ? chunk_off[c + 1] : D.payload_bits;
    const unsigned long long w0 = start >> 5, w1 = (end + 31) >> 5;  // [w0, w1)
    const uint32_t nwords = (uint32_t)(w1 - w0);
    if (nwords > (uint32_t)kStageWords || w1 > words_of(D.payload_bits)) continue;  // cannot happen
    for (uint32_t i = lane; i < nwords; i += 32) buf[i] = 0u;
    __syncwarp();
    // this lane's symbols and bit count
    const unsigned long long slo = lo + (unsigned long long)lane * per;
    const unsigned long long shi = min(hi, slo + per);
    unsigned long long mybits = 0;
    for (unsigned long long i = slo; i < shi; ++i) {
      unsigned long long v = (unsigned long long)vals[i];
      uint32_t sym = v < (unsigned long long)kEsc ? (uint32_t)v : (uint32_t)kEsc;
      mybits += lens[sym] + (sym == kEsc ? D.width : 0u);
    }
    unsigned long long x = mybits;
    for (int o = 1; o < 32; o <<= 1) {
      unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    unsigned long long pos = (start & 31ull) + (x - mybits);  // relative to word w0
    for (unsigned long long i = slo; i < shi; ++i) {
      unsigned long long v = (unsigned long long)vals[i];
      uint32_t sym = v < (unsigned long long)kEsc ? (uint32_t)v : (uint32_t)kEsc;
      uint32_t L = lens[sym];
      put_bits_smem(buf, pos, codes[sym], L);
      pos += L;
      if (sym == kEsc) {
        put_bits_smem(buf, pos, v, D.width);
        pos += D.width;
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
  unsigned long long words_max = (n * 64ull + 31ull) / 32ull;
  unsigned g = (unsigned)std::min<unsigned long long>((words_max + 255) / 256, 8ull * sms);
  if (g == 0) g = 1;
  note_launch();
  k_encode_fixed<T><<<g, 256, 0, s>>>(vals, desc, out, summary);
  // Huffman (no-op unless chosen)
  unsigned long long chunks = (n + (1ull << log2_chunk) - 1ull) >> log2_chunk;
  if (chunks == 0) return;
  unsigned gc = (unsigned)std::min<unsigned long long>((chunks * 32 + 255) / 256, 16ull * sms);
  note_launch();
  k_chunk_bits<T><<<gc, 256, 0, s>>>(vals, desc, lens, log2_chunk, chunk_bits, summary);
  launch_scan_small(chunk_bits, (uint32_t)chunks, chunk_off, s);
  unsigned gt = (unsigned)std::min<unsigned long long>((chunks + 255) / 256, 4ull * sms);
  note_launch();
  k_chunk_table<<<gt, 256, 0, s>>>(chunk_off, desc, out, summary);
  unsigned ge = (unsigned)std::min<unsigned long long>((chunks + kEncWarps - 1) / kEncWarps, 16ull * sms);
  note_launch();
  k_huff_encode<T><<<ge, 32 * kEncWarps, 0, s>>>(vals, desc, codes, lens, log2_chunk, chunk_off,
                                                  out, summary);
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
