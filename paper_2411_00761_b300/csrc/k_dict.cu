// k_dict.cu -- the dictionary stage (last step of the encoding stage, Sec.
// "Block coding"): the LZ77-style LCPZ coder described in lcp_dict.h.
//
// One warp codes one 2^16-byte chunk.  The parse is sequential by nature,
// but its inputs are not: positions enter the hash table 32 at a time (the
// latest earlier lane of the same hash, found with __match_any_sync, is the
// candidate of a position within the batch; the table entry from before the
// batch otherwise), the 4-byte agreement of all 32 candidates is one ballot,
// and the parse jumps from one agreeing position to the next with a
// find-first-set.  Copies are extended 32 bytes per step and sequences are
// written by all lanes at once.  Decoding is one warp per chunk as well:
// literal runs and copies are moved by the 32 lanes, an overlapping copy
// through its period (byte t of a copy at offset o is byte t mod o of the
// o bytes before it).
#include "lcp_dict.h"
#include "lcp_kernels.h"

namespace lcp {
namespace {

constexpr uint32_t kChunk = 1u << kDictLog2Chunk;
constexpr uint32_t kNone = 0xffffu;  // never a table entry: positions are <= 2^16 - 4
constexpr int kWarps = 4;            // chunks per CTA (encode and decode)

__device__ __forceinline__ uint32_t le32(const uint8_t *x) {
  return (uint32_t)__ldg(x) | ((uint32_t)__ldg(x + 1) << 8) | ((uint32_t)__ldg(x + 2) << 16) |
         ((uint32_t)__ldg(x + 3) << 24);
}

__device__ __forceinline__ uint32_t ext_len(uint32_t v) { return v >= 15 ? (v - 15) / 255 + 1 : 0; }

__device__ __forceinline__ uint32_t seq_size(uint32_t ll, uint32_t ml) {
  return 1 + ext_len(ll) + ll + (ml ? 2 + ext_len(ml - 4) : 0);
}

// byte e of the extension of v >= 15: (v - 15) / 255 bytes of 255, then the rest
__device__ __forceinline__ uint32_t ext_byte(uint32_t v, uint32_t e) {
  const uint32_t r = v - 15, full = r / 255;
  return e < full ? 255u : r - 255u * full;
}

// one sequence (ml = 0: literals only), every lane writing bytes lane, lane + 32, ...
__device__ void write_seq(uint8_t *o, const uint8_t *lit, uint32_t ll, uint32_t off, uint32_t ml,
                          uint32_t lane) {
  const uint32_t a = 1 + ext_len(ll), b = a + ll;
  const uint32_t sz = b + (ml ? 2 + ext_len(ml - 4) : 0);
  for (uint32_t t = lane; t < sz; t += 32) {
    uint32_t v;
    if (t == 0)
      v = (min(ll, 15u) << 4) | (ml ? min(ml - 4, 15u) : 0u);
    else if (t < a)
      v = ext_byte(ll, t - 1);
    else if (t < b)
      v = __ldg(lit + (t - a));
    else if (t == b)
      v = off & 0xffu;
    else if (t == b + 1)
      v = off >> 8;
    else
      v = ext_byte(ml - 4, t - b - 2);
    o[t] = (uint8_t)v;
  }
}

__global__ void __launch_bounds__(32 * kWarps)
    k_dict_encode(const uint8_t *__restrict__ in, uint64_t S, uint64_t C,
                  uint8_t *__restrict__ scratch, uint32_t *__restrict__ sizes) {
  __shared__ uint16_t table[kWarps][4096];
  const uint32_t lane = threadIdx.x & 31u, wid = threadIdx.x >> 5;
  uint16_t *tab = table[wid];
  for (uint64_t k = (uint64_t)blockIdx.x * kWarps + wid; k < C; k += (uint64_t)gridDim.x * kWarps) {
    const uint8_t *x = in + (k << kDictLog2Chunk);
    const uint64_t left = S - (k << kDictLog2Chunk);
    const uint32_t m = left < kChunk ? (uint32_t)left : kChunk;
    uint8_t *o = scratch + (k << kDictLog2Chunk);
    for (uint32_t h = lane; h < 4096u; h += 32) tab[h] = (uint16_t)kNone;
    __syncwarp();
    uint32_t size = 0, p = 0, lit = 0;
    bool stored = false;
    for (uint32_t b = 0; b < m && !stored; b += 32) {
      const uint32_t i = b + lane;
      const bool v4 = i + 4 <= m;
      uint32_t key = 0, h = 4096u + lane;  // lanes without four bytes match no other lane
      if (v4) {
        key = le32(x + i);
        h = (key * 2654435761u) >> 20;
      }
      const uint32_t before = v4 ? (uint32_t)tab[h] : kNone;
      const uint32_t grp = __match_any_sync(0xffffffffu, h);
      const uint32_t lower = grp & ((1u << lane) - 1u);
      const uint32_t cand = lower ? b + (31u - (uint32_t)__clz(lower)) : before;
      __syncwarp();
      // the latest lane of each hash leaves its position in the table
      if (v4 && !(grp & ~((2u << lane) - 1u))) tab[h] = (uint16_t)i;
      __syncwarp();
      const bool agree = v4 && cand != kNone && le32(x + cand) == key;
      const uint32_t mask = __ballot_sync(0xffffffffu, agree);
      // the parse over this batch's positions from p on (warp-uniform)
      while (p < b + 32 && p < m) {
        const uint32_t bits = mask & (0xffffffffu << (p - b));
        if (!bits) {
          p = b + 32;
          break;
        }
        const uint32_t q = b + (uint32_t)(__ffs(bits) - 1);
        const uint32_t j = __shfl_sync(0xffffffffu, cand, q - b);
        uint32_t len = 4;
        for (;;) {
          const uint32_t t = len + lane;
          const bool same = q + t < m && __ldg(x + j + t) == __ldg(x + q + t);
          const uint32_t diff = __ballot_sync(0xffffffffu, !same);
          if (diff) {
            len += (uint32_t)(__ffs(diff) - 1);
            break;
          }
          len += 32;
        }
        const uint32_t sz = seq_size(q - lit, len);
        if (size + sz >= m) {
          stored = true;
          break;
        }
        write_seq(o + size, x + lit, q - lit, q - j, len, lane);
        size += sz;
        p = q + len;
        lit = p;
      }
    }
    if (!stored && lit < m) {
      const uint32_t sz = seq_size(m - lit, 0);
      if (size + sz >= m)
        stored = true;
      else {
        write_seq(o + size, x + lit, m - lit, 0, 0, lane);
        size += sz;
      }
    }
    if (lane == 0) sizes[k] = stored ? (m | 0x80000000u) : size;
    __syncwarp();  // the table is reset for the next chunk
  }
}

// exclusive scan of the chunk sizes, one CTA of 1024 threads, tiles of 1024
__global__ void __launch_bounds__(1024)
    k_dict_offsets(const uint32_t *__restrict__ sizes, uint64_t C, unsigned long long base,
                   unsigned long long *__restrict__ off) {
  __shared__ unsigned long long wsum[32];
  __shared__ unsigned long long carry;
  const uint32_t lane = threadIdx.x & 31u, wid = threadIdx.x >> 5;
  if (threadIdx.x == 0) carry = base;
  __syncthreads();
  for (uint64_t t0 = 0; t0 < C; t0 += 1024) {
    const uint64_t k = t0 + threadIdx.x;
    const unsigned long long v = k < C ? (sizes[k] & 0x7fffffffu) : 0ull;
    unsigned long long x = v;
    for (int d = 1; d < 32; d <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xffffffffu, x, d);
      if (lane >= (uint32_t)d) x += y;
    }
    if (lane == 31) wsum[wid] = x;
    __syncthreads();
    if (wid == 0) {
      unsigned long long w = wsum[lane];
      for (int d = 1; d < 32; d <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, w, d);
        if (lane >= (uint32_t)d) w += y;
      }
      wsum[lane] = w;
    }
    __syncthreads();
    const unsigned long long excl = carry + (wid ? wsum[wid - 1] : 0ull) + x - v;
    if (k < C) off[k] = excl;
    __syncthreads();
    if (threadIdx.x == 1023) carry = excl + v;
    __syncthreads();
  }
  if (threadIdx.x == 0) off[C] = carry;
}

__global__ void k_dict_pack(const uint8_t *__restrict__ in, uint64_t S, uint64_t C,
                            const uint8_t *__restrict__ scratch,
                            const uint32_t *__restrict__ sizes,
                            const unsigned long long *__restrict__ off, uint64_t T,
                            uint8_t *__restrict__ out) {
  if (blockIdx.x == 0) {
    for (uint32_t t = threadIdx.x; t < (uint32_t)kDictHead; t += blockDim.x) {
      uint32_t v = 0;
      if (t < 4)
        v = (uint32_t)"LCPZ"[t];
      else if (t == 4)
        v = 1;
      else if (t == 5)
        v = kDictLog2Chunk;
      else if (t >= 8 && t < 32) {
        const unsigned long long f = t < 16 ? S : (t < 24 ? C : T);
        v = (uint32_t)(f >> (8 * (t & 7))) & 0xffu;
      } else if (t >= 32 && (uint64_t)(t - 32) < S)
        v = in[t - 32];
      out[t] = (uint8_t)v;
    }
    const uint64_t body = dict_body(C);
    for (uint64_t t = kDictHead + 4 * C + threadIdx.x; t < body; t += blockDim.x) out[t] = 0;
    for (uint64_t t = off[C] + threadIdx.x; t < T; t += blockDim.x) out[t] = 0;
  }
  for (uint64_t k = blockIdx.x; k < C; k += gridDim.x) {
    const uint32_t e = sizes[k], c = e & 0x7fffffffu;
    if (threadIdx.x == 0) reinterpret_cast<uint32_t *>(out + kDictHead)[k] = e;
    const uint8_t *src = ((e >> 31) ? in : scratch) + (k << kDictLog2Chunk);
    uint8_t *dst = out + off[k];
    for (uint32_t t = threadIdx.x; t < c; t += blockDim.x) dst[t] = src[t];
  }
}

// an extension at z[*q], below c; false when it runs past c
__device__ __forceinline__ bool get_ext(const uint8_t *z, uint32_t &q, uint32_t c, uint32_t &v) {
  for (;;) {
    if (q >= c) return false;
    const uint32_t b = z[q++];
    v += b;
    if (b != 255u) return true;
  }
}

// out is written and read back by the warp: no restrict / non-coherent loads on it
__global__ void __launch_bounds__(32 * kWarps)
    k_dict_decode(const uint8_t *__restrict__ in, uint64_t in_size, uint64_t S, uint64_t T,
                  const unsigned long long *__restrict__ off, uint8_t *out, int *err) {
  const uint32_t lane = threadIdx.x & 31u, wid = threadIdx.x >> 5;
  const uint64_t C = dict_chunks(S);
  // the sizes must add up to the image's total
  if (((off[C] + 15) & ~15ull) != T || T > in_size) {
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicExch(err, 1);
    return;
  }
  const uint32_t *sizes = reinterpret_cast<const uint32_t *>(in + kDictHead);
  for (uint64_t k = (uint64_t)blockIdx.x * kWarps + wid; k < C; k += (uint64_t)gridDim.x * kWarps) {
    const uint32_t e = sizes[k], c = e & 0x7fffffffu;
    const uint64_t left = S - (k << kDictLog2Chunk);
    const uint32_t m = left < kChunk ? (uint32_t)left : kChunk;
    const uint8_t *z = in + off[k];
    uint8_t *y = out + (k << kDictLog2Chunk);
    bool bad = false;
    if (e >> 31) {
      if (c != m)
        bad = true;
      else
        for (uint32_t t = lane; t < m; t += 32) y[t] = z[t];
    } else if (c >= m) {
      bad = true;  // a coded chunk is shorter than its bytes
    } else {
      uint32_t q = 0, w = 0;
      while (w < m) {
        if (q >= c) {
          bad = true;
          break;
        }
        const uint32_t tok = z[q++];
        uint32_t ll = tok >> 4, ml = tok & 15u;
        if (ll == 15 && !get_ext(z, q, c, ll)) {
          bad = true;
          break;
        }
        if (ll > m - w || ll > c - q) {
          bad = true;
          break;
        }
        for (uint32_t t = lane; t < ll; t += 32) y[w + t] = z[q + t];
        w += ll;
        q += ll;
        if (w == m) break;
        if (c - q < 2) {
          bad = true;
          break;
        }
        const uint32_t o = (uint32_t)z[q] | ((uint32_t)z[q + 1] << 8);
        q += 2;
        if (ml == 15 && !get_ext(z, q, c, ml)) {
          bad = true;
          break;
        }
        ml += 4;
        if (o == 0 || o > w || ml > m - w) {
          bad = true;
          break;
        }
        __syncwarp();  // the bytes before w, written by every lane, are visible
        for (uint32_t t = lane; t < ml; t += 32) y[w + t] = y[w - o + (t < o ? t : t % o)];
        __syncwarp();
        w += ml;
      }
      if (!bad && q != c) bad = true;
    }
    if (bad && lane == 0) atomicExch(err, 1);
  }
}

int grid_for(uint64_t C, int sms) {
  const uint64_t need = (C + kWarps - 1) / kWarps;
  const uint64_t cap = (uint64_t)sms * 16;
  return (int)(need < 1 ? 1 : (need < cap ? need : cap));
}

}  // namespace

void launch_dict_encode(const uint8_t *in, uint64_t S, uint8_t *scratch, uint32_t *sizes, int sms,
                        cudaStream_t s) {
  const uint64_t C = dict_chunks(S);
  if (C == 0) return;
  note_launch();
  k_dict_encode<<<grid_for(C, sms), 32 * kWarps, 0, s>>>(in, S, C, scratch, sizes);
}

void launch_dict_offsets(const uint32_t *sizes, uint64_t C, unsigned long long *off,
                         cudaStream_t s) {
  note_launch();
  k_dict_offsets<<<1, 1024, 0, s>>>(sizes, C, dict_body(C), off);
}

void launch_dict_pack(const uint8_t *in, uint64_t S, const uint8_t *scratch, const uint32_t *sizes,
                      const unsigned long long *off, uint64_t T, uint8_t *out, int sms,
                      cudaStream_t s) {
  const uint64_t C = dict_chunks(S);
  const uint64_t cap = (uint64_t)sms * 8;
  note_launch();
  k_dict_pack<<<(int)(C < 1 ? 1 : (C < cap ? C : cap)), 256, 0, s>>>(in, S, C, scratch, sizes, off,
                                                                      T, out);
}

void launch_dict_decode(const uint8_t *in, uint64_t in_size, uint64_t S, uint64_t T,
                        const unsigned long long *off, uint8_t *out, int *err, int sms,
                        cudaStream_t s) {
  note_launch();
  k_dict_decode<<<grid_for(dict_chunks(S), sms), 32 * kWarps, 0, s>>>(in, in_size, S, T, off, out,
                                                                      err);
}

}  // namespace lcp
