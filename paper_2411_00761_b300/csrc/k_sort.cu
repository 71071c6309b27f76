// k_sort.cu -- partition by the key's top bits, per-bucket sort, segmentation.
//
// Sec. "Design of spatial blocks": the non-empty blocks are kept in id order
// with their particle counts and the particles' locations relative to the
// block corner; Sec. "Block coding": each array is delta coded.  The keys
// (block_id * p^d + rel) are sorted with one most-significant-digit partition
// pass into buckets of consecutive block ids, then every bucket is sorted by
// one CTA (in shared memory when it fits) and segmented into blocks in the
// same CTA.  The output bytes depend only on the multiset of keys, so the
// partition pass needs no stable order.
#include "lcp_kernels.h"

namespace lcp {

constexpr int kLocalThreads = 512;
constexpr int kLocalWarps = kLocalThreads / 32;
constexpr int kCap = 4096;  // keys of a unit sorted in shared memory
constexpr int kSubBits = 10; // level-2 split of oversized buckets

// ---------------------------------------------------------------------------
// block-wide exclusive scan of u64 values held one per thread
// ---------------------------------------------------------------------------
template <int THREADS>
__device__ __forceinline__ unsigned long long block_exscan(unsigned long long v,
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
    s_warp[lane] = t;  // inclusive warp totals
  }
  __syncthreads();
  unsigned long long base = w > 0 ? s_warp[w - 1] : 0ull;
  total = s_warp[THREADS / 32 - 1];
  __syncthreads();
  return base + x - v;
}

// ---------------------------------------------------------------------------
// bucket offsets
// ---------------------------------------------------------------------------
__global__ void k_bucket_colsum(const uint32_t *__restrict__ tile_hist, int tiles, uint32_t nb1,
                                unsigned long long *__restrict__ totals) {
  uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb1) return;
  unsigned long long s = 0;
  for (int t = 0; t < tiles; ++t) s += tile_hist[(uint64_t)t * nb1 + b];
  totals[b] = s;
}

// exclusive scan of n values (one CTA); out[n] = total
__global__ void __launch_bounds__(1024) k_scan_small(const unsigned long long *__restrict__ in,
                                                     uint32_t n,
                                                     unsigned long long *__restrict__ out) {
  __shared__ unsigned long long s_warp[32];
  const uint32_t per = (n + 1023) / 1024;
  const uint32_t lo = threadIdx.x * per, hi = min(n, lo + per);
  unsigned long long sum = 0;
  for (uint32_t i = lo; i < hi; ++i) sum += in[i];
  unsigned long long total;
  unsigned long long run = block_exscan<1024>(sum, s_warp, total);
  for (uint32_t i = lo; i < hi; ++i) {
    unsigned long long v = in[i];
    out[i] = run;
    run += v;
  }
  if (threadIdx.x == 0) out[n] = total;
}

__global__ void k_bucket_tileoff(uint32_t *__restrict__ tile_hist, int tiles, uint32_t nb1,
                                 const unsigned long long *__restrict__ bucket_start) {
  uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb1) return;
  uint32_t run = (uint32_t)bucket_start[b];
  for (int t = 0; t < tiles; ++t) {
    uint32_t v = tile_hist[(uint64_t)t * nb1 + b];
    tile_hist[(uint64_t)t * nb1 + b] = run;
    run += v;
  }
}

void launch_bucket_offsets(uint32_t *tile_hist, int tiles, uint32_t nb1,
                           unsigned long long *bucket_start, unsigned long long *totals,
                           cudaStream_t s) {
  unsigned g = (nb1 + 255) / 256;
  note_launch();
  k_bucket_colsum<<<g, 256, 0, s>>>(tile_hist, tiles, nb1, totals);
  note_launch();
  k_scan_small<<<1, 1024, 0, s>>>(totals, nb1, bucket_start);
  note_launch();
  k_bucket_tileoff<<<g, 256, 0, s>>>(tile_hist, tiles, nb1, bucket_start);
}

void launch_scan_small(const unsigned long long *in, uint32_t n, unsigned long long *out,
                       cudaStream_t s) {
  note_launch();
  k_scan_small<<<1, 1024, 0, s>>>(in, n, out);
}

// ---------------------------------------------------------------------------
// scatter: same tiles as the quantize pass; shared-memory cursors per bucket
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(512) k_scatter(const unsigned long long *__restrict__ keys,
                                                 uint64_t n, const Plan *__restrict__ plan,
                                                 uint32_t nb1, uint64_t span,
                                                 const uint32_t *__restrict__ tile_off,
                                                 unsigned long long *__restrict__ keys_out,
                                                 uint32_t *__restrict__ idx_out) {
  extern __shared__ uint32_t s_cur[];
  const uint32_t *to = tile_off + (uint64_t)blockIdx.x * nb1;
  for (uint32_t b = threadIdx.x; b < nb1; b += blockDim.x) s_cur[b] = to[b];
  __syncthreads();
  if (plan->status != OK) return;
  const uint32_t shift = plan->part_shift, nb = nb1 - 1;
  const uint64_t lo = (uint64_t)blockIdx.x * span;
  const uint64_t hi = min(n, lo + span);
  for (uint64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    unsigned long long k = __ldcs(keys + i);
    uint32_t b = (k & kOutlierBit) ? nb : (uint32_t)(k >> shift);
    uint32_t pos = atomicAdd(&s_cur[b], 1u);
    keys_out[pos] = k;
    if (idx_out) idx_out[pos] = (uint32_t)i;
  }
}

void launch_scatter(const unsigned long long *keys, uint64_t n, const Plan *plan, uint32_t nb1,
                    int tiles, const uint32_t *tile_off, unsigned long long *keys_out,
                    uint32_t *idx_out, cudaStream_t s) {
  uint64_t span = (n + tiles - 1) / tiles;
  span = (span + 3) & ~3ull;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr = true;
  }
  note_launch();
  k_scatter<<<tiles, 512, sizeof(uint32_t) * nb1, s>>>(keys, n, plan, nb1, span, tile_off,
                                                      keys_out, idx_out);
}

// ---------------------------------------------------------------------------
// stable CTA radix sort (8-bit digits).  Warp w owns the contiguous element
// range [w*S, (w+1)*S); within a warp elements are ranked in order with
// __match_any_sync, so each pass is stable.  Arrays may live in shared or
// global memory (generic pointers).  Counters are warp-major (w * 256 + digit)
// so the lanes of a warp touch different banks.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

__device__ void radix_pass(const unsigned long long *kin, const uint32_t *iin,
                           unsigned long long *kout, uint32_t *iout, int cnt, int shift,
                           bool by_idx, uint32_t *s_cnt, unsigned long long *s_warp) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < 256 * kLocalWarps; i += kLocalThreads) s_cnt[i] = 0u;
  __syncthreads();
  const int S = (cnt + kLocalWarps - 1) / kLocalWarps;
  const int wlo = min(cnt, w * S), whi = min(cnt, wlo + S);
  const uint32_t lt = lanemask_lt();
  uint32_t *wc = s_cnt + w * 256;
  for (int base = wlo; base < whi; base += 32) {
    int j = base + lane;
    bool valid = j < whi;
    uint32_t dg = 256u + lane;
    if (valid) dg = by_idx ? ((iin[j] >> shift) & 255u) : (uint32_t)((kin[j] >> shift) & 255ull);
    uint32_t peers = __match_any_sync(0xffffffffu, dg);
    if (valid && lane == __ffs(peers) - 1) wc[dg] += __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  // exclusive scan over (digit, warp) in digit-major order: logical index
  // i = digit * warps + warp lives at warp * 256 + digit
  {
    constexpr int per = 256 * kLocalWarps / kLocalThreads;
    uint32_t v[per];
    unsigned long long sum = 0;
#pragma unroll
    for (int k = 0; k < per; ++k) {
      const int i = threadIdx.x * per + k;
      v[k] = s_cnt[(i % kLocalWarps) * 256 + i / kLocalWarps];
      sum += v[k];
    }
    unsigned long long tot;
    unsigned long long run = block_exscan<kLocalThreads>(sum, s_warp, tot);
#pragma unroll
    for (int k = 0; k < per; ++k) {
      const int i = threadIdx.x * per + k;
      s_cnt[(i % kLocalWarps) * 256 + i / kLocalWarps] = (uint32_t)run;
      run += v[k];
    }
  }
  __syncthreads();
  for (int base = wlo; base < whi; base += 32) {
    int j = base + lane;
    bool valid = j < whi;
    uint32_t dg = 256u + lane;
    unsigned long long kv = 0;
    uint32_t iv = 0;
    if (valid) {
      kv = kin[j];
      if (iin) iv = iin[j];
      dg = by_idx ? ((iv >> shift) & 255u) : (uint32_t)((kv >> shift) & 255ull);
    }
    uint32_t peers = __match_any_sync(0xffffffffu, dg);
    uint32_t basepos = valid ? wc[dg] : 0u;
    __syncwarp();
    if (valid) {
      uint32_t pos = basepos + __popc(peers & lt);
      kout[pos] = kv;
      if (iout) iout[pos] = iv;
      if (lane == __ffs(peers) - 1) wc[dg] = basepos + __popc(peers);
    }
    __syncwarp();
  }
  __syncthreads();
}

// sorts (k, i) by key bits [0, kbits), ties by index bits [0, ibits) (LSD:
// index digits first).  Returns 1 when the result ended in the alt buffers.
__device__ int cta_sort(unsigned long long *k, uint32_t *i, unsigned long long *k2, uint32_t *i2,
                        int cnt, int kbits, int ibits, uint32_t *s_cnt,
                        unsigned long long *s_warp) {
  int flip = 0;
  unsigned long long *ka = k, *kb = k2;
  uint32_t *ia = i, *ib = i2;
  for (int sh = 0; sh < ibits; sh += 8) {
    radix_pass(ka, ia, kb, ib, cnt, sh, true, s_cnt, s_warp);
    unsigned long long *t = ka;
    ka = kb;
    kb = t;
    uint32_t *u = ia;
    ia = ib;
    ib = u;
    flip ^= 1;
  }
  for (int sh = 0; sh < kbits; sh += 8) {
    radix_pass(ka, ia, kb, ib, cnt, sh, false, s_cnt, s_warp);
    unsigned long long *t = ka;
    ka = kb;
    kb = t;
    uint32_t *u = ia;
    ia = ib;
    ib = u;
    flip ^= 1;
  }
  return flip;
}

// ---------------------------------------------------------------------------
// level-2 partition of buckets larger than the shared-memory sort: each such
// bucket is split by the next kSubBits key bits (still block-id bits, so no
// block crosses a sub-bucket), one CTA per bucket.  Sort units: the ordered
// list of key ranges that k_local sorts -- consecutive small level-1 buckets
// merged greedily up to kCap keys, split buckets as greedy merges of their
// consecutive sub-buckets, and the outlier bucket.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_seg_plan(const Plan *__restrict__ plan, uint32_t nb1,
                                                   const unsigned long long *__restrict__ bstart,
                                                   uint32_t *__restrict__ big_list,
                                                   int *__restrict__ big_of,
                                                   uint32_t *__restrict__ nbig) {
  __shared__ unsigned long long s_warp[32];
  const Plan &P = *plan;
  const uint32_t nb = nb1 - 1;
  const int sub = min(kSubBits, (int)P.part_shift - (int)P.rel_bits);
  const uint32_t per = (nb1 + 1023) / 1024;
  const uint32_t lo = threadIdx.x * per, hi = min(nb1, lo + per);
  unsigned long long c = 0;
  for (uint32_t b = lo; b < hi; ++b) {
    const bool big = sub > 0 && b < nb && (bstart[b + 1] - bstart[b]) > (unsigned long long)kCap;
    c += big;
  }
  unsigned long long tot;
  unsigned long long run = block_exscan<1024>(c, s_warp, tot);
  for (uint32_t b = lo; b < hi; ++b) {
    const bool big = sub > 0 && b < nb && (bstart[b + 1] - bstart[b]) > (unsigned long long)kCap;
    big_of[b] = big ? (int)run : -1;
    if (big) big_list[run++] = b;
  }
  if (threadIdx.x == 0) *nbig = (uint32_t)tot;
}

// greedy merge of consecutive sub-bucket counts into units of <= kCap keys;
// emit(offset, count) per unit.  Returns the number of units.
template <typename F>
__device__ uint32_t greedy_units(const uint32_t *cnt, uint32_t nsub, F emit) {
  uint32_t units = 0, uoff = 0, ucnt = 0, off = 0;
  for (uint32_t d = 0; d < nsub; ++d) {
    const uint32_t c = cnt[d];
    if (c) {
      if (ucnt && ucnt + c > (uint32_t)kCap) {
        emit(uoff, ucnt);
        ++units;
        ucnt = 0;
      }
      if (!ucnt) uoff = off;
      ucnt += c;
    }
    off += c;
  }
  if (ucnt) {
    emit(uoff, ucnt);
    ++units;
  }
  return units;
}

__global__ void __launch_bounds__(1024) k_split_big(const Plan *__restrict__ plan,
                                                    const unsigned long long *__restrict__ bstart,
                                                    const uint32_t *__restrict__ big_list,
                                                    const uint32_t *__restrict__ nbig,
                                                    const unsigned long long *__restrict__ keys,
                                                    const uint32_t *__restrict__ idx,
                                                    unsigned long long *__restrict__ keys_out,
                                                    uint32_t *__restrict__ idx_out,
                                                    uint32_t *__restrict__ sub_cnt,
                                                    uint32_t *__restrict__ big_units) {
  __shared__ uint32_t h[1 << kSubBits];
  __shared__ uint32_t hc[1 << kSubBits];
  __shared__ unsigned long long s_warp[32];
  const Plan &P = *plan;
  const int sub = min(kSubBits, (int)P.part_shift - (int)P.rel_bits);
  const int shift2 = (int)P.part_shift - sub;
  const uint32_t mask = (1u << sub) - 1u;
  const uint32_t nsub = 1u << sub;
  constexpr int per = (1 << kSubBits) / 1024;
  for (uint32_t j = blockIdx.x; j < *nbig; j += gridDim.x) {
    const uint32_t b = big_list[j];
    const uint64_t lo = bstart[b];
    const uint64_t cnt = bstart[b + 1] - lo;
    for (uint32_t d = threadIdx.x; d < (1u << kSubBits); d += blockDim.x) h[d] = 0u;
    __syncthreads();
    for (uint64_t t = threadIdx.x; t < cnt; t += blockDim.x)
      atomicAdd(&h[(uint32_t)(keys[lo + t] >> shift2) & mask], 1u);
    __syncthreads();
    uint32_t v[per];
    unsigned long long sum = 0;
#pragma unroll
    for (int k = 0; k < per; ++k) {
      const uint32_t d = threadIdx.x * per + k;
      v[k] = d < nsub ? h[d] : 0u;
      sum += v[k];
      if (d < nsub) {
        sub_cnt[(uint64_t)j * (1u << kSubBits) + d] = v[k];
        hc[d] = v[k];
      }
    }
    unsigned long long tot;
    unsigned long long run = block_exscan<1024>(sum, s_warp, tot);
#pragma unroll
    for (int k = 0; k < per; ++k) {
      const uint32_t d = threadIdx.x * per + k;
      if (d < nsub) h[d] = (uint32_t)run;
      run += v[k];
    }
    __syncthreads();
    if (threadIdx.x == 0) big_units[j] = greedy_units(hc, nsub, [](uint32_t, uint32_t) {});
    for (uint64_t t = threadIdx.x; t < cnt; t += blockDim.x) {
      const unsigned long long k = keys[lo + t];
      const uint32_t pos = atomicAdd(&h[(uint32_t)(k >> shift2) & mask], 1u);
      keys_out[lo + pos] = k;
      if (idx_out) idx_out[lo + pos] = idx[lo + t];
    }
    __syncthreads();
  }
}

// Unit list (one CTA).  Thread t owns buckets [t*per, (t+1)*per); within that
// range consecutive small buckets merge greedily up to kCap keys (a single
// bucket above kCap that cannot be split forms its own unit); a split bucket
// contributes its sub-bucket units, written by k_units_big at big_base[j];
// the outlier bucket is a unit of its own.
__global__ void __launch_bounds__(1024) k_units_small(uint32_t nb1,
                                                      const unsigned long long *__restrict__ bstart,
                                                      const int *__restrict__ big_of,
                                                      const uint32_t *__restrict__ big_units,
                                                      uint32_t *__restrict__ big_base,
                                                      uint32_t *__restrict__ u_lo,
                                                      uint32_t *__restrict__ u_cnt,
                                                      uint32_t *__restrict__ u_meta,
                                                      uint32_t *__restrict__ nunit) {
  __shared__ unsigned long long s_warp[32];
  const uint32_t nb = nb1 - 1;
  const uint32_t per = (nb1 + 1023) / 1024;
  const uint32_t lo = threadIdx.x * per, hi = min(nb1, lo + per);
  unsigned long long count = 0;
  uint64_t ucnt = 0;
  for (uint32_t b = lo; b < hi; ++b) {
    const uint64_t c = bstart[b + 1] - bstart[b];
    const int j = big_of[b];
    if (j >= 0 || b == nb) {
      if (ucnt) {
        ++count;
        ucnt = 0;
      }
      if (j >= 0) count += big_units[j];
      else if (c) ++count;
      continue;
    }
    if (!c) continue;
    if (ucnt && ucnt + c > (uint64_t)kCap) {
      ++count;
      ucnt = 0;
    }
    ucnt += c;
  }
  if (ucnt) ++count;
  unsigned long long tot;
  unsigned long long out = block_exscan<1024>(count, s_warp, tot);
  if (threadIdx.x == 0) *nunit = (uint32_t)tot;
  uint64_t ulo = 0;
  ucnt = 0;
  for (uint32_t b = lo; b < hi; ++b) {
    const uint64_t c = bstart[b + 1] - bstart[b];
    const int j = big_of[b];
    if (j >= 0 || b == nb) {
      if (ucnt) {
        u_lo[out] = (uint32_t)ulo;
        u_cnt[out] = (uint32_t)ucnt;
        u_meta[out] = 0u;
        ++out;
        ucnt = 0;
      }
      if (j >= 0) {
        big_base[j] = (uint32_t)out;
        out += big_units[j];
      } else if (c) {
        u_lo[out] = (uint32_t)bstart[b];
        u_cnt[out] = (uint32_t)c;
        u_meta[out] = 2u;  // the outlier bucket
        ++out;
      }
      continue;
    }
    if (!c) continue;
    if (ucnt && ucnt + c > (uint64_t)kCap) {
      u_lo[out] = (uint32_t)ulo;
      u_cnt[out] = (uint32_t)ucnt;
      u_meta[out] = 0u;
      ++out;
      ucnt = 0;
    }
    if (!ucnt) ulo = bstart[b];
    ucnt += c;
  }
  if (ucnt) {
    u_lo[out] = (uint32_t)ulo;
    u_cnt[out] = (uint32_t)ucnt;
    u_meta[out] = 0u;
  }
}

// units of each split bucket (one CTA per bucket, thread 0 walks the
// sub-bucket counts)
__global__ void k_units_big(const unsigned long long *__restrict__ bstart,
                            const uint32_t *__restrict__ big_list,
                            const uint32_t *__restrict__ nbig,
                            const uint32_t *__restrict__ sub_cnt, int nsub_bits_cap,
                            const Plan *__restrict__ plan, const uint32_t *__restrict__ big_base,
                            uint32_t *__restrict__ u_lo, uint32_t *__restrict__ u_cnt,
                            uint32_t *__restrict__ u_meta) {
  (void)nsub_bits_cap;
  const Plan &P = *plan;
  const int sub = min(kSubBits, (int)P.part_shift - (int)P.rel_bits);
  const uint32_t nsub = sub > 0 ? (1u << sub) : 1u;
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < *nbig;
       j += gridDim.x * blockDim.x) {
    const uint64_t lo = bstart[big_list[j]];
    uint32_t o = big_base[j];
    greedy_units(sub_cnt + (uint64_t)j * (1u << kSubBits), nsub, [&](uint32_t off, uint32_t c) {
      u_lo[o] = (uint32_t)(lo + off);
      u_cnt[o] = c;
      u_meta[o] = 1u;  // keys in the level-2 buffer
      ++o;
    });
  }
}

void launch_segments(const Plan *plan, uint32_t nb1, const unsigned long long *bstart,
                     unsigned long long *keys, uint32_t *idx, unsigned long long *keys_alt,
                     uint32_t *idx_alt, uint32_t *big_list, int *big_of, uint32_t *nbig,
                     uint32_t *sub_cnt, uint32_t *big_units, uint32_t *big_base, uint32_t *u_lo,
                     uint32_t *u_cnt, uint32_t *u_meta, uint32_t *nunit, uint64_t n, int sms,
                     cudaStream_t s) {
  (void)n;
  note_launch();
  k_seg_plan<<<1, 1024, 0, s>>>(plan, nb1, bstart, big_list, big_of, nbig);
  note_launch();
  k_split_big<<<sms, 1024, 0, s>>>(plan, bstart, big_list, nbig, keys, idx, keys_alt, idx_alt,
                                   sub_cnt, big_units);
  note_launch();
  k_units_small<<<1, 1024, 0, s>>>(nb1, bstart, big_of, big_units, big_base, u_lo, u_cnt, u_meta,
                                   nunit);
  note_launch();
  k_units_big<<<sms, 128, 0, s>>>(bstart, big_list, nbig, sub_cnt, 0, plan, big_base, u_lo, u_cnt,
                                  u_meta);
}

// ---------------------------------------------------------------------------
// per-unit sort + segmentation into blocks (persistent over units)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kLocalThreads) k_local(LocalArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const bool perm = a.perm != nullptr;
  unsigned long long *sk = reinterpret_cast<unsigned long long *>(smem);
  unsigned long long *sk2 = sk + kCap;
  uint32_t *s_cnt = reinterpret_cast<uint32_t *>(sk2 + kCap);  // 256 * warps
  uint32_t *s_hist = s_cnt + 256 * kLocalWarps;                // 4096
  uint32_t *si = s_hist + kAlpha;                               // perm mode only
  uint32_t *si2 = si + kCap;
  __shared__ unsigned long long s_warp[32];
  __shared__ unsigned long long s_max, s_kmin, s_kmax;
  __shared__ Plan sP;
  if (threadIdx.x == 0) {
    sP = *a.plan;
    s_max = 0ull;
  }
  for (int b = threadIdx.x; b < kAlpha; b += kLocalThreads) s_hist[b] = 0u;
  __syncthreads();
  if (sP.status != OK) return;
  const uint32_t rel_bits = sP.rel_bits;
  const unsigned long long rel_mask = rel_bits >= 64 ? ~0ull : ((1ull << rel_bits) - 1ull);
  const uint64_t chunk_mask = (1ull << a.log2_chunk) - 1ull;
  const int ibits = perm ? (int)bitlen64(a.n > 0 ? a.n - 1 : 0) : 0;
  const uint32_t d = sP.d;
  const uint32_t nseg = *a.nseg;
  unsigned long long my_max = 0ull;

  for (uint32_t sg = blockIdx.x; sg < nseg; sg += gridDim.x) {
    const uint64_t lo = a.seg_lo[sg];
    const int cnt = (int)a.seg_cnt[sg];
    const uint32_t meta = a.seg_meta[sg];
    const bool outl = (meta >> 1) & 1u;
    const bool src_alt = meta & 1u;
    unsigned long long *gk = (src_alt ? a.keys_alt : a.keys) + lo;
    unsigned long long *gk2 = (src_alt ? a.keys : a.keys_alt) + lo;
    uint32_t *gi = nullptr, *gi2 = nullptr;
    if (perm && !outl) {
      gi = (src_alt ? a.idx_alt : a.idx) + lo;
      gi2 = (src_alt ? a.idx : a.idx_alt) + lo;
    }
    // the radix passes cover only the bits where the unit's keys differ
    if (threadIdx.x == 0) {
      s_kmin = ~0ull;
      s_kmax = 0ull;
    }
    __syncthreads();
    const bool in_smem = cnt <= kCap;
    unsigned long long mn = ~0ull, mx = 0ull;
    for (int j = threadIdx.x; j < cnt; j += kLocalThreads) {
      const unsigned long long v = gk[j];
      if (in_smem) {
        sk[j] = v;
        if (gi) si[j] = gi[j];
      }
      mn = v < mn ? v : mn;
      mx = v > mx ? v : mx;
    }
    atomicMin(&s_kmin, mn);
    atomicMax(&s_kmax, mx);
    __syncthreads();
    const int kbits = (int)bitlen64(s_kmin ^ s_kmax);
    const unsigned long long *K;
    const uint32_t *I = nullptr;
    if (in_smem) {
      int fl = cta_sort(sk, gi ? si : nullptr, sk2, gi ? si2 : nullptr, cnt, kbits,
                        outl ? 0 : ibits, s_cnt, s_warp);
      K = fl ? sk2 : sk;
      I = gi ? (fl ? si2 : si) : nullptr;
    } else {
      int fl = cta_sort(gk, gi, gk2, gi2, cnt, kbits, outl ? 0 : ibits, s_cnt, s_warp);
      K = fl ? gk2 : gk;
      I = gi ? (fl ? gi2 : gi) : nullptr;
      __threadfence_block();
    }
    if (outl) {
      const uint64_t imask = ~kOutlierBit;
      for (int j = threadIdx.x; j < cnt; j += kLocalThreads) {
        uint32_t idx = (uint32_t)(K[j] & imask);
        a.outl_idx[j] = idx;
        if (perm) a.perm[lo + j] = idx;
        if (a.q_slot)
          for (uint32_t f = 0; f < d; ++f)
            a.q_slot[(uint64_t)f * a.n + lo + j] = a.q_in[(uint64_t)f * a.n + idx];
      }
      if (threadIdx.x == 0) a.seg_blocks[sg] = 0u;
      __syncthreads();
      continue;
    }
    // segmentation in rounds of one element per thread
    unsigned long long carry = 0ull;  // blocks started in earlier rounds
    for (int r0 = 0; r0 < cnt; r0 += kLocalThreads) {
      const int j = r0 + threadIdx.x;
      const bool valid = j < cnt;
      unsigned long long key = 0ull, prev = 0ull;
      bool start = false;
      if (valid) {
        key = K[j];
        if (j > 0) prev = K[j - 1];
        start = (j == 0) || ((key >> rel_bits) != (prev >> rel_bits));
      }
      unsigned long long tot;
      unsigned long long ord = block_exscan<kLocalThreads>(start ? 1ull : 0ull, s_warp, tot);
      if (valid) {
        const uint64_t g = lo + (uint64_t)j;
        const unsigned long long rel = key & rel_mask;
        unsigned long long v = (start || (g & chunk_mask) == 0) ? rel : rel - (prev & rel_mask);
        a.s_rel[g] = (uint32_t)v;
        atomicAdd(&s_hist[v < (unsigned long long)kEsc ? (uint32_t)v : (uint32_t)kEsc], 1u);
        my_max = v > my_max ? v : my_max;
        if (start) {
          const uint64_t t = lo + carry + ord;
          a.tmp_bid[t] = key >> rel_bits;
          a.tmp_pos[t] = (uint32_t)j;
        }
        if (perm) {
          uint32_t idx = I[j];
          a.perm[g] = idx;
          if (a.q_slot)
            for (uint32_t f = 0; f < d; ++f)
              a.q_slot[(uint64_t)f * a.n + g] = a.q_in[(uint64_t)f * a.n + idx];
        }
      }
      carry += tot;
    }
    if (threadIdx.x == 0) a.seg_blocks[sg] = (uint32_t)carry;
    __syncthreads();
  }
  // stream-2 histogram and max
  for (int s = threadIdx.x; s < kAlpha; s += kLocalThreads)
    if (s_hist[s]) atomicAdd(&a.hist[2 * kAlpha + s], s_hist[s]);
  atomicMax(&s_max, my_max);
  __syncthreads();
  if (threadIdx.x == 0 && s_max) atomicMax(&a.maxv[2], s_max);
}

void launch_local(const LocalArgs &a, int ctas, cudaStream_t s) {
  // keys ping-pong, radix counters, stream histogram; payload ping-pong in perm mode
  const size_t base = (size_t)kCap * 16 + 4ull * 256 * kLocalWarps + 4ull * kAlpha;
  const size_t smem = base + (a.perm ? (size_t)kCap * 8 : 0);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_local, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(base + (size_t)kCap * 8));
    attr = true;
  }
  note_launch();
  k_local<<<a.perm ? ctas / 2 : ctas, kLocalThreads, smem, s>>>(a);
}

// ---------------------------------------------------------------------------
// blocks: compact the per-segment block lists, delta code ids and counts
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_blocks_scan(const uint32_t *__restrict__ seg_blocks,
                                                      const uint32_t *__restrict__ nsegp,
                                                      unsigned long long *__restrict__ block_off,
                                                      int *__restrict__ prev_nonempty,
                                                      unsigned long long *__restrict__ mcount) {
  __shared__ unsigned long long s_warp[32];
  __shared__ int s_last[1024];
  const uint32_t nseg = *nsegp;
  const uint32_t per = (nseg + 1023) / 1024;
  const uint32_t lo = threadIdx.x * per, hi = min(nseg, lo + per);
  unsigned long long sum = 0;
  int last = -1;
  for (uint32_t i = lo; i < hi; ++i) {
    sum += seg_blocks[i];
    if (seg_blocks[i]) last = (int)i;
  }
  s_last[threadIdx.x] = last;
  unsigned long long total;
  unsigned long long run = block_exscan<1024>(sum, s_warp, total);
  __syncthreads();
  if (threadIdx.x == 0) {
    int m = -1;
    for (int t = 0; t < 1024; ++t) {
      int v = s_last[t];
      s_last[t] = m;
      if (v > m) m = v;
    }
    *mcount = total;
  }
  __syncthreads();
  int pl = s_last[threadIdx.x];
  for (uint32_t i = lo; i < hi; ++i) {
    block_off[i] = run;
    run += seg_blocks[i];
    prev_nonempty[i] = pl;
    if (seg_blocks[i]) pl = (int)i;
  }
}

__global__ void __launch_bounds__(512) k_blocks(const Plan *__restrict__ plan,
                                                const uint32_t *__restrict__ nsegp,
                                                const uint32_t *__restrict__ seg_lo,
                                                const uint32_t *__restrict__ seg_cnt,
                                                const uint32_t *__restrict__ sblocks,
                                                const unsigned long long *__restrict__ tmp_bid,
                                                const uint32_t *__restrict__ tmp_pos,
                                                const unsigned long long *__restrict__ block_off,
                                                const int *__restrict__ prev_nonempty,
                                                unsigned long long *__restrict__ s_id,
                                                unsigned long long *__restrict__ s_cnt,
                                                uint32_t *__restrict__ hist,
                                                unsigned long long *__restrict__ maxv) {
  __shared__ uint32_t h0[kAlpha], h1[kAlpha];
  __shared__ unsigned long long m0, m1;
  for (int i = threadIdx.x; i < kAlpha; i += blockDim.x) {
    h0[i] = 0u;
    h1[i] = 0u;
  }
  if (threadIdx.x == 0) {
    m0 = 0ull;
    m1 = 0ull;
  }
  __syncthreads();
  if (plan->status != OK) return;
  const uint32_t nseg = *nsegp;
  unsigned long long x0 = 0ull, x1 = 0ull;
  for (uint32_t b = blockIdx.x; b < nseg; b += gridDim.x) {
    const uint32_t mb = sblocks[b];
    if (mb == 0) continue;
    const uint64_t lo = seg_lo[b];
    const uint32_t cntb = seg_cnt[b];
    for (uint32_t t = threadIdx.x; t < mb; t += blockDim.x) {
      const unsigned long long bid = tmp_bid[lo + t];
      const uint32_t pos = tmp_pos[lo + t];
      const uint32_t end = (t + 1 < mb) ? tmp_pos[lo + t + 1] : cntb;
      const long long c = (long long)(end - pos);
      unsigned long long pbid = 0ull;
      long long pc = 0;
      if (t > 0) {
        pbid = tmp_bid[lo + t - 1];
        pc = (long long)(pos - tmp_pos[lo + t - 1]);
      } else {
        const int pb = prev_nonempty[b];
        if (pb >= 0) {
          const uint32_t pm = sblocks[pb];
          const uint64_t plo = seg_lo[pb];
          const uint32_t pcnt = seg_cnt[pb];
          pbid = tmp_bid[plo + pm - 1];
          pc = (long long)(pcnt - tmp_pos[plo + pm - 1]);
        }
      }
      const uint64_t g = block_off[b] + t;
      const unsigned long long v0 = bid - pbid;
      const unsigned long long v1 = zigzag(c - pc);
      s_id[g] = v0;
      s_cnt[g] = v1;
      atomicAdd(&h0[v0 < (unsigned long long)kEsc ? (uint32_t)v0 : (uint32_t)kEsc], 1u);
      atomicAdd(&h1[v1 < (unsigned long long)kEsc ? (uint32_t)v1 : (uint32_t)kEsc], 1u);
      x0 = v0 > x0 ? v0 : x0;
      x1 = v1 > x1 ? v1 : x1;
    }
  }
  atomicMax(&m0, x0);
  atomicMax(&m1, x1);
  __syncthreads();
  for (int i = threadIdx.x; i < kAlpha; i += blockDim.x) {
    if (h0[i]) atomicAdd(&hist[i], h0[i]);
    if (h1[i]) atomicAdd(&hist[kAlpha + i], h1[i]);
  }
  if (threadIdx.x == 0) {
    if (m0) atomicMax(&maxv[0], m0);
    if (m1) atomicMax(&maxv[1], m1);
  }
}

void launch_blocks(const Plan *plan, const uint32_t *nseg, const uint32_t *seg_lo,
                   const uint32_t *seg_cnt, const uint32_t *seg_blocks,
                   const unsigned long long *tmp_bid, const uint32_t *tmp_pos,
                   unsigned long long *block_off, int *prev_nonempty, unsigned long long *s_id,
                   unsigned long long *s_cnt, uint32_t *hist, unsigned long long *maxv,
                   unsigned long long *mcount, int ctas, cudaStream_t s) {
  note_launch();
  k_blocks_scan<<<1, 1024, 0, s>>>(seg_blocks, nseg, block_off, prev_nonempty, mcount);
  note_launch();
  k_blocks<<<ctas, 512, 0, s>>>(plan, nseg, seg_lo, seg_cnt, seg_blocks, tmp_bid, tmp_pos,
                                block_off, prev_nonempty, s_id, s_cnt, hist, maxv);
}

// value counts: ids and counts have M values, relative locations n - K
__global__ void k_counts_s(const unsigned long long *__restrict__ bucket_start, uint32_t nb,
                           uint64_t n, const unsigned long long *__restrict__ mcount,
                           unsigned long long *__restrict__ nvals,
                           unsigned long long *__restrict__ kcount) {
  const unsigned long long nbk = bucket_start[nb];
  nvals[0] = *mcount;
  nvals[1] = *mcount;
  nvals[2] = nbk;
  *kcount = n - nbk;
}

void launch_counts_s(const unsigned long long *bucket_start, uint32_t nb, uint64_t n,
                     const unsigned long long *mcount, unsigned long long *nvals,
                     unsigned long long *kcount, cudaStream_t s) {
  note_launch();
  k_counts_s<<<1, 1, 0, s>>>(bucket_start, nb, n, mcount, nvals, kcount);
}

// one CTA sorts a device-counted list of (key, payload) pairs by key
__global__ void __launch_bounds__(kLocalThreads, 1) k_sort_pairs(
    unsigned long long *keys, uint32_t *vals, unsigned long long *keys_alt, uint32_t *vals_alt,
    const unsigned long long *cntp, int kbits, unsigned long long *keys_out,
    uint32_t *vals_out) {
  __shared__ uint32_t s_cnt[256 * kLocalWarps];
  __shared__ unsigned long long s_warp[32];
  const int cnt = (int)*cntp;
  if (cnt == 0) return;
  unsigned long long *ka = keys, *kb = keys_alt;
  uint32_t *ia = vals, *ib = vals_alt;
  for (int sh = 0; sh < kbits; sh += 8) {
    radix_pass(ka, ia, kb, ib, cnt, sh, false, s_cnt, s_warp);
    unsigned long long *t = ka;
    ka = kb;
    kb = t;
    uint32_t *u = ia;
    ia = ib;
    ib = u;
  }
  for (int j = threadIdx.x; j < cnt; j += kLocalThreads) {
    keys_out[j] = ka[j];
    vals_out[j] = ia[j];
  }
}

void launch_sort_pairs(unsigned long long *keys, uint32_t *vals, unsigned long long *keys_alt,
                       uint32_t *vals_alt, const unsigned long long *cnt, int kbits,
                       unsigned long long *keys_out, uint32_t *vals_out, cudaStream_t s) {
  note_launch();
  k_sort_pairs<<<1, kLocalThreads, 0, s>>>(keys, vals, keys_alt, vals_alt, cnt, kbits, keys_out,
                                           vals_out);
}

}  // namespace lcp
