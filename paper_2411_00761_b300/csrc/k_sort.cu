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
#include <type_traits>

#include "lcp_kernels.h"

namespace lcp {

constexpr int kLocalThreads = 256;
constexpr int kLocalWarps = kLocalThreads / 32;
constexpr int kCap = kUnitCap;  // keys of a unit sorted in shared memory
constexpr int kSubBits = 10;    // level-2 split of oversized buckets
constexpr int kSplitThreads = 512;
constexpr int kSplitIlp = 4;    // keys in flight per thread in the split passes

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
// block crosses a sub-bucket).  Sort units: the ordered list of key ranges
// that k_local sorts -- consecutive small level-1 buckets merged greedily up
// to kCap keys, runs of consecutive sub-buckets of a split bucket, and the
// outlier bucket.  A split bucket's units start at every sub-bucket whose
// offset enters a new span of kCap/2 slots, so a unit holds fewer than
// kCap/2 keys plus its last sub-bucket.
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
  if (threadIdx.x == 0) {
    nbig[0] = (uint32_t)tot;
    nbig[1] = 0u;  // work counter of k_split_big
  }
}

// One CTA per split bucket (fetched from a work counter): sub-bucket
// histogram, offsets, unit starts (unit_off[j][u], offsets within the
// bucket), then the scatter.  Loads are issued kSplitIlp at a time.
__global__ void __launch_bounds__(kSplitThreads) k_split_big(
    const Plan *__restrict__ plan, const unsigned long long *__restrict__ bstart,
    const uint32_t *__restrict__ big_list, uint32_t *__restrict__ nbig,
    const unsigned long long *__restrict__ keys, const uint32_t *__restrict__ idx,
    unsigned long long *__restrict__ keys_out, uint32_t *__restrict__ idx_out,
    uint32_t *__restrict__ unit_off, uint32_t *__restrict__ big_units) {
  constexpr int kSub = 1 << kSubBits;
  constexpr int per = kSub / kSplitThreads;
  __shared__ uint32_t h[kSub];
  __shared__ unsigned long long s_warp[32];
  __shared__ uint32_t s_j;
  const Plan &P = *plan;
  const int sub = min(kSubBits, (int)P.part_shift - (int)P.rel_bits);
  const int shift2 = (int)P.part_shift - sub;
  const uint32_t mask = (1u << sub) - 1u;
  const uint32_t nsub = 1u << sub;
  const uint32_t total_big = nbig[0];
  const uint32_t G = (uint32_t)kCap / 2;
  for (;;) {
    if (threadIdx.x == 0) s_j = atomicAdd(&nbig[1], 1u);
    for (int d = threadIdx.x; d < kSub; d += kSplitThreads) h[d] = 0u;
    __syncthreads();
    const uint32_t j = s_j;
    if (j >= total_big) break;
    const uint32_t b = big_list[j];
    const uint64_t lo = bstart[b];
    const uint32_t cnt = (uint32_t)(bstart[b + 1] - lo);
    const unsigned long long *kb = keys + lo;
    for (uint32_t t0 = 0; t0 < cnt; t0 += kSplitThreads * kSplitIlp) {
      unsigned long long k[kSplitIlp];
#pragma unroll
      for (int r = 0; r < kSplitIlp; ++r) {
        const uint32_t t = t0 + r * kSplitThreads + threadIdx.x;
        k[r] = t < cnt ? kb[t] : 0ull;
      }
#pragma unroll
      for (int r = 0; r < kSplitIlp; ++r) {
        const uint32_t t = t0 + r * kSplitThreads + threadIdx.x;
        if (t < cnt) atomicAdd(&h[(uint32_t)(k[r] >> shift2) & mask], 1u);
      }
    }
    __syncthreads();
    // offsets and unit starts; thread t owns sub-buckets t*per .. t*per+per-1
    uint32_t c[per], off[per];
    unsigned long long sum = 0;
#pragma unroll
    for (int q = 0; q < per; ++q) {
      const uint32_t dg = threadIdx.x * per + q;
      c[q] = dg < nsub ? h[dg] : 0u;
      sum += c[q];
    }
    unsigned long long tot;
    uint32_t run = (uint32_t)block_exscan<kSplitThreads>(sum, s_warp, tot);
#pragma unroll
    for (int q = 0; q < per; ++q) {
      off[q] = run;
      run += c[q];
    }
    // the offset of the sub-bucket before this thread's first one
    __syncthreads();
    if (threadIdx.x * per + per - 1 < (uint32_t)kSub) h[threadIdx.x * per + per - 1] = off[per - 1];
    __syncthreads();
    const uint32_t prev0 = threadIdx.x > 0 ? h[threadIdx.x * per - 1] : 0u;
    uint32_t ncut = 0;
    bool cut[per];
#pragma unroll
    for (int q = 0; q < per; ++q) {
      const uint32_t dg = threadIdx.x * per + q;
      const uint32_t pv = q ? off[q - 1] : prev0;
      cut[q] = dg < nsub && off[q] < cnt && (dg == 0 || off[q] / G != pv / G);
      ncut += cut[q];
    }
    __syncthreads();
    unsigned long long nunits;
    uint32_t uo = (uint32_t)block_exscan<kSplitThreads>(ncut, s_warp, nunits);
    uint32_t *uj = unit_off + (uint64_t)j * kSub;
#pragma unroll
    for (int q = 0; q < per; ++q)
      if (cut[q]) uj[uo++] = off[q];
    if (threadIdx.x == 0) big_units[j] = (uint32_t)nunits;
#pragma unroll
    for (int q = 0; q < per; ++q) {
      const uint32_t dg = threadIdx.x * per + q;
      if (dg < nsub) h[dg] = off[q];
    }
    __syncthreads();
    for (uint32_t t0 = 0; t0 < cnt; t0 += kSplitThreads * kSplitIlp) {
      unsigned long long k[kSplitIlp];
      uint32_t ix[kSplitIlp];
#pragma unroll
      for (int r = 0; r < kSplitIlp; ++r) {
        const uint32_t t = t0 + r * kSplitThreads + threadIdx.x;
        k[r] = t < cnt ? kb[t] : 0ull;
        ix[r] = (idx_out && t < cnt) ? idx[lo + t] : 0u;
      }
#pragma unroll
      for (int r = 0; r < kSplitIlp; ++r) {
        const uint32_t t = t0 + r * kSplitThreads + threadIdx.x;
        if (t < cnt) {
          const uint32_t pos = atomicAdd(&h[(uint32_t)(k[r] >> shift2) & mask], 1u);
          keys_out[lo + pos] = k[r];
          if (idx_out) idx_out[lo + pos] = ix[r];
        }
      }
    }
    __syncthreads();
  }
}

// Unit list (one CTA).  Thread t owns buckets [t*per, (t+1)*per); within that
// range consecutive small buckets merge greedily up to kCap keys (a single
// bucket above kCap that cannot be split forms its own unit); a split bucket
// contributes its units, written by k_units_big at big_base[j]; the outlier
// bucket is a unit of its own.
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

// units of the split buckets: one warp per bucket, lanes over its units
__global__ void k_units_big(const unsigned long long *__restrict__ bstart,
                            const uint32_t *__restrict__ big_list,
                            const uint32_t *__restrict__ nbig,
                            const uint32_t *__restrict__ unit_off,
                            const uint32_t *__restrict__ big_units,
                            const uint32_t *__restrict__ big_base, uint32_t *__restrict__ u_lo,
                            uint32_t *__restrict__ u_cnt, uint32_t *__restrict__ u_meta) {
  const int lane = threadIdx.x & 31;
  const uint32_t warps = gridDim.x * (blockDim.x >> 5);
  for (uint32_t j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); j < nbig[0]; j += warps) {
    const uint32_t b = big_list[j];
    const uint64_t lo = bstart[b];
    const uint32_t cnt = (uint32_t)(bstart[b + 1] - lo);
    const uint32_t nu = big_units[j], o = big_base[j];
    const uint32_t *uj = unit_off + (uint64_t)j * (1u << kSubBits);
    for (uint32_t u = lane; u < nu; u += 32) {
      const uint32_t a = uj[u], e = u + 1 < nu ? uj[u + 1] : cnt;
      u_lo[o + u] = (uint32_t)(lo + a);
      u_cnt[o + u] = e - a;
      u_meta[o + u] = 1u;  // keys in the level-2 buffer
    }
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
  k_split_big<<<4 * sms, kSplitThreads, 0, s>>>(plan, bstart, big_list, nbig, keys, idx, keys_alt,
                                                idx_alt, sub_cnt, big_units);
  note_launch();
  k_units_small<<<1, 1024, 0, s>>>(nb1, bstart, big_of, big_units, big_base, u_lo, u_cnt, u_meta,
                                   nunit);
  note_launch();
  k_units_big<<<sms, 256, 0, s>>>(bstart, big_list, nbig, sub_cnt, big_units, big_base, u_lo,
                                  u_cnt, u_meta);
}

// ---------------------------------------------------------------------------
// warp bitonic sort of 32*R elements, R per lane in blocked order (lane L
// holds elements L*R .. L*R+R-1), ascending.  Stages that pair lanes run in
// a loop (one shuffle per element); stages inside a lane are unrolled.
// Element types: 32-bit keys, 64-bit keys (or a 32-bit key above a 32-bit
// index), and (key, index) pairs ordered by key, then index.
// ---------------------------------------------------------------------------
struct KeyIdx {
  unsigned long long k;
  uint32_t i;
};
__device__ __forceinline__ bool key_lt(uint32_t a, uint32_t b) { return a < b; }
__device__ __forceinline__ bool key_lt(unsigned long long a, unsigned long long b) { return a < b; }
__device__ __forceinline__ bool key_lt(const KeyIdx &a, const KeyIdx &b) {
  return a.k < b.k || (a.k == b.k && a.i < b.i);
}
__device__ __forceinline__ uint32_t shfl_x(uint32_t v, int m) {
  return __shfl_xor_sync(0xffffffffu, v, m);
}
__device__ __forceinline__ unsigned long long shfl_x(unsigned long long v, int m) {
  return __shfl_xor_sync(0xffffffffu, v, m);
}
__device__ __forceinline__ KeyIdx shfl_x(const KeyIdx &v, int m) {
  return KeyIdx{shfl_x(v.k, m), shfl_x(v.i, m)};
}

template <int R, typename T>
__device__ __forceinline__ void warp_bitonic(T (&v)[R]) {
  const uint32_t lane = threadIdx.x & 31;
#pragma unroll 1
  for (uint32_t k = 2; k <= 32u * R; k <<= 1) {
    if (k > (uint32_t)R) {
      // element i = lane*R + r sorts up when bit k of i is clear; for k > R
      // that bit is bit k/R of the lane
      const bool up = (lane & (k / R)) == 0;
#pragma unroll 1
      for (uint32_t lj = k / (2 * R); lj >= 1; lj >>= 1) {
        const bool keep_max = ((lane & lj) == 0) != up;
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const T o = shfl_x(v[r], (int)lj);
          if (key_lt(o, v[r]) != keep_max) v[r] = o;
        }
      }
    }
#pragma unroll
    for (int j = R / 2; j >= 1; j >>= 1) {
      if ((uint32_t)j < k) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const int p = r ^ j;
          if (p > r) {
            const bool up = ((lane * R + r) & k) == 0;
            if (key_lt(v[p], v[r]) == up) {
              const T t = v[r];
              v[r] = v[p];
              v[p] = t;
            }
          }
        }
      }
    }
  }
}

// Window element forms: 0 the key minus the window base, 32 bits; 1 the
// 64-bit key; 2 the 32-bit form 0 above the 32-bit index; 3 (key, index).
template <int MODE>
struct WinElem {
  using T = typename std::conditional<
      MODE == 0, uint32_t,
      typename std::conditional<MODE == 3, KeyIdx, unsigned long long>::type>::type;
};

template <int MODE>
__device__ __forceinline__ typename WinElem<MODE>::T win_load(const unsigned long long *sk,
                                                              const uint32_t *si, int j,
                                                              unsigned long long base) {
  if constexpr (MODE == 0) return (uint32_t)(sk[j] - base);
  else if constexpr (MODE == 1) return sk[j];
  else if constexpr (MODE == 2) return ((sk[j] - base) << 32) | (unsigned long long)si[j];
  else return KeyIdx{sk[j], si[j]};
}
template <int MODE>
__device__ __forceinline__ typename WinElem<MODE>::T win_pad() {
  if constexpr (MODE == 0) return 0xffffffffu;
  else if constexpr (MODE == 3) return KeyIdx{~0ull, 0xffffffffu};
  else return ~0ull;
}
template <int MODE>
__device__ __forceinline__ void win_store(unsigned long long *sk, uint32_t *si, int j,
                                          const typename WinElem<MODE>::T &v,
                                          unsigned long long base) {
  if constexpr (MODE == 0) {
    sk[j] = base + v;
  } else if constexpr (MODE == 1) {
    sk[j] = v;
  } else if constexpr (MODE == 2) {
    sk[j] = base + (v >> 32);
    si[j] = (uint32_t)v;
  } else {
    sk[j] = v.k;
    si[j] = v.i;
  }
}

template <int R, int MODE>
__device__ __forceinline__ void sort_window_r(unsigned long long *sk, uint32_t *si, int w0, int c,
                                              unsigned long long base) {
  using T = typename WinElem<MODE>::T;
  const int lane = threadIdx.x & 31;
  T v[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int i = lane * R + r;
    v[r] = i < c ? win_load<MODE>(sk, si, w0 + i, base) : win_pad<MODE>();
  }
  warp_bitonic<R>(v);
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int i = lane * R + r;
    if (i < c) win_store<MODE>(sk, si, w0 + i, v[r], base);
  }
}

// largest window one warp sorts in registers
__device__ __forceinline__ int window_cap(int mode) { return mode == 3 ? 256 : 512; }

template <int MODE>
__device__ __noinline__ void sort_window(unsigned long long *sk, uint32_t *si, int w0, int c,
                                         unsigned long long base) {
  if (c <= 32) sort_window_r<1, MODE>(sk, si, w0, c, base);
  else if (c <= 64) sort_window_r<2, MODE>(sk, si, w0, c, base);
  else if (c <= 128) sort_window_r<4, MODE>(sk, si, w0, c, base);
  else if (c <= 256) sort_window_r<8, MODE>(sk, si, w0, c, base);
  else if constexpr (MODE != 3) sort_window_r<16, MODE>(sk, si, w0, c, base);
}

// ---------------------------------------------------------------------------
// per-unit sort + segmentation into blocks (persistent over units).
//
// A unit of up to kCap keys is sorted in shared memory: the keys are loaded
// into registers, partitioned by their top 8 varying bits (one counting
// pass, no order needed inside a digit group), and the digit groups are
// gathered into windows (consecutive groups whose starts share a span of
// kWinSpan slots) that one warp sorts in registers with a bitonic network,
// on 32-bit offsets from the window's base key when its key span allows.
// Windows too large for a warp (a digit group of hundreds of keys) fall back
// to the CTA radix sort.  Sorting each window sorts the unit because the
// windows are ordered by digit.
// ---------------------------------------------------------------------------
constexpr int kPer = kCap / kLocalThreads;  // keys per thread of a unit
constexpr int kWinSpan = 32;
constexpr int kMaxWin = kCap / kWinSpan + 2;

template <bool PERM>
__global__ void __launch_bounds__(kLocalThreads, 4) k_local(LocalArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned long long *sk = reinterpret_cast<unsigned long long *>(smem);  // kCap
  uint32_t *s_cnt = reinterpret_cast<uint32_t *>(sk + kCap);              // 256 * warps
  uint32_t *s_hist = s_cnt + 256 * kLocalWarps;                            // kAlpha
  uint32_t *si = PERM ? s_hist + kAlpha : nullptr;                         // kCap
  __shared__ unsigned long long s_warp[32];
  __shared__ unsigned long long s_max, s_kmin, s_kmax;
  __shared__ uint32_t s_cur[256];
  __shared__ uint32_t s_win[kMaxWin];
  __shared__ uint8_t s_wdg[kMaxWin];
  __shared__ uint32_t s_nwin;
  __shared__ uint32_t s_wcnt[kLocalWarps];
  __shared__ uint32_t s_status;
  __shared__ uint32_t s_relb;
  __shared__ uint32_t s_nseg;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    s_status = (uint32_t)a.plan->status;
    s_relb = a.plan->rel_bits;
    s_nseg = *a.nseg;
    s_max = 0ull;
  }
  for (int b = threadIdx.x; b < kAlpha; b += kLocalThreads) s_hist[b] = 0u;
  __syncthreads();
  if ((int)s_status != OK) return;
  const uint32_t rel_bits = s_relb;
  const unsigned long long rel_mask = rel_bits >= 64 ? ~0ull : ((1ull << rel_bits) - 1ull);
  const uint64_t chunk_mask = (1ull << a.log2_chunk) - 1ull;
  const int ibits = PERM ? (int)bitlen64(a.n > 0 ? a.n - 1 : 0) : 0;
  const uint32_t d = a.plan->d;
  const uint32_t nseg = s_nseg;
  const uint32_t lt = lanemask_lt();
  unsigned long long my_max = 0ull;

  for (uint32_t sg = blockIdx.x; sg < nseg; sg += gridDim.x) {
    const uint64_t lo = a.seg_lo[sg];
    const int cnt = (int)a.seg_cnt[sg];
    const uint32_t meta = a.seg_meta[sg];
    const bool outl = (meta >> 1) & 1u;
    const bool src_alt = meta & 1u;
    const bool use_idx = PERM && !outl;
    unsigned long long *gk = (src_alt ? a.keys_alt : a.keys) + lo;
    unsigned long long *gk2 = (src_alt ? a.keys : a.keys_alt) + lo;
    uint32_t *gi = nullptr, *gi2 = nullptr;
    if (use_idx) {
      gi = (src_alt ? a.idx_alt : a.idx) + lo;
      gi2 = (src_alt ? a.idx : a.idx_alt) + lo;
    }
    if (threadIdx.x == 0) {
      s_kmin = ~0ull;
      s_kmax = 0ull;
    }
    for (int g = threadIdx.x; g < 256; g += kLocalThreads) s_cur[g] = 0u;
    __syncthreads();
    const unsigned long long *K;
    const uint32_t *I = nullptr;
    if (cnt <= kCap) {
      unsigned long long kr[kPer];
      uint32_t ir[kPer];
      unsigned long long mn = ~0ull, mx = 0ull;
#pragma unroll
      for (int r = 0; r < kPer; ++r) {
        const int j = r * kLocalThreads + threadIdx.x;
        kr[r] = 0ull;
        ir[r] = 0u;
        if (j < cnt) {
          kr[r] = gk[j];
          if (PERM && use_idx) ir[r] = gi[j];
          mn = kr[r] < mn ? kr[r] : mn;
          mx = kr[r] > mx ? kr[r] : mx;
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long a1 = __shfl_xor_sync(0xffffffffu, mn, o);
        const unsigned long long b1 = __shfl_xor_sync(0xffffffffu, mx, o);
        mn = a1 < mn ? a1 : mn;
        mx = b1 > mx ? b1 : mx;
      }
      if (lane == 0) {
        atomicMin(&s_kmin, mn);
        atomicMax(&s_kmax, mx);
      }
      __syncthreads();
      const unsigned long long kmin = s_kmin, kmax = s_kmax;
      const int kbits = (int)bitlen64(kmin ^ kmax);
      const int sh = kbits > 8 ? kbits - 8 : 0;
      // digit histogram (one shared atomic per run of equal digits in a warp)
      uint32_t peers[kPer];
#pragma unroll
      for (int r = 0; r < kPer; ++r) {
        const int j = r * kLocalThreads + threadIdx.x;
        const bool valid = j < cnt;
        const uint32_t dg = valid ? (uint32_t)(kr[r] >> sh) & 255u : 256u + lane;
        peers[r] = __match_any_sync(0xffffffffu, dg);
        if (valid && lane == __ffs(peers[r]) - 1) atomicAdd(&s_cur[dg], __popc(peers[r]));
      }
      __syncthreads();
      // group offsets (cursors) and windows, warp 0: lane L owns digits 8L..8L+7
      if (warp == 0) {
        uint32_t offs[8], sum = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          offs[k] = s_cur[lane * 8 + k];
          sum += offs[k];
        }
        uint32_t incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= o) incl += y;
        }
        uint32_t run = incl - sum;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const uint32_t c = offs[k];
          offs[k] = run;
          s_cur[lane * 8 + k] = run;
          run += c;
        }
        const uint32_t p7 = __shfl_up_sync(0xffffffffu, offs[7], 1);
        uint32_t cutm = 0u;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const uint32_t prev = k ? offs[k - 1] : p7;
          const bool first = lane == 0 && k == 0;
          const bool cut = offs[k] < (uint32_t)cnt &&
                           (first || offs[k] / kWinSpan != prev / kWinSpan);
          cutm |= (cut ? 1u : 0u) << k;
        }
        const uint32_t nc = __popc(cutm);
        uint32_t ci = nc;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t y = __shfl_up_sync(0xffffffffu, ci, o);
          if (lane >= o) ci += y;
        }
        uint32_t wpos = ci - nc;
#pragma unroll
        for (int k = 0; k < 8; ++k)
          if ((cutm >> k) & 1u) {
            s_win[wpos] = offs[k];
            s_wdg[wpos] = (uint8_t)(lane * 8 + k);
            ++wpos;
          }
        if (lane == 31) {
          s_nwin = ci;
          s_win[ci] = (uint32_t)cnt;
        }
      }
      __syncthreads();
      // scatter into digit order
#pragma unroll
      for (int r = 0; r < kPer; ++r) {
        const int j = r * kLocalThreads + threadIdx.x;
        const bool valid = j < cnt;
        const uint32_t dg = (uint32_t)(kr[r] >> sh) & 255u;
        const int leader = __ffs(peers[r]) - 1;
        uint32_t base = 0u;
        if (valid && lane == leader) base = atomicAdd(&s_cur[dg], __popc(peers[r]));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (valid) {
          const uint32_t pos = base + __popc(peers[r] & lt);
          sk[pos] = kr[r];
          if (PERM && use_idx) si[pos] = ir[r];
        }
      }
      __syncthreads();
      // windows, one warp each: keys of the window w lie in
      // [top | g0 << sh, top | g1 << sh) for its first and end digits g0, g1
      const uint32_t nwin = s_nwin;
      const unsigned long long top = sh + 8 >= 64 ? 0ull : (kmin >> (sh + 8)) << (sh + 8);
      const uint32_t gend = (uint32_t)((kmax >> sh) & 255ull) + 1u;
      const int wide_mode = use_idx ? 3 : 1;
      for (uint32_t wi = warp; wi < nwin; wi += kLocalWarps) {
        const int w0 = (int)s_win[wi], c = (int)s_win[wi + 1] - w0;
        if (c < 2) continue;
        const uint32_t g0 = s_wdg[wi], g1 = wi + 1 < nwin ? s_wdg[wi + 1] : gend;
        const unsigned long long base = top | ((unsigned long long)g0 << sh);
        const bool narrow = ((unsigned long long)(g1 - g0) << sh) <= (1ull << 32);
        const int mode = narrow ? (use_idx ? 2 : 0) : wide_mode;
        if (c > window_cap(mode)) continue;
        if (mode == 0) {
          sort_window<0>(sk, si, w0, c, base);
        } else if (mode == 1) {
          sort_window<1>(sk, si, w0, c, base);
        } else {
          if constexpr (PERM) {
            if (mode == 2) sort_window<2>(sk, si, w0, c, base);
            else sort_window<3>(sk, si, w0, c, base);
          }
        }
      }
      __syncthreads();
      // windows too large for a warp: CTA radix sort, scratch in global memory
      for (uint32_t wi = 0; wi < nwin; ++wi) {
        const int w0 = (int)s_win[wi], c = (int)s_win[wi + 1] - w0;
        const uint32_t g0 = s_wdg[wi], g1 = wi + 1 < nwin ? s_wdg[wi + 1] : gend;
        const bool narrow = ((unsigned long long)(g1 - g0) << sh) <= (1ull << 32);
        const int mode = narrow ? (use_idx ? 2 : 0) : wide_mode;
        if (c <= window_cap(mode)) continue;
        const int fl = cta_sort(sk + w0, use_idx ? si + w0 : nullptr, gk2 + w0,
                                use_idx ? gi2 + w0 : nullptr, c, kbits, use_idx ? ibits : 0,
                                s_cnt, s_warp);
        if (fl) {
          for (int j = threadIdx.x; j < c; j += kLocalThreads) {
            sk[w0 + j] = gk2[w0 + j];
            if (use_idx) si[w0 + j] = gi2[w0 + j];
          }
        }
        __syncthreads();
      }
      K = sk;
      I = use_idx ? si : nullptr;
    } else {
      // beyond shared memory: CTA radix sort in global memory
      unsigned long long mn = ~0ull, mx = 0ull;
      for (int j = threadIdx.x; j < cnt; j += kLocalThreads) {
        const unsigned long long v = gk[j];
        mn = v < mn ? v : mn;
        mx = v > mx ? v : mx;
      }
      atomicMin(&s_kmin, mn);
      atomicMax(&s_kmax, mx);
      __syncthreads();
      const int kbits = (int)bitlen64(s_kmin ^ s_kmax);
      const int fl = cta_sort(gk, gi, gk2, gi2, cnt, kbits, use_idx ? ibits : 0, s_cnt, s_warp);
      K = fl ? gk2 : gk;
      I = use_idx ? (fl ? gi2 : gi) : nullptr;
    }
    if (outl) {
      const uint64_t imask = ~kOutlierBit;
      for (int j = threadIdx.x; j < cnt; j += kLocalThreads) {
        uint32_t idx = (uint32_t)(K[j] & imask);
        a.outl_idx[j] = idx;
        if (PERM) a.perm[lo + j] = idx;
        if (a.q_slot)
          for (uint32_t f = 0; f < d; ++f)
            a.q_slot[(uint64_t)f * a.n + lo + j] = a.q_in[(uint64_t)f * a.n + idx];
      }
      if (threadIdx.x == 0) a.seg_blocks[sg] = 0u;
      __syncthreads();
      continue;
    }
    // segmentation: warp w owns positions [w*S, (w+1)*S), S a multiple of 32
    const int S = (cnt + kLocalWarps * 32 - 1) / (kLocalWarps * 32) * 32;
    const int wlo = min(cnt, warp * S), whi = min(cnt, wlo + S);
    uint32_t nstart = 0u;
    for (int j0 = wlo; j0 < whi; j0 += 32) {
      const int j = j0 + lane;
      bool start = false;
      if (j < whi) start = j == 0 || (K[j] >> rel_bits) != (K[j - 1] >> rel_bits);
      nstart += __popc(__ballot_sync(0xffffffffu, start));
    }
    if (lane == 0) s_wcnt[warp] = nstart;
    __syncthreads();
    uint32_t run = 0u, total = 0u;
#pragma unroll
    for (int w2 = 0; w2 < kLocalWarps; ++w2) {
      const uint32_t v = s_wcnt[w2];
      run += w2 < warp ? v : 0u;
      total += v;
    }
    for (int j0 = wlo; j0 < whi; j0 += 32) {
      const int j = j0 + lane;
      const bool valid = j < whi;
      unsigned long long key = 0ull, prev = 0ull;
      bool start = false;
      if (valid) {
        key = K[j];
        if (j > 0) prev = K[j - 1];
        start = j == 0 || (key >> rel_bits) != (prev >> rel_bits);
      }
      const uint32_t bal = __ballot_sync(0xffffffffu, start);
      unsigned long long v = 0ull;
      if (valid) {
        const uint64_t g = lo + (uint64_t)j;
        const unsigned long long rel = key & rel_mask;
        v = (start || (g & chunk_mask) == 0) ? rel : rel - (prev & rel_mask);
        a.s_rel[g] = (uint32_t)v;
        my_max = v > my_max ? v : my_max;
        if (start) {
          const uint64_t t = lo + run + __popc(bal & lt);
          a.tmp_bid[t] = key >> rel_bits;
          a.tmp_pos[t] = (uint32_t)j;
        }
        if (PERM) {
          const uint32_t idx = I[j];
          a.perm[g] = idx;
          if (a.q_slot)
            for (uint32_t f = 0; f < d; ++f)
              a.q_slot[(uint64_t)f * a.n + g] = a.q_in[(uint64_t)f * a.n + idx];
        }
      }
      // stream-2 histogram: escapes counted per warp, other values per lane
      const bool esc = valid && v >= (unsigned long long)kEsc;
      const uint32_t nesc = __popc(__ballot_sync(0xffffffffu, esc));
      if (lane == 0 && nesc) atomicAdd(&s_hist[kEsc], nesc);
      if (valid && !esc) atomicAdd(&s_hist[(uint32_t)v], 1u);
      run += __popc(bal);
    }
    if (threadIdx.x == 0) a.seg_blocks[sg] = total;
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
  // unit keys, fallback radix counters, stream histogram; unit indices in perm mode
  const size_t base = (size_t)kCap * 8 + 4ull * 256 * kLocalWarps + 4ull * kAlpha;
  const size_t smem = base + (a.perm ? (size_t)kCap * 4 : 0);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_local<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)base);
    cudaFuncSetAttribute(k_local<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(base + (size_t)kCap * 4));
    attr = true;
  }
  note_launch();
  if (a.perm) k_local<true><<<ctas, kLocalThreads, smem, s>>>(a);
  else k_local<false><<<ctas, kLocalThreads, smem, s>>>(a);
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
