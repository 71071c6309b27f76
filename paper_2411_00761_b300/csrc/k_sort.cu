// k_sort.cu -- partition by the key's top bits, sorting, segmentation.
//
// Sec. "Design of spatial blocks": the non-empty blocks are kept in id order
// with their particle counts and the particles' locations relative to the
// block corner; Sec. "Block coding": each array is delta coded.  The keys
// (block_id * p^d + rel) are sorted most-significant digit first: one
// partition pass into buckets of consecutive block ids; buckets above
// kSplitMin keys are partitioned again by the next block-id bits into
// sub-buckets, and runs of sub-buckets are sorted by one warp each in
// registers; small buckets are merged into units that one CTA sorts in
// shared memory.  Every sorted run starts at a block boundary, so it is
// segmented where it is sorted: a start flag and the block id at each
// block's first particle, the relative-location deltas for every particle.
// A scan of the start flags then numbers the blocks.  The output bytes
// depend only on the multiset of keys, so no partition pass needs a stable
// order.
#include <algorithm>
#include <type_traits>

#include "lcp_kernels.h"

namespace lcp {

constexpr int kLocalThreads = 256;
constexpr int kLocalWarps = kLocalThreads / 32;
constexpr int kCap = kUnitCap;  // keys of a unit sorted in shared memory
constexpr int kSplitMin = 256;  // buckets above this many keys are split again
constexpr int kSubMinBits = 5;  // level-2 digit width: about 8 keys per sub-bucket,
constexpr int kSubMaxBits = 13; // within these bounds
constexpr int kSubMax = 1 << kSubMaxBits;
constexpr int kSplitThreads = 512;
constexpr int kSplitIlp = 4;    // keys in flight per thread in the split passes
constexpr uint32_t kSplitChunk = 16384;  // keys per task (staged in shared memory by k_split_big)
constexpr int kStageThreads = 1024;      // k_split_big: 16 staged keys per thread
constexpr int kSubThreads = 256;
constexpr int kSubCtas = 5;     // resident k_subsort CTAs per SM (48 registers)


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

// exclusive scan of n values (one CTA); out[n] = total.  Tiles of
// kScanTileS values, kScanPer consecutive values per thread read with 16-byte
// loads (all of a tile's loads in flight at once), so a 2^17-value scan takes
// eight tiles.
constexpr int kScanPer = 16;
constexpr int kScanTileS = 1024 * kScanPer;

// one tile's exclusive scan with carry-in; returns the tile's total
__device__ __forceinline__ unsigned long long scan_tile(const unsigned long long *__restrict__ in,
                                                        uint64_t n, uint64_t base,
                                                        unsigned long long carry,
                                                        unsigned long long *__restrict__ out,
                                                        unsigned long long *s_warp, bool vec) {
  const uint64_t i0 = base + (uint64_t)threadIdx.x * kScanPer;
  unsigned long long v[kScanPer];
  if (vec && i0 + kScanPer <= n) {
#pragma unroll
    for (int j = 0; j < kScanPer; j += 2) {
      const ulonglong2 x = *reinterpret_cast<const ulonglong2 *>(in + i0 + j);
      v[j] = x.x;
      v[j + 1] = x.y;
    }
  } else {
#pragma unroll
    for (int j = 0; j < kScanPer; ++j) v[j] = i0 + j < n ? in[i0 + j] : 0ull;
  }
  unsigned long long sum = 0;
#pragma unroll
  for (int j = 0; j < kScanPer; ++j) sum += v[j];
  unsigned long long total;
  unsigned long long run = carry + block_exscan<1024>(sum, s_warp, total);
  if (!out) return total;
  if (vec && i0 + kScanPer <= n) {
#pragma unroll
    for (int j = 0; j < kScanPer; j += 2) {
      const unsigned long long a = run;
      run += v[j];
      *reinterpret_cast<ulonglong2 *>(out + i0 + j) = make_ulonglong2(a, run);
      run += v[j + 1];
    }
  } else {
#pragma unroll
    for (int j = 0; j < kScanPer; ++j) {
      if (i0 + j < n) out[i0 + j] = run;
      run += v[j];
    }
  }
  return total;
}

__global__ void __launch_bounds__(1024) k_scan_small(const unsigned long long *__restrict__ in,
                                                     uint32_t n,
                                                     unsigned long long *__restrict__ out,
                                                     const uint32_t *__restrict__ gate) {
  __shared__ unsigned long long s_warp[32];
  if (gate && *gate != 1u) return;  // the stream this scan serves is not Huffman coded
  const bool vec = ((((uintptr_t)in) | ((uintptr_t)out)) & 15u) == 0;
  unsigned long long carry = 0;
  for (uint64_t base = 0; base < n; base += kScanTileS)
    carry += scan_tile(in, n, base, carry, out, s_warp, vec);
  if (threadIdx.x == 0) out[n] = carry;
}

// longer scans: tile totals (one CTA per tile), their scan, then every tile
// again from its offset
__global__ void __launch_bounds__(1024) k_scan_tiles(const unsigned long long *__restrict__ in,
                                                     uint32_t n,
                                                     const unsigned long long *__restrict__ offs,
                                                     unsigned long long *__restrict__ out,
                                                     const uint32_t *__restrict__ gate) {
  __shared__ unsigned long long s_warp[32];
  if (gate && *gate != 1u) return;
  const bool vec = ((((uintptr_t)in) | ((uintptr_t)out)) & 15u) == 0;
  const uint64_t base = (uint64_t)blockIdx.x * kScanTileS;
  if (!offs) {  // totals
    const unsigned long long t = scan_tile(in, n, base, 0ull, nullptr, s_warp, vec);
    if (threadIdx.x == 0) out[blockIdx.x] = t;
  } else {
    scan_tile(in, n, base, offs[blockIdx.x], out, s_warp, vec);
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = offs[gridDim.x];
  }
}

// per bucket, the running offset over the tiles (eight tiles' counts loaded
// at a time)
__global__ void k_bucket_tileoff(uint32_t *__restrict__ tile_hist, int tiles, uint32_t nb1,
                                 const unsigned long long *__restrict__ bucket_start) {
  uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb1) return;
  uint32_t run = (uint32_t)bucket_start[b];
  for (int t0 = 0; t0 < tiles; t0 += 8) {
    uint32_t v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j)
      v[j] = t0 + j < tiles ? tile_hist[(uint64_t)(t0 + j) * nb1 + b] : 0u;
#pragma unroll
    for (int j = 0; j < 8; ++j)
      if (t0 + j < tiles) {
        tile_hist[(uint64_t)(t0 + j) * nb1 + b] = run;
        run += v[j];
      }
  }
}

void launch_bucket_offsets(uint32_t *tile_hist, int tiles, uint32_t nb1,
                           unsigned long long *bucket_start, unsigned long long *totals,
                           cudaStream_t s) {
  unsigned g = (nb1 + 255) / 256;
  note_launch();
  k_bucket_colsum<<<g, 256, 0, s>>>(tile_hist, tiles, nb1, totals);
  note_launch();
  k_scan_small<<<1, 1024, 0, s>>>(totals, nb1, bucket_start, nullptr);
  note_launch();
  k_bucket_tileoff<<<g, 256, 0, s>>>(tile_hist, tiles, nb1, bucket_start);
}

void launch_scan_small(const unsigned long long *in, uint32_t n, unsigned long long *out,
                       cudaStream_t s, const uint32_t *gate, unsigned long long *tmp) {
  const uint32_t tiles = (uint32_t)(((uint64_t)n + kScanTileS - 1) / kScanTileS);
  if (!tmp || tiles <= 1) {
    note_launch();
    k_scan_small<<<1, 1024, 0, s>>>(in, n, out, gate);
    return;
  }
  unsigned long long *tot = tmp, *offs = tmp + tiles + 1;  // scan_tmp_len(n) entries
  note_launch();
  k_scan_tiles<<<tiles, 1024, 0, s>>>(in, n, nullptr, tot, gate);
  note_launch();
  k_scan_small<<<1, 1024, 0, s>>>(tot, tiles, offs, gate);
  note_launch();
  k_scan_tiles<<<tiles, 1024, 0, s>>>(in, n, offs, out, gate);
}

uint64_t scan_tmp_len(uint64_t n) { return 2 * ((n + kScanTileS - 1) / kScanTileS + 2); }

// ---------------------------------------------------------------------------
// scatter: same tiles as the quantize pass; shared-memory cursors per bucket.
// One launch serves the buckets [blo, bhi) only: every 8-byte key write
// opens or extends a partially written 32-byte sector at its bucket's write
// front in this tile, and all tiles x buckets fronts of a frame exceed L2 at
// 64M keys, so partial sectors would be evicted and rewritten.  Passes over
// bucket ranges keep each pass's fronts L2-resident; keys outside the range
// are read and skipped.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(512) k_scatter(const unsigned long long *__restrict__ keys,
                                                 uint64_t n, const Plan *__restrict__ plan,
                                                 uint32_t nb1, uint64_t span,
                                                 const uint32_t *__restrict__ tile_off,
                                                 unsigned long long *__restrict__ keys_out,
                                                 uint32_t *__restrict__ idx_out,
                                                 const uint32_t *__restrict__ bounds,
                                                 uint32_t pass) {
  extern __shared__ uint32_t s_cur[];
  const uint32_t blo = bounds[pass], bhi = bounds[pass + 1];
  const uint32_t *to = tile_off + (uint64_t)blockIdx.x * nb1;
  for (uint32_t b = threadIdx.x + blo; b < bhi; b += blockDim.x) s_cur[b - blo] = to[b];
  __syncthreads();
  if (plan->status != OK) return;
  const uint32_t shift = plan->part_shift, nb = nb1 - 1;
  const uint64_t lo = (uint64_t)blockIdx.x * span;
  const uint64_t hi = min(n, lo + span);
  // kIlp keys per thread per round; the next round's keys are loaded before
  // this round's cursor updates and stores, so loads stay in flight
  constexpr int kIlp = 4;
  const uint64_t step = (uint64_t)kIlp * blockDim.x;
  unsigned long long kn[kIlp];
#pragma unroll
  for (int r = 0; r < kIlp; ++r) {
    const uint64_t i = lo + (uint64_t)r * blockDim.x + threadIdx.x;
    kn[r] = i < hi ? __ldcs(keys + i) : 0ull;
  }
  for (uint64_t i0 = lo; i0 < hi; i0 += step) {
    unsigned long long k[kIlp];
#pragma unroll
    for (int r = 0; r < kIlp; ++r) {
      k[r] = kn[r];
      const uint64_t i = i0 + step + (uint64_t)r * blockDim.x + threadIdx.x;
      kn[r] = i < hi ? __ldcs(keys + i) : 0ull;
    }
    // one cursor update per run of lanes with the same bucket
    uint32_t pos[kIlp];
    bool in[kIlp];
#pragma unroll
    for (int r = 0; r < kIlp; ++r) {
      const uint64_t i = i0 + (uint64_t)r * blockDim.x + threadIdx.x;
      const uint32_t b = (k[r] & kOutlierBit) ? nb : (uint32_t)(k[r] >> shift);
      const bool valid = i < hi && b >= blo && b < bhi;
      in[r] = valid;
      pos[r] = 0u;
      if (!__any_sync(0xffffffffu, valid)) continue;
      int leader;
      uint32_t rank, len;
      lane_runs(b, valid, leader, rank, len);
      uint32_t base = 0u;
      if (valid && rank == 0u) base = atomicAdd(&s_cur[b - blo], len);
      pos[r] = __shfl_sync(0xffffffffu, base, leader) + rank;
    }
#pragma unroll
    for (int r = 0; r < kIlp; ++r) {
      const uint64_t i = i0 + (uint64_t)r * blockDim.x + threadIdx.x;
      if (in[r]) {
        keys_out[pos[r]] = k[r];
        if (idx_out) idx_out[pos[r]] = (uint32_t)i;
      }
    }
  }
}

// bucket bounds of the scatter passes: pass r takes the buckets whose keys
// start in [r n / passes, (r + 1) n / passes) of the partitioned order
// (bstart: exclusive bucket starts, bstart[nb1] = n), so passes move about
// the same number of keys
__global__ void k_scatter_bounds(const unsigned long long *__restrict__ bstart, uint32_t nb1,
                                 uint64_t n, uint32_t passes, uint32_t *__restrict__ bounds) {
  const uint32_t r = threadIdx.x;
  if (r > passes) return;
  if (r == passes) {
    bounds[r] = nb1;
    return;
  }
  const unsigned long long target = (unsigned long long)((n * (uint64_t)r) / passes);
  uint32_t lo = 0, hi = nb1;  // first bucket with bstart >= target
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (bstart[mid] < target) lo = mid + 1;
    else hi = mid;
  }
  bounds[r] = r == 0 ? 0u : lo;
}

void launch_scatter(const unsigned long long *keys, uint64_t n, const Plan *plan, uint32_t nb1,
                    int tiles, const uint32_t *tile_off, const unsigned long long *bstart,
                    uint32_t *bounds, unsigned long long *keys_out, uint32_t *idx_out,
                    cudaStream_t s) {
  uint64_t span = (n + tiles - 1) / tiles;
  span = (span + 3) & ~3ull;
  static const bool attr =  // once per process, thread-safe
      cudaFuncSetAttribute(k_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024) ==
      cudaSuccess;
  (void)attr;
  // passes: about 40 MB of 32-byte write fronts (tiles x buckets) in all,
  // split by key count
  const uint64_t fronts = (uint64_t)tiles * nb1 * 32ull;
  const uint64_t budget = 40ull << 20;
  const uint32_t passes = (uint32_t)std::min<uint64_t>(
      kScatterPassesMax, std::max<uint64_t>(1, (fronts + budget - 1) / budget));
  note_launch();
  k_scatter_bounds<<<1, 32, 0, s>>>(bstart, nb1, n, passes, bounds);
  for (uint32_t r = 0; r < passes; ++r) {
    note_launch();
    k_scatter<<<tiles, 512, sizeof(uint32_t) * nb1, s>>>(keys, n, plan, nb1, span, tile_off,
                                                         keys_out, idx_out, bounds, r);
  }
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
// level-2 partition of buckets above kSplitMin keys: each such bucket is
// split by the next sub_bits_for(count) key bits (still block-id bits, so no
// block crosses a sub-bucket), one CTA per bucket of up to kSplitChunk keys,
// larger buckets in kSplitChunk-key tasks on several CTAs.  Sort units
// (k_local): the ordered list of key ranges holding consecutive unsplit
// buckets merged greedily up to kCap keys, and the outlier bucket.
// ---------------------------------------------------------------------------
// level-2 digit width of a split bucket of cnt keys (maxsub: block-id bits
// below the level-1 digit)
__device__ __forceinline__ int sub_bits_for(uint64_t cnt, int maxsub) {
  int b = (int)bitlen64(cnt >> 3);
  b = b < kSubMinBits ? kSubMinBits : (b > kSubMaxBits ? kSubMaxBits : b);
  return b < maxsub ? b : maxsub;
}
__device__ __forceinline__ uint32_t sub_chunks(int sub) {
  return sub > 5 ? (1u << (sub - 5)) : 1u;  // 32-digit chunks
}
// tasks of a split bucket of cnt keys: one up to kSplitChunk keys, else one
// per kSplitChunk keys
__device__ __host__ __forceinline__ uint32_t split_tasks(uint32_t cnt) {
  return cnt > kSplitChunk ? (cnt + kSplitChunk - 1) / kSplitChunk : 1u;
}

// split buckets: big_list[j] = bucket, big_cb[j] = first 32-digit chunk of
// its sub-bucket offsets (big_cb[nbig] = all chunks), big_tb[j] = its first
// task (big_tb[nbig] = all tasks), big_hs[j] = first histogram slot of a
// bucket of several tasks; task_owner[t] and slot_owner[h] = the bucket of
// task t and of slot h; multi[m] = the m-th bucket of several tasks.
// nbig: [0] split buckets, [1] work counter, [2] chunks, [3] tasks,
// [4] buckets of several tasks, [5] histogram slots, [6] k_subsort's work
// counter
__global__ void __launch_bounds__(1024) k_seg_plan(const Plan *__restrict__ plan, uint32_t nb1,
                                                   const unsigned long long *__restrict__ bstart,
                                                   SegBufs g) {
  __shared__ unsigned long long s_warp[32];
  const Plan &P = *plan;
  const uint32_t nb = nb1 - 1;
  const int maxsub = (int)P.part_shift - (int)P.rel_bits;
  const uint32_t per = (nb1 + 1023) / 1024;
  const uint32_t lo = threadIdx.x * per, hi = min(nb1, lo + per);
  // c = (chunks << 32) | buckets; e = (tasks << 40) | (slots << 20) | multi
  unsigned long long c = 0, e = 0;
  for (uint32_t b = lo; b < hi; ++b) {
    const uint64_t cnt = bstart[b + 1] - bstart[b];
    if (maxsub > 0 && b < nb && cnt > (uint64_t)kSplitMin) {
      c += ((unsigned long long)sub_chunks(sub_bits_for(cnt, maxsub)) << 32) | 1ull;
      const unsigned long long T = split_tasks((uint32_t)cnt);
      e += (T << 40) | (T > 1 ? (T << 20) | 1ull : 0ull);
    }
  }
  unsigned long long tot, tote;
  unsigned long long run = block_exscan<1024>(c, s_warp, tot);
  unsigned long long rune = block_exscan<1024>(e, s_warp, tote);
  for (uint32_t b = lo; b < hi; ++b) {
    const uint64_t cnt = bstart[b + 1] - bstart[b];
    const bool big = maxsub > 0 && b < nb && cnt > (uint64_t)kSplitMin;
    const uint32_t j = (uint32_t)run;
    g.big_of[b] = big ? (int)j : -1;
    if (big) {
      g.big_list[j] = b;
      g.big_cb[j] = (uint32_t)(run >> 32);
      run += ((unsigned long long)sub_chunks(sub_bits_for(cnt, maxsub)) << 32) | 1ull;
      const uint32_t T = split_tasks((uint32_t)cnt);
      const uint32_t tb = (uint32_t)(rune >> 40), hs = (uint32_t)(rune >> 20) & 0xFFFFFu;
      g.big_tb[j] = tb;
      g.big_hs[j] = hs;
      for (uint32_t k = 0; k < T; ++k) g.task_owner[tb + k] = j;
      if (T > 1) {
        g.multi[(uint32_t)rune & 0xFFFFFu] = j;
        for (uint32_t k = 0; k < T; ++k) g.slot_owner[hs + k] = j;
      }
      rune += ((unsigned long long)T << 40) | (T > 1 ? ((unsigned long long)T << 20) | 1ull : 0ull);
    }
  }
  if (threadIdx.x == 0) {
    g.nbig[0] = (uint32_t)tot;
    g.nbig[1] = 0u;  // work counter of k_split_big
    g.nbig[6] = 0u;  // work counter of k_subsort
    g.nbig[2] = (uint32_t)(tot >> 32);
    g.nbig[3] = (uint32_t)(tote >> 40);
    g.nbig[4] = (uint32_t)tote & 0xFFFFFu;
    g.nbig[5] = (uint32_t)(tote >> 20) & 0xFFFFFu;
    g.big_cb[(uint32_t)tot] = (uint32_t)(tot >> 32);
    g.big_tb[(uint32_t)tot] = (uint32_t)(tote >> 40);
  }
}

// sub-bucket histogram of key range [c0, c1) of a split bucket into h
// (zeroed by the caller), kSplitIlp loads in flight per thread
__device__ __forceinline__ void split_count(const unsigned long long *__restrict__ kb,
                                            uint32_t c0, uint32_t c1, int shift2, uint32_t mask,
                                            uint32_t *h) {
  for (uint32_t t0 = c0; t0 < c1; t0 += kSplitThreads * kSplitIlp) {
    unsigned long long k[kSplitIlp];
#pragma unroll
    for (int r = 0; r < kSplitIlp; ++r) {
      const uint32_t t = t0 + r * kSplitThreads + threadIdx.x;
      k[r] = t < c1 ? kb[t] : 0ull;
    }
#pragma unroll
    for (int r = 0; r < kSplitIlp; ++r) {
      const uint32_t t = t0 + r * kSplitThreads + threadIdx.x;
      const uint32_t dg = (uint32_t)(k[r] >> shift2) & mask;
      int leader;
      uint32_t rank, len;
      lane_runs(dg, t < c1, leader, rank, len);
      if (t < c1 && rank == 0u) atomicAdd(&h[dg], len);
    }
  }
}

// Buckets of several tasks, pass 1: one kSplitChunk-key task per slot, its
// sub-bucket histogram stored densely at shist[slot * kSubMax + digit].
__global__ void __launch_bounds__(kSplitThreads) k_split_hist(
    const Plan *__restrict__ plan, const unsigned long long *__restrict__ bstart, SegBufs g,
    const unsigned long long *__restrict__ keys) {
  __shared__ uint32_t h[kSubMax];
  const Plan &P = *plan;
  const int maxsub = (int)P.part_shift - (int)P.rel_bits;
  const uint32_t nslot = g.nbig[5];
  for (uint32_t sl = blockIdx.x; sl < nslot; sl += gridDim.x) {
    for (int d = threadIdx.x; d < kSubMax; d += kSplitThreads) h[d] = 0u;
    __syncthreads();
    const uint32_t j = g.slot_owner[sl];
    const uint64_t lo = bstart[g.big_list[j]];
    const uint32_t cnt = (uint32_t)(bstart[g.big_list[j] + 1] - lo);
    const int sub = sub_bits_for(cnt, maxsub);
    const uint32_t c0 = (sl - g.big_hs[j]) * kSplitChunk;
    const uint32_t c1 = min(cnt, c0 + kSplitChunk);
    split_count(keys + lo, c0, c1, (int)P.part_shift - sub, (1u << sub) - 1u, h);
    __syncthreads();
    uint32_t *out = g.shist + (uint64_t)sl * kSubMax;
    for (uint32_t d = threadIdx.x; d < (1u << sub); d += kSplitThreads) out[d] = h[d];
    __syncthreads();
  }
}

// Buckets of several tasks, pass 2 (one CTA per bucket): sub-bucket offsets
// from the summed task histograms; each task's slot is replaced by its
// starting position per sub-bucket (the offset plus the earlier tasks'
// counts).  Thread t owns digits 8t .. 8t+7, read and written as vectors.
constexpr int kScanThreads = 1024;
__global__ void __launch_bounds__(kScanThreads) k_split_scan(
    const Plan *__restrict__ plan, const unsigned long long *__restrict__ bstart, SegBufs g) {
  constexpr int per = kSubMax / kScanThreads;
  static_assert(per == 8, "two 16-byte vectors per thread");
  __shared__ unsigned long long s_warp[32];
  const Plan &P = *plan;
  const int maxsub = (int)P.part_shift - (int)P.rel_bits;
  const uint32_t nmulti = g.nbig[4];
  const uint32_t d0 = threadIdx.x * per;
  for (uint32_t m = blockIdx.x; m < nmulti; m += gridDim.x) {
    const uint32_t j = g.multi[m];
    const uint32_t b = g.big_list[j];
    const uint32_t cnt = (uint32_t)(bstart[b + 1] - bstart[b]);
    const int sub = sub_bits_for(cnt, maxsub);
    const uint32_t nsub = 1u << sub;
    const uint32_t T = split_tasks(cnt);
    uint32_t *hj = g.shist + (uint64_t)g.big_hs[j] * kSubMax + d0;
    const bool full = d0 + per <= nsub;  // else only digits below nsub count
    uint32_t c[per];
#pragma unroll
    for (int q = 0; q < per; ++q) c[q] = 0u;
    if (d0 < nsub) {
#pragma unroll 4
      for (uint32_t k = 0; k < T; ++k) {
        const uint32_t *p = hj + (uint64_t)k * kSubMax;
        if (full) {
          const uint4 x = reinterpret_cast<const uint4 *>(p)[0];
          const uint4 y = reinterpret_cast<const uint4 *>(p)[1];
          c[0] += x.x, c[1] += x.y, c[2] += x.z, c[3] += x.w;
          c[4] += y.x, c[5] += y.y, c[6] += y.z, c[7] += y.w;
        } else {
#pragma unroll
          for (int q = 0; q < per; ++q)
            if (d0 + q < nsub) c[q] += p[q];
        }
      }
    }
    unsigned long long sum = 0;
#pragma unroll
    for (int q = 0; q < per; ++q) sum += c[q];
    unsigned long long all;
    uint32_t run = (uint32_t)block_exscan<kScanThreads>(sum, s_warp, all);
    uint32_t o[per];
#pragma unroll
    for (int q = 0; q < per; ++q) {
      o[q] = run;
      run += c[q];
    }
    if (d0 < nsub) {
      uint32_t *so = g.sub_off + (uint64_t)g.big_cb[j] * 32u + d0;
#pragma unroll
      for (int q = 0; q < per; ++q)
        if (full || d0 + q < nsub) so[q] = o[q];
#pragma unroll 4
      for (uint32_t k = 0; k < T; ++k) {
        uint32_t *p = hj + (uint64_t)k * kSubMax;
        if (full) {
          const uint4 x = reinterpret_cast<const uint4 *>(p)[0];
          const uint4 y = reinterpret_cast<const uint4 *>(p)[1];
          reinterpret_cast<uint4 *>(p)[0] = make_uint4(o[0], o[1], o[2], o[3]);
          reinterpret_cast<uint4 *>(p)[1] = make_uint4(o[4], o[5], o[6], o[7]);
          o[0] += x.x, o[1] += x.y, o[2] += x.z, o[3] += x.w;
          o[4] += y.x, o[5] += y.y, o[6] += y.z, o[7] += y.w;
        } else {
#pragma unroll
          for (int q = 0; q < per; ++q)
            if (d0 + q < nsub) {
              const uint32_t x = p[q];
              p[q] = o[q];
              o[q] += x;
            }
        }
      }
    }
    for (uint32_t q = threadIdx.x; q < sub_chunks(sub); q += kScanThreads)
      g.chunk_owner[g.big_cb[j] + q] = j;
  }
}

// Split tasks (fetched from a work counter), one CTA per task of up to
// kSplitChunk keys staged in shared memory: the keys are read once (their
// sub-bucket histogram counted on the way in), put in sub-bucket order
// locally (the slot of each key in a second shared array), then written out
// in that order, so each sub-bucket's keys leave as one contiguous run.  A
// bucket of one task: its sub-bucket offsets (sub_off[32 * big_cb[j] +
// digit], within the bucket) are the local ones.  A task of a bucket of
// several: its starting positions come from k_split_scan.
constexpr size_t kStageSmem = (size_t)kSplitChunk * (8 + 2);  // keys, local order

__global__ void __launch_bounds__(kStageThreads, 1) k_split_big(
    const Plan *__restrict__ plan, const unsigned long long *__restrict__ bstart, SegBufs g,
    const unsigned long long *__restrict__ keys, const uint32_t *__restrict__ idx,
    unsigned long long *__restrict__ keys_out, uint32_t *__restrict__ idx_out) {
  constexpr int per = kSubMax / kStageThreads;        // digits per thread in the scan
  constexpr int kk = (int)kSplitChunk / kStageThreads;  // staged keys per thread
  extern __shared__ __align__(16) unsigned long long sk[];
  uint16_t *lord = reinterpret_cast<uint16_t *>(sk + kSplitChunk);  // key index by local slot
  __shared__ uint32_t h[kSubMax];
  __shared__ unsigned long long s_warp[32];
  __shared__ uint32_t s_t;
  const Plan &P = *plan;
  const int maxsub = (int)P.part_shift - (int)P.rel_bits;
  const uint32_t total = g.nbig[3];
  for (;;) {
    if (threadIdx.x == 0) s_t = atomicAdd(&g.nbig[1], 1u);
    for (int d = threadIdx.x; d < kSubMax; d += kStageThreads) h[d] = 0u;
    __syncthreads();
    const uint32_t t = s_t;
    if (t >= total) break;
    const uint32_t j = g.task_owner[t];
    const uint32_t b = g.big_list[j];
    const uint64_t lo = bstart[b];
    const uint32_t cnt = (uint32_t)(bstart[b + 1] - lo);
    const int sub = sub_bits_for(cnt, maxsub);
    const int shift2 = (int)P.part_shift - sub;
    const uint32_t mask = (1u << sub) - 1u;
    const uint32_t nsub = 1u << sub;
    const bool single = split_tasks(cnt) == 1u;
    const uint32_t k = single ? 0u : t - g.big_tb[j];
    const uint32_t c0 = k * kSplitChunk;
    const uint32_t m = min(cnt, c0 + kSplitChunk) - c0;  // keys of this task
    const unsigned long long *kb = keys + lo + c0;
    if (single)
      for (uint32_t q = threadIdx.x; q < sub_chunks(sub); q += kStageThreads)
        g.chunk_owner[g.big_cb[j] + q] = j;
    // 1. stage the keys (all loads in flight at once) and count the digits
    {
      unsigned long long kv[kk];
#pragma unroll
      for (int r = 0; r < kk; ++r) {
        const uint32_t i = (uint32_t)r * kStageThreads + threadIdx.x;
        kv[r] = i < m ? kb[i] : 0ull;
      }
#pragma unroll
      for (int r = 0; r < kk; ++r) {
        const uint32_t i = (uint32_t)r * kStageThreads + threadIdx.x;
        const uint32_t dg = (uint32_t)(kv[r] >> shift2) & mask;
        if (i < m) sk[i] = kv[r];
        int leader;
        uint32_t rank, len;
        lane_runs(dg, i < m, leader, rank, len);
        if (i < m && rank == 0u) atomicAdd(&h[dg], len);
      }
    }
    __syncthreads();
    // 2. local sub-bucket starts; thread t owns digits t*per .. t*per+per-1
    {
      uint32_t c[per];
      unsigned long long sum = 0;
#pragma unroll
      for (int q = 0; q < per; ++q) {
        const uint32_t dg = threadIdx.x * per + q;
        c[q] = dg < nsub ? h[dg] : 0u;
        sum += c[q];
      }
      unsigned long long tot;
      uint32_t run = (uint32_t)block_exscan<kStageThreads>(sum, s_warp, tot);
      uint32_t *so = g.sub_off + (uint64_t)g.big_cb[j] * 32u;
#pragma unroll
      for (int q = 0; q < per; ++q) {
        const uint32_t dg = threadIdx.x * per + q;
        if (dg < nsub) {
          if (single) so[dg] = run;
          h[dg] = run;
        }
        run += c[q];
      }
    }
    __syncthreads();
    // 3. local order: lord[local slot] = staged index (h[d] ends at the
    // start of digit d + 1)
#pragma unroll 4
    for (int r = 0; r < kk; ++r) {
      const uint32_t i = (uint32_t)r * kStageThreads + threadIdx.x;
      const bool on = i < m;
      const uint32_t dg = on ? (uint32_t)(sk[i] >> shift2) & mask : 0u;
      int leader;
      uint32_t rank, len;
      lane_runs(dg, on, leader, rank, len);
      uint32_t bs = 0u;
      if (on && rank == 0u) bs = atomicAdd(&h[dg], len);
      const uint32_t ls = __shfl_sync(0xffffffffu, bs, leader) + rank;
      if (on) lord[ls] = (uint16_t)i;
    }
    __syncthreads();
    // 4. out in local order: runs of one sub-bucket go to consecutive slots
    const uint32_t *gb = single ? nullptr : g.shist + ((uint64_t)g.big_hs[j] + k) * kSubMax;
    for (uint32_t p = threadIdx.x; p < m; p += kStageThreads) {
      const uint32_t i = lord[p];
      const unsigned long long key = sk[i];
      uint32_t pos = p;
      if (!single) {
        const uint32_t dg = (uint32_t)(key >> shift2) & mask;
        const uint32_t ls = dg ? h[dg - 1] : 0u;  // local start of the digit
        pos = gb[dg] + (p - ls);
      }
      keys_out[lo + pos] = key;
      if (idx_out) idx_out[lo + pos] = idx[lo + c0 + i];
    }
    __syncthreads();
  }
}

// Unit list (one CTA).  Thread t owns buckets [t*per, (t+1)*per); within that
// range consecutive unsplit buckets merge greedily up to kCap keys (a single
// bucket above kCap that cannot be split forms its own unit); a split bucket
// ends the run; the outlier bucket is a unit of its own.
__global__ void __launch_bounds__(1024) k_units_small(uint32_t nb1,
                                                      const unsigned long long *__restrict__ bstart,
                                                      const int *__restrict__ big_of,
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
    if (big_of[b] >= 0 || b == nb) {
      if (ucnt) {
        ++count;
        ucnt = 0;
      }
      if (b == nb && c) ++count;
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
    if (big_of[b] >= 0 || b == nb) {
      if (ucnt) {
        u_lo[out] = (uint32_t)ulo;
        u_cnt[out] = (uint32_t)ucnt;
        u_meta[out] = 0u;
        ++out;
        ucnt = 0;
      }
      if (b == nb && c) {
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

// every split bucket holds more than kSplitMin keys and at most
// max(32, 2^kSubMaxBits) offsets, about one per 4..8 keys
uint64_t sub_off_size(uint64_t n, uint32_t nb1) {
  const uint64_t nbig = std::min<uint64_t>(nb1, n / (kSplitMin + 1) + 1);
  return nbig * 32 + n / 4 + 64;
}

// tasks: every split bucket, plus one per kSplitChunk keys
uint64_t split_tasks_max(uint64_t n, uint32_t nb1) {
  return std::min<uint64_t>(nb1, n / (kSplitMin + 1) + 1) + n / kSplitChunk + 1;
}
// histogram slots: the tasks of the buckets of several tasks (each above
// kSplitChunk keys), fewer than 2 n / kSplitChunk
uint64_t split_slots_max(uint64_t n) { return 2 * (n / kSplitChunk) + 2; }

void launch_segments(const Plan *plan, uint32_t nb1, const unsigned long long *bstart,
                     unsigned long long *keys, uint32_t *idx, unsigned long long *keys_alt,
                     uint32_t *idx_alt, const SegBufs &g, uint32_t *u_lo, uint32_t *u_cnt,
                     uint32_t *u_meta, uint32_t *nunit, uint64_t n, int sms, cudaStream_t s) {
  note_launch();
  k_seg_plan<<<1, 1024, 0, s>>>(plan, nb1, bstart, g);
  if (n > kSplitChunk) {  // a bucket may need several tasks
    const uint64_t mmax = std::min<uint64_t>(nb1, n / (kSplitChunk + 1) + 1);
    note_launch();
    k_split_hist<<<(unsigned)std::min<uint64_t>(split_slots_max(n), 4 * sms), kSplitThreads, 0,
                   s>>>(plan, bstart, g, keys);
    note_launch();
    k_split_scan<<<(unsigned)std::min<uint64_t>(mmax, sms), kScanThreads, 0, s>>>(plan, bstart,
                                                                                 g);
  }
  static const bool attr =  // once per process, thread-safe
      cudaFuncSetAttribute(k_split_big, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)kStageSmem) == cudaSuccess;
  (void)attr;
  note_launch();
  k_split_big<<<sms, kStageThreads, kStageSmem, s>>>(plan, bstart, g, keys, idx, keys_alt,
                                                      idx_alt);
  note_launch();
  k_units_small<<<1, 1024, 0, s>>>(nb1, bstart, g.big_of, u_lo, u_cnt, u_meta, nunit);
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

// kmax (a power of two, 2 <= kmax <= 32R): the elements that matter all lie
// in [0, kmax) (the rest are padding); levels above kmax are skipped, and the
// first kmax elements still end ascending.
template <int R, typename T>
__device__ __forceinline__ void warp_bitonic(T (&v)[R], uint32_t kmax = 32u * R) {
  const uint32_t lane = threadIdx.x & 31;
#pragma unroll 1
  for (uint32_t k = 2; k <= kmax; k <<= 1) {
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

// the same network for one element per lane, every stage unrolled
template <typename T>
__device__ __forceinline__ void warp_bitonic32(T &v) {
  const uint32_t lane = threadIdx.x & 31;
#pragma unroll
  for (uint32_t k = 2; k <= 32; k <<= 1) {
    const bool up = (lane & k) == 0;
#pragma unroll
    for (uint32_t lj = k / 2; lj >= 1; lj >>= 1) {
      const bool keep_max = ((lane & lj) == 0) != up;
      const T o = shfl_x(v, (int)lj);
      if (key_lt(o, v) != keep_max) v = o;
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
__device__ __forceinline__ typename WinElem<MODE>::T win_make(unsigned long long key, uint32_t ix,
                                                              unsigned long long base) {
  if constexpr (MODE == 0) return (uint32_t)(key - base);
  else if constexpr (MODE == 1) return key;
  else if constexpr (MODE == 2) return ((key - base) << 32) | (unsigned long long)ix;
  else return KeyIdx{key, ix};
}
template <int MODE>
__device__ __forceinline__ typename WinElem<MODE>::T win_pad() {
  if constexpr (MODE == 0) return 0xffffffffu;
  else if constexpr (MODE == 3) return KeyIdx{~0ull, 0xffffffffu};
  else return ~0ull;
}
template <int MODE>
__device__ __forceinline__ void win_split(const typename WinElem<MODE>::T &v,
                                          unsigned long long base, unsigned long long &key,
                                          uint32_t &ix) {
  if constexpr (MODE == 0) {
    key = base + v;
    ix = 0u;
  } else if constexpr (MODE == 1) {
    key = v;
    ix = 0u;
  } else if constexpr (MODE == 2) {
    key = base + (v >> 32);
    ix = (uint32_t)v;
  } else {
    key = v.k;
    ix = v.i;
  }
}

// largest window one warp sorts in registers
__host__ __device__ constexpr int window_cap(int mode) { return mode == 3 ? 256 : 512; }

// the element form of a window whose keys lie in [base, base + span)
__device__ __forceinline__ int window_mode(unsigned long long span, bool with_idx) {
  const bool narrow = span <= (1ull << 32);
  return narrow ? (with_idx ? 2 : 0) : (with_idx ? 3 : 1);
}

// sorts the shared-memory window [w0, w0 + c) in place
template <int R, int MODE>
__device__ __forceinline__ void smem_window_r(unsigned long long *sk, uint32_t *si, int w0, int c,
                                              unsigned long long base) {
  using T = typename WinElem<MODE>::T;
  const int lane = threadIdx.x & 31;
  T v[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int i = lane * R + r;
    v[r] = i < c ? win_make<MODE>(sk[w0 + i], MODE >= 2 ? si[w0 + i] : 0u, base)
                 : win_pad<MODE>();
  }
  warp_bitonic<R>(v);
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int i = lane * R + r;
    if (i < c) {
      unsigned long long key;
      uint32_t ix;
      win_split<MODE>(v[r], base, key, ix);
      sk[w0 + i] = key;
      if (MODE >= 2) si[w0 + i] = ix;
    }
  }
}

template <int MODE>
__device__ __noinline__ void smem_window(unsigned long long *sk, uint32_t *si, int w0, int c,
                                         unsigned long long base) {
  if (c <= 32) smem_window_r<1, MODE>(sk, si, w0, c, base);
  else if (c <= 64) smem_window_r<2, MODE>(sk, si, w0, c, base);
  else if (c <= 128) smem_window_r<4, MODE>(sk, si, w0, c, base);
  else if (c <= 256) smem_window_r<8, MODE>(sk, si, w0, c, base);
  else if constexpr (MODE != 3) smem_window_r<16, MODE>(sk, si, w0, c, base);
}

// ---------------------------------------------------------------------------
// segmentation outputs of one sorted particle at slot g (its predecessor in
// sorted order is prev; start: the particle opens a block)
// ---------------------------------------------------------------------------
struct SegOut {
  uint32_t *s_rel;
  uint8_t *bflag;
  unsigned long long *tmp_bid;
  uint32_t *perm;
  const int32_t *q_in;
  int32_t *q_slot;
  uint64_t n;
  uint32_t d, rel_bits;
  unsigned long long rel_mask;
  uint64_t chunk_mask;
};

template <bool PERM>
__device__ __forceinline__ void seg_emit(const SegOut &o, bool valid, uint64_t g,
                                         unsigned long long key, unsigned long long prev,
                                         bool start, uint32_t ix, uint32_t *s_hist,
                                         unsigned long long &my_max) {
  const int lane = threadIdx.x & 31;
  unsigned long long v = 0ull;
  if (valid) {
    const unsigned long long rel = key & o.rel_mask;
    v = (start || (g & o.chunk_mask) == 0) ? rel : rel - (prev & o.rel_mask);
    o.s_rel[g] = (uint32_t)v;
    o.bflag[g] = start ? 1 : 0;
    o.tmp_bid[g] = key >> o.rel_bits;  // every slot: full sectors
    my_max = v > my_max ? v : my_max;
    if (PERM) {
      o.perm[g] = ix;
      if (o.q_slot)
        for (uint32_t f = 0; f < o.d; ++f)
          o.q_slot[(uint64_t)f * o.n + g] = o.q_in[(uint64_t)f * o.n + ix];
    }
  }
  // stream-2 histogram: escapes counted per warp, other values per lane
  const bool esc = valid && v >= (unsigned long long)kEsc;
  const uint32_t nesc = __popc(__ballot_sync(0xffffffffu, esc));
  if (lane == 0 && nesc) atomicAdd(&s_hist[kEsc], nesc);
  if (valid && !esc) atomicAdd(&s_hist[(uint32_t)v], 1u);
}

// ---------------------------------------------------------------------------
// sub-bucket runs of the split buckets: one warp per run, sorted and
// segmented in registers.  Warp tasks are 32 consecutive sub-buckets of a
// split bucket.  Runs are packed greedily: a run opens at a non-empty
// sub-bucket, takes the smallest window of 32, 64 or kRunCap slots that
// holds it, and adds the following sub-buckets while they fit.  Sorting a
// run of whole sub-buckets sorts each of them, since the sub-buckets are
// ordered by digit.  A sub-bucket of more than kRunCap particles becomes a
// k_local unit.
// ---------------------------------------------------------------------------
constexpr int kRunCap = 128;

template <int R, int MODE, bool PERM>
__device__ __forceinline__ void sub_run_r(const unsigned long long *ks, const uint32_t *is, int c,
                                          unsigned long long base, uint64_t g0, const SegOut &o,
                                          uint32_t *s_hist, unsigned long long &my_max) {
  using T = typename WinElem<MODE>::T;
  const int lane = threadIdx.x & 31;
  T v[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int i = lane * R + r;
    v[r] = i < c ? win_make<MODE>(ks[i], PERM ? is[i] : 0u, base) : win_pad<MODE>();
  }
  if constexpr (R == 1) {
    warp_bitonic32(v[0]);
  } else {
    uint32_t kmax = 2u;
    while (kmax < (uint32_t)c) kmax <<= 1;
    warp_bitonic<R>(v, kmax);
  }
  unsigned long long key[R];
  uint32_t ix[R];
#pragma unroll
  for (int r = 0; r < R; ++r) win_split<MODE>(v[r], base, key[r], ix[r]);
  const unsigned long long lp = __shfl_up_sync(0xffffffffu, key[R - 1], 1);
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int i = lane * R + r;
    const unsigned long long prev = r ? key[r - 1] : lp;
    const bool start = i == 0 || (key[r] >> o.rel_bits) != (prev >> o.rel_bits);
    seg_emit<PERM>(o, i < c, g0 + (uint64_t)i, key[r], prev, start, ix[r], s_hist, my_max);
  }
}

template <int MODE, bool PERM>
__device__ __forceinline__ void sub_run(const unsigned long long *ks, const uint32_t *is, int c,
                                        unsigned long long base, uint64_t g0, const SegOut &o,
                                        uint32_t *s_hist, unsigned long long &my_max) {
  if (c <= 32) sub_run_r<1, MODE, PERM>(ks, is, c, base, g0, o, s_hist, my_max);
  else if (c <= 64) sub_run_r<2, MODE, PERM>(ks, is, c, base, g0, o, s_hist, my_max);
  else sub_run_r<4, MODE, PERM>(ks, is, c, base, g0, o, s_hist, my_max);
}

template <bool PERM>
__global__ void __launch_bounds__(kSubThreads, kSubCtas) k_subsort(SubsortArgs A) {
  __shared__ uint32_t s_hist[kAlpha];
  __shared__ unsigned long long s_max;
  __shared__ int s_status;
  __shared__ uint32_t s_part, s_rel, s_d, s_nbig, s_nchunk;
  if (threadIdx.x == 0) {
    s_status = A.plan->status;
    s_part = A.plan->part_shift;
    s_rel = A.plan->rel_bits;
    s_d = A.plan->d;
    s_nbig = A.nbig[0];
    s_nchunk = A.nbig[2];
    s_max = 0ull;
  }
  for (int b = threadIdx.x; b < kAlpha; b += kSubThreads) s_hist[b] = 0u;
  __syncthreads();
  if (s_status != OK) return;
  const int lane = threadIdx.x & 31;
  const uint32_t part_shift = s_part, rel_bits = s_rel;
  const int maxsub = (int)part_shift - (int)rel_bits;
  SegOut o;
  o.s_rel = A.s_rel;
  o.bflag = A.bflag;
  o.tmp_bid = A.tmp_bid;
  o.perm = A.perm;
  o.q_in = A.q_in;
  o.q_slot = A.q_slot;
  o.n = A.n;
  o.d = s_d;
  o.rel_bits = rel_bits;
  o.rel_mask = (1ull << rel_bits) - 1ull;
  o.chunk_mask = (1ull << A.log2_chunk) - 1ull;
  unsigned long long my_max = 0ull;
  const uint32_t ntask = s_nchunk;
  const uint32_t warps = gridDim.x * (kSubThreads / 32);
  // first task by warp id, then from a work counter; the next index is
  // fetched while the current task runs
  uint32_t tn = 0u;
  for (uint32_t t = blockIdx.x * (kSubThreads / 32) + (threadIdx.x >> 5); t < ntask;
       t = __shfl_sync(0xffffffffu, tn, 0)) {
    if (lane == 0) tn = warps + atomicAdd(&A.nbig[6], 1u);
    const uint32_t j = A.chunk_owner[t], ch = t - A.big_cb[j];
    const uint32_t b = A.big_list[j];
    const uint64_t lo = A.bstart[b];
    const uint32_t cnt = (uint32_t)(A.bstart[b + 1] - lo);
    const int sub = sub_bits_for(cnt, maxsub);
    const uint32_t nsub = 1u << sub;
    const int shift2 = (int)part_shift - sub;
    const uint32_t *so = A.sub_off + (uint64_t)A.big_cb[j] * 32u;
    const uint32_t dg = ch * 32u + lane;
    const uint32_t off = dg < nsub ? so[dg] : cnt;
    uint32_t nx = __shfl_down_sync(0xffffffffu, off, 1);
    if (lane == 31) nx = dg + 1 < nsub ? so[dg + 1] : cnt;
    const uint32_t c = nx - off;
    const uint32_t ne = __ballot_sync(0xffffffffu, c > 0);
    if (!ne) continue;
    const unsigned long long bucket_base = (unsigned long long)b << part_shift;
    const unsigned long long *ks = A.keys_alt + lo;
    const uint32_t *is = PERM ? A.idx_alt + lo : nullptr;
    int l0 = __ffs(ne) - 1;
    while (l0 >= 0) {
      // a run: from sub-bucket l0, whole sub-buckets while the run fits the
      // smallest window of 32, 64 or 128 slots that holds sub-bucket l0
      const uint32_t w0 = __shfl_sync(0xffffffffu, off, l0);
      const uint32_t c0 = __shfl_sync(0xffffffffu, c, l0);
      const uint32_t cap = c0 <= 32u ? 32u : (c0 <= 64u ? 64u : (uint32_t)kRunCap);
      const uint32_t fit = __ballot_sync(0xffffffffu, lane >= l0 && nx - w0 <= cap);
      const int L = fit ? 31 - __clz(fit) : l0;
      const uint32_t w1 = __shfl_sync(0xffffffffu, nx, L);
      const uint32_t upto = L == 31 ? 0xffffffffu : ((2u << L) - 1u);
      const uint32_t rest = ne & ~upto;
      const int l_next = rest ? __ffs(rest) - 1 : -1;
      const int wc = (int)(w1 - w0);
      if (c0 > (uint32_t)kRunCap) {  // one sub-bucket too large for a warp: a k_local unit
        if (lane == 0) {
          const uint32_t u = atomicAdd(A.nunit, 1u);
          A.u_lo[u] = (uint32_t)(lo + w0);
          A.u_cnt[u] = (uint32_t)wc;
          A.u_meta[u] = 1u;  // keys in the level-2 buffer
        }
        l0 = l_next;
        continue;
      }
      // digits of the run: [g0, g1), g1 one past its last non-empty sub-bucket
      const uint32_t g0 = ch * 32u + (uint32_t)l0;
      const uint32_t g1 = ch * 32u + (uint32_t)(32 - __clz(ne & upto));
      const unsigned long long base = bucket_base | ((unsigned long long)g0 << shift2);
      const int mode = window_mode((unsigned long long)(g1 - g0) << shift2, PERM);
      const uint64_t g = lo + w0;
      if (mode == 0) {
        sub_run<0, PERM>(ks + w0, PERM ? is + w0 : nullptr, wc, base, g, o, s_hist, my_max);
      } else if (mode == 1) {
        sub_run<1, PERM>(ks + w0, PERM ? is + w0 : nullptr, wc, base, g, o, s_hist, my_max);
      } else {
        if constexpr (PERM) {
          if (mode == 2) sub_run<2, true>(ks + w0, is + w0, wc, base, g, o, s_hist, my_max);
          else sub_run<3, true>(ks + w0, is + w0, wc, base, g, o, s_hist, my_max);
        }
      }
      l0 = l_next;
    }
  }
  __syncthreads();
  for (int s = threadIdx.x; s < kAlpha; s += kSubThreads)
    if (s_hist[s]) atomicAdd(&A.hist[2 * kAlpha + s], s_hist[s]);
  atomicMax(&s_max, my_max);
  __syncthreads();
  if (threadIdx.x == 0 && s_max) atomicMax(&A.maxv[2], s_max);
}

void launch_subsort(const SubsortArgs &a, int sms, cudaStream_t s) {
  note_launch();
  if (a.perm) k_subsort<true><<<kSubCtas * sms, kSubThreads, 0, s>>>(a);
  else k_subsort<false><<<kSubCtas * sms, kSubThreads, 0, s>>>(a);
}

// ---------------------------------------------------------------------------
// per-unit sort + segmentation (persistent over units).
//
// A unit of up to kCap keys is sorted in shared memory: the keys are loaded
// into registers, partitioned by their top 8 varying bits (one counting
// pass, no order needed inside a digit group), and the digit groups are
// gathered into windows (consecutive groups whose starts share a span of
// kWinSpan slots) that one warp sorts in registers with a bitonic network,
// on 32-bit offsets from the window's base key when its key span allows.
// Windows too large for a warp (a digit group of hundreds of keys) fall back
// to the CTA radix sort.  Sorting each window sorts the unit because the
// windows are ordered by digit.  Larger units are sorted by the CTA radix
// sort in global memory.
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
  __shared__ int s_status;
  __shared__ uint32_t s_relb, s_d, s_nseg;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    s_status = a.plan->status;
    s_relb = a.plan->rel_bits;
    s_d = a.plan->d;
    s_nseg = *a.nseg;
    s_max = 0ull;
  }
  for (int b = threadIdx.x; b < kAlpha; b += kLocalThreads) s_hist[b] = 0u;
  __syncthreads();
  if (s_status != OK) return;
  SegOut o;
  o.s_rel = a.s_rel;
  o.bflag = a.bflag;
  o.tmp_bid = a.tmp_bid;
  o.perm = a.perm;
  o.q_in = a.q_in;
  o.q_slot = a.q_slot;
  o.n = a.n;
  o.d = s_d;
  o.rel_bits = s_relb;
  o.rel_mask = (1ull << s_relb) - 1ull;
  o.chunk_mask = (1ull << a.log2_chunk) - 1ull;
  const int ibits = PERM ? (int)bitlen64(a.n > 0 ? a.n - 1 : 0) : 0;
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
      for (int q = 16; q > 0; q >>= 1) {
        const unsigned long long a1 = __shfl_xor_sync(0xffffffffu, mn, q);
        const unsigned long long b1 = __shfl_xor_sync(0xffffffffu, mx, q);
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
        for (int q = 1; q < 32; q <<= 1) {
          const uint32_t y = __shfl_up_sync(0xffffffffu, incl, q);
          if (lane >= q) incl += y;
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
        for (int q = 1; q < 32; q <<= 1) {
          const uint32_t y = __shfl_up_sync(0xffffffffu, ci, q);
          if (lane >= q) ci += y;
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
      // windows, one warp each: keys of window w lie in
      // [top | g0 << sh, top | g1 << sh) for its first and end digits g0, g1
      const uint32_t nwin = s_nwin;
      const unsigned long long top = sh + 8 >= 64 ? 0ull : (kmin >> (sh + 8)) << (sh + 8);
      const uint32_t gend = (uint32_t)((kmax >> sh) & 255ull) + 1u;
      for (uint32_t wi = warp; wi < nwin; wi += kLocalWarps) {
        const int w0 = (int)s_win[wi], c = (int)s_win[wi + 1] - w0;
        if (c < 2) continue;
        const uint32_t g0 = s_wdg[wi], g1 = wi + 1 < nwin ? s_wdg[wi + 1] : gend;
        const unsigned long long base = top | ((unsigned long long)g0 << sh);
        const int mode = window_mode((unsigned long long)(g1 - g0) << sh, use_idx);
        if (c > window_cap(mode)) continue;
        if (mode == 0) {
          smem_window<0>(sk, si, w0, c, base);
        } else if (mode == 1) {
          smem_window<1>(sk, si, w0, c, base);
        } else {
          if constexpr (PERM) {
            if (mode == 2) smem_window<2>(sk, si, w0, c, base);
            else smem_window<3>(sk, si, w0, c, base);
          }
        }
      }
      __syncthreads();
      // windows too large for a warp: CTA radix sort, scratch in global memory
      for (uint32_t wi = 0; wi < nwin; ++wi) {
        const int w0 = (int)s_win[wi], c = (int)s_win[wi + 1] - w0;
        const uint32_t g0 = s_wdg[wi], g1 = wi + 1 < nwin ? s_wdg[wi + 1] : gend;
        const int mode = window_mode((unsigned long long)(g1 - g0) << sh, use_idx);
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
          for (uint32_t f = 0; f < o.d; ++f)
            a.q_slot[(uint64_t)f * a.n + lo + j] = a.q_in[(uint64_t)f * a.n + idx];
      }
      __syncthreads();
      continue;
    }
    // segmentation; the unit's first particle opens a block
    for (int j0 = 0; j0 < cnt; j0 += kLocalThreads) {
      const int j = j0 + threadIdx.x;
      const bool valid = j < cnt;
      unsigned long long key = 0ull, prev = 0ull;
      bool start = false;
      uint32_t ix = 0u;
      if (valid) {
        key = K[j];
        if (j > 0) prev = K[j - 1];
        start = j == 0 || (key >> o.rel_bits) != (prev >> o.rel_bits);
        if (PERM) ix = I[j];
      }
      seg_emit<PERM>(o, valid, lo + (uint64_t)j, key, prev, start, ix, s_hist, my_max);
    }
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
  static const bool attr =  // once per process, thread-safe
      cudaFuncSetAttribute(k_local<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)base) == cudaSuccess &&
      cudaFuncSetAttribute(k_local<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(base + (size_t)kCap * 4)) == cudaSuccess;
  (void)attr;
  note_launch();
  if (a.perm) k_local<true><<<ctas, kLocalThreads, smem, s>>>(a);
  else k_local<false><<<ctas, kLocalThreads, smem, s>>>(a);
}

// ---------------------------------------------------------------------------
// blocks: number the block starts (scan of the start flags over the nbk
// non-outlier slots), then delta code ids and counts (Sec. "Block coding")
// ---------------------------------------------------------------------------
constexpr int kFlagThreads = 256;
constexpr int kFlagPer = 8;  // slots per thread (one 8-byte load)
constexpr int kFlagTile = kFlagThreads * kFlagPer;

__device__ __forceinline__ uint32_t flag_bits8(const uint8_t *flag, uint64_t g, uint64_t nbk) {
  // start flags of slots g .. g+7 (g a multiple of 8) as a bit mask
  if (g >= nbk) return 0u;
  const uint2 w = *reinterpret_cast<const uint2 *>(flag + g);
  uint32_t bits = 0u;
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    bits |= ((w.x >> (8 * b)) & 1u) << b;
    bits |= ((w.y >> (8 * b)) & 1u) << (4 + b);
  }
  const uint64_t left = nbk - g;
  if (left < 8) bits &= (1u << left) - 1u;
  return bits;
}

__global__ void __launch_bounds__(kFlagThreads) k_flag_count(
    const uint8_t *__restrict__ flag, const unsigned long long *__restrict__ nbkp,
    unsigned long long *__restrict__ tile_cnt) {
  __shared__ unsigned long long s_warp[32];
  const uint64_t nbk = *nbkp;
  const uint64_t g = (uint64_t)blockIdx.x * kFlagTile + (uint64_t)threadIdx.x * kFlagPer;
  const uint32_t c = __popc(flag_bits8(flag, g, nbk));
  unsigned long long tot;
  block_exscan<kFlagThreads>(c, s_warp, tot);
  if (threadIdx.x == 0) tile_cnt[blockIdx.x] = tot;
}

// bpos[B] = slot of block B's first particle, bidv[B] = its block id;
// bpos[M] = nbk; mcount = M.  A tile's blocks are gathered in shared memory
// and written out contiguously.
__global__ void __launch_bounds__(kFlagThreads) k_flag_apply(
    const uint8_t *__restrict__ flag, const unsigned long long *__restrict__ nbkp,
    const unsigned long long *__restrict__ tile_base, uint32_t ntiles,
    const unsigned long long *__restrict__ tmp_bid, uint32_t *__restrict__ bpos,
    unsigned long long *__restrict__ bidv, unsigned long long *__restrict__ mcount) {
  __shared__ unsigned long long s_warp[32];
  __shared__ uint32_t s_pos[kFlagTile];
  __shared__ unsigned long long s_bid[kFlagTile];
  const uint64_t nbk = *nbkp;
  const uint64_t g = (uint64_t)blockIdx.x * kFlagTile + (uint64_t)threadIdx.x * kFlagPer;
  uint32_t bits = flag_bits8(flag, g, nbk);
  unsigned long long tot;
  uint32_t t = (uint32_t)block_exscan<kFlagThreads>(__popc(bits), s_warp, tot);
  if (bits) {
    unsigned long long ids[kFlagPer];
    const ulonglong2 *src = reinterpret_cast<const ulonglong2 *>(tmp_bid + g);
#pragma unroll
    for (int q = 0; q < kFlagPer / 2; ++q) {
      const ulonglong2 v = src[q];
      ids[2 * q] = v.x;
      ids[2 * q + 1] = v.y;
    }
#pragma unroll
    for (int b = 0; b < kFlagPer; ++b)
      if ((bits >> b) & 1u) {
        s_pos[t] = (uint32_t)(g + b);
        s_bid[t] = ids[b];
        ++t;
      }
  }
  __syncthreads();
  const unsigned long long B0 = tile_base[blockIdx.x];
  for (uint32_t i = threadIdx.x; i < (uint32_t)tot; i += kFlagThreads) {
    bpos[B0 + i] = s_pos[i];
    bidv[B0 + i] = s_bid[i];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const unsigned long long M = tile_base[ntiles];
    bpos[M] = (uint32_t)nbk;
    *mcount = M;
  }
}

__global__ void __launch_bounds__(512) k_blocks_map(const Plan *__restrict__ plan,
                                                    const uint32_t *__restrict__ bpos,
                                                    const unsigned long long *__restrict__ bidv,
                                                    const unsigned long long *__restrict__ mcount,
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
  const int lane = threadIdx.x & 31;
  const uint64_t M = *mcount;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  unsigned long long x0 = 0ull, x1 = 0ull;
  // trip count uniform across the warp (ballots below); the next round's
  // positions and ids are loaded before this round's are used
  const uint64_t iters = (M + stride - 1) / stride;
  const uint64_t g0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t np = 0u, npn = 0u, npp = 0u;
  unsigned long long nb = 0ull, nbp = 0ull;
  auto fetch = [&](uint64_t B) {
    if (B < M) {
      np = bpos[B];
      npn = bpos[B + 1];
      nb = bidv[B];
      npp = B > 0 ? bpos[B - 1] : 0u;
      nbp = B > 0 ? bidv[B - 1] : 0ull;
    }
  };
  fetch(g0);
  for (uint64_t it = 0; it < iters; ++it) {
    const uint64_t B = it * stride + g0;
    const bool valid = B < M;
    const uint32_t p = np, pn = npn, pp = npp;
    const unsigned long long bid = nb, pbid = nbp;
    fetch(B + stride);
    unsigned long long v0 = 0ull, v1 = 0ull;
    if (valid) {
      const long long c = (long long)(pn - p);
      const long long pc = B > 0 ? (long long)(p - pp) : 0ll;
      v0 = bid - pbid;
      v1 = zigzag(c - pc);
      s_id[B] = v0;
      s_cnt[B] = v1;
      x0 = v0 > x0 ? v0 : x0;
      x1 = v1 > x1 ? v1 : x1;
    }
    const bool e0 = valid && v0 >= (unsigned long long)kEsc;
    const bool e1 = valid && v1 >= (unsigned long long)kEsc;
    const uint32_t n0 = __popc(__ballot_sync(0xffffffffu, e0));
    const uint32_t n1 = __popc(__ballot_sync(0xffffffffu, e1));
    if (lane == 0) {
      if (n0) atomicAdd(&h0[kEsc], n0);
      if (n1) atomicAdd(&h1[kEsc], n1);
    }
    if (valid && !e0) atomicAdd(&h0[(uint32_t)v0], 1u);
    if (valid && !e1) atomicAdd(&h1[(uint32_t)v1], 1u);
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

uint64_t flag_tiles(uint64_t n) { return (n + kFlagTile - 1) / kFlagTile + 1; }

void launch_blocks(const Plan *plan, const uint8_t *bflag, const unsigned long long *nbk,
                   uint64_t n, const unsigned long long *tmp_bid, unsigned long long *tile_cnt,
                   unsigned long long *tile_base, uint32_t *bpos, unsigned long long *bidv,
                   unsigned long long *s_id, unsigned long long *s_cnt, uint32_t *hist,
                   unsigned long long *maxv, unsigned long long *mcount, int sms,
                   cudaStream_t s) {
  const uint32_t ntiles = (uint32_t)((n + kFlagTile - 1) / kFlagTile);
  const uint32_t nt = ntiles ? ntiles : 1u;
  note_launch();
  k_flag_count<<<nt, kFlagThreads, 0, s>>>(bflag, nbk, tile_cnt);
  launch_scan_small(tile_cnt, nt, tile_base, s);
  note_launch();
  k_flag_apply<<<nt, kFlagThreads, 0, s>>>(bflag, nbk, tile_base, nt, tmp_bid, bpos, bidv,
                                            mcount);
  note_launch();
  k_blocks_map<<<2 * sms, 512, 0, s>>>(plan, bpos, bidv, mcount, s_id, s_cnt, hist, maxv);
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
