// k_frame.cu -- frame stage: min/max, plan, quantize + block keys.
//
// Sec. "Error-Bound Aware Quantization" (Eq. quantization) and Sec. "Design
// of spatial blocks" (Eq. block size and id).  Every input value is read once
// for min/max and once for quantization; both passes are HBM-bound streams
// with 128-bit loads.
#include <float.h>

#include "lcp_kernels.h"

namespace lcp {

// ---------------------------------------------------------------------------
// min / max (IEEE totalOrder, so -0 < +0) and a non-finite flag per frame
// ---------------------------------------------------------------------------
__global__ void k_minmax_init(MinMax *mm) {
  int t = threadIdx.x;
  if (t < kMaxD) {
    mm->lo[t] = 0xffffffffu;
    mm->hi[t] = 0u;
  }
  if (t == 0) mm->nonfinite = 0u;
}

__global__ void __launch_bounds__(256) k_minmax(const float *__restrict__ fields, uint64_t n,
                                                MinMax *mm) {
  const int f = blockIdx.y;
  const float *x = fields + (uint64_t)f * n;
  uint32_t lo = 0xffffffffu, hi = 0u, bad = 0u;
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const bool vec = ((n & 3ull) == 0) && ((((uintptr_t)fields) & 15u) == 0);
  if (vec) {
    const float4 *x4 = reinterpret_cast<const float4 *>(x);
    const uint64_t n4 = n >> 2;
    for (uint64_t i = tid; i < n4; i += stride) {
      float4 v = __ldcs(x4 + i);
      float a[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        uint32_t b = __float_as_uint(a[k]);
        bad |= ((b & 0x7f800000u) == 0x7f800000u);
        uint32_t key = order_key(a[k]);
        lo = min(lo, key);
        hi = max(hi, key);
      }
    }
  } else {
    for (uint64_t i = tid; i < n; i += stride) {
      float v = x[i];
      uint32_t b = __float_as_uint(v);
      bad |= ((b & 0x7f800000u) == 0x7f800000u);
      uint32_t key = order_key(v);
      lo = min(lo, key);
      hi = max(hi, key);
    }
  }
  lo = __reduce_min_sync(0xffffffffu, lo);
  hi = __reduce_max_sync(0xffffffffu, hi);
  bad = __reduce_or_sync(0xffffffffu, bad);
  __shared__ uint32_t s_lo[8], s_hi[8], s_bad[8];
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) {
    s_lo[w] = lo;
    s_hi[w] = hi;
    s_bad[w] = bad;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 1; k < (int)(blockDim.x >> 5); ++k) {
      lo = min(lo, s_lo[k]);
      hi = max(hi, s_hi[k]);
      bad |= s_bad[k];
    }
    atomicMin(&mm->lo[f], lo);
    atomicMax(&mm->hi[f], hi);
    if (bad) atomicOr(&mm->nonfinite, 1u);
  }
}

void launch_minmax(const float *fields, uint64_t n, uint32_t d, MinMax *mm, int sms,
                   cudaStream_t s) {
  note_launch();
  k_minmax_init<<<1, 32, 0, s>>>(mm);
  if (n == 0) return;
  uint64_t want = (n + 4095) / 4096;
  int gx = (int)(want < (uint64_t)(4 * sms) ? want : (uint64_t)(4 * sms));
  gx = (gx + (int)d - 1) / (int)d;
  if (gx < 1) gx = 1;
  note_launch();
  k_minmax<<<dim3(gx, d), 256, 0, s>>>(fields, n, mm);
}

// ---------------------------------------------------------------------------
// plan: resolve each field's bound, bins and reconstruction constants; apply
// the domain rules in a fixed order (non-finite, then per field: bound out of
// [2^-100, 2^100] -> ERR_ARG, 2^30 bins or more -> ERR_RANGE, |value| >=
// 2^32 * 2e -> ERR_RANGE; then the 63-bit key space of LCP-S).
// ---------------------------------------------------------------------------
__global__ void k_plan(const MinMax *mm, uint64_t n, uint32_t d, double eb, int mode,
                       uint32_t p, uint32_t nbits_target, uint32_t method, Plan *plan) {
  __shared__ int st[kMaxD];
  const int f = threadIdx.x;
  uint32_t lp = 0;
  while (p > 1 && (1u << lp) < p) ++lp;
  if (f < (int)d) {
    float mn = 0.0f, mx = 0.0f;
    if (n > 0) {
      mn = order_key_inv(mm->lo[f]);
      mx = order_key_inv(mm->hi[f]);
    }
    st[f] = plan_field(mn, mx, eb, mode, lp, plan->f[f]);
  }
  __syncthreads();
  if (f != 0) return;
  plan->d = d;
  plan->lp = lp;
  plan->n = n;
  plan->method = method;
  plan->nbits = 0;
  plan->key_bits = 0;
  plan->part_shift = 0;
  plan->rel_bits = lp * d;
  int status = OK;
  if (n > 0 && mm->nonfinite) status = ERR_NONFINITE;
  for (uint32_t k = 0; status == OK && k < d; ++k) status = st[k];
  if (status == OK && method == 0) {
    // key space: prod(bn_f) * p^d <= 2^63
    unsigned long long blocks = 1ull;
    bool over = false;
    for (uint32_t k = 0; k < d; ++k) {
      plan->f[k].stride = blocks;
      unsigned long long bn = plan->f[k].bn;
      if (blocks > (~0ull) / bn) {
        over = true;
        break;
      }
      blocks *= bn;
    }
    if (!over) over = (lp * d > 63) || (blocks > (1ull << (63 - lp * d)));
    if (over) {
      status = ERR_RANGE;
    } else {
      unsigned long long maxkey = (blocks << (lp * d)) - 1ull;
      uint32_t kb = bitlen64(maxkey);
      uint32_t bid_bits = kb > lp * d ? kb - lp * d : 0u;
      uint32_t nb = nbits_target < bid_bits ? nbits_target : bid_bits;
      plan->key_bits = kb;
      plan->nbits = nb;
      plan->part_shift = kb - nb;
    }
  }
  plan->status = status;
}

void launch_plan(const MinMax *mm, uint64_t n, uint32_t d, double eb, int mode, uint32_t p,
                 uint32_t nbits_target, uint32_t method, Plan *plan, cudaStream_t s) {
  note_launch();
  k_plan<<<1, 32, 0, s>>>(mm, n, d, eb, mode, p, nbits_target, method, plan);
}

// ---------------------------------------------------------------------------
// LCP-S quantize + key.  Tile t (one CTA) owns the contiguous input range
// [t*span, (t+1)*span); it writes each particle's key (block_id * p^d + rel,
// or kOutlierBit | index for particles kept raw) and a histogram of the
// partition buckets of its range.
// ---------------------------------------------------------------------------
template <int D>
__device__ __forceinline__ void quant_particle(const float *xs, const Plan &P, uint64_t i,
                                               unsigned long long &key, int32_t *qs) {
  bool bad = false;
  unsigned long long bid = 0ull, rel = 0ull;
  const uint32_t lp = P.lp;
  const unsigned long long pm = (1ull << lp) - 1ull;
#pragma unroll
  for (int f = 0; f < D; ++f) {
    const FieldPlan &F = P.f[f];
    bool chk;
    int32_t q = quantize(xs[f], F, chk);
    if (chk) bad |= violates(xs[f], reconstruct(q, F), F.e);
    qs[f] = q;
    bid += ((unsigned long long)q >> lp) * F.stride;
    rel |= ((unsigned long long)q & pm) << (f * lp);
  }
  key = bad ? (kOutlierBit | i) : ((bid << P.rel_bits) | rel);
}

template <int D>
__global__ void __launch_bounds__(512, 2) k_quantize_s(const float *__restrict__ fields, uint64_t n,
                                                    const Plan *__restrict__ plan, uint32_t nb1,
                                                    uint64_t span,
                                                    unsigned long long *__restrict__ keys,
                                                    uint32_t *__restrict__ tile_hist,
                                                    int32_t *__restrict__ qout) {
  extern __shared__ uint32_t s_hist[];
  __shared__ Plan sP;
  if (threadIdx.x == 0) sP = *plan;
  for (uint32_t b = threadIdx.x; b < nb1; b += blockDim.x) s_hist[b] = 0u;
  __syncthreads();
  if (sP.status != OK) return;
  const uint64_t lo = (uint64_t)blockIdx.x * span;
  const uint64_t hi = min(n, lo + span);
  const uint32_t shift = sP.part_shift;
  const uint32_t nb = nb1 - 1;
  // one particle per thread per round (loads coalesced across the warp);
  // the trip count is uniform so that bucket counts can be aggregated
  // across lanes: one atomic per run of lanes with the same bucket
  for (uint64_t b0 = lo; b0 < hi; b0 += blockDim.x) {
    const uint64_t i = b0 + threadIdx.x;
    const bool valid = i < hi;
    uint32_t b = 0u;
    if (valid) {
      float xs[D];
#pragma unroll
      for (int f = 0; f < D; ++f) xs[f] = __ldcs(fields + (uint64_t)f * n + i);
      unsigned long long k;
      int32_t qs[D];
      quant_particle<D>(xs, sP, i, k, qs);
      b = (k & kOutlierBit) ? nb : (uint32_t)(k >> shift);
      keys[i] = k;
      if (qout) {
#pragma unroll
        for (int f = 0; f < D; ++f) qout[(uint64_t)f * n + i] = qs[f];
      }
    }
    int leader;
    uint32_t rank, len;
    lane_runs(b, valid, leader, rank, len);
    if (valid && rank == 0u) atomicAdd(&s_hist[b], len);
  }
  __syncthreads();
  uint32_t *th = tile_hist + (uint64_t)blockIdx.x * nb1;
  for (uint32_t b = threadIdx.x; b < nb1; b += blockDim.x) th[b] = s_hist[b];
}

template <int D>
static void launch_q(const float *fields, uint64_t n, const Plan *plan, uint32_t nb1, int tiles,
                     unsigned long long *keys, uint32_t *tile_hist, int32_t *q, cudaStream_t s) {
  uint64_t span = (n + tiles - 1) / tiles;
  span = (span + 3) & ~3ull;
  size_t smem = sizeof(uint32_t) * nb1;
  static const bool attr =  // once per instantiation, thread-safe
      cudaFuncSetAttribute(k_quantize_s<D>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           200 * 1024) == cudaSuccess;
  (void)attr;
  note_launch();
  k_quantize_s<D><<<tiles, 512, smem, s>>>(fields, n, plan, nb1, span, keys, tile_hist, q);
}

void launch_quantize_s(const float *fields, uint64_t n, uint32_t d, const Plan *plan,
                       uint32_t nb1, int tiles, unsigned long long *keys, uint32_t *tile_hist,
                       int32_t *q, cudaStream_t s) {
  switch (d) {
    case 1: launch_q<1>(fields, n, plan, nb1, tiles, keys, tile_hist, q, s); break;
    case 2: launch_q<2>(fields, n, plan, nb1, tiles, keys, tile_hist, q, s); break;
    case 3: launch_q<3>(fields, n, plan, nb1, tiles, keys, tile_hist, q, s); break;
    case 4: launch_q<4>(fields, n, plan, nb1, tiles, keys, tile_hist, q, s); break;
    case 5: launch_q<5>(fields, n, plan, nb1, tiles, keys, tile_hist, q, s); break;
    case 6: launch_q<6>(fields, n, plan, nb1, tiles, keys, tile_hist, q, s); break;
    case 7: launch_q<7>(fields, n, plan, nb1, tiles, keys, tile_hist, q, s); break;
    default: launch_q<8>(fields, n, plan, nb1, tiles, keys, tile_hist, q, s); break;
  }
}

// ---------------------------------------------------------------------------
// element rules (verification entry point)
// ---------------------------------------------------------------------------
__global__ void k_element_rules(const float *__restrict__ x, uint64_t n,
                                const FieldPlan *__restrict__ fp, int32_t *__restrict__ q,
                                float *__restrict__ xr, uint8_t *__restrict__ viol,
                                int *__restrict__ status) {
  const FieldPlan F = *fp;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    bool chk;
    float v = x[i];
    int32_t qq = quantize(v, F, chk);
    float r = reconstruct(qq, F);
    q[i] = qq;
    xr[i] = r;
    viol[i] = violates(v, r, F.e) ? 1 : 0;
    if (qq < 0 || qq >= (1 << 30)) atomicExch(status, ERR_RANGE);  // outside the domain
  }
}

__global__ void k_field_plan(float m, float e, float max_abs, FieldPlan *fp, int *status) {
  // a one-field plan with min m and bound e; the largest value only matters
  // for the guard window, which the element entry point does not use
  FieldPlan F;
  double ebf = (double)e;
  int st = plan_field(m, m, ebf, 0, 0, F);
  (void)max_abs;  // unused: k_element_rules checks every q < 2^30; no rule on |x|
  *fp = F;
  *status = st;
}

void launch_element_rules(const float *x, uint64_t n, FieldPlan *fp_dev, int32_t *q, float *xr,
                          uint8_t *viol, int *status, cudaStream_t s) {
  if (n == 0) return;
  uint64_t blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  note_launch();
  k_element_rules<<<(unsigned)blocks, 256, 0, s>>>(x, n, fp_dev, q, xr, viol, status);
}

void launch_field_plan(float m, float e, float max_abs, FieldPlan *fp, int *status,
                       cudaStream_t s) {
  note_launch();
  k_field_plan<<<1, 1, 0, s>>>(m, e, max_abs, fp, status);
}

}  // namespace lcp
