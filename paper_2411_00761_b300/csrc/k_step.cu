// k_step.cu -- one time step of many trajectories' LCP-T frames (config 4),
// decoded in one persistent launch.
//
// Sec. "LCP-T: The Temporal Compressor" codes a frame as the differences of
// its codes from the reference frame's; the stream is field-major, so symbol
// s = f N + j is exactly element s of the [d][N] reference codes and of the
// decoded frame.  A lane that decodes a chunk of the stream can therefore
// finish every symbol on the spot: q = q_ref[s] + unzigzag(symbol), checked
// against [0, qmax_f], reconstructed by Eq. quantization (reverse) and
// stored.  The planning is on the device as well: one CTA per frame reads
// its container's header and stream section, builds the frame's field plans
// and Huffman tables and counts its work items; a scan places the items of
// all frames in one list that a persistent grid takes from a counter.  With
// fixed grids and descriptors in device memory, the whole step is one CUDA
// graph that the host replays every time step.
#include <algorithm>

#include "lcp_kernels.h"

namespace lcp {

namespace {

__device__ __forceinline__ unsigned long long ld64(const uint8_t *p) {
  unsigned long long v = 0;
  for (int i = 7; i >= 0; --i) v = (v << 8) | p[i];
  return v;
}
__device__ __forceinline__ uint32_t ld32(const uint8_t *p) {
  return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}

constexpr int kStepThreads = 256;
constexpr int kStepR = 8;       // symbols per round and lane
constexpr int kStepRing = 64;   // payload words per lane (ring in shared memory)
static_assert(kStepR * (kLmax + 32) <= 32 * (kStepRing / 2 - 2), "ring covers two rounds");

// parse one LCP-T container (the rules of the host-side header reader)
__device__ int parse_t(const StepIn &J, StepFrame &F) {
  const uint8_t *in = J.in;
  if (!in || J.in_size < 48) return ERR_FORMAT;
  if (in[0] != 'L' || in[1] != 'C' || in[2] != 'P' || in[3] != '1' || in[4] != 1) return ERR_FORMAT;
  if (in[5] != 1) return ERR_FORMAT;  // LCP-T only
  const uint32_t d = in[6], lc = in[7];
  if (d < 1 || d > kMaxD || lc < 5 || lc > 10) return ERR_FORMAT;
  const uint32_t flags = ld32(in + 8);
  if (flags & 4u) return ERR_FORMAT;  // re-quantized reference: not on this path
  const unsigned long long n = ld64(in + 16), K = ld64(in + 24), total = ld64(in + 40);
  const unsigned long long H = 48ull + 16ull * d + 16ull * 1 + 16ull;
  if (total > J.in_size || total < H || n >= (1ull << 32) || n != J.n || d != J.d) return ERR_FORMAT;
  F.d = d;
  F.n = n;
  F.nd = n * d;
  F.K = K;
  F.log2_chunk = lc;
  unsigned long long off[2], bytes[2];
  for (int k = 0; k < 2; ++k) {
    off[k] = ld64(in + 48 + 16 * d + 16 * k);
    bytes[k] = ld64(in + 48 + 16 * d + 16 * k + 8);
    if (off[k] < H || off[k] > total || bytes[k] > total - off[k] || (off[k] & 15)) return ERR_FORMAT;
  }
  if (bytes[1] != pad16(8ull * K) + pad16(4ull * K) || K > n * d) return ERR_FORMAT;
  if (bytes[0] < 32) return ERR_FORMAT;
  const uint8_t *sh = in + off[0];
  F.sec = sh;
  F.patch = in + off[1];
  F.coder = sh[0];
  F.width = sh[1];
  F.used = (uint32_t)sh[2] | ((uint32_t)sh[3] << 8);
  const unsigned long long sn = ld64(sh + 8);
  F.payload_bits = ld64(sh + 16);
  if (sn != n * d || F.width > 32 || F.coder > 1) return ERR_FORMAT;
  F.n_chunks = (F.nd + (1ull << lc) - 1) >> lc;
  if (F.coder == 0) {
    if (F.payload_bits != F.nd * F.width) return ERR_FORMAT;
    if (bytes[0] != 32 + pad16(4 * words_of(F.payload_bits))) return ERR_FORMAT;
    F.ct = nullptr;
    F.pl = reinterpret_cast<const uint32_t *>(sh + 32);
  } else {
    if (F.used == 0 || F.used > (uint32_t)kAlpha) return ERR_FORMAT;
    if (bytes[0] != pad16(80ull + 2ull * F.used) + pad16(8 * F.n_chunks) +
                        pad16(4 * words_of(F.payload_bits)))
      return ERR_FORMAT;
    F.ct = sh + pad16(80ull + 2ull * F.used);
    F.pl = reinterpret_cast<const uint32_t *>(F.ct + pad16(8ull * F.n_chunks));
  }
  F.nwords = words_of(F.payload_bits);
  for (uint32_t f = 0; f < d; ++f) {
    float m, e;
    const uint32_t mb = ld32(in + 48 + 16 * f), eb = ld32(in + 52 + 16 * f);
    m = __uint_as_float(mb);
    e = __uint_as_float(eb);
    const uint32_t qmax = ld32(in + 56 + 16 * f);
    if (qmax >= (1u << 30)) return ERR_FORMAT;
    FieldPlan P;
    if (plan_field(m, m, (double)e, 0, 0, P) != OK) return ERR_FORMAT;
    P.qmax = qmax;
    field_block_grid(P, 0);  // the plan a one-frame decode records, field for field
    F.f[f] = P;
  }
  unsigned long long stride = 1ull;
  for (uint32_t f = 0; f < d; ++f) {
    F.f[f].stride = stride;
    stride *= F.f[f].bn;
  }
  return OK;
}

}  // namespace

// per frame: header, plans, Huffman tables (k_huff_table's construction), items
__global__ void __launch_bounds__(kStepThreads) k_step_plan(const uint32_t *__restrict__ nframes,
                                                            const StepIn *__restrict__ jobs,
                                                            StepFrame *__restrict__ frames,
                                                            HuffTable *__restrict__ tabs) {
  const uint32_t fi = blockIdx.x;
  if (fi >= *nframes) return;
  StepFrame &F = frames[fi];
  __shared__ int s_st;
  if (threadIdx.x == 0) {
    F.err = 0u;
    F.groups = 0ull;
    const int st = parse_t(jobs[fi], F);
    F.status = st;
    if (st == OK) F.groups = (F.n_chunks + 31) / 32;
    s_st = st;
  }
  __syncthreads();
  if (s_st != OK || F.coder != 1) return;
  // canonical decode tables of the frame's stream
  HuffTable *T = tabs + fi;
  const uint8_t *sec = F.sec;
  __shared__ uint32_t cnt[kLmax + 1], first[kLmax + 2], index[kLmax + 2];
  const uint32_t U = F.used;
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
      T->index[L] = idx - cnt[L];
      T->count[L] = cnt[L];
    }
    T->used = U;
    T->ok = (total == U && U > 0 && U <= (uint32_t)kAlpha) ? 1u : 0u;
    if (!T->ok) F.status = ERR_FORMAT;
  }
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < U && i < (uint32_t)kAlpha; i += blockDim.x)
    T->syms[i] = (uint16_t)((uint32_t)sec[80 + 2 * i] | ((uint32_t)sec[81 + 2 * i] << 8));
  __syncthreads();
  huff_fill_fast(first, cnt, index, T->syms, min(U, (uint32_t)kAlpha), T->fast);
}

// places every frame's items in one list (frames of a failed plan get none)
__global__ void k_step_items(const uint32_t *__restrict__ nframes, StepFrame *__restrict__ frames,
                             unsigned long long *__restrict__ items) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  unsigned long long run = 0;
  const uint32_t nf = *nframes;
  for (uint32_t f = 0; f < nf; ++f) {
    frames[f].item0 = run;
    items[f] = run;
    if (frames[f].status == OK) run += frames[f].groups;
  }
  items[nf] = run;
  items[kStepMaxFrames + 1] = 0ull;  // the work counter
}

// the persistent decode: a warp takes an item (32 chunks of one frame), each
// lane decodes its chunk and finishes every symbol
__global__ void __launch_bounds__(kStepThreads) k_step_decode(const uint32_t *__restrict__ nframes,
                                                              const StepIn *__restrict__ jobs,
                                                              StepFrame *__restrict__ frames,
                                                              const HuffTable *__restrict__ tabs,
                                                              unsigned long long *__restrict__ items) {
  extern __shared__ __align__(16) uint32_t st_ring[];
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  uint32_t *myring = st_ring + (size_t)wl * (kStepRing * 32) + lane;
  const uint32_t nf = *nframes;
  const unsigned long long total = items[nf];
  for (;;) {
    unsigned long long it = 0;
    if (lane == 0) it = atomicAdd(&items[kStepMaxFrames + 1], 1ull);
    it = __shfl_sync(0xffffffffu, it, 0);
    if (it >= total) break;
    uint32_t lo = 0, hi = nf;  // the frame: last f with items[f] <= it
    while (hi - lo > 1) {
      const uint32_t mid = (lo + hi) >> 1;
      if (items[mid] <= it) lo = mid;
      else hi = mid;
    }
    const uint32_t fi = lo;
    StepFrame &F = frames[fi];
    const StepIn J = jobs[fi];
    const unsigned long long g = it - F.item0;
    const unsigned long long cs = 1ull << F.log2_chunk;
    const unsigned long long c = g * 32 + lane;
    const bool act = c < F.n_chunks;
    const unsigned long long s0 = c * cs;
    const unsigned long long s1 = act ? min(F.nd, s0 + cs) : s0;
    const uint32_t mine = (uint32_t)(s1 - s0);
    const unsigned long long n = F.n;
    // the field of the first symbol, then counted along
    uint32_t fld = act ? (uint32_t)(s0 / n) : 0u;
    unsigned long long fend = act ? (unsigned long long)(fld + 1) * n : 0ull;
    float fm = F.f[fld].m, fe = F.f[fld].e;
    uint32_t qmax = F.f[fld].qmax;
    bool bad = false;
    const uint32_t width = F.width;
    const uint32_t *pl = F.pl;
    const unsigned long long nwords = F.nwords;
    // Huffman: the lane's payload through the ring; fixed: by position
    const HuffTable *T = tabs + fi;
    unsigned long long pos0 = 0;
    uint32_t bp = 0, issued = 0, avail = 0;
    const uint32_t *src = pl;
    const bool huff = F.coder == 1;
    if (act && huff) {
      const uint32_t *ctw = reinterpret_cast<const uint32_t *>(F.ct);
      pos0 = (unsigned long long)ctw[2 * c] | ((unsigned long long)ctw[2 * c + 1] << 32);
      if (pos0 > F.payload_bits) {
        bad = true;
        pos0 = 0;
      }
      src = pl + (pos0 >> 5);
      const unsigned long long left = nwords - (pos0 >> 5);
      avail = left < 0xffffffffull ? (uint32_t)left : 0xffffffffu;
      bp = (uint32_t)(pos0 & 31);
      for (; issued < (uint32_t)kStepRing; ++issued)
        cp_async4(myring + issued * 32, issued < avail ? src + issued : pl, issued < avail);
    }
    cp_async_commit();
    cp_async_wait0();
    auto peek32 = [&](uint32_t b) {
      const uint32_t wi = b >> 5;
      const uint32_t x = myring[(wi & (kStepRing - 1)) * 32];
      const uint32_t y = myring[((wi + 1) & (kStepRing - 1)) * 32];
      return __funnelshift_l(y, x, b & 31);
    };
    for (uint32_t r0 = 0; r0 < mine; r0 += kStepR) {
      if (huff) {
        if (r0) {
          const uint32_t need = (bp >> 5) + (uint32_t)kStepRing;
          for (; issued < need; ++issued)
            cp_async4(myring + (issued & (kStepRing - 1)) * 32, issued < avail ? src + issued : pl,
                      issued < avail);
        }
        cp_async_commit();
        cp_async_wait1();
      }
      const uint32_t todo = min(mine - r0, (uint32_t)kStepR);
      uint32_t v[kStepR];
#pragma unroll
      for (uint32_t k = 0; k < (uint32_t)kStepR; ++k) {
        const bool on = k < todo;
        uint32_t x = 0u;
        if (huff) {
          const uint32_t win = peek32(bp);
          const uint32_t e = T->fast[win >> (32 - kFastBits)];
          uint32_t sym = e >> 5, len = e & 31u;
          const bool longc = on && e == 0u;
          if (__any_sync(__activemask(), longc)) {
            if (longc) {
              int L = kFastBits + 1;
              uint32_t code = 0;
              for (; L <= kLmax; ++L) {
                code = win >> (32 - L);
                if (code - T->first[L] < T->count[L]) break;
              }
              if (L > kLmax) {
                bad = true;
                sym = 0;
                len = 1;
              } else {
                sym = T->syms[T->index[L] + (code - T->first[L])];
                len = (uint32_t)L;
              }
            }
          }
          const bool esc = on && sym == (uint32_t)kEsc && width > 0;
          const uint32_t hw = peek32(bp + len);
          x = esc ? (hw >> (32u - width)) : sym;
          bp += on ? len + (esc ? width : 0u) : 0u;
        } else if (on && width) {
          const unsigned long long bit = (s0 + r0 + k) * width;
          const unsigned long long wi = bit >> 5;
          const uint32_t a = __ldg(pl + wi), b = wi + 1 < nwords ? __ldg(pl + wi + 1) : 0u;
          x = __funnelshift_l(b, a, (uint32_t)(bit & 31)) >> (32u - width);
        }
        v[k] = x;
      }
      // finish the round's symbols: codes, range, values
      const unsigned long long sb = s0 + r0;
      int32_t q[kStepR];
      float y[kStepR];
      const bool full = todo == (uint32_t)kStepR;
      int32_t qr[kStepR];
      if (full) {
        const int4 a = *reinterpret_cast<const int4 *>(J.qref + sb);
        const int4 b = *reinterpret_cast<const int4 *>(J.qref + sb + 4);
        qr[0] = a.x;
        qr[1] = a.y;
        qr[2] = a.z;
        qr[3] = a.w;
        qr[4] = b.x;
        qr[5] = b.y;
        qr[6] = b.z;
        qr[7] = b.w;
      } else {
#pragma unroll
        for (int k = 0; k < kStepR; ++k) qr[k] = (uint32_t)k < todo ? J.qref[sb + k] : 0;
      }
#pragma unroll
      for (int k = 0; k < kStepR; ++k) {
        const unsigned long long s = sb + k;
        if ((uint32_t)k < todo && s >= fend) {  // the next field
          ++fld;
          fend += n;
          fm = F.f[fld].m;
          fe = F.f[fld].e;
          qmax = F.f[fld].qmax;
        }
        long long qq = (long long)qr[k] + unzigzag((unsigned long long)v[k]);
        if ((uint32_t)k < todo && (qq < 0 || qq > (long long)qmax)) {
          bad = true;
          qq = 0;
        }
        q[k] = (int32_t)qq;
        float z;
        y[k] = recon_rn_f32(qq, fm, fe, z) ? z : reconstruct(qq, F.f[fld]);
      }
      if (full) {
        *reinterpret_cast<float4 *>(J.out + sb) = make_float4(y[0], y[1], y[2], y[3]);
        *reinterpret_cast<float4 *>(J.out + sb + 4) = make_float4(y[4], y[5], y[6], y[7]);
        *reinterpret_cast<int4 *>(J.qnew + sb) = make_int4(q[0], q[1], q[2], q[3]);
        *reinterpret_cast<int4 *>(J.qnew + sb + 4) = make_int4(q[4], q[5], q[6], q[7]);
      } else {
#pragma unroll
        for (int k = 0; k < kStepR; ++k)
          if ((uint32_t)k < todo) {
            J.out[sb + k] = y[k];
            J.qnew[sb + k] = q[k];
          }
      }
    }
    cp_async_wait0();
    if (huff && act && (pos0 & ~31ull) + bp > F.payload_bits) bad = true;
    if (bad) atomicOr(&F.err, 1u);
  }
}

// raw values of the patched symbols (the codes stay the decoded ones)
__global__ void k_step_patches(const uint32_t *__restrict__ nframes,
                               const StepIn *__restrict__ jobs, StepFrame *__restrict__ frames) {
  const uint32_t nf = *nframes;
  for (uint32_t fi = 0; fi < nf; ++fi) {
    StepFrame &F = frames[fi];
    if (F.status != OK || F.K == 0) continue;
    const uint32_t *iw = reinterpret_cast<const uint32_t *>(F.patch);
    const float *v = reinterpret_cast<const float *>(F.patch + pad16(8ull * F.K));
    for (unsigned long long k = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; k < F.K;
         k += (unsigned long long)gridDim.x * blockDim.x) {
      const unsigned long long s = (unsigned long long)iw[2 * k] | ((unsigned long long)iw[2 * k + 1] << 32);
      if (s >= F.nd) {
        atomicOr(&F.err, 1u);
        continue;
      }
      jobs[fi].out[s] = v[k];
    }
  }
}

// statuses and the field plans of every frame, for the host
__global__ void k_step_finish(const uint32_t *__restrict__ nframes,
                              const StepFrame *__restrict__ frames, StepResult *__restrict__ res) {
  const uint32_t nf = *nframes;
  for (uint32_t fi = blockIdx.x * blockDim.x + threadIdx.x; fi < nf; fi += gridDim.x * blockDim.x) {
    const StepFrame &F = frames[fi];
    StepResult R;
    R.status = (F.status == OK && F.err) ? ERR_FORMAT : F.status;
    R.pad = 0;
    for (int f = 0; f < kMaxD; ++f) R.f[f] = F.f[f];
    res[fi] = R;
  }
}

size_t step_decode_smem() { return sizeof(uint32_t) * kStepRing * 32 * (kStepThreads / 32); }

int launch_step(const uint32_t *nframes, const StepIn *jobs, StepFrame *frames, HuffTable *tabs,
                unsigned long long *items, StepResult *res, int sms, cudaStream_t s) {
  static const bool attr =  // once per process, thread-safe
      cudaFuncSetAttribute(k_step_decode, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)step_decode_smem()) == cudaSuccess;
  (void)attr;
  k_step_plan<<<kStepMaxFrames, kStepThreads, 0, s>>>(nframes, jobs, frames, tabs);
  k_step_items<<<1, 32, 0, s>>>(nframes, frames, items);
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_step_decode, kStepThreads,
                                                    step_decode_smem()) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  k_step_decode<<<sms * per_sm, kStepThreads, step_decode_smem(), s>>>(nframes, jobs, frames, tabs,
                                                                      items);
  k_step_patches<<<sms, 256, 0, s>>>(nframes, jobs, frames);
  k_step_finish<<<1, 256, 0, s>>>(nframes, frames, res);
  return 5;  // kernels recorded; counted once per replay by the caller
}

}  // namespace lcp
