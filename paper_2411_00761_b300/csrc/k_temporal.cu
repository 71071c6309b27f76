// k_temporal.cu -- LCP-T kernels (Sec. "LCP-T: The Temporal Compressor").
//
// A temporal frame is quantized like LCP-S (Eq. quantization), every code is
// predicted by the reference frame's code of the same particle, and the
// differences form one stream, field-major: symbol f * n + j is the zigzag
// of q_t[f][pi(j)] - q_ref[f][j], where j is the reference's decoded slot and
// pi(j) the input index of the particle decoded there.  Elements whose
// rounded centre misses the bound are patched with their raw value.
#include <algorithm>

#include "lcp_kernels.h"

namespace lcp {

template <int D_UNUSED>
__global__ void __launch_bounds__(512) k_quantize_t(const float *__restrict__ fields, uint64_t n,
                                                    const Plan *__restrict__ plan,
                                                    const uint32_t *__restrict__ pi,
                                                    const int32_t *__restrict__ qref,
                                                    uint32_t *__restrict__ sym,
                                                    int32_t *__restrict__ qnew,
                                                    uint32_t *__restrict__ hist,
                                                    unsigned long long *__restrict__ maxv,
                                                    unsigned long long *__restrict__ kcount,
                                                    unsigned long long *__restrict__ patch_s,
                                                    float *__restrict__ patch_x) {
  __shared__ uint32_t h[kAlpha];
  __shared__ FieldPlan F;
  __shared__ unsigned long long s_max;
  __shared__ int s_status;
  const int f = blockIdx.y;
  for (int i = threadIdx.x; i < kAlpha; i += blockDim.x) h[i] = 0u;
  if (threadIdx.x == 0) {
    F = plan->f[f];
    s_max = 0ull;
    s_status = plan->status;
  }
  __syncthreads();
  if (s_status != OK) return;
  const float *x = fields + (uint64_t)f * n;
  unsigned long long mymax = 0ull;
  for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
       j += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t s = (uint64_t)f * n + j;
    const float v = __ldg(x + pi[j]);
    bool chk;
    const int32_t q = quantize(v, F, chk);
    if (chk && violates(v, reconstruct(q, F), F.e)) {
      unsigned long long k = atomicAdd(kcount, 1ull);
      patch_s[k] = s;
      patch_x[k] = v;
    }
    const unsigned long long z = zigzag((long long)q - (long long)qref[s]);
    sym[s] = (uint32_t)z;
    qnew[s] = q;
    atomicAdd(&h[z < (unsigned long long)kEsc ? (uint32_t)z : (uint32_t)kEsc], 1u);
    mymax = z > mymax ? z : mymax;
  }
  atomicMax(&s_max, mymax);
  __syncthreads();
  for (int i = threadIdx.x; i < kAlpha; i += blockDim.x)
    if (h[i]) atomicAdd(&hist[i], h[i]);
  if (threadIdx.x == 0 && s_max) atomicMax(maxv, s_max);
}

void launch_quantize_t(const float *fields, uint64_t n, uint32_t d, const Plan *plan,
                       const uint32_t *pi, const int32_t *qref, uint32_t *sym, int32_t *qnew,
                       uint32_t *hist, unsigned long long *maxv, unsigned long long *kcount,
                       unsigned long long *patch_s, float *patch_x, int sms, cudaStream_t s) {
  if (n == 0) return;
  unsigned gx = (unsigned)std::min<unsigned long long>((n + 511) / 512, (unsigned long long)(2 * sms));
  gx = (gx + d - 1) / d;
  if (gx == 0) gx = 1;
  note_launch();
  k_quantize_t<0><<<dim3(gx, d), 512, 0, s>>>(fields, n, plan, pi, qref, sym, qnew, hist, maxv,
                                              kcount, patch_s, patch_x);
}

// patches: sorted (by symbol index) list -> container
__global__ void k_patches_write(const unsigned long long *__restrict__ ps,
                                const uint32_t *__restrict__ order,
                                const float *__restrict__ px, const StreamDesc *__restrict__ od,
                                uint8_t *__restrict__ out, const Summary *__restrict__ summary) {
  const Summary S = *summary;
  if (S.status != OK || S.K == 0) return;
  uint8_t *o = out + od->offset;
  uint32_t *ow = reinterpret_cast<uint32_t *>(o);
  float *ov = reinterpret_cast<float *>(o + pad16(8ull * S.K));
  for (unsigned long long k = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; k < S.K;
       k += (unsigned long long)gridDim.x * blockDim.x) {
    unsigned long long s = ps[k];
    ow[2 * k] = (uint32_t)s;
    ow[2 * k + 1] = (uint32_t)(s >> 32);
    ov[k] = px[order[k]];
  }
}

void launch_patches_write(const unsigned long long *ps, const uint32_t *order, const float *px,
                          const StreamDesc *od, uint8_t *out, const Summary *summary, int sms,
                          cudaStream_t s) {
  note_launch();
  k_patches_write<<<sms, 256, 0, s>>>(ps, order, px, od, out, summary);
}

// decode: q = q_ref + unzigzag(symbol), reconstruct, new reference codes
__global__ void __launch_bounds__(512) k_recon_t(const Plan *__restrict__ plan, uint64_t n,
                                                 const uint32_t *__restrict__ sym,
                                                 const int32_t *__restrict__ qref,
                                                 float *__restrict__ out,
                                                 int32_t *__restrict__ qnew,
                                                 int *__restrict__ err) {
  __shared__ FieldPlan F;
  const int f = blockIdx.y;
  if (threadIdx.x == 0) F = plan->f[f];
  __syncthreads();
  for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
       j += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t s = (uint64_t)f * n + j;
    long long q = (long long)qref[s] + unzigzag(sym[s]);
    if (q < 0 || q > (long long)F.qmax) {
      atomicExch(err, 1);
      q = 0;
    }
    if (out) {  // null: codes only (a reference frame)
      float z;
      out[s] = recon_rn_f32(q, F.m, F.e, z) ? z : reconstruct(q, F);
    }
    qnew[s] = (int32_t)q;
  }
}

// value-space prediction across grids (Sec. "Best error-bound scale for
// anchor frames"): a reference code on the reference's grid (Q2) quantized on
// this frame's grid (Q1), clamped to [0, qmax]
__global__ void __launch_bounds__(512) k_requant(const Plan *__restrict__ plan, uint64_t n,
                                                 const int32_t *__restrict__ qref, RefGrid g,
                                                 int32_t *__restrict__ qout) {
  __shared__ FieldPlan F;
  const int f = blockIdx.y;
  if (threadIdx.x == 0) F = plan->f[f];
  __syncthreads();
  const FieldPlan &R = g.f[f];
  const double inv2e = 0.5 / (double)F.e;
  for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
       j += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t s = (uint64_t)f * n + j;
    const float x = reconstruct((long long)qref[s], R);
    int32_t q = 0;
    if (x >= F.m) {
      if (((double)x - (double)F.m) * inv2e >= (double)F.qmax + 1.0) {
        q = (int32_t)F.qmax;  // beyond the grid: no exact Q1 needed
      } else {
        bool chk;
        const int32_t r = quantize(x, F, chk);
        q = r > (int32_t)F.qmax ? (int32_t)F.qmax : r;
      }
    }
    qout[s] = q;
  }
}

void launch_requant(const Plan *plan, uint64_t n, uint32_t d, const int32_t *qref,
                    const RefGrid &g, int32_t *qout, int sms, cudaStream_t s) {
  if (n == 0) return;
  unsigned gx = (unsigned)std::min<unsigned long long>((n + 511) / 512, (unsigned long long)(4 * sms));
  note_launch();
  k_requant<<<dim3(gx, d), 512, 0, s>>>(plan, n, qref, g, qout);
}

void launch_recon_t(const Plan *plan, uint64_t n, uint32_t d, const uint32_t *sym,
                    const int32_t *qref, float *out, int32_t *qnew, int *err, int sms,
                    cudaStream_t s) {
  if (n == 0) return;
  unsigned gx = (unsigned)std::min<unsigned long long>((n + 511) / 512, (unsigned long long)(4 * sms));
  note_launch();
  k_recon_t<<<dim3(gx, d), 512, 0, s>>>(plan, n, sym, qref, out, qnew, err);
}

__global__ void k_patches_apply(const uint8_t *__restrict__ sec, uint64_t K, uint64_t nd,
                                float *__restrict__ out, int *__restrict__ err) {
  const uint32_t *iw = reinterpret_cast<const uint32_t *>(sec);
  const float *v = reinterpret_cast<const float *>(sec + pad16(8ull * K));
  for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < K;
       k += (uint64_t)gridDim.x * blockDim.x) {
    unsigned long long s = (unsigned long long)iw[2 * k] | ((unsigned long long)iw[2 * k + 1] << 32);
    if (s >= nd) {
      atomicExch(err, 1);
      continue;
    }
    out[s] = v[k];
  }
}

void launch_patches_apply(const uint8_t *sec, uint64_t K, uint64_t nd, float *out, int *err,
                          int sms, cudaStream_t s) {
  if (K == 0) return;
  note_launch();
  k_patches_apply<<<sms, 256, 0, s>>>(sec, K, nd, out, err);
}

}  // namespace lcp
