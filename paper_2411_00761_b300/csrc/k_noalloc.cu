// k_noalloc.cu -- the element rules for callers that cannot allocate.
//
// lcp_quantize() gets a small per-call device buffer for its plan and status.
// Some callers cannot allow that: code that runs inside an application whose
// device memory is owned by the application's own pool (a cudaMalloc there
// would bypass the pool and synchronize the device), or real-time loops that
// forbid allocation once they are running.  lcp_quantize_noalloc() computes
// the same results with all of its scratch in one fixed, file-scope device
// array, so it allocates nothing; the caller still provides inputs and
// outputs.
#include <stddef.h>

#include <mutex>

#include "../../include/lcp.h"
#include "lcp_kernels.h"

using namespace lcp;

namespace {

constexpr int kNaThreads = 256;
constexpr int kNaPerThread = 16;
constexpr uint32_t kNaMaxCtas = 4096;
static_assert((unsigned long long)kNaMaxCtas * kNaThreads * kNaPerThread ==
                  LCP_NOALLOC_MAX_ELEMENTS,
              "limit stated in lcp.h");

// Scratch of every call: a completion counter (must be zero when a call
// starts), the per-CTA violation counts, and the call's status and total.
// 16.5 KB, held by every GPU that loads the library until the process exits.
struct NoallocScratch {
  unsigned int done;
  int status;
  unsigned long long total;
  unsigned int partial[kNaMaxCtas];
};
static __device__ __align__(256) NoallocScratch g_noalloc_scratch;

__global__ void __launch_bounds__(kNaThreads) k_element_rules_noalloc(
    const float *__restrict__ x, uint64_t n, float m, float e, float max_abs,
    int32_t *__restrict__ q, float *__restrict__ xr, uint8_t *__restrict__ viol,
    NoallocScratch *scr) {
  __shared__ FieldPlan F;
  __shared__ int st;
  __shared__ unsigned int s_cnt;
  __shared__ bool s_last;
  if (threadIdx.x == 0) {
    st = plan_field(m, m, (double)e, 0, 0, F);
    (void)max_abs;  // unused: the kernel checks q < 2^30 on every value
    s_cnt = 0u;
  }
  __syncthreads();
  unsigned int c = 0;
  if (st == OK) {
    const uint64_t base = (uint64_t)blockIdx.x * kNaThreads * kNaPerThread;
#pragma unroll 4
    for (int k = 0; k < kNaPerThread; ++k) {
      const uint64_t i = base + (uint64_t)k * kNaThreads + threadIdx.x;
      if (i < n) {
        bool chk;
        const float v = x[i];
        const int32_t qq = quantize(v, F, chk);
        const float r = reconstruct(qq, F);
        const bool bad = violates(v, r, F.e);
        q[i] = qq;
        xr[i] = r;
        viol[i] = bad ? 1 : 0;
        c += bad;
        if (qq < 0 || qq >= (1 << 30)) c |= 0x80000000u;  // outside the domain
      }
    }
  }
  const bool out_of_range = __any_sync(0xffffffffu, (c & 0x80000000u) != 0u);
  c = __reduce_add_sync(0xffffffffu, c & 0x7fffffffu);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(&s_cnt, c);
  if ((threadIdx.x & 31) == 0 && out_of_range) atomicOr(&s_cnt, 0x80000000u);
  __syncthreads();
  if (threadIdx.x == 0) {
    scr->partial[blockIdx.x] = s_cnt;
    __threadfence();
    s_last = atomicAdd(&scr->done, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (s_last && threadIdx.x == 0) {
    __threadfence();
    unsigned long long t = 0;
    bool range = false;
    for (unsigned int b = 0; b < gridDim.x; ++b) {
      const unsigned int v = *(volatile unsigned int *)&scr->partial[b];
      t += v & 0x7fffffffu;
      range |= (v & 0x80000000u) != 0u;
    }
    scr->total = t;
    scr->status = (st == OK && range) ? ERR_RANGE : st;
  }
}

// device address of the scratch array, resolved once per device
std::mutex g_na_mutex;
NoallocScratch *g_na_ptr[128] = {};

int noalloc_scratch(NoallocScratch **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) {
    cudaGetLastError();
    return ERR_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_na_mutex);
  if (!g_na_ptr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return ERR_CUDA;
    }
    g_na_ptr[dev] = reinterpret_cast<NoallocScratch *>(p);
  }
  *out = g_na_ptr[dev];
  return OK;
}

}  // namespace

extern "C" lcp_status lcp_quantize_noalloc(const float *d_x, uint64_t n, float m, float e,
                                           float max_abs, int32_t *d_q, float *d_xr,
                                           uint8_t *d_viol, uint64_t *n_violations,
                                           void *stream) {
  if (n > LCP_NOALLOC_MAX_ELEMENTS) return LCP_ERR_ARG;
  if (n > 0 && (!d_x || !d_q || !d_xr || !d_viol)) return LCP_ERR_ARG;
  if (!(e > 0.0f)) return LCP_ERR_ARG;
  NoallocScratch *scr = nullptr;
  int st = noalloc_scratch(&scr);
  if (st != OK) return (lcp_status)st;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemsetAsync(&scr->done, 0, sizeof(unsigned int), s) != cudaSuccess) {
    cudaGetLastError();
    return LCP_ERR_CUDA;
  }
  const uint64_t per = (uint64_t)kNaThreads * kNaPerThread;
  unsigned grid = (unsigned)((n + per - 1) / per);
  if (grid == 0) grid = 1;
  note_launch();
  k_element_rules_noalloc<<<grid, kNaThreads, 0, s>>>(d_x, n, m, e, max_abs, d_q, d_xr, d_viol,
                                                      scr);
  struct {  // same layout as the head of NoallocScratch
    unsigned int done;
    int status;
    unsigned long long total;
  } res;
  static_assert(offsetof(NoallocScratch, total) == 8, "scratch head layout");
  if (cudaGetLastError() != cudaSuccess ||
      cudaMemcpyAsync(&res, scr, sizeof(res), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return LCP_ERR_CUDA;
  }
  if (n_violations) *n_violations = res.status == OK ? res.total : 0;
  return (lcp_status)res.status;
}
