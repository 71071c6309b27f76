// lcp_api.cu -- C ABI of the B300 LCP library: contexts, workspace,
// LCP-S / LCP-T compression and decompression, trajectories (Algorithm 1)
// with the LCP-FSM selection.
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <array>
#include <vector>

#include "../../include/lcp.h"
#include "lcp_dict.h"
#include "lcp_kernels.h"

using namespace lcp;

unsigned long long lcp::g_launches = 0;

namespace {

constexpr uint32_t kFlagFirst = 1u, kFlagRefAnchor = 2u;
constexpr uint32_t kFlagRequant = 4u;  // reference codes re-quantized on the frame's grid

struct DevBuf {
  void *p = nullptr;
  size_t cap = 0;
};

int grow(DevBuf &b, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (b.cap >= bytes) return OK;
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.cap = 0;
  bytes = (bytes + 255) & ~(size_t)255;
  if (cudaMalloc(&b.p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return ERR_NOMEM;
  }
  b.cap = bytes;
  return OK;
}

template <typename T>
T *P(DevBuf &b) {
  return reinterpret_cast<T *>(b.p);
}

struct Workspace {
  DevBuf big_list, big_cb, big_tb, big_hs, task_owner, slot_owner, multi, shist, chunk_owner, big_of, nbig, sub_cnt, seg_lo, seg_cnt, seg_meta, nseg, bflag, ftile, fbase;
  DevBuf mm, plan, keys, keys2, idx2, idx_alt, tile_hist, btot, bstart, s_rel, tmp_bid, tmp_pos,
      s_id, s_cnt, hist, maxv, nvals, mcount, kcount, desc, codes, lens,
      tables, chunk_bits, chunk_off, outl_idx, summary, q_in, q_slot, perm, sym, patch_s,
      patch_i, patch_x, patch_s2, patch_i2, patch_so, patch_io, dec_fields, hufft, err,
      scan_tmp, cand, tq, fplan, fstatus, cbwork, sample, rq, lut, sbounds;
  DevBuf host_in, host_out;  // device copies for the host-buffer entry points
  DevBuf hstage;             // container header bytes gathered for one copy
  DevBuf hpad;               // a short container, zero padded to the largest header
  // dictionary stage: coded chunks, size table, chunk offsets, the image
  // (compress) and the decoded container (decompress of an LCPZ image)
  DevBuf dict_scratch, dict_sizes, dict_off, dict_img, dict_raw;
};

__global__ void k_set_u64(unsigned long long *p, unsigned long long v) { *p = v; }
__global__ void k_iota(uint32_t *p, const unsigned long long *cnt) {
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < *cnt;
       i += (unsigned long long)gridDim.x * blockDim.x)
    p[i] = (uint32_t)i;
}

struct DeviceGuard {
  int prev = -1;
  bool ok = true;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev && cudaSetDevice(dev) != cudaSuccess) {
      ok = false;
      cudaGetLastError();  // leave no stale error for the next call
    }
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

thread_local char g_last_error[256] = "";

void note_cuda_error(cudaError_t e, const char *what, int line) {
  snprintf(g_last_error, sizeof g_last_error, "%s at lcp_api.cu:%d: %s", what, line,
           cudaGetErrorString(e));
}

#define CK(expr)                                  \
  do {                                            \
    cudaError_t _ce = (expr);                     \
    if (_ce != cudaSuccess) {                     \
      note_cuda_error(_ce, #expr, __LINE__);      \
      cudaGetLastError();                         \
      return ERR_CUDA;                            \
    }                                             \
  } while (0)
#define TRY(expr)            \
  do {                       \
    int _s = (expr);         \
    if (_s != OK) return _s; \
  } while (0)

// level-1 partition bits: about 2048 keys per bucket at most, up to 2^14
// buckets, shifted by the schedule's delta (0 .. 15)
uint32_t bits_target(uint64_t n, int delta = 0) {
  uint32_t b = 0;
  while (b < 14 && ((2048ull << b) < n)) ++b;
  const int t = (int)b + delta;
  return (uint32_t)(t < 0 ? 0 : (t > 15 ? 15 : t));
}

bool aligned16(const void *p) { return (((uintptr_t)p) & 15u) == 0; }

}  // namespace

namespace {
// Stage marks: prof_begin(c, name, s) ... prof_end(c, s) around one kernel
void prof_reset(lcp_ctx *c);
void prof_begin(lcp_ctx *c, const char *name, cudaStream_t s);
void prof_end(lcp_ctx *c, cudaStream_t s);
}  // namespace

// per-kernel timing (events recorded on the call's stream): of the last
// call, or accumulated over calls until read (lcp_ctx_profile mode 2)
constexpr int kProfCall = 32;     // stages kept per call
constexpr int kProfAccum = 4096;  // stages kept while accumulating
struct Profile {
  bool on = false, accumulate = false;
  int n = 0;
  std::vector<std::array<char, 32>> names;
  std::vector<cudaEvent_t> ev;  // two per stage
  int cap() const { return (int)names.size(); }
};

struct lcp_ctx {
  int device = 0;
  int sms = 148;
  // schedule (lcp_ctx_set_schedule): chunk size of the streams (recorded in
  // every container), shift of the level-1 partition bits (never changes the
  // bytes)
  uint32_t log2_chunk = 10;
  int bucket_delta = 0;
  // dictionary stage after every compression (lcp_ctx_set_dict)
  bool dict = false;
  Workspace ws;
  Profile prof;
  Plan *h_plan = nullptr;
  Summary *h_sum = nullptr;
  uint8_t *h_stage = nullptr;  // header staging (pinned)
  int *h_err = nullptr;
};

struct lcp_traj {
  lcp_ctx *ctx = nullptr;
  int device = 0;  // the device of its buffers (the context may be destroyed first)
  uint32_t batch = 1, p = 8;
  uint64_t t = 0;
  uint64_t n = 0;
  uint32_t d = 0;
  bool has_prev = false, has_anchor = false;
  // LCP-FSM: state 0 = T, else k of S{k}
  int state = 2, counter = 0;
  bool s_known = false;
  uint64_t s_est = 0;
  // anchor bound scaling: anchors coded at eb / anchor_scale (1: off); the
  // grids of the previous frame and the anchor, and whether each is a scaled
  // anchor (frames predicted from it re-quantize its codes)
  uint32_t anchor_scale = 1;
  bool prev_scaled = false, anc_scaled = false;
  FieldPlan prev_F[kMaxD] = {}, anc_F[kMaxD] = {};
  DevBuf prev_q, prev_pi, anc_q, anc_pi, new_q, new_pi;
};

namespace {
void prof_reset(lcp_ctx *c) {
  if (!c->prof.accumulate) c->prof.n = 0;
}
void prof_begin(lcp_ctx *c, const char *name, cudaStream_t s) {
  Profile &P = c->prof;
  if (!P.on || P.n >= P.cap()) return;
  strncpy(P.names[P.n].data(), name, 31);
  P.names[P.n][31] = 0;
  cudaEventRecord(P.ev[2 * P.n], s);
}
void prof_end(lcp_ctx *c, cudaStream_t s) {
  Profile &P = c->prof;
  if (!P.on || P.n >= P.cap()) return;
  cudaEventRecord(P.ev[2 * P.n + 1], s);
  ++P.n;
}
}  // namespace

// ===========================================================================
// internal: LCP-S compression of one frame
// ===========================================================================
namespace {

int read_plan(lcp_ctx *c, cudaStream_t s) {
  CK(cudaMemcpyAsync(c->h_plan, c->ws.plan.p, sizeof(Plan), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return c->h_plan->status;
}

int read_summary(lcp_ctx *c, cudaStream_t s) {
  CK(cudaMemcpyAsync(c->h_sum, c->ws.summary.p, sizeof(Summary), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return OK;
}

int ws_common(lcp_ctx *c, uint64_t n, uint32_t d) {
  Workspace &w = c->ws;
  TRY(grow(w.mm, sizeof(MinMax)));
  TRY(grow(w.plan, sizeof(Plan)));
  TRY(grow(w.hist, 3ull * kAlpha * 4));
  TRY(grow(w.maxv, 4 * 8));
  TRY(grow(w.nvals, 4 * 8));
  TRY(grow(w.mcount, 8));
  TRY(grow(w.kcount, 8));
  TRY(grow(w.desc, 4 * sizeof(StreamDesc)));
  TRY(grow(w.codes, 3ull * kAlpha * 4));
  TRY(grow(w.lens, 3ull * kAlpha));
  TRY(grow(w.tables, 3ull * (kAlpha + 32) * 2));
  TRY(grow(w.summary, sizeof(Summary)));
  TRY(grow(w.cbwork, codebook_work_size(3)));
  const uint64_t nd = n * d;
  // per-chunk bit counts and offsets of the longest stream (n d values in
  // LCP-T) at the context's chunk size
  const uint64_t chunks = (std::max<uint64_t>(nd, n) >> c->log2_chunk) + 2;
  TRY(grow(w.chunk_bits, (chunks + scan_tmp_len(chunks)) * 8));  // counts, scan scratch
  TRY(grow(w.chunk_off, (chunks + 1) * 8));
  return OK;
}

int compress_s_impl(lcp_ctx *c, const float *X, uint64_t n, uint32_t d, double eb, int mode,
                    uint32_t p, uint32_t flags, uint8_t *out, size_t cap, bool size_only,
                    uint32_t *perm_out, int32_t *q_slot_out, uint64_t *total_out,
                    cudaStream_t s) {
  Workspace &w = c->ws;
  const int sms = c->sms;
  TRY(ws_common(c, n, d));
  const bool want_perm = perm_out != nullptr;
  const bool want_q = q_slot_out != nullptr;
  // 1-2. min/max and plan
  prof_begin(c, "s.minmax", s);
  launch_minmax(X, n, d, P<MinMax>(w.mm), sms, s);
  prof_end(c, s);
  launch_plan(P<MinMax>(w.mm), n, d, eb, mode, p, bits_target(n, c->bucket_delta), 0,
              P<Plan>(w.plan), s);
  CK(cudaGetLastError());
  int st = read_plan(c, s);
  if (st != OK) return st;
  const uint32_t nb = 1u << c->h_plan->nbits;
  const uint32_t nb1 = nb + 1;
  int tiles = (int)std::min<uint64_t>((uint64_t)(2 * sms), std::max<uint64_t>(1, n / 2048));
  if ((size_t)nb1 * 4 > 100 * 1024) tiles = std::min(tiles, sms);
  const uint64_t nn = std::max<uint64_t>(n, 1);
  TRY(grow(w.keys, nn * 8));
  TRY(grow(w.keys2, nn * 8));
  TRY(grow(w.tile_hist, (size_t)tiles * nb1 * 4));
  TRY(grow(w.btot, (size_t)nb1 * 8));
  TRY(grow(w.bstart, (size_t)(nb1 + 1) * 8));
  TRY(grow(w.sbounds, (size_t)(kScatterPassesMax + 1) * 4));
  TRY(grow(w.s_rel, nn * 4));
  TRY(grow(w.tmp_bid, nn * 8));
  TRY(grow(w.tmp_pos, (nn + 1) * 4));  // block start slots
  TRY(grow(w.bflag, (nn + 4096) & ~(uint64_t)4095));
  TRY(grow(w.ftile, flag_tiles(nn) * 8));
  TRY(grow(w.fbase, (flag_tiles(nn) + 1) * 8));
  // split buckets (each above 256 keys) and the units: unsplit buckets
  // merged, the outlier bucket, runs of sub-buckets too large for a warp
  const uint64_t segcap = nb1 + n / 128 + 2;
  TRY(grow(w.big_list, (size_t)(nb1 + 1) * 4));
  TRY(grow(w.big_cb, (size_t)(nb1 + 1) * 4));
  TRY(grow(w.big_tb, (size_t)(nb1 + 1) * 4));
  TRY(grow(w.big_hs, (size_t)(nb1 + 1) * 4));
  TRY(grow(w.task_owner, (size_t)split_tasks_max(n, nb1) * 4));
  TRY(grow(w.slot_owner, (size_t)split_slots_max(n) * 4));
  TRY(grow(w.multi, (size_t)nb1 * 4));
  TRY(grow(w.shist, (size_t)split_slots_max(n) * 8192 * 4));
  TRY(grow(w.big_of, (size_t)nb1 * 4));
  TRY(grow(w.nbig, 32));
  TRY(grow(w.sub_cnt, (size_t)sub_off_size(n, nb1) * 4));
  TRY(grow(w.chunk_owner, (size_t)(sub_off_size(n, nb1) / 32 + 1) * 4));
  TRY(grow(w.seg_lo, (size_t)segcap * 4));
  TRY(grow(w.seg_cnt, (size_t)segcap * 4));
  TRY(grow(w.seg_meta, (size_t)segcap * 4));
  TRY(grow(w.nseg, 16));
  TRY(grow(w.s_id, nn * 8));
  TRY(grow(w.s_cnt, nn * 8));
  TRY(grow(w.outl_idx, nn * 4));
  if (want_perm) {
    TRY(grow(w.idx2, nn * 4));
    TRY(grow(w.idx_alt, nn * 4));
  }
  if (want_q) TRY(grow(w.q_in, nn * 4 * d));
  // 3. quantize + keys + bucket histograms
  prof_begin(c, "s.quantize", s);
  launch_quantize_s(X, n, d, P<Plan>(w.plan), nb1, tiles, P<unsigned long long>(w.keys),
                    P<uint32_t>(w.tile_hist), want_q ? P<int32_t>(w.q_in) : nullptr, s);
  prof_end(c, s);
  // 4. bucket offsets, 5. scatter
  prof_begin(c, "s.bucket_offsets", s);
  launch_bucket_offsets(P<uint32_t>(w.tile_hist), tiles, nb1, P<unsigned long long>(w.bstart),
                        P<unsigned long long>(w.btot), s);
  prof_end(c, s);
  prof_begin(c, "s.scatter", s);
  launch_scatter(P<unsigned long long>(w.keys), n, P<Plan>(w.plan), nb1, tiles,
                 P<uint32_t>(w.tile_hist), P<unsigned long long>(w.bstart),
                 P<uint32_t>(w.sbounds), P<unsigned long long>(w.keys2),
                 want_perm ? P<uint32_t>(w.idx2) : nullptr, s);
  prof_end(c, s);
  CK(cudaGetLastError());
  // 6. level-2 split of the large buckets, sorting + segmentation
  prof_begin(c, "s.split", s);
  SegBufs sg;
  sg.big_list = P<uint32_t>(w.big_list);
  sg.big_cb = P<uint32_t>(w.big_cb);
  sg.big_tb = P<uint32_t>(w.big_tb);
  sg.big_hs = P<uint32_t>(w.big_hs);
  sg.task_owner = P<uint32_t>(w.task_owner);
  sg.slot_owner = P<uint32_t>(w.slot_owner);
  sg.multi = P<uint32_t>(w.multi);
  sg.big_of = P<int>(w.big_of);
  sg.nbig = P<uint32_t>(w.nbig);
  sg.sub_off = P<uint32_t>(w.sub_cnt);
  sg.chunk_owner = P<uint32_t>(w.chunk_owner);
  sg.shist = P<uint32_t>(w.shist);
  launch_segments(P<Plan>(w.plan), nb1, P<unsigned long long>(w.bstart),
                  P<unsigned long long>(w.keys2), want_perm ? P<uint32_t>(w.idx2) : nullptr,
                  P<unsigned long long>(w.keys), want_perm ? P<uint32_t>(w.idx_alt) : nullptr, sg,
                  P<uint32_t>(w.seg_lo), P<uint32_t>(w.seg_cnt), P<uint32_t>(w.seg_meta),
                  P<uint32_t>(w.nseg), n, sms, s);
  prof_end(c, s);
  CK(cudaMemsetAsync(w.hist.p, 0, 3ull * kAlpha * 4, s));
  CK(cudaMemsetAsync(w.maxv.p, 0, 4 * 8, s));
  SubsortArgs sa;
  sa.plan = P<Plan>(w.plan);
  sa.big_list = P<uint32_t>(w.big_list);
  sa.big_cb = P<uint32_t>(w.big_cb);
  sa.chunk_owner = P<uint32_t>(w.chunk_owner);
  sa.nbig = P<uint32_t>(w.nbig);
  sa.bstart = P<unsigned long long>(w.bstart);
  sa.sub_off = P<uint32_t>(w.sub_cnt);
  sa.keys_alt = P<unsigned long long>(w.keys);
  sa.idx_alt = want_perm ? P<uint32_t>(w.idx_alt) : nullptr;
  sa.nunit = P<uint32_t>(w.nseg);
  sa.u_lo = P<uint32_t>(w.seg_lo);
  sa.u_cnt = P<uint32_t>(w.seg_cnt);
  sa.u_meta = P<uint32_t>(w.seg_meta);
  sa.s_rel = P<uint32_t>(w.s_rel);
  sa.bflag = P<uint8_t>(w.bflag);
  sa.tmp_bid = P<unsigned long long>(w.tmp_bid);
  sa.hist = P<uint32_t>(w.hist);
  sa.maxv = P<unsigned long long>(w.maxv);
  sa.perm = want_perm ? perm_out : nullptr;
  sa.q_in = want_q ? P<int32_t>(w.q_in) : nullptr;
  sa.q_slot = want_q ? q_slot_out : nullptr;
  sa.log2_chunk = c->log2_chunk;
  sa.n = n;
  prof_begin(c, "s.subsort", s);
  launch_subsort(sa, sms, s);
  prof_end(c, s);
  LocalArgs la;
  la.plan = P<Plan>(w.plan);
  la.nseg = P<uint32_t>(w.nseg);
  la.seg_lo = P<uint32_t>(w.seg_lo);
  la.seg_cnt = P<uint32_t>(w.seg_cnt);
  la.seg_meta = P<uint32_t>(w.seg_meta);
  la.keys = P<unsigned long long>(w.keys2);
  la.idx = want_perm ? P<uint32_t>(w.idx2) : nullptr;
  la.keys_alt = P<unsigned long long>(w.keys);  // free after the scatter
  la.idx_alt = want_perm ? P<uint32_t>(w.idx_alt) : nullptr;
  la.s_rel = P<uint32_t>(w.s_rel);
  la.bflag = P<uint8_t>(w.bflag);
  la.tmp_bid = P<unsigned long long>(w.tmp_bid);
  la.hist = P<uint32_t>(w.hist);
  la.maxv = P<unsigned long long>(w.maxv);
  la.perm = want_perm ? perm_out : nullptr;
  la.q_in = want_q ? P<int32_t>(w.q_in) : nullptr;
  la.q_slot = want_q ? q_slot_out : nullptr;
  la.outl_idx = P<uint32_t>(w.outl_idx);
  la.log2_chunk = c->log2_chunk;
  la.n = n;
  prof_begin(c, "s.local_sort", s);
  launch_local(la, 4 * sms, s);
  prof_end(c, s);
  CK(cudaGetLastError());
  // 7. blocks: ids and counts (the level-1 keys are free: block ids there)
  prof_begin(c, "s.blocks", s);
  launch_blocks(P<Plan>(w.plan), P<uint8_t>(w.bflag), P<unsigned long long>(w.bstart) + nb, n,
                P<unsigned long long>(w.tmp_bid), P<unsigned long long>(w.ftile),
                P<unsigned long long>(w.fbase), P<uint32_t>(w.tmp_pos),
                P<unsigned long long>(w.keys2), P<unsigned long long>(w.s_id),
                P<unsigned long long>(w.s_cnt), P<uint32_t>(w.hist),
                P<unsigned long long>(w.maxv), P<unsigned long long>(w.mcount), sms, s);
  launch_counts_s(P<unsigned long long>(w.bstart), nb, n, P<unsigned long long>(w.mcount),
                  P<unsigned long long>(w.nvals), P<unsigned long long>(w.kcount), s);
  prof_end(c, s);
  // 8. codebooks and the container layout
  prof_begin(c, "s.codebook", s);
  launch_codebook(3, P<uint32_t>(w.hist), P<unsigned long long>(w.maxv),
                  P<unsigned long long>(w.nvals), c->log2_chunk, P<uint8_t>(w.cbwork),
                  P<StreamDesc>(w.desc),
                  P<uint32_t>(w.codes), P<uint8_t>(w.lens), P<uint16_t>(w.tables), s);
  LayoutArgs L;
  L.method = 0;
  L.d = d;
  L.log2_chunk = c->log2_chunk;
  L.flags = flags;
  L.p = p;
  L.n = n;
  L.plan = P<Plan>(w.plan);
  L.desc = P<StreamDesc>(w.desc);
  L.tables = P<uint16_t>(w.tables);
  L.mcount = P<unsigned long long>(w.mcount);
  L.kcount = P<unsigned long long>(w.kcount);
  L.out = out;
  L.cap = size_only ? ~0ull : cap;
  L.summary = P<Summary>(w.summary);
  launch_layout(L, sms, size_only, s);
  prof_end(c, s);
  CK(cudaGetLastError());
  if (!size_only) {
    // 9. payloads
    StreamDesc *D = P<StreamDesc>(w.desc);
    prof_begin(c, "s.encode_ids", s);
    launch_encode_u64(P<unsigned long long>(w.s_id), n, D + 0, P<uint32_t>(w.codes),
                      P<uint8_t>(w.lens), c->log2_chunk, out, P<Summary>(w.summary),
                      P<unsigned long long>(w.chunk_bits), P<unsigned long long>(w.chunk_off), sms,
                      s);
    prof_end(c, s);
    prof_begin(c, "s.encode_counts", s);
    launch_encode_u64(P<unsigned long long>(w.s_cnt), n, D + 1, P<uint32_t>(w.codes) + kAlpha,
                      P<uint8_t>(w.lens) + kAlpha, c->log2_chunk, out, P<Summary>(w.summary),
                      P<unsigned long long>(w.chunk_bits), P<unsigned long long>(w.chunk_off), sms,
                      s);
    prof_end(c, s);
    prof_begin(c, "s.encode_rel", s);
    launch_encode_u32(P<uint32_t>(w.s_rel), n, D + 2, P<uint32_t>(w.codes) + 2 * kAlpha,
                      P<uint8_t>(w.lens) + 2 * kAlpha, c->log2_chunk, out, P<Summary>(w.summary),
                      P<unsigned long long>(w.chunk_bits), P<unsigned long long>(w.chunk_off), sms,
                      s);
    prof_end(c, s);
    prof_begin(c, "s.outliers", s);
    launch_outliers_s(X, n, d, P<uint32_t>(w.outl_idx), D + 3, out, P<Summary>(w.summary), sms, s);
    prof_end(c, s);
    CK(cudaGetLastError());
  }
  TRY(read_summary(c, s));
  *total_out = c->h_sum->total;
  return c->h_sum->status;
}

// ===========================================================================
// internal: LCP-T compression of one frame against (qref, pi)
// ===========================================================================
int compress_t_impl(lcp_ctx *c, const float *X, uint64_t n, uint32_t d, double eb, int mode,
                    const uint32_t *pi, const int32_t *qref, uint32_t flags, uint8_t *out,
                    size_t cap, bool size_only, int32_t *qnew, uint64_t *total_out,
                    cudaStream_t s, const FieldPlan *ref_grid = nullptr) {
  Workspace &w = c->ws;
  const int sms = c->sms;
  TRY(ws_common(c, n, d));
  const uint64_t nd = std::max<uint64_t>(n * d, 1);
  TRY(grow(w.sym, nd * 4));
  TRY(grow(w.patch_s, nd * 8));
  TRY(grow(w.patch_x, nd * 4));
  launch_minmax(X, n, d, P<MinMax>(w.mm), sms, s);
  launch_plan(P<MinMax>(w.mm), n, d, eb, mode, 0, 0, 1, P<Plan>(w.plan), s);
  CK(cudaGetLastError());
  int st = read_plan(c, s);
  if (st != OK) return st;
  if (ref_grid) {  // the reference is on another grid: predict in value space
    TRY(grow(w.rq, nd * 4));
    RefGrid g;
    for (uint32_t f = 0; f < d; ++f) g.f[f] = ref_grid[f];
    launch_requant(P<Plan>(w.plan), n, d, qref, g, P<int32_t>(w.rq), sms, s);
    CK(cudaGetLastError());
    qref = P<int32_t>(w.rq);
  }
  CK(cudaMemsetAsync(w.hist.p, 0, 3ull * kAlpha * 4, s));
  CK(cudaMemsetAsync(w.maxv.p, 0, 4 * 8, s));
  CK(cudaMemsetAsync(w.kcount.p, 0, 8, s));
  CK(cudaMemsetAsync(w.mcount.p, 0, 8, s));
  prof_begin(c, "t.quantize", s);
  launch_quantize_t(X, n, d, P<Plan>(w.plan), pi, qref, P<uint32_t>(w.sym), qnew,
                    P<uint32_t>(w.hist), P<unsigned long long>(w.maxv),
                    P<unsigned long long>(w.kcount), P<unsigned long long>(w.patch_s),
                    P<float>(w.patch_x), sms, s);
  prof_end(c, s);
  note_launch();
  k_set_u64<<<1, 1, 0, s>>>(P<unsigned long long>(w.nvals), (unsigned long long)(n * d));
  launch_codebook(1, P<uint32_t>(w.hist), P<unsigned long long>(w.maxv),
                  P<unsigned long long>(w.nvals), c->log2_chunk, P<uint8_t>(w.cbwork),
                  P<StreamDesc>(w.desc),
                  P<uint32_t>(w.codes), P<uint8_t>(w.lens), P<uint16_t>(w.tables), s);
  LayoutArgs L;
  L.method = 1;
  L.d = d;
  L.log2_chunk = c->log2_chunk;
  L.flags = flags;
  L.p = 0;
  L.n = n;
  L.plan = P<Plan>(w.plan);
  L.desc = P<StreamDesc>(w.desc);
  L.tables = P<uint16_t>(w.tables);
  L.mcount = P<unsigned long long>(w.mcount);
  L.kcount = P<unsigned long long>(w.kcount);
  L.out = out;
  L.cap = size_only ? ~0ull : cap;
  L.summary = P<Summary>(w.summary);
  launch_layout(L, sms, size_only, s);
  CK(cudaGetLastError());
  if (!size_only) {
    StreamDesc *D = P<StreamDesc>(w.desc);
    launch_encode_u32(P<uint32_t>(w.sym), n * d, D + 0, P<uint32_t>(w.codes), P<uint8_t>(w.lens),
                      c->log2_chunk, out, P<Summary>(w.summary),
                      P<unsigned long long>(w.chunk_bits), P<unsigned long long>(w.chunk_off), sms,
                      s);
    // patches in increasing symbol index
    TRY(grow(w.patch_i, nd * 4));
    TRY(grow(w.patch_s2, nd * 8));
    TRY(grow(w.patch_i2, nd * 4));
    TRY(grow(w.patch_so, nd * 8));
    TRY(grow(w.patch_io, nd * 4));
    note_launch();
    k_iota<<<sms, 256, 0, s>>>(P<uint32_t>(w.patch_i), P<unsigned long long>(w.kcount));
    int kbits = (int)bitlen64(n * d > 0 ? n * d - 1 : 0);
    launch_sort_pairs(P<unsigned long long>(w.patch_s), P<uint32_t>(w.patch_i),
                      P<unsigned long long>(w.patch_s2), P<uint32_t>(w.patch_i2),
                      P<unsigned long long>(w.kcount), kbits, P<unsigned long long>(w.patch_so),
                      P<uint32_t>(w.patch_io), s);
    launch_patches_write(P<unsigned long long>(w.patch_so), P<uint32_t>(w.patch_io),
                         P<float>(w.patch_x), D + 1, out, P<Summary>(w.summary), sms, s);
    CK(cudaGetLastError());
  }
  TRY(read_summary(c, s));
  *total_out = c->h_sum->total;
  return c->h_sum->status;
}

int check_frame_args(const void *X, uint64_t n, uint32_t d, double eb, int mode) {
  if (d < 1 || d > 8) return ERR_ARG;
  if (n >= (1ull << 32)) return ERR_ARG;
  if (n > 0 && (!X || !aligned16(X))) return ERR_ARG;
  if (!(eb > 0.0) || eb != eb || eb > 1e308) return ERR_ARG;
  if (mode != LCP_EB_ABS && mode != LCP_EB_REL) return ERR_ARG;
  return OK;
}

int check_p(uint32_t p, uint32_t d) {
  if (p == 0 || p > 65536 || (p & (p - 1))) return ERR_ARG;
  uint32_t lp = 0;
  while ((1u << lp) < p) ++lp;
  if (lp * d > 32) return ERR_ARG;
  return OK;
}

// p == 0: exact size for each candidate, smallest wins, ties to the smaller p
// one container (below, with the decompression entry points); codes_only: a
// frame decoded only as the reference of later frames; floats_cap > 0: the
// output's capacity in values (d n of them needed) instead of n_cap
int decompress_impl(lcp_ctx *c, lcp_traj *t, const uint8_t *in, size_t in_size, float *out,
                    uint64_t n_cap, uint64_t *n_out, uint32_t *d_out, cudaStream_t s,
                    bool codes_only = false, uint64_t floats_cap = 0);

int choose_p(lcp_ctx *c, const float *X, uint64_t n, uint32_t d, double eb, int mode,
             uint32_t *best, cudaStream_t s) {
  const uint32_t cands[5] = {2, 4, 8, 16, 32};
  uint64_t best_size = ~0ull;
  int last = ERR_RANGE;
  *best = 0;
  for (uint32_t p : cands) {
    if (check_p(p, d) != OK) continue;
    uint64_t total = 0;
    int st = compress_s_impl(c, X, n, d, eb, mode, p, 0, nullptr, 0, true, nullptr, nullptr,
                             &total, s);
    if (st == ERR_RANGE || st == ERR_ARG) {
      last = st;
      continue;
    }
    if (st != OK) return st;
    if (total < best_size) {
      best_size = total;
      *best = p;
    }
  }
  return *best ? OK : last;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

const char *lcp_status_str(lcp_status s) {
  switch (s) {
    case LCP_OK: return "ok";
    case LCP_ERR_ARG: return "invalid argument";
    case LCP_ERR_NONFINITE: return "non-finite input value";
    case LCP_ERR_RANGE: return "frame outside the codec's domain";
    case LCP_ERR_CAPACITY: return "output buffer too small";
    case LCP_ERR_FORMAT: return "malformed container";
    case LCP_ERR_STATE: return "temporal frame without a matching reference";
    case LCP_ERR_NOMEM: return "device allocation failed";
    case LCP_ERR_TIMEOUT: return "bounded device wait expired";
    case LCP_ERR_CUDA: return "CUDA runtime error";
  }
  return "unknown status";
}

lcp_status lcp_ctx_create(int device, lcp_ctx **out) {
  if (!out) return LCP_ERR_ARG;
  *out = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
    cudaGetLastError();
    return LCP_ERR_CUDA;
  }
  DeviceGuard g(device);
  if (!g.ok) return LCP_ERR_CUDA;
  lcp_ctx *c = new lcp_ctx();
  c->device = device;
  cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, device);
  if (cudaMallocHost(&c->h_plan, sizeof(Plan)) != cudaSuccess ||
      cudaMallocHost(&c->h_sum, sizeof(Summary)) != cudaSuccess ||
      cudaMallocHost(&c->h_stage, 8192) != cudaSuccess ||
      cudaMallocHost(&c->h_err, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    lcp_ctx_destroy(c);
    return LCP_ERR_NOMEM;
  }
  *out = c;
  return LCP_OK;
}

uint64_t lcp_ctx_device_bytes(const lcp_ctx *c) {
  if (!c) return 0;
  const DevBuf *bufs = reinterpret_cast<const DevBuf *>(&c->ws);
  uint64_t b = 0;
  for (size_t i = 0; i < sizeof(Workspace) / sizeof(DevBuf); ++i) b += bufs[i].cap;
  return b;
}

uint64_t lcp_traj_device_bytes(const lcp_traj *t) {
  if (!t) return 0;
  const DevBuf *bufs[] = {&t->prev_q, &t->prev_pi, &t->anc_q, &t->anc_pi, &t->new_q, &t->new_pi};
  uint64_t b = 0;
  for (const DevBuf *x : bufs) b += x->cap;
  return b;
}

lcp_status lcp_ctx_destroy(lcp_ctx *c) {
  if (!c) return LCP_ERR_ARG;
  DeviceGuard g(c->device);
  DevBuf *bufs = reinterpret_cast<DevBuf *>(&c->ws);
  for (size_t i = 0; i < sizeof(Workspace) / sizeof(DevBuf); ++i)
    if (bufs[i].p) cudaFree(bufs[i].p);
  if (c->h_plan) cudaFreeHost(c->h_plan);
  if (c->h_sum) cudaFreeHost(c->h_sum);
  if (c->h_stage) cudaFreeHost(c->h_stage);
  if (c->h_err) cudaFreeHost(c->h_err);
  for (cudaEvent_t e : c->prof.ev) cudaEventDestroy(e);
  delete c;
  return LCP_OK;
}

size_t lcp_max_compressed_size(uint64_t n, uint32_t d) {
  return (size_t)(48ull + 16ull * d + 64ull + 256ull + (24ull + 16ull * d) * n);
}

lcp_status lcp_ctx_reserve(lcp_ctx *c, uint64_t n, uint32_t d) {
  if (!c || d < 1 || d > 8) return LCP_ERR_ARG;
  DeviceGuard g(c->device);
  if (!g.ok) return LCP_ERR_CUDA;
  int st = ws_common(c, n, d);
  Workspace &w = c->ws;
  const uint64_t nn = std::max<uint64_t>(n, 1);
  if (st == OK) st = grow(w.keys, nn * 8);
  if (st == OK) st = grow(w.keys2, nn * 8);
  if (st == OK) st = grow(w.s_rel, nn * 4);
  if (st == OK) st = grow(w.tmp_bid, nn * 8);
  if (st == OK) st = grow(w.tmp_pos, nn * 4);
  if (st == OK) st = grow(w.s_id, nn * 8);
  if (st == OK) st = grow(w.s_cnt, nn * 8);
  if (st == OK) st = grow(w.outl_idx, nn * 4);
  return (lcp_status)st;
}

// ---------------------------------------------------------------------------
// trajectories
// ---------------------------------------------------------------------------
lcp_status lcp_traj_create(lcp_ctx *c, uint32_t batch_size, uint32_t p, lcp_traj **out) {
  if (!c || !out || batch_size == 0 || p == 0 || (p & (p - 1)) || p > 65536) return LCP_ERR_ARG;
  lcp_traj *t = new lcp_traj();
  t->ctx = c;
  t->device = c->device;
  t->batch = batch_size;
  t->p = p;
  *out = t;
  return LCP_OK;
}

lcp_status lcp_traj_destroy(lcp_traj *t) {
  if (!t) return LCP_ERR_ARG;
  DeviceGuard g(t->device);
  DevBuf *bufs[] = {&t->prev_q, &t->prev_pi, &t->anc_q, &t->anc_pi, &t->new_q, &t->new_pi};
  for (DevBuf *b : bufs)
    if (b->p) cudaFree(b->p);
  delete t;
  return LCP_OK;
}

namespace {
// trajectory image: this header, then prev_q [d][n] int32, prev_pi [n]
// uint32 (when bit0 of flags), anc_q, anc_pi (when bit1), then the grids of
// the previous frame and of the anchor (d field plans each)
constexpr uint32_t kTrajMagic = 0x5354434cu;  // "LCTS"
constexpr uint32_t kTrajVersion = 2;
struct TrajImage {
  uint32_t magic, version;
  uint32_t batch, p;
  uint64_t t, n;
  uint32_t d, flags;  // bit0 previous frame, bit1 anchor, bit2 S size known,
                      // bit3 previous frame is a scaled anchor, bit4 anchor is
  int32_t state, counter;
  uint64_t s_est;
  uint32_t anchor_scale, pad;
};
static_assert(sizeof(TrajImage) == 64, "image header layout");

size_t traj_image_size(uint64_t n, uint32_t d, uint32_t flags) {
  const size_t per = (size_t)n * d * 4 + (size_t)n * 4;
  return sizeof(TrajImage) + ((flags & 1u) ? per : 0) + ((flags & 2u) ? per : 0) +
         2 * (size_t)d * sizeof(FieldPlan);
}
}  // namespace

lcp_status lcp_traj_export(const lcp_traj *t, void *host_out, size_t cap, size_t *size,
                           void *stream) {
  if (!t || !size) return LCP_ERR_ARG;
  const uint32_t flags = (t->has_prev ? 1u : 0u) | (t->has_anchor ? 2u : 0u) |
                         (t->s_known ? 4u : 0u) | (t->prev_scaled ? 8u : 0u) |
                         (t->anc_scaled ? 16u : 0u);
  const size_t need = traj_image_size(t->n, t->d, flags);
  *size = need;
  if (!host_out || cap < need) return LCP_ERR_CAPACITY;
  DeviceGuard g(t->device);
  if (!g.ok) return LCP_ERR_CUDA;
  TrajImage h{kTrajMagic, kTrajVersion, t->batch, t->p, t->t, t->n, t->d, flags,
              t->state, t->counter, t->s_est, t->anchor_scale, 0u};
  memcpy(host_out, &h, sizeof h);
  uint8_t *o = reinterpret_cast<uint8_t *>(host_out) + sizeof h;
  const size_t qb = (size_t)t->n * t->d * 4, pb = (size_t)t->n * 4;
  cudaStream_t s = (cudaStream_t)stream;
  const DevBuf *src[4] = {&t->prev_q, &t->prev_pi, &t->anc_q, &t->anc_pi};
  const bool have[4] = {t->has_prev, t->has_prev, t->has_anchor, t->has_anchor};
  for (int k = 0; k < 4; ++k) {
    if (!have[k]) continue;
    const size_t b = (k & 1) ? pb : qb;
    if (b && cudaMemcpyAsync(o, src[k]->p, b, cudaMemcpyDeviceToHost, s) != cudaSuccess) {
      cudaGetLastError();
      return LCP_ERR_CUDA;
    }
    o += b;
  }
  memcpy(o, t->prev_F, (size_t)t->d * sizeof(FieldPlan));
  memcpy(o + (size_t)t->d * sizeof(FieldPlan), t->anc_F, (size_t)t->d * sizeof(FieldPlan));
  if (cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return LCP_ERR_CUDA;
  }
  return LCP_OK;
}

lcp_status lcp_traj_import(lcp_ctx *c, const void *host_in, size_t size, lcp_traj **out,
                           void *stream) {
  if (!c || !host_in || !out) return LCP_ERR_ARG;
  *out = nullptr;
  TrajImage h;
  if (size < sizeof h) return LCP_ERR_FORMAT;
  memcpy(&h, host_in, sizeof h);
  const bool shape_ok = h.n == 0 ? h.d <= 8 : (h.d >= 1 && h.d <= 8 && h.n < (1ull << 32));
  if (h.magic != kTrajMagic || h.version != kTrajVersion || h.batch == 0 || h.p == 0 ||
      (h.p & (h.p - 1)) || h.p > 65536 || (h.flags & ~31u) || !shape_ok || h.state < 0 ||
      h.anchor_scale == 0 || h.anchor_scale > 1024 ||
      h.state > 16 || h.counter < 0 || h.counter > 16 ||
      size != traj_image_size(h.n, h.d, h.flags))
    return LCP_ERR_FORMAT;
  DeviceGuard g(c->device);
  if (!g.ok) return LCP_ERR_CUDA;
  lcp_traj *t = new lcp_traj();
  t->ctx = c;
  t->device = c->device;
  t->batch = h.batch;
  t->p = h.p;
  t->t = h.t;
  t->n = h.n;
  t->d = h.d;
  t->has_prev = (h.flags & 1u) != 0;
  t->has_anchor = (h.flags & 2u) != 0;
  t->s_known = (h.flags & 4u) != 0;
  t->prev_scaled = (h.flags & 8u) != 0;
  t->anc_scaled = (h.flags & 16u) != 0;
  t->anchor_scale = h.anchor_scale;
  t->state = h.state;
  t->counter = h.counter;
  t->s_est = h.s_est;
  const uint8_t *in = reinterpret_cast<const uint8_t *>(host_in) + sizeof h;
  const size_t qb = (size_t)h.n * h.d * 4, pb = (size_t)h.n * 4;
  cudaStream_t s = (cudaStream_t)stream;
  DevBuf *dst[4] = {&t->prev_q, &t->prev_pi, &t->anc_q, &t->anc_pi};
  const bool have[4] = {t->has_prev, t->has_prev, t->has_anchor, t->has_anchor};
  int st = OK;
  for (int k = 0; k < 4 && st == OK; ++k) {
    if (!have[k]) continue;
    const size_t b = (k & 1) ? pb : qb;
    st = grow(*dst[k], b);
    if (st == OK && b &&
        cudaMemcpyAsync(dst[k]->p, in, b, cudaMemcpyHostToDevice, s) != cudaSuccess) {
      cudaGetLastError();
      st = ERR_CUDA;
    }
    in += b;
  }
  if (st == OK) {
    memcpy(t->prev_F, in, (size_t)h.d * sizeof(FieldPlan));
    memcpy(t->anc_F, in + (size_t)h.d * sizeof(FieldPlan), (size_t)h.d * sizeof(FieldPlan));
  }
  if (st == OK && cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    st = ERR_CUDA;
  }
  if (st != OK) {
    lcp_traj_destroy(t);
    return (lcp_status)st;
  }
  *out = t;
  return LCP_OK;
}

lcp_status lcp_traj_set_anchor_scale(lcp_traj *t, uint32_t scale) {
  if (!t || scale == 0 || scale > 1024) return LCP_ERR_ARG;
  t->anchor_scale = scale;
  return LCP_OK;
}

namespace {

enum Action { A_SPATIAL, A_COMPARE, A_TEST, A_TEMPORAL };

struct FsmCopy {
  int state, counter;
  bool s_known;
  uint64_t s_est;
};

// the LCP-FSM decision for the next frame (mutates only the copy)
Action fsm_plan(FsmCopy &f, bool has_ref) {
  if (!has_ref) return A_SPATIAL;
  if (!f.s_known) return A_COMPARE;
  if (f.state == 0) return A_TEST;
  f.counter += 1;
  if (f.counter >= f.state) {
    f.counter = 0;
    return A_TEST;
  }
  return A_SPATIAL;
}

int traj_buffers(lcp_traj *t, uint64_t n, uint32_t d) {
  const size_t qb = std::max<uint64_t>(n * d, 1) * 4, pb = std::max<uint64_t>(n, 1) * 4;
  DevBuf *bufs[6] = {&t->prev_q, &t->prev_pi, &t->anc_q, &t->anc_pi, &t->new_q, &t->new_pi};
  const size_t need[6] = {qb, pb, qb, pb, qb, pb};
  bool fresh = false;
  for (int k = 0; k < 6; ++k) {
    const void *old = bufs[k]->p;
    TRY(grow(*bufs[k], need[k]));
    if (bufs[k]->p != old) {  // new memory starts zeroed: checkpoint images are
      fresh = true;            // defined even for arrays a decoder never writes
      if (cudaMemset(bufs[k]->p, 0, bufs[k]->cap) != cudaSuccess) {
        cudaGetLastError();
        return ERR_CUDA;
      }
    }
  }
  if (fresh && cudaStreamSynchronize(cudaStreamLegacy) != cudaSuccess) {
    cudaGetLastError();
    return ERR_CUDA;
  }
  return OK;
}

// compress the next frame of a trajectory (Algorithm 1)
int traj_compress(lcp_ctx *c, lcp_traj *t, const float *X, uint64_t n, uint32_t d, double eb,
                  int mode, int method, uint8_t *out, size_t cap, size_t *out_size,
                  int *chosen, bool commit, uint64_t *est_s, uint64_t *est_t, cudaStream_t s) {
  if (t->has_prev && (n != t->n || d != t->d)) return ERR_STATE;
  TRY(check_p(t->p, d));
  TRY(traj_buffers(t, n, d));
  Workspace &w = c->ws;
  const bool first = (t->t % t->batch) == 0;
  const bool ref_anchor = first;
  const bool has_ref = first ? t->has_anchor : t->has_prev;
  const int32_t *rq = ref_anchor ? P<int32_t>(t->anc_q) : P<int32_t>(t->prev_q);
  const uint32_t *rpi = ref_anchor ? P<uint32_t>(t->anc_pi) : P<uint32_t>(t->prev_pi);
  const uint32_t sflags = first ? kFlagFirst : 0u;
  // a reference that is a scaled anchor is on another grid: value-space
  // prediction (Sec. "Best error-bound scale for anchor frames")
  const bool ref_scaled = has_ref && (ref_anchor ? t->anc_scaled : t->prev_scaled);
  const FieldPlan *rgrid = ref_scaled ? (ref_anchor ? t->anc_F : t->prev_F) : nullptr;
  const uint32_t tflags =
      sflags | (ref_anchor ? kFlagRefAnchor : 0u) | (ref_scaled ? kFlagRequant : 0u);
  // temporal correlation as the LCP-FSM sees it when the frame is planned
  const bool correlated = t->state == 0 || t->state == 2;
  FsmCopy f{t->state, t->counter, t->s_known, t->s_est};
  Action a;
  if (method == LCP_SPATIAL) a = A_SPATIAL;
  else if (method == LCP_TEMPORAL) {
    if (!has_ref) return ERR_STATE;
    a = A_TEMPORAL;
  } else a = fsm_plan(f, has_ref);
  const size_t qb = std::max<uint64_t>(n * d, 1) * 4;
  TRY(grow(w.tq, qb));
  TRY(grow(w.cand, lcp_max_compressed_size(n, d)));
  bool use_t = false;
  uint64_t s_size = 0, t_size = 0;
  const bool size_only = !commit;
  if (a == A_SPATIAL) {
    TRY(compress_s_impl(c, X, n, d, eb, mode, t->p, sflags, out, cap, size_only,
                        P<uint32_t>(t->new_pi), P<int32_t>(t->new_q), &s_size, s));
    if (a == A_SPATIAL && method == LCP_AUTO) f.s_known = true, f.s_est = s_size;
    if (method != LCP_AUTO) f.s_known = true, f.s_est = s_size;
  } else if (a == A_TEMPORAL) {
    TRY(compress_t_impl(c, X, n, d, eb, mode, rpi, rq, tflags, out, cap, size_only,
                        P<int32_t>(w.tq), &t_size, s, rgrid));
    use_t = true;
  } else if (a == A_COMPARE) {
    TRY(compress_s_impl(c, X, n, d, eb, mode, t->p, sflags, out, cap, size_only,
                        P<uint32_t>(t->new_pi), P<int32_t>(t->new_q), &s_size, s));
    int st = compress_t_impl(c, X, n, d, eb, mode, rpi, rq, tflags, P<uint8_t>(w.cand),
                             w.cand.cap, size_only, P<int32_t>(w.tq), &t_size, s, rgrid);
    if (st != OK) return st;
    use_t = t_size < s_size;
    f.s_known = true;
    f.s_est = s_size;
    f.state = use_t ? 0 : 2;
    f.counter = 0;
    if (use_t && commit) {
      if (t_size > cap) {
        *out_size = t_size;
        return ERR_CAPACITY;
      }
      CK(cudaMemcpyAsync(out, w.cand.p, t_size, cudaMemcpyDeviceToDevice, s));
    }
  } else {  // A_TEST: LCP-T against the LCP-S estimate
    int st = compress_t_impl(c, X, n, d, eb, mode, rpi, rq, tflags, out, cap, size_only,
                             P<int32_t>(w.tq), &t_size, s, rgrid);
    if (st != OK && st != ERR_CAPACITY) return st;
    use_t = t_size <= f.s_est;
    if (use_t && st == ERR_CAPACITY) {
      *out_size = t_size;
      return ERR_CAPACITY;
    }
    if (!use_t) {
      TRY(compress_s_impl(c, X, n, d, eb, mode, t->p, sflags, out, cap, size_only,
                          P<uint32_t>(t->new_pi), P<int32_t>(t->new_q), &s_size, s));
      f.s_est = s_size;
    }
    if (use_t) f.state = 0;
    else f.state = (f.state == 0) ? 2 : std::min(2 * f.state, 16);
    f.counter = 0;
  }
  *out_size = use_t ? t_size : s_size;
  if (chosen) *chosen = use_t ? LCP_TEMPORAL : LCP_SPATIAL;
  if (est_s) *est_s = (a == A_COMPARE) ? s_size : (f.s_known ? t->s_est : 0);
  if (est_t) *est_t = t_size;
  if (!commit) return OK;
  // an anchor while the frames are temporally correlated: coded again at
  // eb / anchor_scale (kept at eb when that bound leaves the domain); the
  // LCP-FSM has decided on the size at eb
  bool scaled = false;
  if (!use_t && first && t->anchor_scale > 1 && correlated) {
    uint64_t s2 = 0;
    const int st = compress_s_impl(c, X, n, d, eb / (double)t->anchor_scale, mode, t->p, sflags,
                                   out, cap, false, P<uint32_t>(t->new_pi), P<int32_t>(t->new_q),
                                   &s2, s);
    if (st == OK) {
      scaled = true;
      *out_size = s2;
    } else if (st == ERR_CAPACITY) {
      *out_size = s2;
      return st;
    } else if (st != ERR_RANGE && st != ERR_ARG) {
      return st;
    }
  }
  // commit the reference state
  if (use_t) {
    std::swap(t->prev_q, w.tq);
    if (ref_anchor)
      CK(cudaMemcpyAsync(t->prev_pi.p, t->anc_pi.p, std::max<uint64_t>(n, 1) * 4,
                         cudaMemcpyDeviceToDevice, s));
    t->prev_scaled = false;
  } else {
    std::swap(t->prev_q, t->new_q);
    std::swap(t->prev_pi, t->new_pi);
    t->prev_scaled = scaled;
    if (scaled)  // the grid of the scaled anchor, from its plan
      for (uint32_t k = 0; k < d; ++k) t->prev_F[k] = c->h_plan->f[k];
    if (first) {
      CK(cudaMemcpyAsync(t->anc_q.p, t->prev_q.p, qb, cudaMemcpyDeviceToDevice, s));
      CK(cudaMemcpyAsync(t->anc_pi.p, t->prev_pi.p, std::max<uint64_t>(n, 1) * 4,
                         cudaMemcpyDeviceToDevice, s));
      t->has_anchor = true;
      t->anc_scaled = scaled;
      for (uint32_t k = 0; k < d; ++k) t->anc_F[k] = t->prev_F[k];
    }
  }
  CK(cudaStreamSynchronize(s));
  t->has_prev = true;
  t->n = n;
  t->d = d;
  t->t += 1;
  t->state = f.state;
  t->counter = f.counter;
  t->s_known = f.s_known;
  t->s_est = f.s_est;
  return OK;
}

// ---------------------------------------------------------------------------
// dictionary stage (Sec. "Block coding", its last step): LCPZ images, see
// lcp_dict.h
// ---------------------------------------------------------------------------
inline uint64_t le64(const uint8_t *p) {
  uint64_t v;
  memcpy(&v, p, 8);
  return v;
}

bool overlap(const void *a, uint64_t na, const void *b, uint64_t nb) {
  const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
  return na && nb && x < y + nb && y < x + na;
}

// workspace for the image of up to S raw bytes
int dict_reserve(lcp_ctx *c, uint64_t S) {
  Workspace &w = c->ws;
  const uint64_t C = dict_chunks(S);
  TRY(grow(w.dict_scratch, S));
  TRY(grow(w.dict_sizes, 4 * C));
  TRY(grow(w.dict_off, 8 * (C + 1)));
  TRY(grow(w.dict_img, dict_max_size(S)));
  return OK;
}

// codes in[0, S) chunk by chunk; *T the image's size (one synchronization)
int dict_encode(lcp_ctx *c, const uint8_t *in, uint64_t S, uint64_t *T, cudaStream_t s) {
  Workspace &w = c->ws;
  const uint64_t C = dict_chunks(S);
  TRY(grow(w.dict_scratch, S));
  TRY(grow(w.dict_sizes, 4 * C));
  TRY(grow(w.dict_off, 8 * (C + 1)));
  prof_begin(c, "dict.encode", s);
  launch_dict_encode(in, S, P<uint8_t>(w.dict_scratch), P<uint32_t>(w.dict_sizes), c->sms, s);
  CK(cudaGetLastError());
  launch_dict_offsets(P<uint32_t>(w.dict_sizes), C, P<unsigned long long>(w.dict_off), s);
  CK(cudaGetLastError());
  prof_end(c, s);
  CK(cudaMemcpyAsync(c->h_stage, P<unsigned long long>(w.dict_off) + C, 8,
                     cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  *T = pad16(le64(c->h_stage));
  return OK;
}

// the image (T bytes) of in[0, S) after dict_encode, into out
int dict_pack(lcp_ctx *c, const uint8_t *in, uint64_t S, uint64_t T, uint8_t *out,
              cudaStream_t s) {
  Workspace &w = c->ws;
  prof_begin(c, "dict.pack", s);
  launch_dict_pack(in, S, P<uint8_t>(w.dict_scratch), P<uint32_t>(w.dict_sizes),
                   P<unsigned long long>(w.dict_off), T, out, c->sms, s);
  CK(cudaGetLastError());
  prof_end(c, s);
  return OK;
}

// a container replaced in place by its image when that is shorter
int dict_apply(lcp_ctx *c, uint8_t *buf, size_t *size, cudaStream_t s) {
  const uint64_t S = *size;
  uint64_t T = 0;
  TRY(grow(c->ws.dict_img, dict_max_size(S)));
  TRY(dict_encode(c, buf, S, &T, s));
  if (T >= S) return OK;
  TRY(dict_pack(c, buf, S, T, P<uint8_t>(c->ws.dict_img), s));
  CK(cudaMemcpyAsync(buf, c->ws.dict_img.p, T, cudaMemcpyDeviceToDevice, s));
  *size = T;
  return OK;
}

// decodes an image into dst (dst_cap bytes), or into the workspace buffer
// dict_raw when to_ws; *raw_size = the raw bytes (set once the header is read)
int dict_decode(lcp_ctx *c, const uint8_t *in, size_t in_size, uint8_t *dst, uint64_t dst_cap,
                uint64_t *raw_size, bool to_ws, cudaStream_t s) {
  if (!in || !aligned16(in) || in_size < kDictHead) return ERR_FORMAT;
  Workspace &w = c->ws;
  uint8_t *st = c->h_stage;
  CK(cudaMemcpyAsync(st, in, 32, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (st[0] != 'L' || st[1] != 'C' || st[2] != 'P' || st[3] != 'Z' || st[4] != 1 ||
      st[5] != kDictLog2Chunk)
    return ERR_FORMAT;
  const uint64_t S = le64(st + 8), C = le64(st + 16), T = le64(st + 24);
  if (C != dict_chunks(S) || T > in_size || dict_body(C) > T) return ERR_FORMAT;
  *raw_size = S;
  if (to_ws) {
    TRY(grow(w.dict_raw, S));
    dst = P<uint8_t>(w.dict_raw);
  } else {
    if (S > dst_cap) return ERR_CAPACITY;
    if (S && !dst) return ERR_ARG;
  }
  TRY(grow(w.dict_off, 8 * (C + 1)));
  TRY(grow(w.err, 8));
  int *err = P<int>(w.err);
  CK(cudaMemsetAsync(err, 0, 4, s));
  prof_begin(c, "dict.decode", s);
  launch_dict_offsets(reinterpret_cast<const uint32_t *>(in + kDictHead), C,
                      P<unsigned long long>(w.dict_off), s);
  CK(cudaGetLastError());
  launch_dict_decode(in, in_size, S, T, P<unsigned long long>(w.dict_off), dst, err, c->sms, s);
  CK(cudaGetLastError());
  prof_end(c, s);
  CK(cudaMemcpyAsync(c->h_err, err, 4, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return *c->h_err ? ERR_FORMAT : OK;
}

int compress_entry(lcp_ctx *c, lcp_traj *traj, const float *d_fields, uint64_t n, uint32_t d,
                   double eb, lcp_eb_mode mode, uint32_t p, lcp_method method, void *d_out,
                   size_t out_cap, size_t *out_size, lcp_method *chosen, uint32_t *d_perm,
                   cudaStream_t s);

}  // namespace

lcp_status lcp_compress(lcp_ctx *c, lcp_traj *traj, const float *d_fields, uint64_t n, uint32_t d,
                        double eb, lcp_eb_mode mode, uint32_t p, lcp_method method, void *d_out,
                        size_t out_cap, size_t *out_size, lcp_method *chosen, uint32_t *d_perm,
                        void *stream) {
  if (!c || !out_size) return LCP_ERR_ARG;
  *out_size = 0;
  DeviceGuard g(c->device);
  if (!g.ok) return LCP_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  // the stage's workspace comes first: once a trajectory has taken the frame
  // the call can no longer fail for memory
  if (c->dict && d < 1 + (uint32_t)kMaxD &&
      dict_reserve(c, std::min<uint64_t>(out_cap, lcp_max_compressed_size(n, d))) != OK)
    return LCP_ERR_NOMEM;
  int st = compress_entry(c, traj, d_fields, n, d, eb, mode, p, method, d_out, out_cap, out_size,
                          chosen, d_perm, s);
  if (st == OK && c->dict) st = dict_apply(c, (uint8_t *)d_out, out_size, s);
  return (lcp_status)st;
}

namespace {

int compress_entry(lcp_ctx *c, lcp_traj *traj, const float *d_fields, uint64_t n, uint32_t d,
                   double eb, lcp_eb_mode mode, uint32_t p, lcp_method method, void *d_out,
                   size_t out_cap, size_t *out_size, lcp_method *chosen, uint32_t *d_perm,
                   cudaStream_t s) {
  int st = check_frame_args(d_fields, n, d, eb, mode);
  if (st != OK) return (lcp_status)st;
  if (!d_out || !aligned16(d_out)) return LCP_ERR_ARG;
  if (method != LCP_SPATIAL && method != LCP_TEMPORAL && method != LCP_AUTO) return LCP_ERR_ARG;
  if (!traj && method == LCP_TEMPORAL) return LCP_ERR_STATE;
  prof_reset(c);
  if (traj) {
    int ch = LCP_SPATIAL;
    st = traj_compress(c, traj, d_fields, n, d, eb, mode, method, (uint8_t *)d_out, out_cap,
                       out_size, &ch, true, nullptr, nullptr, s);
    if (chosen) *chosen = (lcp_method)ch;
    if (st == OK && d_perm) {
      const void *src = (ch == LCP_SPATIAL) ? traj->prev_pi.p : traj->prev_pi.p;
      if (cudaMemcpyAsync(d_perm, src, n * 4, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
          cudaStreamSynchronize(s) != cudaSuccess)
        return LCP_ERR_CUDA;
    }
    return (lcp_status)st;
  }
  if (p == 0) {
    st = choose_p(c, d_fields, n, d, eb, mode, &p, s);
    if (st != OK) return (lcp_status)st;
  } else {
    st = check_p(p, d);
    if (st != OK) return (lcp_status)st;
  }
  uint64_t total = 0;
  st = compress_s_impl(c, d_fields, n, d, eb, mode, p, 0, (uint8_t *)d_out, out_cap, false, d_perm,
                       nullptr, &total, s);
  *out_size = total;
  if (chosen) *chosen = LCP_SPATIAL;
  return (lcp_status)st;
}

}  // namespace

lcp_status lcp_ctx_set_dict(lcp_ctx *c, int on) {
  if (!c) return LCP_ERR_ARG;
  c->dict = on != 0;
  return LCP_OK;
}

size_t lcp_dict_max_size(uint64_t raw_bytes) { return (size_t)dict_max_size(raw_bytes); }

lcp_status lcp_dict_compress(lcp_ctx *c, const void *d_in, size_t in_size, void *d_out,
                             size_t out_cap, size_t *out_size, void *stream) {
  if (!c || !out_size || (in_size && !d_in) || !d_out || !aligned16(d_out)) return LCP_ERR_ARG;
  *out_size = 0;
  if (overlap(d_in, in_size, d_out, out_cap)) return LCP_ERR_ARG;
  DeviceGuard g(c->device);
  if (!g.ok) return LCP_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  prof_reset(c);
  uint64_t T = 0;
  int st = dict_encode(c, (const uint8_t *)d_in, in_size, &T, s);
  if (st != OK) return (lcp_status)st;
  *out_size = T;
  if (T > out_cap) return LCP_ERR_CAPACITY;
  return (lcp_status)dict_pack(c, (const uint8_t *)d_in, in_size, T, (uint8_t *)d_out, s);
}

lcp_status lcp_dict_decompress(lcp_ctx *c, const void *d_in, size_t in_size, void *d_out,
                               size_t out_cap, size_t *out_size, void *stream) {
  if (!c || !out_size) return LCP_ERR_ARG;
  *out_size = 0;
  if (overlap(d_in, in_size, d_out, out_cap)) return LCP_ERR_ARG;
  DeviceGuard g(c->device);
  if (!g.ok) return LCP_ERR_CUDA;
  prof_reset(c);
  uint64_t raw = 0;
  int st = dict_decode(c, (const uint8_t *)d_in, in_size, (uint8_t *)d_out, out_cap, &raw, false,
                       (cudaStream_t)stream);
  *out_size = (size_t)raw;
  return (lcp_status)st;
}

lcp_status lcp_ctx_set_schedule(lcp_ctx *c, const lcp_schedule *sc) {
  if (!c) return LCP_ERR_ARG;
  if (!sc) {
    c->log2_chunk = 10;
    c->bucket_delta = 0;
    return LCP_OK;
  }
  if (sc->log2_chunk < 5 || sc->log2_chunk > 10 || sc->bucket_delta < -4 ||
      sc->bucket_delta > 1)
    return LCP_ERR_ARG;
  c->log2_chunk = sc->log2_chunk;
  c->bucket_delta = sc->bucket_delta;
  return LCP_OK;
}

lcp_status lcp_ctx_get_schedule(const lcp_ctx *c, lcp_schedule *out) {
  if (!c || !out) return LCP_ERR_ARG;
  memset(out, 0, sizeof(*out));
  out->log2_chunk = c->log2_chunk;
  out->bucket_delta = c->bucket_delta;
  return LCP_OK;
}

lcp_status lcp_tune_schedule(lcp_ctx *c, const float *d_fields, uint64_t n, uint32_t d, double eb,
                             lcp_eb_mode mode, uint32_t p, double max_growth, int reps,
                             lcp_schedule *best, float *best_ms, void *stream) {
  if (!c || !best) return LCP_ERR_ARG;
  int st = check_frame_args(d_fields, n, d, eb, mode);
  if (st != OK) return (lcp_status)st;
  if (!(max_growth >= 0.0) || reps < 1 || reps > 100 || n == 0) return LCP_ERR_ARG;
  DeviceGuard g(c->device);
  if (!g.ok) return LCP_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  const uint32_t keep_lc = c->log2_chunk;
  const int keep_bd = c->bucket_delta;
  if (p == 0) {  // the exact block-size search, once
    c->log2_chunk = 10;
    c->bucket_delta = 0;
    st = choose_p(c, d_fields, n, d, eb, mode, &p, s);
    if (st != OK) {
      c->log2_chunk = keep_lc;
      c->bucket_delta = keep_bd;
      return (lcp_status)st;
    }
  } else if (check_p(p, d) != OK) {
    return LCP_ERR_ARG;
  }
  const size_t cap = lcp_max_compressed_size(n, d);
  void *buf = nullptr;
  float *y = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaMallocAsync(&buf, cap, s) != cudaSuccess ||
      cudaMallocAsync((void **)&y, (size_t)n * d * 4, s) != cudaSuccess ||
      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    if (buf) cudaFreeAsync(buf, s);
    if (y) cudaFreeAsync(y, s);
    if (e0) cudaEventDestroy(e0);
    return LCP_ERR_NOMEM;
  }
  // candidates: chunk sizes 2^8 .. 2^10 (smaller chunks decode with more
  // lanes but cost table bytes), level-1 partition widths around the default
  const uint32_t lcs[3] = {10, 9, 8};
  const int bds[4] = {0, -1, -2, 1};
  uint64_t base_size = 0;
  float best_t = 0.0f;
  bool have = false;
  for (uint32_t lc : lcs) {
    for (int bd : bds) {
      c->log2_chunk = lc;
      c->bucket_delta = bd;
      float tmin = 0.0f;  // the fastest of the timed rounds (least disturbed)
      uint64_t size = 0;
      for (int r = 0; r <= reps && st == OK; ++r) {  // the first round warms up
        size_t sz = 0;
        uint64_t total = 0;
        st = cudaEventRecord(e0, s) == cudaSuccess ? OK : ERR_CUDA;
        if (st == OK)
          st = compress_s_impl(c, d_fields, n, d, eb, mode, p, 0, (uint8_t *)buf, cap, false,
                               nullptr, nullptr, &total, s);
        if (st == OK) {
          sz = (size_t)total;
          uint64_t no = 0;
          uint32_t dd = 0;
          st = decompress_impl(c, nullptr, (const uint8_t *)buf, sz, y, n, &no, &dd, s);
        }
        if (st == OK && (cudaEventRecord(e1, s) != cudaSuccess ||
                         cudaEventSynchronize(e1) != cudaSuccess))
          st = ERR_CUDA;
        if (st == OK && r > 0) {
          float ms = 0.0f;
          cudaEventElapsedTime(&ms, e0, e1);
          tmin = r == 1 ? ms : std::min(tmin, ms);
        }
        size = sz;
      }
      if (st != OK) break;
      if (lc == 10 && bd == 0) base_size = size;
      const float t = tmin;
      const bool fits = (double)size <= (1.0 + max_growth) * (double)base_size;
      if (fits && (!have || t < best_t)) {
        have = true;
        best_t = t;
        memset(best, 0, sizeof(*best));
        best->log2_chunk = lc;
        best->bucket_delta = bd;
      }
    }
    if (st != OK) break;
  }
  cudaFreeAsync(buf, s);
  cudaFreeAsync(y, s);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamSynchronize(s);
  c->log2_chunk = keep_lc;
  c->bucket_delta = keep_bd;
  if (st != OK) return (lcp_status)st;
  if (best_ms) *best_ms = best_t;
  return LCP_OK;
}

lcp_status lcp_choose_block_size(lcp_ctx *c, const float *d_fields, uint64_t n, uint32_t d,
                                 double eb, lcp_eb_mode mode, uint64_t sample, uint32_t *p_best,
                                 uint64_t *sizes, void *stream) {
  if (!c || !p_best) return LCP_ERR_ARG;
  int st = check_frame_args(d_fields, n, d, eb, mode);
  if (st != OK) return (lcp_status)st;
  if (sample > n) return LCP_ERR_ARG;
  DeviceGuard g(c->device);
  if (!g.ok) return LCP_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  const uint64_t S = sample ? sample : std::min<uint64_t>(n, std::max<uint64_t>(65536, (n + 7) / 8));
  const float *Xs = d_fields;
  if (S < n) {  // the first S particles of every field, contiguous
    st = grow(c->ws.sample, (size_t)S * d * 4);
    if (st != OK) return (lcp_status)st;
    if (cudaMemcpy2DAsync(c->ws.sample.p, S * 4, d_fields, n * 4, S * 4, d,
                          cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
      cudaGetLastError();
      return LCP_ERR_CUDA;
    }
    Xs = reinterpret_cast<const float *>(c->ws.sample.p);
  }
  uint64_t best = ~0ull;
  int last = ERR_RANGE;
  *p_best = 0;
  for (uint32_t k = 0; k <= 16; ++k) {
    const uint32_t p = 1u << k;
    if (sizes) sizes[k] = 0;
    if (check_p(p, d) != OK) continue;
    uint64_t total = 0;
    st = compress_s_impl(c, Xs, S, d, eb, mode, p, 0, nullptr, 0, true, nullptr, nullptr, &total,
                         s);
    if (st == ERR_RANGE || st == ERR_ARG) {
      last = st;
      continue;
    }
    if (st != OK) return (lcp_status)st;
    if (sizes) sizes[k] = total;
    if (total < best) {
      best = total;
      *p_best = p;
    }
  }
  return *p_best ? LCP_OK : (lcp_status)last;
}

lcp_status lcp_select(lcp_ctx *c, lcp_traj *traj, const float *d_fields, uint64_t n, uint32_t d,
                      double eb, lcp_eb_mode mode, lcp_method *chosen, uint64_t *est_s,
                      uint64_t *est_t, void *stream) {
  if (!c || !traj || !chosen) return LCP_ERR_ARG;
  int st = check_frame_args(d_fields, n, d, eb, mode);
  if (st != OK) return (lcp_status)st;
  DeviceGuard g(c->device);
  if (!g.ok) return LCP_ERR_CUDA;
  size_t sz = 0;
  int ch = LCP_SPATIAL;
  uint64_t es = 0, et = 0;
  st = traj_compress(c, traj, d_fields, n, d, eb, mode, LCP_AUTO, nullptr, 0, &sz, &ch, false,
                     &es, &et, (cudaStream_t)stream);
  if (st != OK) return (lcp_status)st;
  *chosen = (lcp_method)ch;
  if (est_s) *est_s = es;
  if (est_t) *est_t = et;
  return LCP_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// decompression
// ---------------------------------------------------------------------------
namespace {

inline uint64_t rd64(const uint8_t *p) {
  uint64_t v;
  memcpy(&v, p, 8);
  return v;
}
inline uint32_t rd32(const uint8_t *p) {
  uint32_t v;
  memcpy(&v, p, 4);
  return v;
}

struct Header {
  int method;
  uint32_t d, log2_chunk, flags, p, lp;
  uint64_t n, K, M, total;
  float m[kMaxD], e[kMaxD];
  uint32_t qmax[kMaxD];
  uint64_t off[4], bytes[4];
  StreamInfo si[3];
  int ns;
};

// read_header's answer for an LCPZ image (not a status)
constexpr int kDictImage = 1;

int read_header(lcp_ctx *c, const uint8_t *in, size_t in_size, Header &h, cudaStream_t s) {
  if (!in || !aligned16(in) || in_size < 48) return ERR_FORMAT;
  uint8_t *st = c->h_stage;
  // the fixed header with the largest field table and directory (8 fields, 4
  // sections) and the stream section headers it names, gathered on the
  // device: one copy, one synchronization
  const size_t head = std::min<size_t>(in_size, (size_t)kHeadBytes);
  TRY(grow(c->ws.hstage, kHeadStage));
  const uint8_t *src = in;
  if (in_size < (size_t)kHeadBytes) {
    // a buffer shorter than the largest header: gathered from a zero-padded
    // copy, so the gather's directory reads (up to kHeadBytes) stay in
    // memory this call owns; the bytes read are the same below in_size
    TRY(grow(c->ws.hpad, kHeadBytes));
    CK(cudaMemsetAsync(c->ws.hpad.p, 0, kHeadBytes, s));
    CK(cudaMemcpyAsync(c->ws.hpad.p, in, in_size, cudaMemcpyDeviceToDevice, s));
    src = P<uint8_t>(c->ws.hpad);
  }
  launch_head_gather(src, in_size, P<uint8_t>(c->ws.hstage), s);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(st, c->ws.hstage.p, kHeadStage, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (st[0] == 'L' && st[1] == 'C' && st[2] == 'P' && st[3] == 'Z') return kDictImage;
  if (st[0] != 'L' || st[1] != 'C' || st[2] != 'P' || st[3] != '1' || st[4] != 1) return ERR_FORMAT;
  h.method = st[5];
  h.d = st[6];
  h.log2_chunk = st[7];
  if (h.method > 1 || h.d < 1 || h.d > 8) return ERR_FORMAT;
  if (h.log2_chunk < 5 || h.log2_chunk > 10) return ERR_FORMAT;
  h.flags = rd32(st + 8);
  h.p = rd32(st + 12);
  h.n = rd64(st + 16);
  h.K = rd64(st + 24);
  h.M = rd64(st + 32);
  h.total = rd64(st + 40);
  h.ns = h.method == 0 ? 3 : 1;
  const uint64_t H = 48ull + 16ull * h.d + 16ull * h.ns + 16ull;
  if (h.total > in_size || h.total < H || h.n >= (1ull << 32) || H > head) return ERR_FORMAT;
  for (uint32_t f = 0; f < h.d; ++f) {
    memcpy(&h.m[f], st + 48 + 16 * f, 4);
    memcpy(&h.e[f], st + 52 + 16 * f, 4);
    h.qmax[f] = rd32(st + 56 + 16 * f);
    if (h.qmax[f] >= (1u << 30)) return ERR_FORMAT;
  }
  for (int k = 0; k <= h.ns; ++k) {
    h.off[k] = rd64(st + 48 + 16 * h.d + 16 * k);
    h.bytes[k] = rd64(st + 48 + 16 * h.d + 16 * k + 8);
    if (h.off[k] < H || h.off[k] > h.total || h.bytes[k] > h.total - h.off[k] || (h.off[k] & 15))
      return ERR_FORMAT;
  }
  h.lp = 0;
  if (h.method == 0) {
    if (h.p == 0 || (h.p & (h.p - 1)) || h.p > 65536) return ERR_FORMAT;
    while ((1u << h.lp) < h.p) ++h.lp;
    if (h.lp * h.d > 32 || h.K > h.n || h.M > h.n - h.K) return ERR_FORMAT;
    if (h.bytes[3] != pad16(4ull * h.d * h.K)) return ERR_FORMAT;
    if ((h.M == 0) != (h.n == h.K)) return ERR_FORMAT;
  } else {
    if (h.bytes[1] != pad16(8ull * h.K) + pad16(4ull * h.K) || h.K > h.n * h.d) return ERR_FORMAT;
  }
  for (int k = 0; k < h.ns; ++k)
    if (h.bytes[k] < 32) return ERR_FORMAT;
  for (int k = 0; k < h.ns; ++k) {
    const uint8_t *sh = st + kHeadBytes + 32 * k;
    StreamInfo &I = h.si[k];
    I.coder = sh[0];
    I.width = sh[1];
    I.used = (uint32_t)sh[2] | ((uint32_t)sh[3] << 8);
    I.n = rd64(sh + 8);
    I.payload_bits = rd64(sh + 16);
    I.maxv = rd64(sh + 24);
    I.log2_chunk = h.log2_chunk;
    const uint64_t want = h.method == 0 ? (k < 2 ? h.M : h.n - h.K) : h.n * h.d;
    if (I.n != want || I.width > 64 || I.coder > 1) return ERR_FORMAT;
    if (h.method == 0 && k == 2 && I.width > 32) return ERR_FORMAT;  // relative codes < 2^32
    if (h.method == 1 && I.width > 32) return ERR_FORMAT;
    if (I.coder == 0) {
      I.n_chunks = 0;
      if (I.payload_bits != I.n * I.width) return ERR_FORMAT;
      if (h.bytes[k] != 32 + pad16(4 * words_of(I.payload_bits))) return ERR_FORMAT;
    } else {
      if (I.used == 0 || I.used > (uint32_t)kAlpha) return ERR_FORMAT;
      I.n_chunks = (I.n + (1ull << h.log2_chunk) - 1) >> h.log2_chunk;
      if (h.bytes[k] != pad16(80ull + 2ull * I.used) + pad16(8 * I.n_chunks) +
                            pad16(4 * words_of(I.payload_bits)))
        return ERR_FORMAT;
    }
  }
  return OK;
}

// codes_only: a frame decoded only as the reference of later frames (its
// codes into the trajectory, no values; out is ignored)
int decompress_impl(lcp_ctx *c, lcp_traj *t, const uint8_t *in, size_t in_size, float *out,
                    uint64_t n_cap, uint64_t *n_out, uint32_t *d_out, cudaStream_t s,
                    bool codes_only, uint64_t floats_cap) {
  Header h;
  int rh = read_header(c, in, in_size, h, s);
  if (rh == kDictImage) {
    // the dictionary stage first: its container, decoded into the workspace
    uint64_t raw = 0;
    TRY(dict_decode(c, in, in_size, nullptr, 0, &raw, true, s));
    in = P<uint8_t>(c->ws.dict_raw);
    in_size = raw;
    rh = read_header(c, in, in_size, h, s);
    if (rh == kDictImage) rh = ERR_FORMAT;  // one stage only
  }
  TRY(rh);
  if (floats_cap) n_cap = floats_cap / std::max<uint32_t>(h.d, 1u);
  if (n_out) *n_out = h.n;
  if (d_out) *d_out = h.d;
  if (codes_only) {
    if (!t) return ERR_ARG;
    out = nullptr;
  } else {
    if (h.n > n_cap) return ERR_CAPACITY;
    if (h.n > 0 && (!out || !aligned16(out))) return ERR_ARG;
  }
  const bool first = (h.flags & kFlagFirst) != 0;
  const bool ra = (h.flags & kFlagRefAnchor) != 0;
  if (h.method == 1) {
    if (!t) return ERR_STATE;
    if (!(ra ? t->has_anchor : t->has_prev) || t->n != h.n || t->d != h.d) return ERR_STATE;
  }
  Workspace &w = c->ws;
  const int sms = c->sms;
  const uint64_t n = h.n, nn = std::max<uint64_t>(n, 1);
  TRY(grow(w.plan, sizeof(Plan)));
  TRY(grow(w.dec_fields, sizeof(DecodeFields)));
  TRY(grow(w.hufft, 3 * sizeof(HuffTable)));
  TRY(grow(w.err, 8));
  if (t) TRY(traj_buffers(t, n, h.d));
  DecodeFields *hf = reinterpret_cast<DecodeFields *>(c->h_stage + 6144);
  memset(hf, 0, sizeof(DecodeFields));
  for (uint32_t f = 0; f < h.d; ++f) {
    hf->m[f] = h.m[f];
    hf->e[f] = h.e[f];
    hf->qmax[f] = h.qmax[f];
  }
  hf->lp = h.lp;
  CK(cudaMemsetAsync(w.plan.p, 0, sizeof(Plan), s));
  CK(cudaMemsetAsync(w.err.p, 0, 8, s));
  CK(cudaMemcpyAsync(w.dec_fields.p, hf, sizeof(DecodeFields), cudaMemcpyHostToDevice, s));
  launch_decode_plan(P<DecodeFields>(w.dec_fields), h.d, P<Plan>(w.plan), s);
  CK(cudaGetLastError());
  int *err = P<int>(w.err);
  HuffTable *ht = P<HuffTable>(w.hufft);
  int32_t *qout = t ? P<int32_t>(t->new_q) : nullptr;
  if (h.method == 0) {
    const uint64_t nb = n - h.K, M = h.M, mm = std::max<uint64_t>(M, 1);
    // block-id and count deltas in 4 bytes unless a stream's largest value
    // needs 8; relative-location deltas of a fixed-width stream are read by
    // the expand straight from the container
    const bool wide = h.si[0].maxv >= (1ull << 32) || h.si[1].maxv >= (1ull << 32);
    const bool rel_fixed = h.si[2].coder == 0;
    TRY(grow(w.s_id, mm * (wide ? 8 : 4)));
    TRY(grow(w.s_cnt, mm * (wide ? 8 : 4)));
    if (!rel_fixed) TRY(grow(w.s_rel, nn * 4));
    // block-scan aggregates: one per chunk from the Huffman decode when both
    // block streams are Huffman-coded, else one per 1024 blocks
    const bool fused = h.si[0].coder == 1 && h.si[1].coder == 1;
    const uint32_t agg_log2 = fused ? h.log2_chunk : 10u;
    TRY(grow(w.scan_tmp, block_bases_bytes(mm, agg_log2)));
    LutOffsets lo;
    lo.off[0] = 0;
    for (uint32_t f = 0; f < h.d; ++f)
      lo.off[f + 1] = (uint32_t)std::min<uint64_t>((uint64_t)lo.off[f] + h.qmax[f] + 1ull,
                                                  0xffffffffull);
    const bool lut = out && lo.off[h.d] <= kLutMax;
    if (lut) TRY(grow(w.lut, (size_t)lo.off[h.d] * 4));
    prof_begin(c, "d.streams", s);
    {
      const uint8_t *secs[3] = {in + h.off[0], in + h.off[1], in + h.off[2]};
      void *outs[3] = {w.s_id.p, w.s_cnt.p, rel_fixed ? nullptr : w.s_rel.p};
      const int wd[3] = {wide ? 1 : 0, wide ? 1 : 0, 0};
      const int am[3] = {fused ? 1 : 0, fused ? 2 : 0, 0};
      launch_decode_streams(3, secs, h.si, ht, outs, wd, am, w.scan_tmp.p, err, sms, s);
      CK(cudaGetLastError());
    }
    prof_end(c, s);
    if (M > 0) {
      prof_begin(c, "d.block_scans", s);
      if (!fused) launch_block_sums(w.s_id.p, w.s_cnt.p, wide ? 1 : 0, M, w.scan_tmp.p, s);
      launch_block_bases(M, agg_log2, w.scan_tmp.p, s);
      if (lut) launch_recon_lut(P<Plan>(w.plan), h.d, lo, P<float>(w.lut), sms, s);
      CK(cudaGetLastError());
      prof_end(c, s);
      ExpandArgs ea;
      ea.plan = P<Plan>(w.plan);
      ea.sid = w.s_id.p;
      ea.scnt = w.s_cnt.p;
      ea.wide = wide ? 1 : 0;
      ea.M = M;
      ea.tiles = (M + 1023) / 1024;
      ea.agg = w.scan_tmp.p;
      ea.agg_log2 = agg_log2;
      ea.rel = rel_fixed ? nullptr : P<uint32_t>(w.s_rel);
      ea.rel_pl = reinterpret_cast<const uint32_t *>(in + h.off[2] + 32);
      ea.rel_w = h.si[2].width;
      ea.rel_words = words_of(h.si[2].payload_bits);
      ea.nb = nb;
      ea.n = n;
      ea.log2_chunk = h.log2_chunk;
      ea.lut = lut ? P<float>(w.lut) : nullptr;
      ea.lut_off = lo;
      for (uint32_t f = 0; f < kMaxD; ++f) ea.qmax[f] = f < h.d ? h.qmax[f] : 0u;
      ea.lp = h.lp;
      ea.out = out;
      ea.qout = qout;
      ea.err = err;
      prof_begin(c, "d.expand", s);
      launch_expand(h.d, ea, lut, sms, s);
      CK(cudaGetLastError());
      prof_end(c, s);
    }
    launch_outliers_decode(P<Plan>(w.plan), reinterpret_cast<const float *>(in + h.off[3]), h.K,
                           n, h.d, out, qout, sms, s);
  } else {
    const uint64_t nd = std::max<uint64_t>(n * h.d, 1);
    TRY(grow(w.sym, nd * 4));
    prof_begin(c, "t.decode_stream", s);
    {
      const uint8_t *secs[1] = {in + h.off[0]};
      void *outs[1] = {w.sym.p};
      const int wide[1] = {0};
      launch_decode_streams(1, secs, h.si, ht, outs, wide, nullptr, nullptr, err, sms, s);
    }
    prof_end(c, s);
    const int32_t *qref = ra ? P<int32_t>(t->anc_q) : P<int32_t>(t->prev_q);
    if (h.flags & kFlagRequant) {  // the reference is on another grid
      TRY(grow(w.rq, nd * 4));
      RefGrid g;
      const FieldPlan *rg = ra ? t->anc_F : t->prev_F;
      for (uint32_t f = 0; f < h.d; ++f) g.f[f] = rg[f];
      launch_requant(P<Plan>(w.plan), n, h.d, qref, g, P<int32_t>(w.rq), sms, s);
      qref = P<int32_t>(w.rq);
    }
    prof_begin(c, "t.recon", s);
    launch_recon_t(P<Plan>(w.plan), n, h.d, P<uint32_t>(w.sym), qref, out, qout, err, sms, s);
    prof_end(c, s);
    if (out) launch_patches_apply(in + h.off[1], h.K, n * h.d, out, err, sms, s);
  }
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(c->h_err, w.err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(c->h_plan, w.plan.p, sizeof(Plan), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (*c->h_err || c->h_plan->status != OK) return ERR_FORMAT;
  if (t) {
    std::swap(t->prev_q, t->new_q);
    for (uint32_t k = 0; k < h.d; ++k) t->prev_F[k] = c->h_plan->f[k];  // this frame's grid
    if (h.method == 0 && first) {
      CK(cudaMemcpyAsync(t->anc_q.p, t->prev_q.p, std::max<uint64_t>(n * h.d, 1) * 4,
                         cudaMemcpyDeviceToDevice, s));
      CK(cudaStreamSynchronize(s));
      t->has_anchor = true;
      for (uint32_t k = 0; k < h.d; ++k) t->anc_F[k] = t->prev_F[k];
    }
    t->has_prev = true;
    t->n = n;
    t->d = h.d;
    t->t += 1;
  }
  return OK;
}

}  // namespace

extern "C" {

lcp_status lcp_decompress(lcp_ctx *c, lcp_traj *traj, const void *d_in, size_t in_size,
                          float *d_out, uint64_t n_cap, uint64_t *n_out, uint32_t *d_fields,
                          void *stream) {
  if (!c) return LCP_ERR_ARG;
  DeviceGuard g(c->device);
  if (!g.ok) return LCP_ERR_CUDA;
  prof_reset(c);
  return (lcp_status)decompress_impl(c, traj, (const uint8_t *)d_in, in_size, d_out, n_cap, n_out,
                                     d_fields, (cudaStream_t)stream);
}

lcp_status lcp_compress_host(lcp_ctx *c, lcp_traj *traj, const float *h_fields, uint64_t n,
                             uint32_t d, double eb, lcp_eb_mode mode, uint32_t p,
                             lcp_method method, void *h_out, size_t out_cap, size_t *out_size,
                             lcp_method *chosen, void *stream) {
  if (!c || !out_size || (n > 0 && !h_fields) || !h_out || d < 1 || d > kMaxD) return LCP_ERR_ARG;
  *out_size = 0;
  DeviceGuard g(c->device);
  if (!g.ok) return LCP_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  Workspace &w = c->ws;
  const size_t fb = (size_t)std::max<uint64_t>(n, 1) * d * 4;
  if (grow(w.host_in, fb) != OK || grow(w.host_out, std::max<size_t>(out_cap, 16)) != OK)
    return LCP_ERR_NOMEM;
  if (n > 0 && cudaMemcpyAsync(w.host_in.p, h_fields, (size_t)n * d * 4, cudaMemcpyHostToDevice,
                               s) != cudaSuccess) {
    cudaGetLastError();
    return LCP_ERR_CUDA;
  }
  lcp_status st = lcp_compress(c, traj, P<float>(w.host_in), n, d, eb, mode, p, method,
                               w.host_out.p, out_cap, out_size, chosen, nullptr, stream);
  if (st != LCP_OK) return st;
  if (cudaMemcpyAsync(h_out, w.host_out.p, *out_size, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return LCP_ERR_CUDA;
  }
  return LCP_OK;
}

lcp_status lcp_decompress_host(lcp_ctx *c, lcp_traj *traj, const void *h_in, size_t in_size,
                               float *h_out, uint64_t out_values, uint64_t *n_out,
                               uint32_t *d_fields, void *stream) {
  if (!c || !h_in || !h_out) return LCP_ERR_ARG;
  DeviceGuard g(c->device);
  if (!g.ok) return LCP_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  Workspace &w = c->ws;
  if (grow(w.host_in, std::max<size_t>(in_size, 16)) != OK ||
      grow(w.host_out, (size_t)std::max<uint64_t>(out_values, 4) * 4) != OK)
    return LCP_ERR_NOMEM;
  if (cudaMemcpyAsync(w.host_in.p, h_in, in_size, cudaMemcpyHostToDevice, s) != cudaSuccess) {
    cudaGetLastError();
    return LCP_ERR_CUDA;
  }
  uint64_t no = 0;
  uint32_t dd = 0;
  lcp_status st = lcp_decompress_into(c, traj, w.host_in.p, in_size, P<float>(w.host_out),
                                      out_values, &no, &dd, stream);
  if (n_out) *n_out = no;
  if (d_fields) *d_fields = dd;
  if (st != LCP_OK) return st;
  if (cudaMemcpyAsync(h_out, w.host_out.p, (size_t)no * dd * 4, cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return LCP_ERR_CUDA;
  }
  return LCP_OK;
}

lcp_status lcp_decompress_into(lcp_ctx *c, lcp_traj *traj, const void *d_in, size_t in_size,
                               float *d_out, uint64_t out_values, uint64_t *n_out,
                               uint32_t *d_fields, void *stream) {
  if (!c) return LCP_ERR_ARG;
  DeviceGuard g(c->device);
  if (!g.ok) return LCP_ERR_CUDA;
  prof_reset(c);
  return (lcp_status)decompress_impl(c, traj, (const uint8_t *)d_in, in_size, d_out, 0, n_out,
                                     d_fields, (cudaStream_t)stream, false,
                                     std::max<uint64_t>(out_values, 1));
}

}  // extern "C"

namespace {

// method (0 S, 1 T) and flags of container i, read in rounds of up to 64
// headers per synchronization, newest first
struct ChainPeek {
  lcp_ctx *c;
  const void *const *ins;
  const size_t *sizes;
  cudaStream_t s;
  std::vector<int> method;  // -1: not read yet
  std::vector<uint32_t> flags;
  int get(uint64_t i, int &m, uint32_t &f) {
    if (method[i] < 0) {
      const uint64_t lo = i >= 63 ? i - 63 : 0;
      uint8_t *st = c->h_stage;
      for (uint64_t k = lo; k <= i; ++k) {
        if (!ins[k] || sizes[k] < 48) continue;
        CK(cudaMemcpyAsync(st + 48 * (k - lo), ins[k], 48, cudaMemcpyDeviceToHost, s));
      }
      CK(cudaStreamSynchronize(s));
      for (uint64_t k = lo; k <= i; ++k) {
        if (method[k] >= 0) continue;
        const uint8_t *h = st + 48 * (k - lo);
        // an LCPZ image: its container's header from byte 32
        if (h[0] == 'L' && h[1] == 'C' && h[2] == 'P' && h[3] == 'Z') h += 32;
        if (!ins[k] || sizes[k] < 48) {
          method[k] = 2;  // absent
          continue;
        }
        if (h[0] != 'L' || h[1] != 'C' || h[2] != 'P' || h[3] != '1' || h[5] > 1)
          return ERR_FORMAT;
        method[k] = h[5];
        flags[k] = rd32(h + 8);
      }
    }
    m = method[i];
    f = flags[i];
    return OK;
  }
};

// Frames first..last of one trajectory (Algorithm 1 stream order) through
// the recursive rule of Sec. "Spatial-Anchor-Frame-Based Batch Compression":
// a frame depends on the frames of its batch before it and, when its batch
// opens with an LCP-T frame, on the batch's anchor (the latest earlier batch
// opening coded LCP-S; frame t opens a batch when t % batch = 0, batch
// being the decoder trajectory's).  Decoding starts at the latest LCP-S
// frame of first's batch at or before first, else at the anchor; frames
// before first are decoded to codes only.
int decompress_range(lcp_ctx *c, lcp_traj *t, const void *const *ins, const size_t *sizes,
                     uint64_t count, uint64_t first, uint64_t last, float *const *outs,
                     uint64_t n_cap, uint64_t *n_out, uint32_t *d_out, cudaStream_t s) {
  if (!t || !ins || !sizes || !outs || first > last || last >= count) return ERR_ARG;
  for (uint64_t i = first; i <= last; ++i)
    if (!ins[i] || !outs[i - first]) return ERR_ARG;
  ChainPeek pk{c, ins, sizes, s, std::vector<int>(last + 1, -1),
               std::vector<uint32_t>(last + 1, 0u)};
  const uint64_t B = t->batch;
  int m;
  uint32_t f;
  // back from `first` to the latest LCP-S frame, or to a batch opening coded
  // LCP-T (which needs the anchor)
  uint64_t start = first;
  bool need_anchor = false;
  for (;;) {
    TRY(pk.get(start, m, f));
    if (m == 2) return ERR_STATE;  // a frame the chain needs is absent
    if (((f & kFlagFirst) != 0) != (start % B == 0)) return ERR_ARG;  // batch size differs
    if (m == 0) break;
    if (f & kFlagFirst) {
      need_anchor = true;
      break;
    }
    if (start == 0) return ERR_FORMAT;
    --start;
  }
  std::vector<uint64_t> chain;
  if (need_anchor) {  // the latest earlier batch opening coded LCP-S
    uint64_t a = start;
    bool found = false;
    while (a >= B) {
      a -= B;
      TRY(pk.get(a, m, f));
      if (m == 2) return ERR_STATE;  // cannot tell whether it was the anchor
      if (!(f & kFlagFirst)) return ERR_ARG;
      if (m == 0) {
        found = true;
        break;
      }
    }
    if (!found) return ERR_STATE;
    chain.push_back(a);
  }
  for (uint64_t i = start; i <= last; ++i) chain.push_back(i);
  // a fresh decoder state
  t->has_prev = t->has_anchor = false;
  t->prev_scaled = t->anc_scaled = false;
  t->t = 0;
  for (uint64_t i : chain) {
    const bool want = i >= first;
    uint64_t no = 0;
    uint32_t dd = 0;
    TRY(decompress_impl(c, t, reinterpret_cast<const uint8_t *>(ins[i]), sizes[i],
                        want ? outs[i - first] : nullptr, n_cap, &no, &dd, s, !want));
    if (want) {
      if (n_out) *n_out = no;
      if (d_out) *d_out = dd;
    }
  }
  return OK;
}

}  // namespace

namespace lcp {
// The frames of a chain the caller has already determined (the serving
// loop's own bookkeeping), in stream order: all but the last decoded to
// codes only, the last into out.  t is reset first.
int decode_chain(lcp_ctx *c, lcp_traj *t, const void *const *ins, const size_t *sizes, int k,
                 float *out, uint64_t n_cap, uint64_t *n_out, uint32_t *d_out, cudaStream_t s) {
  if (!c || !t || !ins || !sizes || k < 1) return ERR_ARG;
  DeviceGuard g(c->device);
  if (!g.ok) return ERR_CUDA;
  prof_reset(c);
  t->has_prev = t->has_anchor = false;
  t->prev_scaled = t->anc_scaled = false;
  t->t = 0;
  for (int i = 0; i < k; ++i) {
    const bool last = i == k - 1;
    TRY(decompress_impl(c, t, reinterpret_cast<const uint8_t *>(ins[i]), sizes[i],
                        last ? out : nullptr, n_cap, n_out, d_out, s, !last));
  }
  return OK;
}
}  // namespace lcp

extern "C" {

lcp_status lcp_decompress_frames(lcp_ctx *c, lcp_traj *dec, const void *const *d_containers,
                                 const size_t *sizes, uint64_t count, uint64_t first,
                                 uint64_t last, float *const *d_outs, uint64_t n_cap,
                                 uint64_t *n_out, uint32_t *d_fields, void *stream) {
  if (!c) return LCP_ERR_ARG;
  DeviceGuard g(c->device);
  if (!g.ok) return LCP_ERR_CUDA;
  prof_reset(c);
  return (lcp_status)decompress_range(c, dec, d_containers, sizes, count, first, last, d_outs,
                                      n_cap, n_out, d_fields, (cudaStream_t)stream);
}

lcp_status lcp_decompress_frame(lcp_ctx *c, lcp_traj *dec, const void *const *d_containers,
                                const size_t *sizes, uint64_t count, uint64_t target,
                                float *d_out, uint64_t n_cap, uint64_t *n_out,
                                uint32_t *d_fields, void *stream) {
  float *outs[1] = {d_out};
  return lcp_decompress_frames(c, dec, d_containers, sizes, count, target, target, outs, n_cap,
                               n_out, d_fields, stream);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// one time step of many trajectories (config 4): the LCP-T frames in one
// persistent launch, planned on the device, replayed as a CUDA graph
// ---------------------------------------------------------------------------
struct lcp_step {
  lcp_ctx *ctx = nullptr;
  int max_frames = 0;
  // the graph runs on the step's own stream (a capture cannot use the legacy
  // default stream), ordered after the caller's stream and before its next
  // work by events
  cudaStream_t own = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  cudaGraphExec_t exec = nullptr;
  int graph_kernels = 0;  // kernel nodes of the graph
  // optional lanes for the frames the step does not fuse
  std::vector<lcp_ctx *> lane_ctx;
  std::vector<void *> lane_stream;
  // device
  uint32_t *d_nf = nullptr;
  StepIn *d_jobs = nullptr;
  StepFrame *d_frames = nullptr;
  HuffTable *d_tabs = nullptr;
  unsigned long long *d_items = nullptr;
  StepResult *d_res = nullptr;
  // pinned host: the step's jobs in, results out
  uint32_t *h_nf = nullptr;
  StepIn *h_jobs = nullptr;
  StepResult *h_res = nullptr;
  uint8_t *h_head = nullptr;  // container headers (16 bytes each)
};

extern "C" {

lcp_status lcp_step_create(lcp_ctx *c, int max_frames, lcp_step **out) {
  if (!c || !out || max_frames < 1 || max_frames > kStepMaxFrames) return LCP_ERR_ARG;
  *out = nullptr;
  DeviceGuard g(c->device);
  if (!g.ok) return LCP_ERR_CUDA;
  lcp_step *S = new lcp_step();
  S->ctx = c;
  S->max_frames = max_frames;
  const int F = kStepMaxFrames;
  if (cudaMalloc(&S->d_nf, 16) != cudaSuccess ||
      cudaMalloc(&S->d_jobs, sizeof(StepIn) * F) != cudaSuccess ||
      cudaMalloc(&S->d_frames, sizeof(StepFrame) * F) != cudaSuccess ||
      cudaMalloc(&S->d_tabs, sizeof(HuffTable) * F) != cudaSuccess ||
      cudaMalloc(&S->d_items, sizeof(unsigned long long) * (F + 2)) != cudaSuccess ||
      cudaMalloc(&S->d_res, sizeof(StepResult) * F) != cudaSuccess ||
      cudaMallocHost(&S->h_nf, 16) != cudaSuccess ||
      cudaMallocHost(&S->h_jobs, sizeof(StepIn) * F) != cudaSuccess ||
      cudaMallocHost(&S->h_res, sizeof(StepResult) * F) != cudaSuccess ||
      cudaMallocHost(&S->h_head, 16 * (size_t)F) != cudaSuccess ||
      cudaStreamCreateWithFlags(&S->own, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&S->ev_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&S->ev_out, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    lcp_step_destroy(S);
    return LCP_ERR_NOMEM;
  }
  *out = S;
  return LCP_OK;
}

lcp_status lcp_step_destroy(lcp_step *S) {
  if (!S) return LCP_ERR_ARG;
  DeviceGuard g(S->ctx ? S->ctx->device : 0);
  if (S->exec) cudaGraphExecDestroy(S->exec);
  if (S->own) {
    cudaStreamSynchronize(S->own);
    cudaStreamDestroy(S->own);
  }
  if (S->ev_in) cudaEventDestroy(S->ev_in);
  if (S->ev_out) cudaEventDestroy(S->ev_out);
  cudaFree(S->d_nf);
  cudaFree(S->d_jobs);
  cudaFree(S->d_frames);
  cudaFree(S->d_tabs);
  cudaFree(S->d_items);
  cudaFree(S->d_res);
  cudaFreeHost(S->h_nf);
  cudaFreeHost(S->h_jobs);
  cudaFreeHost(S->h_res);
  cudaFreeHost(S->h_head);
  delete S;
  return LCP_OK;
}

lcp_status lcp_step_set_lanes(lcp_step *S, lcp_ctx *const *ctxs, void *const *streams,
                              int lanes) {
  if (!S || lanes < 0 || (lanes > 0 && !ctxs)) return LCP_ERR_ARG;
  for (int k = 0; k < lanes; ++k)
    if (!ctxs[k] || ctxs[k]->device != S->ctx->device) return LCP_ERR_ARG;
  S->lane_ctx.assign(ctxs, ctxs + lanes);
  S->lane_stream.assign(lanes, nullptr);
  if (streams) S->lane_stream.assign(streams, streams + lanes);
  return LCP_OK;
}

}  // extern "C"

namespace {

// the step's device work, recorded once on the step's own stream as a
// graph: jobs in, planning, the persistent decode, patches, results out
int step_graph(lcp_step *S) {
  if (S->exec) return OK;
  cudaStream_t s = S->own;
  cudaGraph_t graph = nullptr;
  CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  cudaMemcpyAsync(S->d_nf, S->h_nf, 16, cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(S->d_jobs, S->h_jobs, sizeof(StepIn) * S->max_frames, cudaMemcpyHostToDevice, s);
  S->graph_kernels =
      launch_step(S->d_nf, S->d_jobs, S->d_frames, S->d_tabs, S->d_items, S->d_res, S->ctx->sms, s);
  cudaMemcpyAsync(S->h_res, S->d_res, sizeof(StepResult) * S->max_frames, cudaMemcpyDeviceToHost,
                  s);
  const cudaError_t e = cudaStreamEndCapture(s, &graph);
  if (e != cudaSuccess || !graph) {
    note_cuda_error(e, "cudaStreamEndCapture", __LINE__);
    cudaGetLastError();
    if (graph) cudaGraphDestroy(graph);
    return ERR_CUDA;
  }
  const cudaError_t ei = cudaGraphInstantiate(&S->exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ei != cudaSuccess) {
    note_cuda_error(ei, "cudaGraphInstantiate", __LINE__);
    cudaGetLastError();
    S->exec = nullptr;
    return ERR_CUDA;
  }
  return OK;
}

}  // namespace

extern "C" {

lcp_status lcp_decompress_step(lcp_step *S, lcp_decompress_job *jobs, int njobs, void *stream) {
  if (!S || njobs < 0 || (njobs > 0 && !jobs)) return LCP_ERR_ARG;
  lcp_ctx *c = S->ctx;
  DeviceGuard g(c->device);
  if (!g.ok) return LCP_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<uint32_t> meth(njobs, 0u), flg(njobs, 0u);
  // headers of every container (method, flags, n, d): rounds of up to 128
  // copies, one synchronization each
  constexpr int kRound = kStepMaxFrames / 2;  // 32-byte slots of h_head
  for (int base = 0; base < njobs; base += kRound) {
    const int end = std::min(njobs, base + kRound);
    for (int k = base; k < end; ++k) {
      lcp_decompress_job &J = jobs[k];
      J.status = LCP_OK;
      J.n_out = 0;
      J.d_fields = 0;
      J.ms = 0.0f;
      if (!J.d_in || J.in_size < 48 || !aligned16(J.d_in)) {
        J.status = LCP_ERR_FORMAT;
        continue;
      }
      if (cudaMemcpyAsync(S->h_head + 32 * (size_t)(k - base), J.d_in, 32, cudaMemcpyDeviceToHost,
                          s) != cudaSuccess) {
        cudaGetLastError();
        return LCP_ERR_CUDA;
      }
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) {
      cudaGetLastError();
      return LCP_ERR_CUDA;
    }
    for (int k = base; k < end; ++k) {
      lcp_decompress_job &J = jobs[k];
      if (J.status != LCP_OK) continue;
      const uint8_t *h = S->h_head + 32 * (size_t)(k - base);
      if (h[0] == 'L' && h[1] == 'C' && h[2] == 'P' && h[3] == 'Z') {
        meth[k] = 2;  // an LCPZ image: decoded one by one
        continue;
      }
      if (h[0] != 'L' || h[1] != 'C' || h[2] != 'P' || h[3] != '1') {
        J.status = LCP_ERR_FORMAT;
        continue;
      }
      J.d_fields = h[6];
      J.n_out = rd64(h + 16);
      meth[k] = h[5];
      flg[k] = rd32(h + 8);
    }
  }
  // the LCP-T frames whose reference is on their own grid go to the fused
  // step; the others are decoded one by one
  std::vector<int> fused;
  std::vector<unsigned char> seen_traj;
  int nf = 0;
  for (int k = 0; k < njobs; ++k) {
    lcp_decompress_job &J = jobs[k];
    if (J.status != LCP_OK) continue;
    const bool is_t = meth[k] == 1u;
    const uint32_t flags = flg[k];
    lcp_traj *t = J.traj;
    bool ok = is_t && t && !(flags & kFlagRequant) && nf < S->max_frames &&
              J.n_out <= J.n_cap && J.d_out && aligned16(J.d_out) &&
              ((flags & kFlagRefAnchor) ? t->has_anchor : t->has_prev) && t->n == J.n_out &&
              t->d == J.d_fields;
    for (int i : fused) ok = ok && jobs[i].traj != t;  // one frame per trajectory
    if (!ok) continue;
    if (traj_buffers(t, J.n_out, J.d_fields) != OK) continue;
    StepIn &I = S->h_jobs[nf];
    I.in = reinterpret_cast<const uint8_t *>(J.d_in);
    I.in_size = J.in_size;
    I.qref = (flags & kFlagRefAnchor) ? P<int32_t>(t->anc_q) : P<int32_t>(t->prev_q);
    I.out = J.d_out;
    I.qnew = P<int32_t>(t->new_q);
    I.n = J.n_out;
    I.d = J.d_fields;
    I.pad = 0;
    fused.push_back(k);
    ++nf;
  }
  if (nf > 0) {
    *S->h_nf = (uint32_t)nf;
    int st = step_graph(S);
    if (st != OK) return (lcp_status)st;
    if (cudaEventRecord(S->ev_in, s) != cudaSuccess ||
        cudaStreamWaitEvent(S->own, S->ev_in, 0) != cudaSuccess ||
        cudaGraphLaunch(S->exec, S->own) != cudaSuccess ||
        cudaEventRecord(S->ev_out, S->own) != cudaSuccess ||
        cudaStreamWaitEvent(s, S->ev_out, 0) != cudaSuccess ||
        cudaStreamSynchronize(S->own) != cudaSuccess) {
      cudaGetLastError();
      return LCP_ERR_CUDA;
    }
    for (int i = 0; i < S->graph_kernels; ++i) note_launch();
    for (int i = 0; i < nf; ++i) {
      lcp_decompress_job &J = jobs[fused[i]];
      const StepResult &R = S->h_res[i];
      J.status = (lcp_status)R.status;
      if (R.status != OK) continue;
      lcp_traj *t = J.traj;
      std::swap(t->prev_q, t->new_q);
      for (uint32_t k = 0; k < J.d_fields; ++k) t->prev_F[k] = R.f[k];
      t->prev_scaled = false;
      t->has_prev = true;
      t->t += 1;
    }
  }
  // the rest: over the step's lanes when it has them and no trajectory
  // comes twice among these frames, else one at a time in job order
  std::vector<int> rest;
  for (int k = 0; k < njobs; ++k)
    if (jobs[k].status == LCP_OK && std::find(fused.begin(), fused.end(), k) == fused.end())
      rest.push_back(k);
  bool spread = S->lane_ctx.size() > 1 && rest.size() > 1;
  for (size_t i = 0; spread && i < rest.size(); ++i)
    for (size_t j = 0; j < i && spread; ++j)
      if (jobs[rest[i]].traj && jobs[rest[i]].traj == jobs[rest[j]].traj) spread = false;
  if (spread) {
    std::vector<lcp_decompress_job> sub(rest.size());
    for (size_t i = 0; i < rest.size(); ++i) sub[i] = jobs[rest[i]];
    lcp_decompress_batch(S->lane_ctx.data(), S->lane_stream.data(), (int)S->lane_ctx.size(),
                         sub.data(), (int)sub.size());
    for (size_t i = 0; i < rest.size(); ++i) jobs[rest[i]] = sub[i];
  } else {
    for (int k : rest) {
      lcp_decompress_job &J = jobs[k];
      uint64_t no = 0;
      uint32_t dd = 0;
      J.status = (lcp_status)decompress_impl(c, J.traj, reinterpret_cast<const uint8_t *>(J.d_in),
                                             J.in_size, J.d_out, J.n_cap, &no, &dd, s);
      J.n_out = no;
      J.d_fields = dd;
    }
  }
  for (int k = 0; k < njobs; ++k)
    if (jobs[k].status != LCP_OK) return LCP_ERR_STATE;  // per-job statuses tell which
  return LCP_OK;
}

lcp_status lcp_peek(const void *d_in, size_t in_size, uint64_t *n, uint32_t *d,
                    lcp_method *method, uint32_t *flags, void *stream) {
  if (!d_in || in_size < 48) return LCP_ERR_FORMAT;
  uint8_t img[80];
  const size_t nb = in_size >= kDictHead ? kDictHead : 48;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemcpyAsync(img, d_in, nb, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return LCP_ERR_CUDA;
  }
  // an LCPZ image carries its container's header at byte 32
  const bool dict = nb == kDictHead && img[0] == 'L' && img[1] == 'C' && img[2] == 'P' &&
                    img[3] == 'Z' && img[4] == 1;
  const uint8_t *h = dict ? img + 32 : img;
  if (h[0] != 'L' || h[1] != 'C' || h[2] != 'P' || h[3] != '1' || h[4] != 1 || h[5] > 1 ||
      h[6] < 1 || h[6] > 8)
    return LCP_ERR_FORMAT;
  if (n) *n = rd64(h + 16);
  if (d) *d = h[6];
  if (method) *method = h[5] ? LCP_TEMPORAL : LCP_SPATIAL;
  if (flags) *flags = rd32(h + 8);
  return LCP_OK;
}

lcp_status lcp_quantize(const float *d_x, uint64_t n, float m, float e, float max_abs,
                        int32_t *d_q, float *d_xr, uint8_t *d_viol, void *stream) {
  if (n > 0 && (!d_x || !d_q || !d_xr || !d_viol)) return LCP_ERR_ARG;
  if (!(e > 0.0f)) return LCP_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  // the plan lives in a small per-call device buffer
  FieldPlan *fp = nullptr;
  int *stp = nullptr;
  if (cudaMallocAsync((void **)&fp, sizeof(FieldPlan) + 16, s) != cudaSuccess) {
    cudaGetLastError();
    return LCP_ERR_NOMEM;
  }
  stp = reinterpret_cast<int *>(fp + 1);
  launch_field_plan(m, e, max_abs, fp, stp, s);
  int hst = 0;
  lcp_status r = LCP_OK;
  if (cudaMemcpyAsync(&hst, stp, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    r = LCP_ERR_CUDA;
  } else if (hst != OK) {
    r = (lcp_status)hst;
  } else {
    // every q must stay below 2^30: checked by the kernel on every value
    launch_element_rules(d_x, n, fp, d_q, d_xr, d_viol, stp, s);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(&hst, stp, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      r = LCP_ERR_CUDA;
    else if (hst != OK)
      r = (lcp_status)hst;
  }
  cudaFreeAsync(fp, s);
  cudaStreamSynchronize(s);
  return r;
}

const char *lcp_last_error(void) { return g_last_error; }

uint64_t lcp_kernel_launches(void) { return __atomic_load_n(&g_launches, __ATOMIC_RELAXED); }

lcp_status lcp_ctx_profile(lcp_ctx *c, int enable) {
  if (!c || enable < 0 || enable > 2) return LCP_ERR_ARG;
  DeviceGuard g(c->device);
  if (!g.ok) return LCP_ERR_CUDA;
  Profile &P = c->prof;
  P.on = enable != 0;
  P.accumulate = enable == 2;
  P.n = 0;
  const int want = P.on ? (P.accumulate ? kProfAccum : kProfCall) : 0;
  while (P.cap() < want) {  // events made here, not while timing
    cudaEvent_t a = nullptr, b = nullptr;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
      cudaGetLastError();
      if (a) cudaEventDestroy(a);
      P.on = false;
      return LCP_ERR_CUDA;
    }
    P.ev.push_back(a);
    P.ev.push_back(b);
    P.names.push_back({});
  }
  return LCP_OK;
}

int lcp_ctx_profile_read(lcp_ctx *c, char *names, float *ms, int cap) {
  if (!c || !c->prof.on) return 0;
  DeviceGuard g(c->device);
  Profile &P = c->prof;
  int k = 0;
  for (; k < P.n && k < cap; ++k) {
    float t = 0.0f;
    if (cudaEventSynchronize(P.ev[2 * k + 1]) != cudaSuccess ||
        cudaEventElapsedTime(&t, P.ev[2 * k], P.ev[2 * k + 1]) != cudaSuccess) {
      cudaGetLastError();
      t = -1.0f;
    }
    if (ms) ms[k] = t;
    if (names) memcpy(names + 32 * k, P.names[k].data(), 32);
  }
  if (P.accumulate) P.n = 0;  // read out: the next stages start a new list
  return k;
}

}  // extern "C"
