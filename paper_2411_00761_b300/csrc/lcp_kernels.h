// lcp_kernels.h -- host-side launchers of the LCP kernels (internal).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "lcp_common.cuh"

namespace lcp {

// largest sort unit held in shared memory; partition buckets above it are
// split by further key bits
constexpr int kUnitCap = 2048;

// kernels launched by this library in this process (all threads)
extern unsigned long long g_launches;
inline void note_launch() { __atomic_add_fetch(&g_launches, 1ull, __ATOMIC_RELAXED); }

// container header fields the decoder needs per field
struct DecodeFields {
  float m[kMaxD];
  float e[kMaxD];
  uint32_t qmax[kMaxD];
  uint32_t lp;
};

// one stream section as read from its 32-byte header
struct StreamInfo {
  unsigned long long n, payload_bits, n_chunks, maxv;
  uint32_t coder, width, used, log2_chunk;
};

// canonical Huffman decode tables
struct HuffTable {
  uint32_t fast[1u << kFastBits];  // sym << 5 | len, 0 when the code is longer
  uint32_t first[kLmax + 2], index[kLmax + 2], count[kLmax + 2];
  uint16_t syms[kAlpha];
  uint32_t used, ok;
};

#ifdef __CUDACC__
// First-level table, one entry per kFastBits-bit window, filled by all the
// block's threads entry by entry: in canonical order the window starts with
// a code of length L for the smallest L whose codes end above it, i.e.
// window < (first[L] + count[L]) 2^(kFastBits - L); that code is the
// window's top L bits and its symbol the (code - first[L])-th of length L.
// Windows whose code is longer than kFastBits get 0.  first, count and
// index are the canonical tables (1 .. kLmax), syms the symbols (U of them).
__device__ inline void huff_fill_fast(const uint32_t *first, const uint32_t *count,
                                      const uint32_t *index, const uint16_t *syms, uint32_t U,
                                      uint32_t *fast) {
  for (uint32_t e = threadIdx.x; e < (1u << kFastBits); e += blockDim.x) {
    uint32_t v = 0u;
    for (int L = 1; L <= kFastBits; ++L) {
      const uint32_t code = e >> (kFastBits - L);
      if (code < first[L] + count[L]) {
        const uint32_t i = index[L] + (code - first[L]);
        if (code >= first[L] && i < U) v = ((uint32_t)syms[i] << 5) | (uint32_t)L;
        break;
      }
    }
    fast[e] = v;
  }
}
#endif

// --- frame stage (k_frame.cu) -------------------------------------------
void launch_minmax(const float *fields, uint64_t n, uint32_t d, MinMax *mm, int sms,
                   cudaStream_t s);
void launch_plan(const MinMax *mm, uint64_t n, uint32_t d, double eb, int mode, uint32_t p,
                 uint32_t nbits_target, uint32_t method, Plan *plan, cudaStream_t s);
void launch_quantize_s(const float *fields, uint64_t n, uint32_t d, const Plan *plan,
                       uint32_t nb1, int tiles, unsigned long long *keys, uint32_t *tile_hist,
                       int32_t *q, cudaStream_t s);
void launch_field_plan(float m, float e, float max_abs, FieldPlan *fp, int *status,
                       cudaStream_t s);
// status: set to ERR_RANGE when a code falls outside [0, 2^30)
void launch_element_rules(const float *x, uint64_t n, FieldPlan *fp_dev, int32_t *q, float *xr,
                          uint8_t *viol, int *status, cudaStream_t s);

// --- partition and segmentation (k_sort.cu) -----------------------------
// exclusive scan, out[n] = total; skipped when gate is given and *gate != 1.
// With tmp (scan_tmp_len(n) entries) a long scan runs one CTA per tile.
void launch_scan_small(const unsigned long long *in, uint32_t n, unsigned long long *out,
                       cudaStream_t s, const uint32_t *gate = nullptr,
                       unsigned long long *tmp = nullptr);
uint64_t scan_tmp_len(uint64_t n);
void launch_bucket_offsets(uint32_t *tile_hist, int tiles, uint32_t nb1,
                           unsigned long long *bucket_start, unsigned long long *totals,
                           cudaStream_t s);
// bounds: kScatterPassesMax + 1 entries (device scratch)
constexpr uint32_t kScatterPassesMax = 16;
void launch_scatter(const unsigned long long *keys, uint64_t n, const Plan *plan, uint32_t nb1,
                    int tiles, const uint32_t *tile_off, const unsigned long long *bstart,
                    uint32_t *bounds, unsigned long long *keys_out, uint32_t *idx_out,
                    cudaStream_t s);
// level-2 split of the buckets above the split threshold (sub_off: per
// split bucket, the offset of each sub-bucket) and the unit list of the
// unsplit buckets and the outlier bucket
// Buffers (device): big_list, big_cb, big_tb, big_hs, big_of: nb1 + 1
// entries; task_owner: split_tasks_max; slot_owner: split_slots_max; multi:
// nb1; nbig: 8; sub_off: sub_off_size; chunk_owner (split bucket of each
// 32-digit chunk): sub_off_size / 32 + 1; shist: split_slots_max * 8192.
struct SegBufs {
  uint32_t *big_list, *big_cb, *big_tb, *big_hs, *task_owner, *slot_owner, *multi;
  int *big_of;
  uint32_t *nbig, *sub_off, *chunk_owner, *shist;
};
uint64_t sub_off_size(uint64_t n, uint32_t nb1);
uint64_t split_tasks_max(uint64_t n, uint32_t nb1);
uint64_t split_slots_max(uint64_t n);
void launch_segments(const Plan *plan, uint32_t nb1, const unsigned long long *bstart,
                     unsigned long long *keys, uint32_t *idx, unsigned long long *keys_alt,
                     uint32_t *idx_alt, const SegBufs &g, uint32_t *u_lo, uint32_t *u_cnt,
                     uint32_t *u_meta, uint32_t *nunit, uint64_t n, int sms, cudaStream_t s);
// sorting and segmentation outputs, per sorted slot g: s_rel[g] (relative
// location deltas), bflag[g] (1 where a block starts), tmp_bid[g] (the block
// id, at block starts only), perm[g] and q_slot (perm mode)
struct LocalArgs {
  const Plan *plan;
  const uint32_t *nseg;                    // units (device count)
  const uint32_t *seg_lo, *seg_cnt, *seg_meta;
  unsigned long long *keys;                // partitioned keys (level 1)
  uint32_t *idx;                           // partitioned input indices (perm mode)
  unsigned long long *keys_alt;            // level-2 split keys / scratch
  uint32_t *idx_alt;
  uint32_t *s_rel;                         // [n]
  uint8_t *bflag;                          // [n]
  unsigned long long *tmp_bid;             // [n]
  uint32_t *hist;                          // [3][4096]
  unsigned long long *maxv;                // [3]
  uint32_t *perm;                          // [n] slot -> input index (perm mode) or null
  const int32_t *q_in;                     // [d][n] codes by input index, or null
  int32_t *q_slot;                         // [d][n] codes by slot, or null
  uint32_t *outl_idx;                      // [n] outlier input indices, ascending
  uint32_t log2_chunk;
  uint64_t n;
};
void launch_local(const LocalArgs &a, int ctas, cudaStream_t s);
// runs of sub-buckets of the split buckets, sorted and segmented by warps;
// runs too large for a warp are appended to the unit list
struct SubsortArgs {
  const Plan *plan;
  const uint32_t *big_list, *big_cb, *chunk_owner;
  uint32_t *nbig;  // [6]: work counter (zeroed by the split)
  const unsigned long long *bstart;
  const uint32_t *sub_off;
  const unsigned long long *keys_alt;      // split keys
  const uint32_t *idx_alt;                 // split input indices (perm mode)
  uint32_t *nunit, *u_lo, *u_cnt, *u_meta;
  uint32_t *s_rel;
  uint8_t *bflag;
  unsigned long long *tmp_bid;
  uint32_t *hist;
  unsigned long long *maxv;
  uint32_t *perm;
  const int32_t *q_in;
  int32_t *q_slot;
  uint32_t log2_chunk;
  uint64_t n;
};
void launch_subsort(const SubsortArgs &a, int sms, cudaStream_t s);
// block numbering from the start flags of the nbk = *nbk non-outlier slots
// and the delta-coded ids and counts with their histograms; tile_cnt and
// tile_base hold flag_tiles(n) values, bpos n + 1, bidv n
uint64_t flag_tiles(uint64_t n);
void launch_blocks(const Plan *plan, const uint8_t *bflag, const unsigned long long *nbk,
                   uint64_t n, const unsigned long long *tmp_bid, unsigned long long *tile_cnt,
                   unsigned long long *tile_base, uint32_t *bpos, unsigned long long *bidv,
                   unsigned long long *s_id, unsigned long long *s_cnt, uint32_t *hist,
                   unsigned long long *maxv, unsigned long long *mcount, int sms,
                   cudaStream_t s);
// value counts of the three LCP-S streams and K
void launch_counts_s(const unsigned long long *bucket_start, uint32_t nb, uint64_t n,
                     const unsigned long long *mcount, unsigned long long *nvals,
                     unsigned long long *kcount, cudaStream_t s);
// sorts cnt (device count) (key, payload) pairs by key with one CTA
void launch_sort_pairs(unsigned long long *keys, uint32_t *vals, unsigned long long *keys_alt,
                       uint32_t *vals_alt, const unsigned long long *cnt, int kbits,
                       unsigned long long *keys_out, uint32_t *vals_out, cudaStream_t s);

// --- coding (k_code.cu) --------------------------------------------------
// work: codebook_work_size(ns) bytes
size_t codebook_work_size(int ns);
void launch_codebook(int ns, const uint32_t *hist, const unsigned long long *maxv,
                     const unsigned long long *n_vals, uint32_t log2_chunk, uint8_t *work,
                     StreamDesc *desc, uint32_t *codes, uint8_t *lens, uint16_t *tables,
                     cudaStream_t s);
struct LayoutArgs {
  int method;  // 0 S, 1 T
  uint32_t d, log2_chunk, flags, p;
  uint64_t n;
  const Plan *plan;
  StreamDesc *desc;  // [ns + 1], the last one is the outlier / patch section
  const uint16_t *tables;
  const unsigned long long *mcount;  // M (S)
  const unsigned long long *kcount;  // K
  uint8_t *out;
  unsigned long long cap;
  Summary *summary;
};
// size_only: offsets and total only (no writes to out)
void launch_layout(const LayoutArgs &a, int sms, bool size_only, cudaStream_t s);
void launch_encode_u64(const unsigned long long *vals, uint64_t n, const StreamDesc *desc,
                       const uint32_t *codes, const uint8_t *lens, uint32_t log2_chunk,
                       uint8_t *out, const Summary *summary, unsigned long long *chunk_bits,
                       unsigned long long *chunk_off, int sms, cudaStream_t s);
void launch_encode_u32(const uint32_t *vals, uint64_t n, const StreamDesc *desc,
                       const uint32_t *codes, const uint8_t *lens, uint32_t log2_chunk,
                       uint8_t *out, const Summary *summary, unsigned long long *chunk_bits,
                       unsigned long long *chunk_off, int sms, cudaStream_t s);
void launch_outliers_s(const float *fields, uint64_t n, uint32_t d, const uint32_t *outl_idx,
                       const StreamDesc *desc_outl, uint8_t *out, const Summary *summary,
                       int sms, cudaStream_t s);

// --- temporal (k_temporal.cu) --------------------------------------------
void launch_quantize_t(const float *fields, uint64_t n, uint32_t d, const Plan *plan,
                       const uint32_t *pi, const int32_t *qref, uint32_t *sym, int32_t *qnew,
                       uint32_t *hist, unsigned long long *maxv, unsigned long long *kcount,
                       unsigned long long *patch_s, float *patch_x, int sms, cudaStream_t s);
void launch_patches_write(const unsigned long long *ps, const uint32_t *order, const float *px,
                          const StreamDesc *od, uint8_t *out, const Summary *summary, int sms,
                          cudaStream_t s);
void launch_recon_t(const Plan *plan, uint64_t n, uint32_t d, const uint32_t *sym,
                    const int32_t *qref, float *out, int32_t *qnew, int *err, int sms,
                    cudaStream_t s);
void launch_patches_apply(const uint8_t *sec, uint64_t K, uint64_t nd, float *out, int *err,
                          int sms, cudaStream_t s);
// reference codes re-quantized on the frame's grid (plan): q' =
// clamp(Q1_frame(Q2_ref(q)), 0, qmax), per field, [d][n] int32
struct RefGrid {
  FieldPlan f[kMaxD];
};
void launch_requant(const Plan *plan, uint64_t n, uint32_t d, const int32_t *qref,
                    const RefGrid &g, int32_t *qout, int sms, cudaStream_t s);

// --- decode (k_decode.cu) --------------------------------------------------
// container bytes the host needs before decoding, gathered on the device:
// [0, kHeadBytes) the fixed header, field table and section directory, then
// 32 bytes per stream section header (up to 3)
constexpr int kHeadBytes = 48 + 16 * kMaxD + 16 * 4 + 16;
constexpr int kHeadStage = kHeadBytes + 3 * 32;
void launch_head_gather(const uint8_t *in, uint64_t in_size, uint8_t *stage, cudaStream_t s);
void launch_decode_plan(const DecodeFields *df, uint32_t d, Plan *plan, cudaStream_t s);
void launch_huff_table(const uint8_t *sec, HuffTable *T, cudaStream_t s);
// decodes ns streams (secs[k], infos[k]) into outs[k] (8-byte values when
// wide[k], else 4-byte; a null outs[k] skips the stream); Huffman streams
// share one launch (tables ht[k]).  agg_mode[k] (optional): 1 = the stream
// holds LCP-S block-id deltas, 2 = count deltas; its Huffman lanes then also
// write one block-scan aggregate per chunk into agg
void launch_decode_streams(int ns, const uint8_t *const *secs, const StreamInfo *infos,
                           HuffTable *ht, void *const *outs, const int *wide, const int *agg_mode,
                           void *agg, int *err, int sms, cudaStream_t s);
// LCP-S block scans: aggregates of 2^agg_log2 blocks each (agg:
// block_bases_bytes(M, agg_log2) bytes), their sums when the decode did not
// write them (agg_log2 = 10), and their bases
uint64_t block_bases_bytes(uint64_t M, uint32_t agg_log2);
void launch_block_sums(const void *sid, const void *scnt, int wide, uint64_t M, void *agg,
                       cudaStream_t s);
void launch_block_bases(uint64_t M, uint32_t agg_log2, void *agg, cudaStream_t s);
// reconstruction table of every code of every field: field f's codes
// 0..qmax_f at off[f]; off[d] entries in all
struct LutOffsets {
  uint32_t off[kMaxD + 1];
};
constexpr uint32_t kLutMax = 16384;  // largest table the expand keeps in shared memory
void launch_recon_lut(const Plan *plan, uint32_t d, const LutOffsets &lo, float *lut, int sms,
                      cudaStream_t s);
// the LCP-S expand over block tiles (see k_decode.cu)
struct ExpandArgs {
  const Plan *plan;
  const void *sid, *scnt;  // id deltas, zigzag count deltas: u64 when wide, else u32
  int wide;
  uint64_t M, tiles;       // tiles = ceil(M / 1024)
  const void *agg;         // block_bases_bytes(M, agg_log2) bytes, bases formed
  uint32_t agg_log2;       // blocks per aggregate = 2^agg_log2 (<= 10)
  const uint32_t *rel;     // decoded relative-location deltas [nb], or null:
  const uint32_t *rel_pl;  // then the fixed-width payload (rel_w <= 32 bits per value)
  uint32_t rel_w;
  uint64_t rel_words;
  uint64_t nb, n;
  uint32_t log2_chunk;
  const float *lut;        // with a table: its values and offsets
  LutOffsets lut_off;
  uint32_t qmax[kMaxD];    // largest code of each field (host copy)
  uint32_t lp;             // log2 p
  // filled by launch_expand: blocks per axis, floor(r / bn) = umulhi(r,
  // bmagic) >> bshift (bshift 255 when bn = 1), whether block ids need 64
  // bits, and the pairs (qmax_2i | qmax_2i+1 << 16)
  uint32_t bn[kMaxD];
  unsigned long long bmagic[kMaxD];
  uint32_t bshift[kMaxD];
  // the same quotient for r < 2^31: umulhi(r, bmagic32) >> bshift (Thm. 4.2
  // with 31-bit dividends: bmagic32 = ceil(2^(31 + l) / bn) < 2^32)
  uint32_t bmagic32[kMaxD];
  int div0_64;
  uint32_t qmax2[kMaxD / 2];
  float *out;              // [d][n], or null (codes only)
  int32_t *qout;           // [d][n] codes, or null
  int *err;
};
void launch_expand(uint32_t d, const ExpandArgs &a, bool lut, int sms, cudaStream_t s);
void launch_outliers_decode(const Plan *plan, const float *raw, uint64_t K, uint64_t n, uint32_t d,
                            float *out, int32_t *qout, int sms, cudaStream_t s);

// --- one time step of LCP-T frames in one persistent launch (k_step.cu) ---
constexpr int kStepMaxFrames = 256;
struct StepIn {             // per frame, from the host
  const uint8_t *in;        // container (device)
  unsigned long long in_size;
  const int32_t *qref;      // reference codes [d][n]
  float *out;               // decoded frame [d][n]
  int32_t *qnew;            // its codes [d][n]
  unsigned long long n;
  uint32_t d, pad;
};
struct StepFrame {          // per frame, planned on the device
  int status;
  uint32_t d, coder, width, used, log2_chunk;
  unsigned long long n, nd, K, n_chunks, payload_bits, nwords, groups, item0;
  const uint8_t *sec, *ct, *patch;
  const uint32_t *pl;
  unsigned int err;
  FieldPlan f[kMaxD];
};
struct StepResult {         // per frame, to the host
  int status;
  uint32_t pad;
  FieldPlan f[kMaxD];
};
// nframes (device) <= kStepMaxFrames; items: kStepMaxFrames + 2 entries
int launch_step(const uint32_t *nframes, const StepIn *jobs, StepFrame *frames, HuffTable *tabs,
                unsigned long long *items, StepResult *res, int sms, cudaStream_t s);

}  // namespace lcp
