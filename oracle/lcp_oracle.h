/*
 * lcp_oracle.h -- CPU oracle of the LCP hot path (arXiv 2411.00761).
 *
 * TEST INFRASTRUCTURE ONLY.  This header and lcp_oracle.c are a plain,
 * slow, single-threaded restatement of what LCP-S (Sec. "LCP-S", Eq.
 * quantization, Eq. block size and id, Sec. "Block coding") and LCP-T
 * (Sec. "LCP-T: The Temporal Compressor") compute.  Only tests/, the smoke
 * check and the bench's CPU-baseline leg may load it.  It shares no code,
 * header, table or constant generator with the CUDA library; the container
 * layout both sides produce is written out in prose in the design notes.
 *
 * All arithmetic on coordinates is exact: quantization, reconstruction and
 * the error guard are evaluated on exact dyadic rationals (multi-limb
 * integers), never in rounded floating point.
 */
#ifndef LCP_ORACLE_H
#define LCP_ORACLE_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes (same numbering as the library's public header, restated) */
#define ORC_OK 0
#define ORC_ERR_ARG (-1)
#define ORC_ERR_NONFINITE (-2)
#define ORC_ERR_RANGE (-3)
#define ORC_ERR_CAPACITY (-4)
#define ORC_ERR_FORMAT (-5)
#define ORC_ERR_STATE (-6)
#define ORC_ERR_NOMEM (-7)

/* error-bound modes */
#define ORC_EB_ABS 0
#define ORC_EB_REL 1

/* ---- element-wise rules (exact) ---------------------------------------- */

/* Q1: q = floor((x - m) / (2 e)) over the reals (Eq. quantization). */
int64_t orc_q1(float x, float m, float e);
/* Q2: RN32(m + (2q + 1) e), one rounding of the exact value (Eq. quantization,
 * reverse quantization). */
float orc_q2(int64_t q, float m, float e);
/* Q3: 1 when |x - x'| > e over the reals (Eq. abs violated), else 0. */
int orc_q3_violates(float x, float xr, float e);
/* Largest binary32 value <= d (round toward -inf); d > 0 finite. */
float orc_round_down_f32(double d);

/* vectorised forms for tests */
void orc_q1_many(const float *x, size_t n, float m, float e, int64_t *q);
void orc_q2_many(const int64_t *q, size_t n, float m, float e, float *xr);
void orc_q3_many(const float *x, const float *xr, size_t n, float e, uint8_t *v);

/* ---- Huffman code lengths (Sec. "Block coding") ------------------------ */
/* freq[4096] in, len[4096] out (0 for unused symbols).  Returns max length. */
int orc_huffman_lengths(const uint64_t *freq, uint8_t *len);

/* ---- frame plan --------------------------------------------------------- */
typedef struct {
  float min_f, max_f;
  double eb_f;   /* resolved error bound (ABS or REL x range) */
  float e;       /* effective bound: largest f32 <= eb_f */
  uint32_t qmax; /* floor((max - min) / 2e) */
} orc_field_plan;

/* Resolves per-field min/max, bounds and qmax.  fields is [d][n] f32. */
int orc_plan(const float *fields, uint64_t n, uint32_t d, double eb, int eb_mode,
             orc_field_plan *plan /* [d] */);

/* ---- LCP-S -------------------------------------------------------------- */
/* Upper bound on the container size for n particles of d fields. */
size_t orc_max_compressed_size(uint64_t n, uint32_t d, uint32_t log2_chunk);

/* Compresses one frame with LCP-S.  p: block multiplier (power of two).
 * flags: stored in the header (bit0 = first frame of a batch).
 * pi_out [n] (optional): original index of each decoded slot.
 * q_out [d][n] (optional): quantization code of each decoded slot.
 * streams (optional, for intermediate diffing): if ids/cnts/rels are non-NULL
 * they receive the three stream value arrays (sizes M, M, n-K). */
int orc_compress_s(const float *fields, uint64_t n, uint32_t d, double eb, int eb_mode,
                   uint32_t p, uint32_t log2_chunk, uint32_t flags, uint8_t *out,
                   size_t out_cap, size_t *out_size, uint32_t *pi_out, int32_t *q_out,
                   uint64_t *ids, uint64_t *cnts, uint64_t *rels, uint64_t *m_out,
                   uint64_t *k_out);

/* ---- LCP-T -------------------------------------------------------------- */
/* ref_q [d][n]: reference codes in decoded-slot order; ref_pi [n]: original
 * index of each slot.  q_out [d][n] receives this frame's codes (slot order). */
int orc_compress_t(const float *fields, uint64_t n, uint32_t d, double eb, int eb_mode,
                   const int32_t *ref_q, const uint32_t *ref_pi, uint32_t log2_chunk,
                   uint32_t flags, uint8_t *out, size_t out_cap, size_t *out_size,
                   int32_t *q_out, uint64_t *syms, uint64_t *k_out);

/* ---- decode ------------------------------------------------------------- */
/* Reads the fixed header.  Returns method (0 S, 1 T) or a negative status. */
int orc_peek(const uint8_t *in, size_t in_size, uint64_t *n, uint32_t *d, uint32_t *flags,
             uint32_t *p);
/* Decodes a container.  T frames need ref_q [d][n] (slot order).  out [d][n]
 * receives decoded values in slot order; q_out [d][n] (optional) the codes. */
int orc_decompress(const uint8_t *in, size_t in_size, const int32_t *ref_q, float *out,
                   uint64_t n_cap, int32_t *q_out);

/* ---- dictionary stage (Sec. "Block coding", its last step) ------------- */
/* The paper ends the encoding stage with a dictionary coder (Zstd).  This
 * is the library's own LZ77-style coder of a byte string (normally a whole
 * container), the "LCPZ" format written out in prose in the design notes:
 * 2^16-byte chunks coded independently; per chunk a greedy parse in which
 * position i may copy from the latest earlier position j of the chunk whose
 * four bytes hash alike (every position enters the table, also those
 * inside a copy), a copy being kept when at least four bytes agree; a chunk
 * whose coding is not strictly shorter is stored as it is. */
#define ORC_DICT_LOG2_CHUNK 16
#define ORC_DICT_HEAD 80
/* Size of the LCPZ image of raw_bytes bytes when every chunk is stored. */
size_t orc_dict_max_size(uint64_t raw_bytes);
int orc_dict_compress(const uint8_t *in, uint64_t in_size, uint8_t *out, size_t out_cap,
                      size_t *out_size);
/* out receives the raw bytes; *out_size their count (the header's). */
int orc_dict_decompress(const uint8_t *in, size_t in_size, uint8_t *out, size_t out_cap,
                        size_t *out_size);

#ifdef __cplusplus
}
#endif
#endif
