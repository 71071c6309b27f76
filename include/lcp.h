/*
 * lcp.h -- C ABI of the B300 LCP library (liblcp.so).
 *
 * LCP (arXiv 2411.00761) is an error-bounded lossy compressor for particle
 * frames.  This library runs its hot path on one GPU:
 *
 *   LCP-S  (Sec. "LCP-S: the Error-Bound Aware Block-wise Spatial
 *          Compressor"): quantize every field into bins of width 2*eb (Eq.
 *          quantization), group particles into blocks of p bins per axis (Eq.
 *          block size and id), keep per non-empty block its id, particle count
 *          and the particles' locations relative to the block corner, delta
 *          code the three arrays and code each with Huffman or fixed-length
 *          bits, whichever is shorter (Sec. "Block coding", Table 3).
 *   LCP-T  (Sec. "LCP-T: The Temporal Compressor"): quantize as LCP-S, predict
 *          every code from the previous (or anchor) frame, code the
 *          differences.
 *   LCP    (Sec. "Hybrid Compression with LCP-S & T", Algorithm 1): per frame
 *          choice between the two with the LCP-FSM, spatial anchor frames
 *          opening each batch.
 *
 * Conventions shared by every entry point:
 *   - Frames are field-major ("SoA") float32 arrays [d][n] in DEVICE memory:
 *     field f of particle i is fields[f * n + i].  d is 1..8 (3 for x, y, z;
 *     further fields are extra dimensions of the block space, Sec. "Problem
 *     formulation").  Pointers must be 16-byte aligned.
 *   - The caller owns every input and output buffer.  The library owns only
 *     the context's workspace and the trajectory state.
 *   - Work is queued on the CUDA stream passed as `stream` (a cudaStream_t,
 *     NULL for the legacy default stream).  Calls that return a size or a
 *     status computed on the device synchronize that stream before returning.
 *   - No call aborts or exits.  Every failure is an lcp_status; a failed call
 *     leaves the output buffer contents unspecified and the trajectory state
 *     unchanged.
 *   - A context is not thread-safe: use one per host thread.
 *
 * The compressed container ("LCP1") is a byte string in device memory; its
 * layout is fixed and documented with the library.  Output bytes are a pure
 * function of the input values, eb, eb mode, p, method and reference state.
 */
#ifndef LCP_H
#define LCP_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define LCP_API __attribute__((visibility("default")))
#else
#define LCP_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LCP_OK = 0,
  LCP_ERR_ARG = -1,       /* invalid argument (d, eb, mode, p, pointer, alignment) */
  LCP_ERR_NONFINITE = -2, /* a NaN or infinity in the input frame */
  LCP_ERR_RANGE = -3,     /* frame outside the codec's domain: a field needs
                             2^30 or more bins, |value| >= 2^32 * 2 eb, or the
                             block key needs more than 63 bits */
  LCP_ERR_CAPACITY = -4,  /* output buffer too small; *out_size holds the need */
  LCP_ERR_FORMAT = -5,    /* malformed container */
  LCP_ERR_STATE = -6,     /* temporal frame without a matching reference */
  LCP_ERR_NOMEM = -7,     /* device allocation failed */
  LCP_ERR_TIMEOUT = -8,   /* a bounded device wait expired */
  LCP_ERR_CUDA = -9       /* a CUDA runtime call failed */
} lcp_status;

typedef enum {
  LCP_EB_ABS = 0, /* eb is the absolute bound of every field (Eq. abs) */
  LCP_EB_REL = 1  /* eb_f = eb * (max_f - min_f), or eb when the range is 0 */
} lcp_eb_mode;

typedef enum {
  LCP_SPATIAL = 0,  /* LCP-S */
  LCP_TEMPORAL = 1, /* LCP-T against the trajectory's reference */
  LCP_AUTO = 2      /* LCP-FSM choice (Sec. "Hybrid Compression"), Algorithm 1 */
} lcp_method;

typedef struct lcp_ctx lcp_ctx;   /* device workspace of one GPU */
typedef struct lcp_traj lcp_traj; /* per-trajectory reference state (device) */

/* Human-readable name of a status. */
LCP_API const char *lcp_status_str(lcp_status s);

/* Creates a context on CUDA device `device`.  The workspace grows on demand
 * (cudaMalloc, which synchronizes the device).  ERR_CUDA if the device is
 * unusable. */
LCP_API lcp_status lcp_ctx_create(int device, lcp_ctx **out);
LCP_API lcp_status lcp_ctx_destroy(lcp_ctx *ctx);
/* Pre-sizes the workspace for frames of up to n particles of d fields. */
LCP_API lcp_status lcp_ctx_reserve(lcp_ctx *ctx, uint64_t n, uint32_t d);

/* Upper bound on the container size of a frame of n particles and d fields
 * (any method). */
LCP_API size_t lcp_max_compressed_size(uint64_t n, uint32_t d);

/*
 * Compresses one frame.
 *   traj == NULL: stateless LCP-S; method must be LCP_SPATIAL or LCP_AUTO
 *                 (which then means spatial).
 *   traj != NULL: the frame is the next frame of that trajectory (Algorithm
 *                 1); LCP_AUTO applies the LCP-FSM, the other methods force
 *                 one (LCP_TEMPORAL needs a reference: ERR_STATE otherwise).
 *   eb, mode:     error bound (Eq. abs); the bound used per field is the
 *                 largest float32 not above eb_f, stored in the container.
 *   p:            block edge in bins, block_size = 2 eb p (Eq. block size
 *                 and id); a power of two, p^d <= 2^32.  p == 0 picks the
 *                 smallest container over p = 2, 4, 8, 16, 32 (Sec. "Best
 *                 block size"), ties to the smaller p.
 *   d_out:        device buffer of out_cap bytes; *out_size receives the
 *                 container size (also on ERR_CAPACITY, then the need).
 *   chosen:       optional; receives the method used.
 *   d_perm:       optional device uint32 [n]: for each decoded slot j, the
 *                 input index of the particle decoded there (the container
 *                 stores no permutation; decoded order is block order).
 * Synchronizes `stream`.
 */
LCP_API lcp_status lcp_compress(lcp_ctx *ctx, lcp_traj *traj, const float *d_fields, uint64_t n,
                        uint32_t d, double eb, lcp_eb_mode mode, uint32_t p, lcp_method method,
                        void *d_out, size_t out_cap, size_t *out_size, lcp_method *chosen,
                        uint32_t *d_perm, void *stream);

/*
 * Decompresses one container into d_out [d][n_cap] (field-major, stride n of
 * the container).  traj (decoder-side trajectory) is needed for LCP-T frames,
 * whose reference is the previous decoded frame or the last anchor as the
 * container's flags say; it is updated for the frames that follow.  Decoded
 * values are in slot order (blocks in id order, then raw outliers).
 * *n_out / *d_fields receive the frame's shape.  Synchronizes `stream`.
 */
LCP_API lcp_status lcp_decompress(lcp_ctx *ctx, lcp_traj *traj, const void *d_in, size_t in_size,
                          float *d_out, uint64_t n_cap, uint64_t *n_out, uint32_t *d_fields,
                          void *stream);
/* The same, for a caller that does not know the frame's shape beforehand:
 * d_out holds out_values floats, and the frame needs d n of them (values
 * [f][n], stride n); LCP_ERR_CAPACITY (nothing written) when it needs more. */
LCP_API lcp_status lcp_decompress_into(lcp_ctx *ctx, lcp_traj *traj, const void *d_in,
                                       size_t in_size, float *d_out, uint64_t out_values,
                                       uint64_t *n_out, uint32_t *d_fields, void *stream);

/*
 * Host-buffer variants of lcp_compress and lcp_decompress_into: the frame
 * h_fields [d][n] (compress) or the container h_in (decompress) is in host
 * memory, and so is the result (h_out: out_cap bytes of container, or
 * out_values floats of frame).  The library copies the input to the device,
 * makes the device call and copies the result back, all on `stream`; the
 * device copies live in the context's workspace (grown on demand, kept).
 * Host memory should be pinned (cudaHostAlloc / cudaHostRegister) for full
 * copy speed; pageable memory works but is staged by the driver.  Statuses
 * as for the device calls; synchronizes `stream`.
 */
LCP_API lcp_status lcp_compress_host(lcp_ctx *ctx, lcp_traj *traj, const float *h_fields,
                                     uint64_t n, uint32_t d, double eb, lcp_eb_mode mode,
                                     uint32_t p, lcp_method method, void *h_out, size_t out_cap,
                                     size_t *out_size, lcp_method *chosen, void *stream);
LCP_API lcp_status lcp_decompress_host(lcp_ctx *ctx, lcp_traj *traj, const void *h_in,
                                       size_t in_size, float *h_out, uint64_t out_values,
                                       uint64_t *n_out, uint32_t *d_fields, void *stream);

/*
 * Random-access retrieval (Sec. "Spatial-Anchor-Frame-Based Batch
 * Compression", its recursive decompression): frames first..last of one
 * trajectory, decoded into d_outs[0 .. last - first] ([d][n_cap] each).
 *   d_containers / sizes: host arrays of `count` entries, entry i the
 *     container of the trajectory's frame i (device pointer) in stream order,
 *     as lcp_compress wrote them.  Frames the request does not need may be
 *     NULL (e.g. evicted).
 *   A frame depends on its batch's frames before it and, when its batch
 *   opens with an LCP-T frame, on the batch's anchor (the latest earlier
 *   batch opening coded LCP-S).  The call decodes from the latest LCP-S frame
 *   of first's batch at or before first (else from the anchor); frames
 *   before `first` are decoded to codes only (no values written).  Besides
 *   those frames, the batch openings between the anchor and first's batch
 *   must be present (their headers show which one is the anchor).
 *   dec: a decoder-side trajectory created with the stream's batch size
 *     (frame t opens a batch when t % batch = 0), used as scratch state; the
 *     call resets it and leaves it holding frame `last` as its previous frame.
 *   ERR_STATE when a frame the chain needs is NULL or no anchor precedes an
 *   LCP-T batch opening; ERR_ARG when the stream's batch openings do not
 *   match dec's batch size; ERR_FORMAT for a container that is not LCP1.
 * *n_out / *d_fields receive the shape of the frames returned.  Synchronizes
 * `stream` (once per header round and per decoded frame).
 */
LCP_API lcp_status lcp_decompress_frames(lcp_ctx *ctx, lcp_traj *dec,
                                 const void *const *d_containers, const size_t *sizes,
                                 uint64_t count, uint64_t first, uint64_t last,
                                 float *const *d_outs, uint64_t n_cap, uint64_t *n_out,
                                 uint32_t *d_fields, void *stream);
/* One frame (first = last = target) of lcp_decompress_frames. */
LCP_API lcp_status lcp_decompress_frame(lcp_ctx *ctx, lcp_traj *dec,
                                const void *const *d_containers, const size_t *sizes,
                                uint64_t count, uint64_t target, float *d_out, uint64_t n_cap,
                                uint64_t *n_out, uint32_t *d_fields, void *stream);

/*
 * Schedule of a context: knobs of how its compressions run.
 *   log2_chunk   5..10 (default 10): every stream is cut into chunks of
 *                2^log2_chunk symbols that decode independently (Sec. "Block
 *                coding" names the coders; the chunking is this library's).
 *                Recorded in each container's header, so it is part of the
 *                bytes like p: smaller chunks cost chunk-table bytes and buy
 *                decoding parallelism.  Decoders accept every value.
 *   bucket_delta -4..1 (default 0): shift of the width of the first sort
 *                partition (up to 2^15 buckets).  Never changes the bytes.
 * The paper's own tuning is its block-size choice (lcp_choose_block_size);
 * these knobs are GPU schedule parameters with no counterpart there.
 */
typedef struct {
  uint32_t log2_chunk;
  int32_t bucket_delta;
  uint32_t reserved[6]; /* zero */
} lcp_schedule;
/* Applies a schedule to the context's later compressions (NULL: defaults);
 * ERR_ARG outside the ranges above. */
LCP_API lcp_status lcp_ctx_set_schedule(lcp_ctx *ctx, const lcp_schedule *schedule);
LCP_API lcp_status lcp_ctx_get_schedule(const lcp_ctx *ctx, lcp_schedule *out);
/*
 * Autotuner of the schedule for one frame shape: LCP-S round trips
 * (compress then decompress) of d_fields at bound eb and block multiplier p
 * (0: the exact block-size search first, Sec. "Best block size"), for
 * log2_chunk in {8, 9, 10} and bucket_delta in {-2, -1, 0, 1}, each timed
 * with CUDA events over `reps` round trips after one untimed; a candidate's
 * time is its fastest round (the least disturbed).  The fastest schedule
 * whose container is at most (1 + max_growth) times the default schedule's
 * size is returned in *best (and that round-trip ms in *best_ms, optional);
 * the context's own schedule is left as it was.
 * Allocates a worst-case container and an [d][n] output buffer for the
 * duration of the call (stream-ordered).  Synchronizes `stream`.
 */
LCP_API lcp_status lcp_tune_schedule(lcp_ctx *ctx, const float *d_fields, uint64_t n, uint32_t d,
                             double eb, lcp_eb_mode mode, uint32_t p, double max_growth,
                             int reps, lcp_schedule *best, float *best_ms, void *stream);

/*
 * Dictionary stage (Sec. "Block coding": dictionary coding is the last step
 * of the encoding stage; the paper uses Zstd).  The library's own LZ77-style
 * coder turns a byte string -- normally a container -- into an "LCPZ" image:
 *   - the input is cut into chunks of 2^16 bytes (the last one shorter),
 *     each coded alone by one warp: a greedy parse that copies from the
 *     latest earlier position whose four bytes hash alike when at least four
 *     bytes agree, written as LZ4-like sequences (token, literals, u16
 *     offset, length extensions); a chunk whose coding is not strictly
 *     shorter is stored as it is;
 *   - the image opens with an 80-byte header (magic "LCPZ", raw bytes S,
 *     chunk count, total bytes, and a copy of the first 48 raw bytes so a
 *     container's header stays readable), then one u32 size per chunk, then
 *     the chunks.  Its size is at most lcp_dict_max_size(S).
 * The layout is fixed and documented with the library; the bytes are a pure
 * function of the input bytes.
 *
 * lcp_ctx_set_dict(ctx, 1) applies the stage after every lcp_compress /
 * lcp_compress_host / lcp_compress_batch lane call of that context, keeping
 * the image only when it is shorter than the container; the capacity rule of
 * those calls is unchanged (out_cap must hold the container before the
 * stage).  Every decompression entry point, lcp_peek and the random-access
 * calls accept an image wherever a container is accepted, with or without
 * the option (lcp_decompress_step decodes images one by one, not fused).
 */
LCP_API lcp_status lcp_ctx_set_dict(lcp_ctx *ctx, int on);
LCP_API size_t lcp_dict_max_size(uint64_t raw_bytes);
/* The image of d_in[0, in_size) into d_out (16-byte aligned, not overlapping
 * d_in).  *out_size = the image's size, also on ERR_CAPACITY.  Synchronizes
 * `stream` once (the size); the image is written asynchronously after it. */
LCP_API lcp_status lcp_dict_compress(lcp_ctx *ctx, const void *d_in, size_t in_size, void *d_out,
                                     size_t out_cap, size_t *out_size, void *stream);
/* The raw bytes of an image (d_in 16-byte aligned) into d_out (out_cap
 * bytes, not overlapping d_in).  *out_size = the raw size once the header is
 * read (also on ERR_CAPACITY).  ERR_FORMAT for a malformed image: bad
 * header, size table, token, offset or length.  Synchronizes `stream`. */
LCP_API lcp_status lcp_dict_decompress(lcp_ctx *ctx, const void *d_in, size_t in_size,
                                       void *d_out, size_t out_cap, size_t *out_size,
                                       void *stream);

/* Reads n, d, method and flags from a container's header (device memory);
 * for an LCPZ image, from the container header it carries. */
LCP_API lcp_status lcp_peek(const void *d_in, size_t in_size, uint64_t *n, uint32_t *d,
                    lcp_method *method, uint32_t *flags, void *stream);

/*
 * LCP-FSM query (Sec. "Hybrid Compression"): the method the trajectory's next
 * frame would get, without coding it or changing any state.  *est_s is the
 * LCP-S size estimate (the size of the most recent LCP-S frame, 0 if none),
 * *est_t the exact LCP-T size when the FSM tests LCP-T for this frame (0
 * otherwise).  Both are sizes at the trajectory's bound eb: with anchor
 * scaling on (lcp_traj_set_anchor_scale), a frame that becomes an anchor is
 * written at eb / scale and its container is larger than est_s, so size the
 * output buffer with lcp_max_compressed_size, not with est_s.
 */
LCP_API lcp_status lcp_select(lcp_ctx *ctx, lcp_traj *traj, const float *d_fields, uint64_t n,
                      uint32_t d, double eb, lcp_eb_mode mode, lcp_method *chosen,
                      uint64_t *est_s, uint64_t *est_t, void *stream);

/*
 * Block-size search on a sample (Sec. "Best block size"): the candidates are
 * p = 2^k, 0 <= k <= 16, within the domain (p^d <= 2^32), each judged by the
 * exact LCP-S container size of a sample of the frame coded with that p;
 * the smallest wins, ties to the smaller p.  The sample is the frame's first
 * S particles in storage order, coded with the same eb and mode: S = sample
 * when 0 < sample <= n, S = min(n, max(65536, ceil(n / 8))) when sample == 0.
 *   d_fields:  device float32 [d][n], field-major, 16-byte aligned.
 *   p_best:    receives the chosen p.
 *   sizes:     optional host array of 17 entries; sizes[k] receives the
 *              sample's container size for p = 2^k, 0 where that p is
 *              outside the domain.
 * Returns ERR_RANGE when no candidate is in the domain.  Synchronizes
 * `stream`.
 */
LCP_API lcp_status lcp_choose_block_size(lcp_ctx *ctx, const float *d_fields, uint64_t n,
                                         uint32_t d, double eb, lcp_eb_mode mode,
                                         uint64_t sample, uint32_t *p_best, uint64_t *sizes,
                                         void *stream);

/*
 * Trajectory state for Algorithm 1: batch_size frames per batch (the first
 * frame of a batch is predicted from the last spatial anchor frame).  p is
 * the block multiplier its LCP-S frames use (nonzero).  A trajectory object
 * is used either for compressing or for decompressing one frame sequence.
 */
LCP_API lcp_status lcp_traj_create(lcp_ctx *ctx, uint32_t batch_size, uint32_t p, lcp_traj **out);
LCP_API lcp_status lcp_traj_destroy(lcp_traj *traj);

/*
 * Anchor bound scaling (Sec. "Best error-bound scale for anchor frames";
 * the paper picks 5).  With scale > 1, an anchor -- a first-in-batch frame
 * the LCP-FSM codes LCP-S -- is written with bound eb / scale while the FSM
 * sees temporal correlation (its state is T or S2 when the frame is planned;
 * a trajectory's first frame counts as correlated); the bound stays eb when
 * eb / scale leaves the codec's domain, and the FSM keeps deciding on sizes
 * at eb.  A T frame whose reference is such an anchor is predicted in value
 * space: every reference code is reconstructed on the anchor's grid (Q2),
 * quantized on the frame's grid (Q1) and clamped to [0, qmax]; its container
 * sets flag bit2 so that decoders do the same.  scale == 1 (the default)
 * turns it off.  scale in [1, 1024], else ERR_ARG.  Set it before the first
 * frame; encoder and decoder trajectories need no matching setting (the
 * containers carry the bounds and the flag).
 */
LCP_API lcp_status lcp_traj_set_anchor_scale(lcp_traj *traj, uint32_t scale);

/*
 * Checkpoint and resume of a trajectory (encoder or decoder side).  A frame
 * depends only on its batch and the batch's anchor (Sec. "Batch
 * compression", Algorithm 1), so the whole reference state is: the previous
 * frame's and the last anchor's slot codes and slot permutation, the LCP-FSM
 * state with its S-size estimate, and the frame counter.  The paper has no
 * checkpoint format; this one is the library's own.
 *
 * lcp_traj_export writes that state as a self-contained byte image into
 * host memory (little-endian; a 64-byte header, then the previous frame's
 * codes [d][n] int32 and permutation [n] uint32, then the anchor's, each
 * present only when the trajectory has it, then the two frames' grids in the
 * library's internal form, so an image is read back by the same library
 * version only).  *size receives the image size;
 * with host_out NULL or cap below it nothing is written and ERR_CAPACITY is
 * returned.  The trajectory is unchanged.  Synchronizes `stream`.
 *
 * lcp_traj_import creates a trajectory on ctx from such an image (the
 * context may be another one, on another device): frames coded or decoded
 * through it continue exactly as through the exported one.  A malformed
 * image returns ERR_FORMAT; *out is NULL on any error.  Synchronizes
 * `stream`.
 */
LCP_API lcp_status lcp_traj_export(const lcp_traj *traj, void *host_out, size_t cap,
                                   size_t *size, void *stream);
LCP_API lcp_status lcp_traj_import(lcp_ctx *ctx, const void *host_in, size_t size,
                                   lcp_traj **out, void *stream);

/* Device memory a context's workspace / a trajectory's state holds (bytes). */
LCP_API uint64_t lcp_ctx_device_bytes(const lcp_ctx *ctx);
LCP_API uint64_t lcp_traj_device_bytes(const lcp_traj *traj);

/*
 * Batched frames (the multi-frame layer around Algorithm 1: all frames of one
 * time step of many trajectories at once).  lcp_compress_batch runs the jobs
 * on `lanes` host threads; lane k uses ctxs[k] and streams[k] (streams may be
 * NULL: every lane then uses the legacy default stream), so
 * frames of different lanes overlap on the GPU.  Jobs are taken largest first
 * (n * d) from a shared counter.  Each job is exactly one lcp_compress call:
 * its bytes equal those of the same call made alone.  Two jobs of one batch
 * must not share a trajectory.  Per job, status, out_size, chosen and ms
 * (host wall time of the call) are filled in.  Returns LCP_OK when every job
 * succeeded, else the status of the first failed job in job order.  The paper
 * batches frames per trajectory (Sec. "Batch compression"); running many
 * trajectories' frames concurrently is this library's.
 */
typedef struct {
  lcp_traj *traj;         /* NULL: stateless LCP-S */
  const float *d_fields;  /* [d][n], device */
  uint64_t n;
  uint32_t d;
  double eb;
  lcp_eb_mode mode;
  uint32_t p;
  lcp_method method;
  void *d_out;            /* container buffer, out_cap bytes, device */
  size_t out_cap;
  size_t out_size;        /* out */
  lcp_method chosen;      /* out */
  lcp_status status;      /* out */
  float ms;               /* out */
} lcp_compress_job;

typedef struct {
  lcp_traj *traj;         /* decoder-side trajectory, or NULL for LCP-S frames */
  const void *d_in;       /* container, device */
  size_t in_size;
  float *d_out;           /* [d][n_cap], device */
  uint64_t n_cap;
  uint64_t n_out;         /* out */
  uint32_t d_fields;      /* out */
  lcp_status status;      /* out */
  float ms;               /* out */
} lcp_decompress_job;

/*
 * One time step of many trajectories (config 4; Algorithm 1 per trajectory)
 * decoded together.  Every LCP-T job whose reference is on its own grid is
 * planned on the device (one CTA per frame reads its header and stream
 * section, builds its field plans and Huffman tables) and decoded by one
 * persistent kernel over the chunks of all these frames, each symbol
 * finished on the spot (code, range check, Eq. quantization reversed); the
 * step's device work is recorded once as a CUDA graph on the step's own
 * stream and replayed there, ordered after the work already queued on
 * `stream` and before anything queued on it later.  Other jobs (LCP-S frames, references
 * re-quantized from a scaled anchor, a second frame of one trajectory) are
 * decoded one by one after the fused ones, in job order.
 *   - A job's traj is its trajectory's decoder state (as for
 *     lcp_decompress); each job's status, n_out and d_fields are set; the
 *     call returns LCP_OK when every job succeeded, else LCP_ERR_STATE.
 *   - One host synchronization for the headers, one after the graph.
 *   - A step serves at most max_frames fused frames per call (<= 256).
 *   - A step object is not thread-safe (one caller at a time).
 *   - lcp_step_set_lanes gives the step lanes (contexts and streams, as for
 *     lcp_decompress_batch; the arrays are copied, the contexts must outlive
 *     the step and be used by nothing else during its calls): the frames it
 *     does not fuse are then spread over them, unless a trajectory comes
 *     twice among those frames (then one at a time).  0 lanes: none.
 */
typedef struct lcp_step lcp_step;
LCP_API lcp_status lcp_step_create(lcp_ctx *ctx, int max_frames, lcp_step **out);
LCP_API lcp_status lcp_step_destroy(lcp_step *step);
LCP_API lcp_status lcp_step_set_lanes(lcp_step *step, lcp_ctx *const *ctxs,
                                      void *const *streams, int lanes);

LCP_API lcp_status lcp_compress_batch(lcp_ctx *const *ctxs, void *const *streams, int lanes,
                                      lcp_compress_job *jobs, int njobs);
LCP_API lcp_status lcp_decompress_batch(lcp_ctx *const *ctxs, void *const *streams, int lanes,
                                        lcp_decompress_job *jobs, int njobs);
LCP_API lcp_status lcp_decompress_step(lcp_step *step, lcp_decompress_job *jobs, int njobs,
                                       void *stream);

/*
 * Serving: a request loop around the codec.  Producers submit requests as
 * they arrive; the server runs them on `lanes` host threads, each with its own
 * context and CUDA stream, so requests of different producers overlap on the
 * GPU, while one producer's requests run one at a time in submission order.
 *   - LCP_REQ_COMPRESS codes the producer's next frame (d_fields [d][n],
 *     device, valid until the request completes) through the producer's
 *     trajectory: LCP-FSM and Algorithm 1 with batch `batch`, block multiplier
 *     p (0: 8).  The container is kept on the device (and copied to d_bytes
 *     when given); the response gives its frame index, size and method.  A
 *     producer's frames all have one shape.
 *   - LCP_REQ_DECOMPRESS decodes the producer's frame `frame` into d_out
 *     [d][n_cap] (device): from the latest LCP-S frame of its batch, or from
 *     the batch's anchor when the batch opens with LCP-T, the frames before
 *     `frame` to codes only.  Containers older than the last 2 * batch frames
 *     are freed (anchors still needed are kept); lcp_server_frames gives the
 *     decodable range [first, next).  A frame that is not decodable when the
 *     request is submitted is refused then (ERR_STATE); otherwise the frames
 *     the request needs are pinned until it completes, so it cannot fail for
 *     want of them.  Containers use stream-ordered device memory from the
 *     device's default pool (freed memory is kept for reuse), so requests
 *     never synchronize the device to allocate.
 *   - Admission: lcp_server_submit returns LCP_ERR_NOMEM when the device
 *     memory the server holds (workspaces, reference states, containers, and
 *     what admitted requests may still add) plus this request's worst case
 *     would exceed hbm_budget (0: no budget).
 *   - lcp_server_wait blocks until the ticket's request is done and returns
 *     its response once; times are ms since lcp_server_create (enqueue: at
 *     submission, start: a lane took it, done: its result is in device memory).
 * The paper has no serving layer; this is the library's.
 */
typedef struct lcp_server lcp_server;
typedef enum { LCP_REQ_COMPRESS = 0, LCP_REQ_DECOMPRESS = 1 } lcp_req_op;
typedef struct {
  lcp_req_op op;
  uint32_t producer;
  const float *d_fields;  /* compress */
  uint64_t n;
  uint32_t d;
  double eb;
  lcp_eb_mode mode;
  uint32_t p;
  uint64_t frame;         /* decompress */
  float *d_out;
  uint64_t n_cap;
  void *d_bytes;          /* compress, optional: a copy of the container */
  size_t bytes_cap;       /* (ERR_CAPACITY in the response when too small) */
} lcp_request;
typedef struct {
  lcp_status status;
  uint64_t frame;
  size_t size;
  lcp_method method;
  double enqueue_ms, start_ms, done_ms;
} lcp_response;

LCP_API lcp_status lcp_server_create(int device, int lanes, uint32_t batch, uint64_t hbm_budget,
                                     lcp_server **out);
LCP_API lcp_status lcp_server_submit(lcp_server *srv, const lcp_request *req, uint64_t *ticket);
LCP_API lcp_status lcp_server_wait(lcp_server *srv, uint64_t ticket, lcp_response *out);
LCP_API lcp_status lcp_server_frames(lcp_server *srv, uint32_t producer, uint64_t *first,
                                     uint64_t *next);
LCP_API uint64_t lcp_server_device_bytes(lcp_server *srv);
LCP_API lcp_status lcp_server_destroy(lcp_server *srv);

/*
 * Per-kernel timing (tracing).  With profiling on, every entry point records
 * a CUDA event pair on its stream around each major kernel (stage names such
 * as "s.quantize", "s.local_sort", "d.expand").
 *   - enable 1: each call's stages replace the previous call's (up to 32).
 *   - enable 2: stages accumulate over calls (up to 4096) until read, so a
 *     timed loop needs no read between its calls; the read empties the list.
 *   - enable 0: off.  Enabling makes the events (outside any timed region).
 * lcp_ctx_profile_read returns the number of stages listed (at most cap),
 * their names in names[32 * k] (NUL-terminated) and durations in ms[k]; it
 * waits for those events.  The paper has no counterpart: this is measurement
 * plumbing.
 */
LCP_API lcp_status lcp_ctx_profile(lcp_ctx *ctx, int enable);
/* Description of the last failed CUDA runtime call on this thread (empty if
 * none): the call, its place in the library and CUDA's error string. */
LCP_API const char *lcp_last_error(void);
/* Number of CUDA kernels this library has launched in this process. */
LCP_API uint64_t lcp_kernel_launches(void);
LCP_API int lcp_ctx_profile_read(lcp_ctx *ctx, char *names, float *ms, int cap);

/*
 * Element rules, exposed for verification.  For x[i] (device, n values) of a
 * field with minimum m and bound e (float32, e > 0 normal):
 *   q[i]    = floor((x[i] - m) / (2 e))            (Eq. quantization)
 *   xr[i]   = RN32(m + (2 q[i] + 1) e)             (reverse quantization)
 *   viol[i] = |x[i] - xr[i]| > e                   (Eq. abs violated)
 * all over the reals, bit-exact.  Requires x[i] >= m (results are
 * unspecified otherwise) and q < 2^30 (ERR_RANGE otherwise, checked on the
 * device for every value).  max_abs is unused; it is kept so that the
 * signature stays stable.
 */
LCP_API lcp_status lcp_quantize(const float *d_x, uint64_t n, float m, float e, float max_abs,
                        int32_t *d_q, float *d_xr, uint8_t *d_viol, void *stream);

/*
 * The element rules of lcp_quantize for callers that cannot allocate device
 * memory: code that runs inside an application which owns the GPU's memory
 * through its own pool (a cudaMalloc would bypass the pool and synchronize
 * the device), or loops that forbid allocation once running.  The paper has
 * no counterpart; this is library plumbing.
 *
 * Same inputs and outputs as lcp_quantize, bit for bit, plus *n_violations
 * (optional, host): how many values break the bound.  The call allocates
 * nothing: its scratch (per-block counts, a completion counter, the status)
 * is one fixed device array of about 16.5 KB inside the library, which every
 * GPU that loads the library holds until the process exits.
 *   - n may be at most LCP_NOALLOC_MAX_ELEMENTS; larger n returns LCP_ERR_ARG
 *     before any work is queued.
 *   - The first call on each device resolves the device address of that
 *     array (cudaGetSymbolAddress).
 *   - No call can be recorded inside a stream capture: every call
 *     synchronizes `stream` and copies its status to the host.
 *   - All calls share the array: the call clears the counter it needs, but
 *     two calls whose work overlaps on the GPU (on different streams, or
 *     from different threads) race on it.  Serialize them.
 * Synchronizes `stream`.
 */
#define LCP_NOALLOC_MAX_ELEMENTS 16777216ull
LCP_API lcp_status lcp_quantize_noalloc(const float *d_x, uint64_t n, float m, float e,
                                        float max_abs, int32_t *d_q, float *d_xr,
                                        uint8_t *d_viol, uint64_t *n_violations, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* LCP_H */
