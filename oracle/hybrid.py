"""Oracle of the multi-frame layer -- TEST INFRASTRUCTURE ONLY.

* ``Fsm``: LCP-FSM, the per-frame choice between LCP-S and LCP-T (Sec.
  "Hybrid Compression with LCP-S & T").  The state diagram (Fig. 3) is not in
  the text; the reading implemented here is: states T and S{k} (k = 2, 4, 8,
  16).  The LCP-S estimate is the size of the most recent LCP-S frame.  With
  no reference frame the choice is spatial; with a reference but no estimate
  yet both are run and the smaller wins (ties to spatial), entering T or S2.
  In T every frame tests LCP-T; it stays when T <= estimate, else the frame
  is coded spatially and the state becomes S2.  In S{k} frames are coded
  spatially without a test until the k-th, which tests LCP-T: a win enters T,
  a loss doubles k (capped at 16).  PARITY UNPINNED against the paper (the
  figure is missing); pinned only by its own definition in tests.
* ``encode_trajectory`` / ``decode_trajectory``: Algorithm 1 (spatial anchor
  frames): the first frame of each batch is predicted from the last anchor,
  other frames from the previous frame, and a first frame coded spatially
  becomes the new anchor.  Decoding follows the recursive rule of Sec.
  "Spatial-Anchor-Frame-Based Batch Compression" in stream order.
* ``choose_block_size``: Sec. "Best block size": exact sizes for each
  candidate p, smallest wins, ties to the smaller p.
"""
from __future__ import annotations

import numpy as np

import oracle

FLAG_FIRST_IN_BATCH = 1
FLAG_REF_ANCHOR = 2
FLAG_REF_REQUANT = 4  # the reference codes were re-quantized on this frame's grid
BLOCK_CANDIDATES = (2, 4, 8, 16, 32)


class Fsm:
    def __init__(self):
        self.state = 2  # "T" or k of S{k}
        self.counter = 0
        self.s_est = None

    def plan(self, has_ref: bool) -> str:
        """'spatial', 'compare' or 'test' (test LCP-T against the estimate)."""
        if not has_ref:
            return "spatial"
        if self.s_est is None:
            return "compare"
        if self.state == "T":
            return "test"
        self.counter += 1
        if self.counter >= self.state:
            self.counter = 0
            return "test"
        return "spatial"

    def after_compare(self, t_wins: bool, s_size: int):
        self.s_est = s_size
        self.state = "T" if t_wins else 2
        self.counter = 0

    def after_test(self, t_wins: bool, s_size: int | None):
        if s_size is not None:
            self.s_est = s_size
        if t_wins:
            self.state = "T"
        elif self.state == "T":
            self.state = 2
        else:
            self.state = min(2 * self.state, 16)
        self.counter = 0

    def after_spatial(self, s_size: int):
        self.s_est = s_size


def grid_of_frame(X, eb: float, mode="abs") -> list[tuple[float, float, int]]:
    """(min, e, qmax) per field of the grid the frame is coded on."""
    return [(g["min"], g["e"], g["qmax"]) for g in oracle.plan(X, eb, mode)]


def grid_of_container(buf: bytes) -> list[tuple[float, float, int]]:
    """(min, e, qmax) per field, from a container header (f32 min, f32 e,
    u32 qmax at byte 48 + 16 f)."""
    d = buf[6]
    return [(float(np.frombuffer(buf, np.float32, 1, 48 + 16 * f)[0]),
             float(np.frombuffer(buf, np.float32, 1, 52 + 16 * f)[0]),
             int(np.frombuffer(buf, np.uint32, 1, 56 + 16 * f)[0])) for f in range(d)]


def requantize(ref_q, ref_grid, grid) -> np.ndarray:
    """Value-space prediction across grids (Sec. "Best error-bound scale for
    anchor frames"): each reference code is reconstructed on the reference's
    grid (Q2) and quantized on the frame's grid (Q1), clamped to [0, qmax]."""
    ref_q = np.asarray(ref_q)
    out = np.empty(ref_q.shape, dtype=np.int32)
    for f, ((mr, er, _), (mt, et, qmax)) in enumerate(zip(ref_grid, grid)):
        x = oracle.q2(ref_q[f].astype(np.int64), mr, er)
        q = np.where(x < np.float32(mt), 0, oracle.q1(np.maximum(x, np.float32(mt)), mt, et))
        out[f] = np.minimum(q, qmax)
    return out


def encode_trajectory(frames, eb: float, mode="abs", p: int = 8, batch: int = 10,
                      log2_chunk: int = 10, anchor_scale: int = 1):
    """Algorithm 1 over an iterable of frames [D, N].  Returns a list of
    (container bytes, method 'S'/'T') in frame order.

    anchor_scale > 1 (Sec. "Best error-bound scale for anchor frames"): an
    anchor -- a first-in-batch frame the LCP-FSM codes S -- is written with
    bound eb / anchor_scale while the FSM sees temporal correlation, i.e. its
    state is T or S2 (LCP-T has not lost twice in a row) when the frame is
    planned; the bound stays eb when eb / anchor_scale leaves the codec's
    domain.  The FSM still decides on the frame's size at eb.  A T frame whose
    reference is such an anchor predicts from the reference codes re-quantized
    on its own grid and sets FLAG_REF_REQUANT."""
    fsm = Fsm()
    prev = None    # dict(q, pi, grid, scaled) of the previous frame, slot order
    anchor = None  # the same for the last spatial anchor frame
    out = []
    for t, X in enumerate(frames):
        first = (t % batch) == 0
        ref = anchor if first else prev
        flags = FLAG_FIRST_IN_BATCH if first else 0
        tflags = flags | (FLAG_REF_ANCHOR if first else 0)
        ref_q = None
        if ref is not None:
            ref_q = ref["q"]
            if ref["scaled"]:
                ref_q = requantize(ref["q"], ref["grid"], grid_of_frame(X, eb, mode))
                tflags |= FLAG_REF_REQUANT
        correlated = fsm.state in ("T", 2)
        action = fsm.plan(ref is not None)
        s_res = t_res = None
        if action == "spatial":
            s_res = oracle.compress_s(X, eb, mode, p, log2_chunk, flags)
            fsm.after_spatial(len(s_res["bytes"]))
            use_t = False
        elif action == "compare":
            s_res = oracle.compress_s(X, eb, mode, p, log2_chunk, flags)
            t_res = oracle.compress_t(X, eb, mode, ref_q, ref["pi"], log2_chunk, tflags)
            use_t = len(t_res["bytes"]) < len(s_res["bytes"])
            fsm.after_compare(use_t, len(s_res["bytes"]))
        else:  # test LCP-T against the estimate
            t_res = oracle.compress_t(X, eb, mode, ref_q, ref["pi"], log2_chunk, tflags)
            use_t = len(t_res["bytes"]) <= fsm.s_est
            if not use_t:
                s_res = oracle.compress_s(X, eb, mode, p, log2_chunk, flags)
            fsm.after_test(use_t, None if use_t else len(s_res["bytes"]))
        if use_t:
            prev = dict(q=t_res["q"], pi=ref["pi"], grid=None, scaled=False)
            out.append((t_res["bytes"], "T"))
        else:
            scaled = False
            if first and anchor_scale > 1 and correlated:
                try:
                    s_res = oracle.compress_s(X, eb / anchor_scale, mode, p, log2_chunk, flags)
                    scaled = True
                except oracle.OracleError as err:
                    if err.status not in (oracle.ERR_ARG, oracle.ERR_RANGE):
                        raise
            prev = dict(q=s_res["q"], pi=s_res["pi"], scaled=scaled,
                        grid=grid_of_container(s_res["bytes"]) if scaled else None)
            if first:
                anchor = prev
            out.append((s_res["bytes"], "S"))
    return out


def decode_trajectory(containers):
    """Decodes containers in stream order; returns the list of decoded frames
    [D, N] in slot order (the slot order of each frame's chain)."""
    prev = None    # dict(q, grid)
    anchor = None
    frames = []
    for buf in containers:
        h = oracle.peek(buf)
        if h["method"] == 0:
            X, q = oracle.decompress(buf)
            cur = dict(q=q, grid=grid_of_container(buf))
            if h["flags"] & FLAG_FIRST_IN_BATCH:
                anchor = cur
        else:
            ref = anchor if h["flags"] & FLAG_REF_ANCHOR else prev
            ref_q = ref["q"]
            if h["flags"] & FLAG_REF_REQUANT:
                ref_q = requantize(ref["q"], ref["grid"], grid_of_container(buf))
            X, q = oracle.decompress(buf, ref_q)
            cur = dict(q=q, grid=grid_of_container(buf))
        prev = cur
        frames.append(X)
    return frames


# Sec. "Best block size": the candidates p = 2^k, 0 <= k <= 16
BLOCK_CANDIDATES_ALL = tuple(1 << k for k in range(17))


def sample_size(n: int) -> int:
    """Particles in the search sample when the caller gives none: an eighth
    of the frame, at least 65536 (all of a smaller frame)."""
    return min(n, max(65536, -(-n // 8)))


def choose_block_size_sampled(X, eb: float, mode="abs", sample: int = 0,
                              log2_chunk: int = 10) -> tuple[int, dict]:
    """Sec. "Best block size": each candidate p = 2^k (0 <= k <= 16) within
    the domain is judged by the exact LCP-S container size of a sample of the
    frame; the smallest wins, ties to the smaller p.  The paper leaves the
    sampling open; here the sample is the frame's first S particles in
    storage order, coded with the same bound and mode (S = sample, or
    sample_size(n) when 0)."""
    X = np.asarray(X, dtype=np.float32)
    n = X.shape[1]
    S = sample if sample else sample_size(n)
    return choose_block_size(np.ascontiguousarray(X[:, :S]), eb, mode, BLOCK_CANDIDATES_ALL,
                             log2_chunk)


def choose_block_size(X, eb: float, mode="abs", candidates=BLOCK_CANDIDATES,
                      log2_chunk: int = 10) -> tuple[int, dict]:
    """Exact compressed size per candidate p; returns (best p, sizes)."""
    sizes = {}
    for p in candidates:
        try:
            sizes[p] = oracle.compressed_size_s(X, eb, mode, p, log2_chunk)
        except oracle.OracleError as err:
            if err.status not in (oracle.ERR_ARG, oracle.ERR_RANGE):
                raise
    if not sizes:
        raise oracle.OracleError(oracle.ERR_RANGE, "choose_block_size")
    best = min(sizes, key=lambda k: (sizes[k], k))
    return best, sizes
