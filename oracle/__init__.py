"""CPU oracle of the LCP hot path (arXiv 2411.00761) -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  The product path (``paper_2411_00761_b300``)
never does: it shares no code with the oracle and fails loudly when its own
CUDA library is missing.

The numerical core is ``lcp_oracle.c`` (single-threaded, exact arithmetic);
this module builds it with gcc and wraps it with ctypes over numpy arrays.
The LCP-FSM / Algorithm 1 driver is plain Python in ``oracle.hybrid``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lcp_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liblcp_oracle.so")

OK, ERR_ARG, ERR_NONFINITE, ERR_RANGE, ERR_CAPACITY, ERR_FORMAT, ERR_STATE, ERR_NOMEM = (
    0, -1, -2, -3, -4, -5, -6, -7)
EB_ABS, EB_REL = 0, 1


class OracleError(RuntimeError):
    def __init__(self, status: int, where: str):
        super().__init__(f"oracle {where} failed with status {status}")
        self.status = status


def build(force: bool = False) -> str:
    """Compiles lcp_oracle.c into liblcp_oracle.so (plain gcc, -O2, no FMA
    contraction, no fast-math)."""
    hdr = os.path.join(_HERE, "lcp_oracle.h")
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(_SRC), os.path.getmtime(hdr))):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                           "-fno-fast-math", "-Wall", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _declare(_lib)
    return _lib


_fp = C.POINTER(C.c_float)
_u8p = C.POINTER(C.c_uint8)
_u32p = C.POINTER(C.c_uint32)
_i32p = C.POINTER(C.c_int32)
_u64p = C.POINTER(C.c_uint64)
_i64p = C.POINTER(C.c_int64)
_szp = C.POINTER(C.c_size_t)


class _FieldPlan(C.Structure):
    """orc_field_plan (lcp_oracle.h)."""
    _fields_ = [("min_f", C.c_float), ("max_f", C.c_float), ("eb_f", C.c_double),
                ("e", C.c_float), ("qmax", C.c_uint32)]


def _declare(L):
    L.orc_q1.restype = C.c_int64
    L.orc_q1.argtypes = [C.c_float, C.c_float, C.c_float]
    L.orc_q2.restype = C.c_float
    L.orc_q2.argtypes = [C.c_int64, C.c_float, C.c_float]
    L.orc_q3_violates.restype = C.c_int
    L.orc_q3_violates.argtypes = [C.c_float, C.c_float, C.c_float]
    L.orc_round_down_f32.restype = C.c_float
    L.orc_round_down_f32.argtypes = [C.c_double]
    L.orc_q1_many.argtypes = [_fp, C.c_size_t, C.c_float, C.c_float, _i64p]
    L.orc_q2_many.argtypes = [_i64p, C.c_size_t, C.c_float, C.c_float, _fp]
    L.orc_q3_many.argtypes = [_fp, _fp, C.c_size_t, C.c_float, _u8p]
    L.orc_huffman_lengths.restype = C.c_int
    L.orc_huffman_lengths.argtypes = [_u64p, _u8p]
    L.orc_max_compressed_size.restype = C.c_size_t
    L.orc_max_compressed_size.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32]
    L.orc_compress_s.restype = C.c_int
    L.orc_compress_s.argtypes = [_fp, C.c_uint64, C.c_uint32, C.c_double, C.c_int, C.c_uint32,
                                 C.c_uint32, C.c_uint32, _u8p, C.c_size_t, _szp, _u32p, _i32p,
                                 _u64p, _u64p, _u64p, _u64p, _u64p]
    L.orc_compress_t.restype = C.c_int
    L.orc_compress_t.argtypes = [_fp, C.c_uint64, C.c_uint32, C.c_double, C.c_int, _i32p, _u32p,
                                 C.c_uint32, C.c_uint32, _u8p, C.c_size_t, _szp, _i32p, _u64p,
                                 _u64p]
    L.orc_peek.restype = C.c_int
    L.orc_peek.argtypes = [_u8p, C.c_size_t, _u64p, _u32p, _u32p, _u32p]
    L.orc_plan.restype = C.c_int
    L.orc_plan.argtypes = [_fp, C.c_uint64, C.c_uint32, C.c_double, C.c_int,
                           C.POINTER(_FieldPlan)]
    L.orc_decompress.restype = C.c_int
    L.orc_decompress.argtypes = [_u8p, C.c_size_t, _i32p, _fp, C.c_uint64, _i32p]
    L.orc_dict_max_size.restype = C.c_size_t
    L.orc_dict_max_size.argtypes = [C.c_uint64]
    L.orc_dict_compress.restype = C.c_int
    L.orc_dict_compress.argtypes = [_u8p, C.c_uint64, _u8p, C.c_size_t, _szp]
    L.orc_dict_decompress.restype = C.c_int
    L.orc_dict_decompress.argtypes = [_u8p, C.c_size_t, _u8p, C.c_size_t, _szp]


def _ptr(a, t):
    return a.ctypes.data_as(t) if a is not None else None


def _mode(mode) -> int:
    if mode in ("abs", EB_ABS):
        return EB_ABS
    if mode in ("rel", EB_REL):
        return EB_REL
    raise ValueError(mode)


def _fields(X) -> np.ndarray:
    X = np.ascontiguousarray(X, dtype=np.float32)
    if X.ndim != 2:
        raise ValueError("fields must be [D, N]")
    return X


# ---- element rules --------------------------------------------------------
def q1(x, m: float, e: float) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float32).ravel()
    q = np.empty(x.size, dtype=np.int64)
    lib().orc_q1_many(_ptr(x, _fp), x.size, m, e, _ptr(q, _i64p))
    return q


def q2(q, m: float, e: float) -> np.ndarray:
    q = np.ascontiguousarray(q, dtype=np.int64).ravel()
    xr = np.empty(q.size, dtype=np.float32)
    lib().orc_q2_many(_ptr(q, _i64p), q.size, m, e, _ptr(xr, _fp))
    return xr


def q3(x, xr, e: float) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float32).ravel()
    xr = np.ascontiguousarray(xr, dtype=np.float32).ravel()
    v = np.empty(x.size, dtype=np.uint8)
    lib().orc_q3_many(_ptr(x, _fp), _ptr(xr, _fp), x.size, e, _ptr(v, _u8p))
    return v.astype(bool)


def round_down_f32(d: float) -> float:
    return float(np.float32(lib().orc_round_down_f32(d)))


def huffman_lengths(freq) -> np.ndarray:
    f = np.zeros(4096, dtype=np.uint64)
    freq = np.asarray(freq, dtype=np.uint64)
    f[: freq.size] = freq
    ln = np.zeros(4096, dtype=np.uint8)
    lib().orc_huffman_lengths(_ptr(f, _u64p), _ptr(ln, _u8p))
    return ln[: max(freq.size, 1)]


def plan(X, eb: float, mode="abs") -> list[dict]:
    """Per-field grid of a frame (orc_plan): min, max, resolved bound eb_f,
    effective bound e (largest f32 <= eb_f) and qmax."""
    X = _fields(X)
    d, n = X.shape
    out = (_FieldPlan * d)()
    st = lib().orc_plan(_ptr(X, _fp), n, d, eb, _mode(mode), out)
    if st != OK:
        raise OracleError(st, "plan")
    return [dict(min=out[f].min_f, max=out[f].max_f, eb=out[f].eb_f, e=out[f].e,
                 qmax=int(out[f].qmax)) for f in range(d)]


def max_compressed_size(n: int, d: int) -> int:
    return int(lib().orc_max_compressed_size(n, d, 10))


# ---- frames ---------------------------------------------------------------
def compress_s(X, eb: float, mode="abs", p: int = 8, log2_chunk: int = 10, flags: int = 0,
               streams: bool = False) -> dict:
    """LCP-S compression of one frame X [D, N] (f32).  Returns the container
    bytes, the slot permutation pi, the slot codes q [D, N], M, K and (when
    asked) the three stream value arrays."""
    X = _fields(X)
    d, n = X.shape
    cap = max_compressed_size(n, d)
    out = np.zeros(cap, dtype=np.uint8)
    size = C.c_size_t(0)
    pi = np.zeros(max(n, 1), dtype=np.uint32)
    q = np.zeros((d, max(n, 1)), dtype=np.int32)
    ids = np.zeros(max(n, 1), dtype=np.uint64) if streams else None
    cnts = np.zeros(max(n, 1), dtype=np.uint64) if streams else None
    rels = np.zeros(max(n, 1), dtype=np.uint64) if streams else None
    m_out = np.zeros(1, dtype=np.uint64)
    k_out = np.zeros(1, dtype=np.uint64)
    st = lib().orc_compress_s(_ptr(X, _fp), n, d, eb, _mode(mode), p, log2_chunk, flags,
                              _ptr(out, _u8p), cap, C.byref(size), _ptr(pi, _u32p),
                              _ptr(q, _i32p), _ptr(ids, _u64p), _ptr(cnts, _u64p),
                              _ptr(rels, _u64p), _ptr(m_out, _u64p), _ptr(k_out, _u64p))
    if st != OK:
        raise OracleError(st, "compress_s")
    M, K = int(m_out[0]), int(k_out[0])
    res = dict(bytes=out[: size.value].tobytes(), pi=pi[:n], q=q[:, :n], M=M, K=K)
    if streams:
        res.update(ids=ids[:M], cnts=cnts[:M], rels=rels[: n - K])
    return res


def compressed_size_s(X, eb: float, mode="abs", p: int = 8, log2_chunk: int = 10) -> int:
    return len(compress_s(X, eb, mode, p, log2_chunk)["bytes"])


def compress_t(X, eb: float, mode, ref_q, ref_pi, log2_chunk: int = 10, flags: int = 0) -> dict:
    """LCP-T compression of X [D, N] against a reference held as slot codes
    ref_q [D, N] and slot permutation ref_pi [N]."""
    X = _fields(X)
    d, n = X.shape
    ref_q = np.ascontiguousarray(ref_q, dtype=np.int32)
    ref_pi = np.ascontiguousarray(ref_pi, dtype=np.uint32)
    if ref_q.shape != (d, n) or ref_pi.shape != (n,):
        raise OracleError(ERR_STATE, "compress_t")
    cap = max_compressed_size(n, d)
    out = np.zeros(cap, dtype=np.uint8)
    size = C.c_size_t(0)
    q = np.zeros((d, max(n, 1)), dtype=np.int32)
    syms = np.zeros(max(n * d, 1), dtype=np.uint64)
    k_out = np.zeros(1, dtype=np.uint64)
    st = lib().orc_compress_t(_ptr(X, _fp), n, d, eb, _mode(mode), _ptr(ref_q, _i32p),
                              _ptr(ref_pi, _u32p), log2_chunk, flags, _ptr(out, _u8p), cap,
                              C.byref(size), _ptr(q, _i32p), _ptr(syms, _u64p),
                              _ptr(k_out, _u64p))
    if st != OK:
        raise OracleError(st, "compress_t")
    return dict(bytes=out[: size.value].tobytes(), q=q[:, :n], syms=syms[: n * d],
                K=int(k_out[0]))


def peek(buf: bytes) -> dict:
    b = np.frombuffer(buf, dtype=np.uint8)
    n = np.zeros(1, dtype=np.uint64)
    d = np.zeros(1, dtype=np.uint32)
    fl = np.zeros(1, dtype=np.uint32)
    p = np.zeros(1, dtype=np.uint32)
    m = lib().orc_peek(_ptr(b, _u8p), b.size, _ptr(n, _u64p), _ptr(d, _u32p), _ptr(fl, _u32p),
                       _ptr(p, _u32p))
    if m < 0:
        raise OracleError(m, "peek")
    return dict(method=m, n=int(n[0]), d=int(d[0]), flags=int(fl[0]), p=int(p[0]))


def decompress(buf: bytes, ref_q=None) -> tuple[np.ndarray, np.ndarray]:
    """Decodes a container; returns (values [D, N] f32, codes [D, N] i32) in
    decoded-slot order.  T frames need the reference slot codes."""
    h = peek(buf)
    d, n = h["d"], h["n"]
    b = np.frombuffer(buf, dtype=np.uint8).copy()
    out = np.zeros((d, max(n, 1)), dtype=np.float32)
    q = np.zeros((d, max(n, 1)), dtype=np.int32)
    rq = None if ref_q is None else np.ascontiguousarray(ref_q, dtype=np.int32)
    st = lib().orc_decompress(_ptr(b, _u8p), b.size, _ptr(rq, _i32p), _ptr(out, _fp), n,
                              _ptr(q, _i32p))
    if st != OK:
        raise OracleError(st, "decompress")
    return out[:, :n], q[:, :n]


def dict_max_size(raw_bytes: int) -> int:
    """Size of the LCPZ image when every chunk is stored (lcp_oracle.h)."""
    return int(lib().orc_dict_max_size(raw_bytes))


def dict_compress(raw: bytes) -> bytes:
    """The dictionary stage (Sec. "Block coding", its last step): the LCPZ
    image of a byte string, normally a container."""
    b = np.frombuffer(raw, dtype=np.uint8)
    out = np.zeros(dict_max_size(b.size), dtype=np.uint8)
    sz = np.zeros(1, dtype=np.uint64)
    st = lib().orc_dict_compress(_ptr(b, _u8p) if b.size else None, b.size, _ptr(out, _u8p),
                                 out.size, sz.ctypes.data_as(_szp))
    if st != OK:
        raise OracleError(st, "dict_compress")
    return out[:int(sz[0])].tobytes()


def dict_decompress(img: bytes) -> bytes:
    """Inverse of dict_compress."""
    b = np.frombuffer(img, dtype=np.uint8)
    raw = int(np.frombuffer(img[8:16], dtype="<u8")[0]) if b.size >= 16 else 0
    out = np.zeros(max(raw, 1), dtype=np.uint8)
    sz = np.zeros(1, dtype=np.uint64)
    st = lib().orc_dict_decompress(_ptr(b, _u8p), b.size, _ptr(out, _u8p), raw,
                                   sz.ctypes.data_as(_szp))
    if st != OK:
        raise OracleError(st, "dict_decompress")
    return out[:int(sz[0])].tobytes()
