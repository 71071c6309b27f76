"""Python binding of liblcp.so (the B300 LCP library).

Argument marshalling only: every step of compression and decompression runs
in the library's CUDA kernels.  Tensors are torch CUDA tensors (device memory
and streams come from PyTorch); frames are float32 [d, n], field-major.
There is no CPU fallback: importing this module without the built library,
or calling it without a GPU, raises.
"""
from __future__ import annotations

import ctypes as C
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblcp.so")

OK, ERR_ARG, ERR_NONFINITE, ERR_RANGE, ERR_CAPACITY, ERR_FORMAT, ERR_STATE, ERR_NOMEM, \
    ERR_TIMEOUT, ERR_CUDA = 0, -1, -2, -3, -4, -5, -6, -7, -8, -9
EB_ABS, EB_REL = 0, 1
SPATIAL, TEMPORAL, AUTO = 0, 1, 2
FLAG_FIRST_IN_BATCH, FLAG_REF_ANCHOR = 1, 2

# every entry point include/lcp.h declares, with its ctypes signature
_vp, _u64, _u32, _sz = C.c_void_p, C.c_uint64, C.c_uint32, C.c_size_t
SIGNATURES = {
    "lcp_status_str": (C.c_char_p, [C.c_int]),
    "lcp_ctx_create": (C.c_int, [C.c_int, C.POINTER(C.c_void_p)]),
    "lcp_ctx_destroy": (C.c_int, [_vp]),
    "lcp_ctx_reserve": (C.c_int, [_vp, _u64, _u32]),
    "lcp_max_compressed_size": (_sz, [_u64, _u32]),
    "lcp_compress": (C.c_int, [_vp, _vp, _vp, _u64, _u32, C.c_double, C.c_int, _u32, C.c_int, _vp,
                               _sz, C.POINTER(_sz), C.POINTER(C.c_int), _vp, _vp]),
    "lcp_decompress": (C.c_int, [_vp, _vp, _vp, _sz, _vp, _u64, C.POINTER(_u64), C.POINTER(_u32),
                                 _vp]),
    "lcp_decompress_into": (C.c_int, [_vp, _vp, _vp, _sz, _vp, _u64, C.POINTER(_u64),
                                      C.POINTER(_u32), _vp]),
    "lcp_compress_host": (C.c_int, [_vp, _vp, _vp, _u64, _u32, C.c_double, C.c_int, _u32,
                                    C.c_int, _vp, _sz, C.POINTER(_sz), C.POINTER(C.c_int),
                                    _vp]),
    "lcp_decompress_host": (C.c_int, [_vp, _vp, _vp, _sz, _vp, _u64, C.POINTER(_u64),
                                      C.POINTER(_u32), _vp]),
    "lcp_peek": (C.c_int, [_vp, _sz, C.POINTER(_u64), C.POINTER(_u32), C.POINTER(C.c_int),
                           C.POINTER(_u32), _vp]),
    "lcp_select": (C.c_int, [_vp, _vp, _vp, _u64, _u32, C.c_double, C.c_int, C.POINTER(C.c_int),
                             C.POINTER(_u64), C.POINTER(_u64), _vp]),
    "lcp_choose_block_size": (C.c_int, [_vp, _vp, _u64, _u32, C.c_double, C.c_int, _u64,
                                        C.POINTER(_u32), C.POINTER(_u64), _vp]),
    "lcp_traj_create": (C.c_int, [_vp, _u32, _u32, C.POINTER(C.c_void_p)]),
    "lcp_traj_destroy": (C.c_int, [_vp]),
    "lcp_traj_set_anchor_scale": (C.c_int, [_vp, _u32]),
    "lcp_traj_export": (C.c_int, [_vp, _vp, _sz, C.POINTER(_sz), _vp]),
    "lcp_traj_import": (C.c_int, [_vp, _vp, _sz, C.POINTER(C.c_void_p), _vp]),
    "lcp_quantize": (C.c_int, [_vp, _u64, C.c_float, C.c_float, C.c_float, _vp, _vp, _vp, _vp]),
    "lcp_ctx_profile": (C.c_int, [_vp, C.c_int]),
    "lcp_kernel_launches": (_u64, []),
    "lcp_last_error": (C.c_char_p, []),
    "lcp_quantize_noalloc": (C.c_int, [_vp, _u64, C.c_float, C.c_float, C.c_float, _vp, _vp, _vp,
                                       C.POINTER(_u64), _vp]),
    "lcp_ctx_profile_read": (C.c_int, [_vp, C.c_char_p, C.POINTER(C.c_float), C.c_int]),
    "lcp_ctx_device_bytes": (_u64, [_vp]),
    "lcp_traj_device_bytes": (_u64, [_vp]),
    "lcp_server_create": (C.c_int, [C.c_int, C.c_int, _u32, _u64, C.POINTER(C.c_void_p)]),
    "lcp_server_submit": (C.c_int, [_vp, _vp, C.POINTER(_u64)]),
    "lcp_server_wait": (C.c_int, [_vp, _u64, _vp]),
    "lcp_server_frames": (C.c_int, [_vp, _u32, C.POINTER(_u64), C.POINTER(_u64)]),
    "lcp_server_device_bytes": (_u64, [_vp]),
    "lcp_server_destroy": (C.c_int, [_vp]),
    "lcp_compress_batch": (C.c_int, [C.POINTER(_vp), C.POINTER(_vp), C.c_int, _vp, C.c_int]),
    "lcp_decompress_batch": (C.c_int, [C.POINTER(_vp), C.POINTER(_vp), C.c_int, _vp, C.c_int]),
    "lcp_step_create": (C.c_int, [_vp, C.c_int, C.POINTER(_vp)]),
    "lcp_step_destroy": (C.c_int, [_vp]),
    "lcp_decompress_step": (C.c_int, [_vp, _vp, C.c_int, _vp]),
    "lcp_step_set_lanes": (C.c_int, [_vp, _vp, _vp, C.c_int]),
    "lcp_ctx_set_schedule": (C.c_int, [_vp, _vp]),
    "lcp_ctx_get_schedule": (C.c_int, [_vp, _vp]),
    "lcp_tune_schedule": (C.c_int, [_vp, _vp, _u64, _u32, C.c_double, C.c_int, _u32, C.c_double,
                                    C.c_int, _vp, C.POINTER(C.c_float), _vp]),
    "lcp_decompress_frames": (C.c_int, [_vp, _vp, C.POINTER(_vp), C.POINTER(_sz), _u64, _u64, _u64,
                                        C.POINTER(_vp), _u64, C.POINTER(_u64), C.POINTER(_u32),
                                        _vp]),
    "lcp_decompress_frame": (C.c_int, [_vp, _vp, C.POINTER(_vp), C.POINTER(_sz), _u64, _u64, _vp,
                                       _u64, C.POINTER(_u64), C.POINTER(_u32), _vp]),
    "lcp_ctx_set_dict": (C.c_int, [_vp, C.c_int]),
    "lcp_dict_max_size": (_sz, [_u64]),
    "lcp_dict_compress": (C.c_int, [_vp, _vp, _sz, _vp, _sz, C.POINTER(_sz), _vp]),
    "lcp_dict_decompress": (C.c_int, [_vp, _vp, _sz, _vp, _sz, C.POINTER(_sz), _vp]),
}


class CompressJob(C.Structure):
    """lcp_compress_job (include/lcp.h)."""
    _fields_ = [("traj", _vp), ("d_fields", _vp), ("n", _u64), ("d", _u32), ("eb", C.c_double),
                ("mode", C.c_int), ("p", _u32), ("method", C.c_int), ("d_out", _vp),
                ("out_cap", _sz), ("out_size", _sz), ("chosen", C.c_int), ("status", C.c_int),
                ("ms", C.c_float)]


class Schedule(C.Structure):
    """lcp_schedule (include/lcp.h)."""
    _fields_ = [("log2_chunk", _u32), ("bucket_delta", C.c_int32), ("reserved", _u32 * 6)]


class Request(C.Structure):
    """lcp_request (include/lcp.h)."""
    _fields_ = [("op", C.c_int), ("producer", _u32), ("d_fields", _vp), ("n", _u64), ("d", _u32),
                ("eb", C.c_double), ("mode", C.c_int), ("p", _u32), ("frame", _u64),
                ("d_out", _vp), ("n_cap", _u64), ("d_bytes", _vp), ("bytes_cap", _sz)]


class Response(C.Structure):
    """lcp_response (include/lcp.h)."""
    _fields_ = [("status", C.c_int), ("frame", _u64), ("size", _sz), ("method", C.c_int),
                ("enqueue_ms", C.c_double), ("start_ms", C.c_double), ("done_ms", C.c_double)]


REQ_COMPRESS, REQ_DECOMPRESS = 0, 1


class DecompressJob(C.Structure):
    """lcp_decompress_job (include/lcp.h)."""
    _fields_ = [("traj", _vp), ("d_in", _vp), ("in_size", _sz), ("d_out", _vp), ("n_cap", _u64),
                ("n_out", _u64), ("d_fields", _u32), ("status", C.c_int), ("ms", C.c_float)]


class LcpError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = _lib.lcp_status_str(status).decode() if _lib is not None else str(status)
        if _lib is not None and status == ERR_CUDA:
            msg += " [" + _lib.lcp_last_error().decode() + "]"
        super().__init__(f"{where}: {msg} ({status})")
        self.status = status


_lib = None


def load() -> C.CDLL:
    """Loads the in-tree liblcp.so; raises when it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"liblcp.so is not built ({LIB_PATH}); run "
                               "python -m paper_2411_00761_b300.build")
        lib = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _check(st: int, where: str):
    if st != OK:
        raise LcpError(st, where)


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _mode(mode) -> int:
    return {"abs": EB_ABS, "rel": EB_REL, EB_ABS: EB_ABS, EB_REL: EB_REL}[mode]


def _method(m) -> int:
    return {"spatial": SPATIAL, "temporal": TEMPORAL, "auto": AUTO,
            SPATIAL: SPATIAL, TEMPORAL: TEMPORAL, AUTO: AUTO}[m]


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def kernel_launches() -> int:
    """CUDA kernels the library has launched in this process."""
    return int(load().lcp_kernel_launches())


def max_compressed_size(n: int, d: int) -> int:
    return int(load().lcp_max_compressed_size(n, d))


def dict_max_size(raw_bytes: int) -> int:
    """Largest LCPZ image of raw_bytes bytes (every chunk stored)."""
    return int(load().lcp_dict_max_size(raw_bytes))


class Context:
    """Device workspace of one GPU (lcp_ctx)."""

    def __init__(self, device: int = 0):
        load()
        if not torch.cuda.is_available():
            raise RuntimeError("the LCP library needs a CUDA GPU")
        self.device = device
        h = C.c_void_p()
        _check(_lib.lcp_ctx_create(device, C.byref(h)), "lcp_ctx_create")
        self.h = h

    def close(self):
        if self.h:
            _lib.lcp_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def profile(self, enable: bool = True, accumulate: bool = False):
        """Per-kernel CUDA-event timing of subsequent calls; with accumulate,
        every call's stages are kept until profile_read."""
        mode = (2 if accumulate else 1) if enable else 0
        _check(_lib.lcp_ctx_profile(self.h, mode), "lcp_ctx_profile")

    def profile_read(self, cap: int = 32) -> list[tuple[str, float]]:
        """(stage, ms) of the most recent call, or of every call since the
        last read when accumulating."""
        names = C.create_string_buffer(32 * cap)
        ms = (C.c_float * cap)()
        k = _lib.lcp_ctx_profile_read(self.h, names, ms, cap)
        raw = names.raw
        return [(raw[32 * i:32 * i + 32].split(b"\0")[0].decode(), float(ms[i])) for i in range(k)]

    def reserve(self, n: int, d: int):
        _check(_lib.lcp_ctx_reserve(self.h, n, d), "lcp_ctx_reserve")

    def compress(self, X: torch.Tensor, eb: float, mode="abs", p: int = 8, method="spatial",
                 traj: "Trajectory | None" = None, out: torch.Tensor | None = None,
                 perm: bool = False, stream=None) -> dict:
        """Compresses X [d, n] (float32, CUDA, contiguous).  Returns the
        container (a uint8 view of `out`), its size, the method used and,
        when asked, the slot permutation (int32 [n])."""
        assert X.is_cuda and X.dtype == torch.float32 and X.dim() == 2 and X.is_contiguous()
        d, n = X.shape
        if out is None:
            out = torch.empty(max_compressed_size(n, d), dtype=torch.uint8, device=X.device)
        pm = torch.empty(max(n, 1), dtype=torch.int32, device=X.device) if perm else None
        size = C.c_size_t(0)
        chosen = C.c_int(0)
        st = _lib.lcp_compress(self.h, traj.h if traj is not None else None, _ptr(X), n, d,
                               float(eb), _mode(mode), p, _method(method), _ptr(out),
                               out.numel(), C.byref(size), C.byref(chosen), _ptr(pm),
                               _stream(stream))
        if st == ERR_CAPACITY:
            raise LcpError(st, f"lcp_compress (needs {size.value} bytes)")
        _check(st, "lcp_compress")
        return dict(bytes=out[: size.value], size=size.value,
                    method="temporal" if chosen.value == TEMPORAL else "spatial",
                    perm=pm[:n] if perm else None)

    def decompress(self, buf: torch.Tensor, size: int | None = None,
                   traj: "Trajectory | None" = None, out: torch.Tensor | None = None,
                   stream=None) -> torch.Tensor:
        """Decodes a container (uint8 CUDA tensor) into float32 [d, n] in slot
        order."""
        assert buf.is_cuda and buf.dtype == torch.uint8
        size = buf.numel() if size is None else size
        if out is None:
            n, d, _, _ = self.peek(buf, size, stream)
            out = torch.empty((d, n), dtype=torch.float32, device=buf.device)
        assert out.is_cuda and out.dtype == torch.float32 and out.is_contiguous()
        # the output's capacity in values: the call checks d n against it, so
        # no header read is needed here
        nn = C.c_uint64(0)
        dd = C.c_uint32(0)
        st = _lib.lcp_decompress_into(self.h, traj.h if traj is not None else None, _ptr(buf),
                                      size, _ptr(out), out.numel(), C.byref(nn), C.byref(dd),
                                      _stream(stream))
        _check(st, "lcp_decompress")
        n, d = nn.value, dd.value
        return out.view(-1)[: d * n].view(d, n)

    def compress_host(self, X: torch.Tensor, eb: float, mode="abs", p: int = 8,
                      method="spatial", traj: "Trajectory | None" = None,
                      out: torch.Tensor | None = None, stream=None) -> dict:
        """lcp_compress_host: X [d, n] float32 in host memory (pinned for full
        speed), the container into the host uint8 tensor out."""
        assert not X.is_cuda and X.dtype == torch.float32 and X.dim() == 2 and X.is_contiguous()
        d, n = X.shape
        if out is None:
            out = torch.empty(max_compressed_size(n, d), dtype=torch.uint8)
        assert not out.is_cuda and out.dtype == torch.uint8
        size = C.c_size_t(0)
        chosen = C.c_int(0)
        st = _lib.lcp_compress_host(self.h, traj.h if traj is not None else None, X.data_ptr(), n,
                                    d, float(eb), _mode(mode), p, _method(method),
                                    out.data_ptr(), out.numel(), C.byref(size), C.byref(chosen),
                                    _stream(stream))
        _check(st, "lcp_compress_host")
        return dict(bytes=out[: size.value], size=size.value,
                    method="temporal" if chosen.value == TEMPORAL else "spatial")

    def decompress_host(self, buf: torch.Tensor, size: int | None = None,
                        traj: "Trajectory | None" = None, out: torch.Tensor | None = None,
                        stream=None) -> torch.Tensor:
        """lcp_decompress_host: a container in host memory decoded into the
        host float32 tensor out (capacity out.numel() values)."""
        assert not buf.is_cuda and buf.dtype == torch.uint8
        assert out is not None and not out.is_cuda and out.dtype == torch.float32
        assert out.is_contiguous()
        size = buf.numel() if size is None else size
        nn = C.c_uint64(0)
        dd = C.c_uint32(0)
        st = _lib.lcp_decompress_host(self.h, traj.h if traj is not None else None,
                                      buf.data_ptr(), size, out.data_ptr(), out.numel(),
                                      C.byref(nn), C.byref(dd), _stream(stream))
        _check(st, "lcp_decompress_host")
        n, d = nn.value, dd.value
        return out.view(-1)[: d * n].view(d, n)

    def set_schedule(self, log2_chunk: int = 10, bucket_delta: int = 0):
        """lcp_ctx_set_schedule."""
        sc = Schedule(log2_chunk, bucket_delta)
        _check(_lib.lcp_ctx_set_schedule(self.h, C.byref(sc)), "lcp_ctx_set_schedule")

    def schedule(self) -> dict:
        sc = Schedule()
        _check(_lib.lcp_ctx_get_schedule(self.h, C.byref(sc)), "lcp_ctx_get_schedule")
        return dict(log2_chunk=sc.log2_chunk, bucket_delta=sc.bucket_delta)

    def tune(self, X: torch.Tensor, eb: float, mode="abs", p: int = 0, max_growth: float = 0.01,
             reps: int = 2, stream=None) -> dict:
        """lcp_tune_schedule: the fastest schedule for this frame shape (the
        context's own schedule is unchanged)."""
        d, n = X.shape
        sc = Schedule()
        ms = C.c_float(0.0)
        _check(_lib.lcp_tune_schedule(self.h, _ptr(X), n, d, float(eb), _mode(mode), p,
                                      float(max_growth), reps, C.byref(sc), C.byref(ms),
                                      _stream(stream)), "lcp_tune_schedule")
        return dict(log2_chunk=sc.log2_chunk, bucket_delta=sc.bucket_delta, ms=ms.value)

    def decompress_frames(self, containers: list, first: int, last: int | None = None,
                          batch: int | None = None, traj: "Trajectory | None" = None,
                          stream=None) -> list[torch.Tensor]:
        """lcp_decompress_frames: frames first..last (default: first only) of
        one trajectory whose containers (uint8 CUDA tensors, frame i at index
        i; None where absent) are given in stream order.  The decoder state is
        traj, else a fresh trajectory of the stream's batch size `batch`.
        Returns float32 [d, n] frames in slot order."""
        last = first if last is None else last
        n, d, _, _ = self.peek(containers[first], None, stream)
        outs = [torch.empty((d, n), dtype=torch.float32, device=containers[first].device)
                for _ in range(first, last + 1)]
        cnt = len(containers)
        ptrs = (_vp * cnt)(*[_ptr(b) if b is not None else None for b in containers])
        sizes = (_sz * cnt)(*[b.numel() if b is not None else 0 for b in containers])
        op = (_vp * len(outs))(*[_ptr(o) for o in outs])
        dec = traj if traj is not None else Trajectory(self, batch, 8)
        nn = C.c_uint64(0)
        dd = C.c_uint32(0)
        _check(_lib.lcp_decompress_frames(self.h, dec.h, ptrs, sizes, cnt, first, last, op, n,
                                          C.byref(nn), C.byref(dd), _stream(stream)),
               "lcp_decompress_frames")
        return outs

    def decompress_frame(self, containers: list, target: int, batch: int | None = None,
                         traj: "Trajectory | None" = None, stream=None) -> torch.Tensor:
        """lcp_decompress_frame: one frame of a trajectory by random access
        (decoder state as in decompress_frames)."""
        n, d, _, _ = self.peek(containers[target], None, stream)
        out = torch.empty((d, n), dtype=torch.float32, device=containers[target].device)
        cnt = len(containers)
        ptrs = (_vp * cnt)(*[_ptr(b) if b is not None else None for b in containers])
        sizes = (_sz * cnt)(*[b.numel() if b is not None else 0 for b in containers])
        dec = traj if traj is not None else Trajectory(self, batch, 8)
        nn = C.c_uint64(0)
        dd = C.c_uint32(0)
        _check(_lib.lcp_decompress_frame(self.h, dec.h, ptrs, sizes, cnt, target, _ptr(out), n,
                                         C.byref(nn), C.byref(dd), _stream(stream)),
               "lcp_decompress_frame")
        return out

    def set_dict(self, on: bool = True):
        """The dictionary stage after every compression of this context (an
        LCPZ image kept when shorter than the container)."""
        _check(_lib.lcp_ctx_set_dict(self.h, int(bool(on))), "lcp_ctx_set_dict")

    def dict_compress(self, buf: torch.Tensor, size: int | None = None,
                      out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """The LCPZ image of buf[:size] (uint8 CUDA), a uint8 view of out."""
        assert buf.is_cuda and buf.dtype == torch.uint8
        size = buf.numel() if size is None else size
        if out is None:
            out = torch.empty(dict_max_size(size), dtype=torch.uint8, device=buf.device)
        n = C.c_size_t(0)
        _check(_lib.lcp_dict_compress(self.h, _ptr(buf), size, _ptr(out), out.numel(), C.byref(n),
                                      _stream(stream)), "lcp_dict_compress")
        return out[:n.value]

    def dict_decompress(self, img: torch.Tensor, size: int | None = None,
                        out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """The raw bytes of an LCPZ image; without out, the size is read from
        the image's header first."""
        assert img.is_cuda and img.dtype == torch.uint8
        size = img.numel() if size is None else size
        if out is None:
            raw = int.from_bytes(bytes(img[8:16].cpu().numpy()), "little") if size >= 16 else 0
            out = torch.empty(max(raw, 1), dtype=torch.uint8, device=img.device)
        n = C.c_size_t(0)
        _check(_lib.lcp_dict_decompress(self.h, _ptr(img), size, _ptr(out), out.numel(),
                                        C.byref(n), _stream(stream)), "lcp_dict_decompress")
        return out[:n.value]

    def peek(self, buf: torch.Tensor, size: int | None = None, stream=None):
        n = C.c_uint64(0)
        d = C.c_uint32(0)
        m = C.c_int(0)
        fl = C.c_uint32(0)
        size = buf.numel() if size is None else size
        _check(_lib.lcp_peek(_ptr(buf), size, C.byref(n), C.byref(d), C.byref(m), C.byref(fl),
                             _stream(stream)), "lcp_peek")
        return n.value, d.value, ("temporal" if m.value == TEMPORAL else "spatial"), fl.value

    def select(self, traj: "Trajectory", X: torch.Tensor, eb: float, mode="abs", stream=None):
        d, n = X.shape
        ch = C.c_int(0)
        es = C.c_uint64(0)
        et = C.c_uint64(0)
        _check(_lib.lcp_select(self.h, traj.h, _ptr(X), n, d, float(eb), _mode(mode),
                               C.byref(ch), C.byref(es), C.byref(et), _stream(stream)),
               "lcp_select")
        return ("temporal" if ch.value == TEMPORAL else "spatial"), es.value, et.value

    def choose_block_size(self, X: torch.Tensor, eb: float, mode="abs", sample: int = 0,
                          stream=None):
        """lcp_choose_block_size: (best p, {p: sample container size}) over
        p = 2^0 .. 2^16 within the domain."""
        d, n = X.shape
        pb = C.c_uint32(0)
        sizes = (C.c_uint64 * 17)()
        _check(_lib.lcp_choose_block_size(self.h, _ptr(X), n, d, float(eb), _mode(mode), sample,
                                          C.byref(pb), sizes, _stream(stream)),
               "lcp_choose_block_size")
        return pb.value, {1 << k: sizes[k] for k in range(17) if sizes[k]}


class Trajectory:
    """Reference state of one frame sequence (lcp_traj), for compressing or for
    decompressing it."""

    def __init__(self, ctx: Context, batch: int = 10, p: int = 8, anchor_scale: int = 1):
        self.ctx = ctx
        h = C.c_void_p()
        _check(_lib.lcp_traj_create(ctx.h, batch, p, C.byref(h)), "lcp_traj_create")
        self.h = h
        if anchor_scale != 1:
            _check(_lib.lcp_traj_set_anchor_scale(h, anchor_scale), "lcp_traj_set_anchor_scale")

    def export(self, stream=None) -> bytes:
        """lcp_traj_export: the reference state as a host byte image."""
        size = C.c_size_t(0)
        st = _lib.lcp_traj_export(self.h, None, 0, C.byref(size), _stream(stream))
        if st != ERR_CAPACITY:
            _check(st, "lcp_traj_export")
        buf = C.create_string_buffer(max(size.value, 1))
        _check(_lib.lcp_traj_export(self.h, buf, size.value, C.byref(size), _stream(stream)),
               "lcp_traj_export")
        return buf.raw[: size.value]

    @classmethod
    def restore(cls, ctx: Context, image: bytes, stream=None) -> "Trajectory":
        """lcp_traj_import: a trajectory on ctx continuing an exported one."""
        self = cls.__new__(cls)
        self.ctx = ctx
        self.h = None
        h = C.c_void_p()
        _check(_lib.lcp_traj_import(ctx.h, image, len(image), C.byref(h), _stream(stream)),
               "lcp_traj_import")
        self.h = h
        return self

    def close(self):
        if self.h:
            _lib.lcp_traj_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Lanes:
    """Contexts and CUDA streams for the batch calls: lane k runs its jobs on
    its own context and stream, so frames of different lanes overlap."""

    def __init__(self, lanes: int, device: int = 0):
        self.ctxs = [Context(device) for _ in range(lanes)]
        self.streams = [torch.cuda.Stream(device=device) for _ in range(lanes)]
        self._c = (_vp * lanes)(*[c.h.value for c in self.ctxs])
        self._s = (_vp * lanes)(*[st.cuda_stream for st in self.streams])

    def __len__(self):
        return len(self.ctxs)

    def compress(self, jobs: list[dict]) -> list[dict]:
        """jobs: dicts with X [d, n] (CUDA float32), eb, mode, p, method, traj
        (Trajectory or None) and out (uint8 CUDA buffer).  Returns per job the
        container view, its size, the method used and the call's ms."""
        arr = (CompressJob * len(jobs))()
        for j, J in zip(arr, jobs):
            X = J["X"]
            assert X.is_cuda and X.dtype == torch.float32 and X.dim() == 2 and X.is_contiguous()
            j.traj = J["traj"].h.value if J.get("traj") is not None else None
            j.d_fields = X.data_ptr()
            j.d, j.n = X.shape
            j.eb = float(J["eb"])
            j.mode = _mode(J.get("mode", "abs"))
            j.p = int(J.get("p", 8))
            j.method = _method(J.get("method", "spatial"))
            j.d_out = J["out"].data_ptr()
            j.out_cap = J["out"].numel()
        torch.cuda.synchronize()  # inputs written on other streams are complete
        st = _lib.lcp_compress_batch(self._c, self._s, len(self), arr, len(jobs))
        res = []
        for j, J in zip(arr, jobs):
            res.append(dict(bytes=J["out"][: j.out_size], size=int(j.out_size),
                            method="temporal" if j.chosen == TEMPORAL else "spatial",
                            status=int(j.status), ms=float(j.ms)))
        _check(st, "lcp_compress_batch")
        return res

    def decompress(self, jobs: list[dict]) -> list[dict]:
        """jobs: dicts with buf (uint8 CUDA), size, traj (decoder Trajectory or
        None) and out (float32 CUDA [d, n_cap]).  Returns per job n, d and ms."""
        arr = (DecompressJob * len(jobs))()
        for j, J in zip(arr, jobs):
            j.traj = J["traj"].h.value if J.get("traj") is not None else None
            j.d_in = J["buf"].data_ptr()
            j.in_size = int(J["size"])
            j.d_out = J["out"].data_ptr()
            j.n_cap = J["out"].shape[-1]
        torch.cuda.synchronize()
        st = _lib.lcp_decompress_batch(self._c, self._s, len(self), arr, len(jobs))
        res = [dict(n=int(j.n_out), d=int(j.d_fields), status=int(j.status), ms=float(j.ms))
               for j in arr]
        _check(st, "lcp_decompress_batch")
        return res


class Step:
    """lcp_step: one time step of many trajectories' LCP-T frames decoded in
    one persistent launch, replayed as a CUDA graph (see include/lcp.h)."""

    def __init__(self, ctx: Context, max_frames: int = 64, lanes: "Lanes | None" = None):
        """lanes: contexts and streams for the frames the step does not fuse
        (lcp_step_set_lanes); they must not serve other calls meanwhile."""
        self.ctx = ctx
        h = C.c_void_p()
        _check(_lib.lcp_step_create(ctx.h, max_frames, C.byref(h)), "lcp_step_create")
        self.h = h
        self.lanes = lanes
        if lanes is not None:
            _check(_lib.lcp_step_set_lanes(h, lanes._c, lanes._s, len(lanes)),
                   "lcp_step_set_lanes")

    def decompress(self, jobs: list[dict], stream=None) -> list[dict]:
        """jobs: dicts with buf (uint8 CUDA), size, traj (decoder Trajectory)
        and out (float32 CUDA [d, n]).  Returns per job n, d and status."""
        arr = (DecompressJob * len(jobs))()
        for j, J in zip(arr, jobs):
            j.traj = J["traj"].h.value if J.get("traj") is not None else None
            j.d_in = J["buf"].data_ptr()
            j.in_size = int(J["size"])
            j.d_out = J["out"].data_ptr()
            j.n_cap = J["out"].shape[-1]
        st = _lib.lcp_decompress_step(self.h, arr, len(jobs), _stream(stream))
        res = [dict(n=int(j.n_out), d=int(j.d_fields), status=int(j.status)) for j in arr]
        _check(st, "lcp_decompress_step")
        return res

    def close(self):
        if self.h:
            _lib.lcp_step_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """The request loop (lcp_server): producers submit compress / decompress
    requests, lanes run them; see include/lcp.h."""

    def __init__(self, lanes: int = 8, batch: int = 10, hbm_budget: int = 0, device: int = 0):
        load()
        if not torch.cuda.is_available():
            raise RuntimeError("the LCP library needs a CUDA GPU")
        h = C.c_void_p()
        _check(_lib.lcp_server_create(device, lanes, batch, hbm_budget, C.byref(h)),
               "lcp_server_create")
        self.h = h

    def submit_compress(self, producer: int, X: torch.Tensor, eb: float, mode="rel",
                        p: int = 8, out: torch.Tensor | None = None) -> int | None:
        """Queues the producer's next frame; returns a ticket, or None when the
        memory budget does not admit it.  X (and out, a uint8 buffer that
        receives a copy of the container) must stay alive until it is done."""
        assert X.is_cuda and X.dtype == torch.float32 and X.dim() == 2 and X.is_contiguous()
        r = Request(op=REQ_COMPRESS, producer=producer, d_fields=X.data_ptr(), n=X.shape[1],
                    d=X.shape[0], eb=float(eb), mode=_mode(mode), p=p)
        if out is not None:
            r.d_bytes = out.data_ptr()
            r.bytes_cap = out.numel()
        return self._submit(r)

    def submit_decompress(self, producer: int, frame: int, out: torch.Tensor) -> int | None:
        """Queues decoding of the producer's frame `frame` into out [d, n]."""
        assert out.is_cuda and out.dtype == torch.float32 and out.dim() == 2
        r = Request(op=REQ_DECOMPRESS, producer=producer, frame=frame, d_out=out.data_ptr(),
                    n_cap=out.shape[1])
        return self._submit(r)

    def _submit(self, r: Request) -> int | None:
        t = C.c_uint64(0)
        st = _lib.lcp_server_submit(self.h, C.byref(r), C.byref(t))
        if st == ERR_NOMEM:
            return None
        _check(st, "lcp_server_submit")
        return t.value

    def wait(self, ticket: int) -> dict:
        """Blocks until the request is done; returns its response."""
        r = Response()
        _check(_lib.lcp_server_wait(self.h, ticket, C.byref(r)), "lcp_server_wait")
        return dict(status=r.status, frame=r.frame, size=r.size,
                    method="temporal" if r.method == TEMPORAL else "spatial",
                    enqueue_ms=r.enqueue_ms, start_ms=r.start_ms, done_ms=r.done_ms)

    def frames(self, producer: int) -> tuple[int, int]:
        """Decodable frame range [first, next) of a producer."""
        a, b = C.c_uint64(0), C.c_uint64(0)
        _check(_lib.lcp_server_frames(self.h, producer, C.byref(a), C.byref(b)),
               "lcp_server_frames")
        return a.value, b.value

    def device_bytes(self) -> int:
        return int(_lib.lcp_server_device_bytes(self.h))

    def close(self):
        if self.h:
            _lib.lcp_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def quantize(x: torch.Tensor, m: float, e: float, max_abs: float | None = None, stream=None):
    """Element rules on the GPU: (q, x', violation) for values x >= m."""
    assert x.is_cuda and x.dtype == torch.float32 and x.is_contiguous()
    load()
    n = x.numel()
    q = torch.empty(n, dtype=torch.int32, device=x.device)
    xr = torch.empty(n, dtype=torch.float32, device=x.device)
    v = torch.empty(n, dtype=torch.uint8, device=x.device)
    if max_abs is None:
        max_abs = 0.0  # unused by the library (kept in the C signature)
    _check(_lib.lcp_quantize(_ptr(x), n, m, e, max_abs, _ptr(q), _ptr(xr), _ptr(v),
                             _stream(stream)), "lcp_quantize")
    return q, xr, v.bool()


NOALLOC_MAX_ELEMENTS = 16777216


def quantize_noalloc(x: torch.Tensor, m: float, e: float, max_abs: float, q: torch.Tensor,
                     xr: torch.Tensor, viol: torch.Tensor, stream=None) -> int:
    """The element rules without any device allocation (lcp_quantize_noalloc),
    for callers that cannot allocate: writes into the caller's q (int32), xr
    (float32) and viol (uint8) and returns how many values break the bound.
    At most NOALLOC_MAX_ELEMENTS values per call; calls must not overlap on
    the GPU (they share one fixed scratch array)."""
    load()
    nv = C.c_uint64(0)
    _check(_lib.lcp_quantize_noalloc(_ptr(x), x.numel(), m, e, max_abs, _ptr(q), _ptr(xr),
                                     _ptr(viol), C.byref(nv), _stream(stream)),
           "lcp_quantize_noalloc")
    return nv.value
