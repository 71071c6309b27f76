"""Independent pure-Python reading of the LCP1 container and of the LCP-S
stream construction, written from the format description (tests only).

Slow (bit by bit); use on small frames.  Shares no code with the oracle or
the CUDA library.
"""
from __future__ import annotations

import struct

import numpy as np

from tests import exact_ref as X

ESC = 4095
LMAX = 24


def pad16(b: int) -> int:
    return (b + 15) // 16 * 16


def bits_of(v: int) -> int:
    return int(v).bit_length()


class BitReader:
    def __init__(self, buf: bytes, off: int):
        self.buf = buf
        self.off = off

    def bit(self, b: int) -> int:
        word = struct.unpack_from("<I", self.buf, self.off + 4 * (b // 32))[0]
        return (word >> (31 - b % 32)) & 1

    def read(self, pos: int, n: int) -> tuple[int, int]:
        v = 0
        for i in range(n):
            v = (v << 1) | self.bit(pos + i)
        return v, pos + n


def parse_stream(buf: bytes, off: int, size: int, log2_chunk: int) -> dict:
    coder, width, U = struct.unpack_from("<BBH", buf, off)
    n, pbits, maxv = struct.unpack_from("<QQQ", buf, off + 8)
    out = dict(coder=coder, width=width, U=U, n=n, payload_bits=pbits, maxv=maxv)
    vals = []
    if coder == 0:
        assert size == 32 + pad16(4 * ((pbits + 31) // 32))
        br = BitReader(buf, off + 32)
        pos = 0
        for _ in range(n):
            v, pos = br.read(pos, width)
            vals.append(v)
    else:
        counts = struct.unpack_from("<24H", buf, off + 32)
        syms = struct.unpack_from(f"<{U}H", buf, off + 80)
        # rebuild canonical codes from (length, symbol) order
        table = {}
        code, k, prev = 0, 0, 0
        lens = {}
        for L in range(1, LMAX + 1):
            for _ in range(counts[L - 1]):
                if k > 0:
                    code = (code + 1) << (L - prev)
                table[(L, code)] = syms[k]
                lens[syms[k]] = L
                prev = L
                k += 1
        assert k == U
        n_chunks = (n + (1 << log2_chunk) - 1) >> log2_chunk
        ct = off + pad16(80 + 2 * U)
        pl = ct + pad16(8 * n_chunks)
        assert size == pad16(80 + 2 * U) + pad16(8 * n_chunks) + pad16(4 * ((pbits + 31) // 32))
        chunk_offsets = list(struct.unpack_from(f"<{n_chunks}Q", buf, ct)) if n_chunks else []
        br = BitReader(buf, pl)
        pos = 0
        for i in range(n):
            if i % (1 << log2_chunk) == 0:
                assert chunk_offsets[i >> log2_chunk] == pos
            c, L = 0, 0
            while True:
                b, pos = br.read(pos, 1)
                c = (c << 1) | b
                L += 1
                if (L, c) in table:
                    s = table[(L, c)]
                    break
                assert L < LMAX
            if s == ESC:
                s, pos = br.read(pos, width)
            vals.append(s)
        assert pos == pbits
        out["lengths"] = lens
    out["values"] = vals
    return out


def parse(buf: bytes) -> dict:
    assert buf[:4] == b"LCP1" and buf[4] == 1
    method, d, log2_chunk = buf[5], buf[6], buf[7]
    flags, p = struct.unpack_from("<II", buf, 8)
    n, k, m, total = struct.unpack_from("<QQQQ", buf, 16)
    assert total == len(buf)
    fields = []
    for f in range(d):
        mn, e = struct.unpack_from("<ff", buf, 48 + 16 * f)
        qmax, z = struct.unpack_from("<II", buf, 48 + 16 * f + 8)
        assert z == 0
        fields.append(dict(min=np.float32(mn), e=np.float32(e), qmax=qmax))
    ns = 3 if method == 0 else 1
    sd = 48 + 16 * d
    secs = [struct.unpack_from("<QQ", buf, sd + 16 * s) for s in range(ns + 1)]
    assert secs[0][0] == 48 + 16 * d + 16 * ns + 16
    for s in range(ns):
        assert secs[s][0] + secs[s][1] == secs[s + 1][0]
    streams = [parse_stream(buf, o, b, log2_chunk) for (o, b) in secs[:ns]]
    res = dict(method=method, d=d, log2_chunk=log2_chunk, flags=flags, p=p, n=n, K=k, M=m,
               total=total, fields=fields, streams=streams)
    oo, ob = secs[ns]
    if method == 0:
        assert ob == pad16(4 * d * k)
        raw = np.frombuffer(buf, dtype=np.float32, count=d * k, offset=oo).reshape(d, k)
        res["outliers"] = raw.copy()
    else:
        assert ob == pad16(8 * k) + pad16(4 * k)
        res["patch_index"] = np.frombuffer(buf, dtype=np.uint64, count=k, offset=oo).copy()
        res["patch_raw"] = np.frombuffer(buf, dtype=np.float32, count=k,
                                         offset=oo + pad16(8 * k)).copy()
    return res


def zigzag(v: int) -> int:
    return 2 * v if v >= 0 else -2 * v - 1


def streams_s_bruteforce(Xf: np.ndarray, e_list, p: int, log2_chunk: int = 10):
    """LCP-S streams of a tiny frame from the paper's equations with exact
    rationals: returns (ids, cnts, rels, outlier indices, slot order)."""
    d, n = Xf.shape
    lp = p.bit_length() - 1
    mins = [min(Xf[f], key=X.total_order_key) for f in range(d)]
    maxs = [max(Xf[f], key=X.total_order_key) for f in range(d)]
    qmax = [X.q1(maxs[f], mins[f], e_list[f]) for f in range(d)]
    bn = [qm // p + 1 for qm in qmax]
    keyed, outl = [], []
    for i in range(n):
        qs = [X.q1(Xf[f][i], mins[f], e_list[f]) for f in range(d)]
        bad = any(X.q3(Xf[f][i], X.q2(qs[f], mins[f], e_list[f]), e_list[f]) for f in range(d))
        if bad:
            outl.append(i)
            continue
        bid, stride, rel = 0, 1, 0
        for f in range(d):
            bid += (qs[f] // p) * stride
            stride *= bn[f]
            rel += (qs[f] % p) * p ** f
        keyed.append((bid * p ** d + rel, i))
    keyed.sort()
    ids, cnts, rels = [], [], []
    prev_b, prev_c, cur = 0, 0, 0
    for k, (key, i) in enumerate(keyed):
        b, r = divmod(key, p ** d)
        start = k == 0 or b != keyed[k - 1][0] // p ** d
        if start:
            if k > 0:
                cnts.append(zigzag(cur - prev_c))
                prev_c = cur
            ids.append(b - prev_b)
            prev_b = b
            cur = 0
        cur += 1
        if start or k % (1 << log2_chunk) == 0:
            rels.append(r)
        else:
            rels.append(r - keyed[k - 1][0] % p ** d)
    if keyed:
        cnts.append(zigzag(cur - prev_c))
    slots = [i for _, i in keyed] + outl
    return ids, cnts, rels, outl, slots


def coder_sizes(values, log2_chunk: int, lengths) -> tuple[int, int]:
    """(fixed bytes, huffman bytes) of a stream given Huffman lengths per
    symbol (a dict); recomputed from the container rules."""
    n = len(values)
    maxv = max(values) if values else 0
    w = bits_of(maxv)
    fixed = 32 + pad16(4 * ((n * w + 31) // 32))
    if n == 0:
        return fixed, None
    any_esc = any(v >= ESC for v in values)
    wesc = bits_of(maxv) if any_esc else 0
    bits = sum(lengths[min(v, ESC)] + (wesc if v >= ESC else 0) for v in values)
    U = len(lengths)
    chunks = (n + (1 << log2_chunk) - 1) >> log2_chunk
    huff = pad16(80 + 2 * U) + pad16(8 * chunks) + pad16(4 * ((bits + 31) // 32))
    return fixed, huff
