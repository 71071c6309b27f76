"""Pins of the oracle's dictionary stage (the last step of the encoding
stage, Sec. "Block coding"; LCPZ layout in lcp_oracle.c).

Hand-worked chunks (tests/golden/dict_worked_examples.txt), closed forms of
runs and periodic strings, the stored-chunk rule, the container header, the
decoder's rejection of malformed input and round trips of real containers.
"""
import os
import struct

import numpy as np
import pytest

import oracle
from paper_2411_00761_b300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden", "dict_worked_examples.txt")
CH = 1 << 16


def examples():
    out = []
    for line in open(GOLD):
        if line.startswith("#") or not line.strip():
            continue
        name, text, hexs = (f.strip() for f in line.split("|"))
        out.append((name, text.encode(), bytes.fromhex(hexs.replace(" ", ""))))
    return out


def head(img):
    magic, ver, lc, _, S, C, T = struct.unpack_from("<4sBBHQQQ", img, 0)
    assert magic == b"LCPZ" and ver == 1 and lc == 16
    return S, C, T


def chunks(img):
    """(coded, stored) per chunk, split by the size table."""
    S, C, T = head(img)
    sizes = struct.unpack_from(f"<{C}I", img, 80)
    at = (80 + 4 * C + 15) // 16 * 16
    out = []
    for e in sizes:
        c = e & 0x7FFFFFFF
        out.append((img[at:at + c], bool(e >> 31)))
        at += c
    assert (at + 15) // 16 * 16 == T == len(img)
    return out


def pad16(b):
    return (b + 15) // 16 * 16


@pytest.mark.parametrize("name,raw,coded", examples(), ids=[e[0] for e in examples()])
def test_worked_examples(name, raw, coded):
    img = oracle.dict_compress(raw)
    (c, stored), = chunks(img)
    assert not stored and c == coded, (name, c.hex())
    assert oracle.dict_decompress(img) == raw


def test_worked_example_container():
    # abcabcabcabcX: header 80 bytes, one table entry, pad to 96, 8 coded
    # bytes, pad to 112
    raw = b"abcabcabcabcX"
    img = oracle.dict_compress(raw)
    want = (b"LCPZ" + bytes([1, 16, 0, 0]) + struct.pack("<QQQ", 13, 1, 112) +
            raw + bytes(48 - 13) + struct.pack("<I", 8) + bytes(12) +
            bytes.fromhex("3561626303001058") + bytes(8))
    assert img == want


def zeros_chunk(k):
    """k >= 5 zero bytes: one literal, then a copy of k - 1 from offset 1."""
    v = k - 1 - 4
    tok = 0x10 | min(v, 15)
    ext = b""
    if v >= 15:
        r = v - 15
        ext = b"\xff" * (r // 255) + bytes([r % 255])
    return bytes([tok, 0, 1, 0]) + ext


@pytest.mark.parametrize("k", [5, 18, 19, 20, 274, 275, 276, 529, 530, 1000, CH])
def test_zero_runs_closed_form(k):
    # ext boundaries: copy-4 = 14 (no ext), 15 (ext 00), 269/270 (fe / ff 00),
    # 525 (ff ff 00); a whole chunk is 1f 00 01 00, 256 x ff, ec (261 bytes)
    (c, stored), = chunks(oracle.dict_compress(bytes(k)))
    assert not stored and c == zeros_chunk(k)
    if k == CH:
        assert len(c) == 261 and c[-1] == 0xEC and c[4:260] == b"\xff" * 256


def test_periodic_closed_form():
    raw = b"abcd" * (CH // 4)
    (c, stored), = chunks(oracle.dict_compress(raw))
    assert not stored
    assert c == b"\x4fabcd\x04\x00" + b"\xff" * 256 + b"\xe9"


def test_chunks_are_independent_and_ragged():
    raw = bytes(2 * CH + 100)
    img = oracle.dict_compress(raw)
    S, C, T = head(img)
    assert (S, C) == (len(raw), 3)
    cs = chunks(img)
    # the second chunk cannot copy from the first: it repeats its coding
    assert cs[0] == (zeros_chunk(CH), False) and cs[1] == (zeros_chunk(CH), False)
    assert cs[2] == (zeros_chunk(100), False)
    assert T == pad16(pad16(80 + 12) + 261 + 261 + 5) == 624
    assert oracle.dict_decompress(img) == raw


@pytest.mark.parametrize("raw", [b"", b"a", b"ab", b"abc", b"abcd", bytes(4)])
def test_tiny_inputs_stored(raw):
    img = oracle.dict_compress(raw)
    S, C, T = head(img)
    assert S == len(raw) and C == (1 if raw else 0)
    assert img[32:32 + len(raw)] == raw and img[32 + len(raw):80] == bytes(48 - len(raw))
    if raw:
        (c, stored), = chunks(img)
        assert stored and c == raw  # 1 + m coded bytes are not shorter than m
    else:
        assert T == 80 == len(img)
    assert oracle.dict_decompress(img) == raw


def test_random_bytes_stored_and_bound():
    raw = np.random.default_rng(5).integers(0, 256, 3 * CH + 777, dtype=np.uint8).tobytes()
    img = oracle.dict_compress(raw)
    assert all(st for _, st in chunks(img))
    assert len(img) == oracle.dict_max_size(len(raw))
    assert img[32:80] == raw[:48]
    assert oracle.dict_decompress(img) == raw


def test_round_trip_containers():
    X = synth.cosmology(1 << 16, 2)
    c_s = oracle.compress_s(X, 1.0, "abs", 8)["bytes"]
    X2 = synth.md_fcc(1 << 15, 1, cells=32)
    c_m = oracle.compress_s(X2, 1e-3, "abs", 4)["bytes"]
    for raw in (c_s, c_m):
        img = oracle.dict_compress(raw)
        assert len(img) < len(raw)  # both frames have redundancy left
        assert img[32:80] == raw[:48]  # the container header preview
        back = oracle.dict_decompress(img)
        assert back == raw
        np.testing.assert_array_equal(oracle.decompress(back)[1], oracle.decompress(raw)[1])


def test_mixed_round_trip():
    rng = np.random.default_rng(9)
    parts = []
    for _ in range(40):
        k = int(rng.integers(1, 9000))
        kind = int(rng.integers(0, 3))
        if kind == 0:
            parts.append(rng.integers(0, 256, k, dtype=np.uint8).tobytes())
        elif kind == 1:
            parts.append(bytes([int(rng.integers(0, 256))]) * k)
        else:
            base = rng.integers(0, 4, int(rng.integers(1, 40)), dtype=np.uint8).tobytes()
            parts.append((base * (k // len(base) + 1))[:k])
    raw = b"".join(parts)
    img = oracle.dict_compress(raw)
    assert oracle.dict_decompress(img) == raw
    assert len(img) <= oracle.dict_max_size(len(raw))


def corrupt(img, at, val):
    b = bytearray(img)
    b[at] = val
    return bytes(b)


def test_decoder_rejects_malformed():
    raw = b"abcabcabcabcX"
    img = oracle.dict_compress(raw)
    p0 = 96
    bad = [
        corrupt(img, 3, ord("1")),                 # magic
        corrupt(img, 5, 15),                       # chunk size
        corrupt(img, p0 + 4, 0),                   # copy offset 0
        corrupt(img, p0 + 4, 4),                   # offset beyond the output (3 bytes so far)
        corrupt(img, p0, 0x3F),                    # copy length past the chunk end
        corrupt(img, 80, 9),                       # chunk size beyond its sequences
        corrupt(img, 80, 7),                       # truncated chunk
        corrupt(img, 24, 96),                      # total bytes
        img[:100],                                 # truncated image
    ]
    for b in bad:
        with pytest.raises(oracle.OracleError) as ei:
            oracle.dict_decompress(b)
        assert ei.value.status == oracle.ERR_FORMAT


def py_read(img: bytes) -> bytes:
    """An independent reader of the LCPZ layout, written from its description
    (it shares nothing with the oracle's C decoder): sizes table, stored
    chunks, sequences with their extensions and overlapping copies."""
    S, C, T = head(img)
    sizes = struct.unpack_from(f"<{C}I", img, 80)
    at = pad16(80 + 4 * C)
    out = bytearray()

    def ext(body, q, v):
        while True:
            b = body[q]
            q += 1
            v += b
            if b != 255:
                return q, v

    for k, e in enumerate(sizes):
        c, m = e & 0x7FFFFFFF, min(CH, S - CH * k)
        body = img[at:at + c]
        at += c
        if e >> 31:
            assert c == m
            out += body
            continue
        y, q = bytearray(), 0
        while len(y) < m:
            tok = body[q]
            q += 1
            ll, ml = tok >> 4, tok & 15
            if ll == 15:
                q, ll = ext(body, q, ll)
            y += body[q:q + ll]
            q += ll
            if len(y) == m:
                break
            o = body[q] | (body[q + 1] << 8)
            q += 2
            if ml == 15:
                q, ml = ext(body, q, ml)
            for _ in range(ml + 4):
                y.append(y[-o])
        assert q == c and len(y) == m
        out += y
    assert pad16(at) == T
    return bytes(out)


def test_independent_reader():
    rng = np.random.default_rng(12)
    X = synth.cosmology(1 << 14, 2)
    inputs = [b"", b"abc", bytes(2 * CH + 100), b"abcd" * 5000, mixed_bytes(rng),
              rng.integers(0, 256, CH + 5, dtype=np.uint8).tobytes(),
              oracle.compress_s(X, 1.0, "abs", 8)["bytes"]]
    for g in examples():
        inputs.append(g[1])
    for raw in inputs:
        assert py_read(oracle.dict_compress(raw)) == raw


def mixed_bytes(rng, parts=30):
    out = []
    for _ in range(parts):
        k = int(rng.integers(1, 5000))
        kind = int(rng.integers(0, 3))
        if kind == 0:
            out.append(rng.integers(0, 256, k, dtype=np.uint8).tobytes())
        elif kind == 1:
            out.append(bytes([int(rng.integers(0, 256))]) * k)
        else:
            base = rng.integers(0, 5, int(rng.integers(1, 30)), dtype=np.uint8).tobytes()
            out.append((base * (k // len(base) + 1))[:k])
    return b"".join(out)
