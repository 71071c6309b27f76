"""Pins of the oracle's LCP-S / LCP-T frames.

* the hand-worked frame in tests/golden/lcp_s_worked_example.txt;
* brute force on tiny frames: the streams rebuilt from the paper's equations
  with exact rationals (tests/container_py.py) equal the oracle's;
* an independent pure-Python reading of every container agrees with the
  oracle's own decoder;
* structural invariants (counts >= 1, block-id deltas >= 1 after the first,
  counts sum to N - K), the error bound on every particle, the coder choice
  being the smaller of the two, and the degenerate cases.
"""
import os

import numpy as np
import pytest

from paper_2411_00761_b300 import synth
from tests import container_py as CP
from tests import exact_ref as X

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "lcp_s_worked_example.txt")


def _golden():
    g = {}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        k, *v = line.split()
        g[k] = v
    return g


def check_bound(Xf, res, Y):
    """every decoded value within eb of its original particle (Eq. abs)"""
    pi = res["pi"]
    hdr = CP.parse(res["bytes"])
    for f in range(Xf.shape[0]):
        e = np.float64(hdr["fields"][f]["e"])
        err = np.abs(Xf[f, pi].astype(np.float64) - Y[f].astype(np.float64))
        assert err.max(initial=0.0) <= e


def test_golden_worked_example(orc):
    g = _golden()
    Xf = np.array([[float(v) for v in g[a]] for a in ("x", "y", "z")], np.float32)
    r = orc.compress_s(Xf, float(g["eb"][0]), "abs", int(g["p"][0]), streams=True)
    assert list(r["pi"]) == [int(v) for v in g["slots"]]
    assert list(r["ids"]) == [int(v) for v in g["ids"]]
    assert list(r["cnts"]) == [int(v) for v in g["cnts"]]
    assert list(r["rels"]) == [int(v) for v in g["rels"]]
    assert r["M"] == int(g["M"][0]) and r["K"] == int(g["K"][0])
    assert len(r["bytes"]) == int(g["total_bytes"][0])
    h = CP.parse(r["bytes"])
    for s, w, word in zip(h["streams"], g["widths"], g["first_words"]):
        assert s["coder"] == 0 and s["width"] == int(w)
    import struct
    offs = [48 + 16 * 3 + 16 * s for s in range(3)]
    for s, word in enumerate(g["first_words"]):
        sec = struct.unpack_from("<Q", r["bytes"], offs[s])[0]
        assert struct.unpack_from("<I", r["bytes"], sec + 32)[0] == int(word, 16)
    for a, name in enumerate(("q_x", "q_y", "q_z")):
        assert list(r["q"][a]) == [int(v) for v in np.array(g[name], int)[r["pi"]]]
    Y, q = orc.decompress(r["bytes"])
    for a, name in enumerate(("decoded_x", "decoded_y", "decoded_z")):
        assert list(Y[a]) == [float(v) for v in g[name]]


@pytest.mark.parametrize("seed", range(8))
def test_bruteforce_tiny_frames(orc, seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(1, 48))
    d = int(rng.integers(1, 5))
    p = int(2 ** rng.integers(0, 4))
    Xf = (rng.normal(size=(d, n)) * rng.choice([0.01, 1.0, 100.0])).astype(np.float32)
    if seed % 3 == 0:  # many duplicate and near-edge values
        Xf = np.round(Xf, 1).astype(np.float32)
    eb = float(rng.choice([1e-3, 0.05, 0.3]))
    log2_chunk = 5
    e_list = [X.round_down_f32(eb)] * d
    blocks = 1
    for f in range(d):
        mn = min(Xf[f], key=X.total_order_key)
        mx = max(Xf[f], key=X.total_order_key)
        blocks *= X.q1(mx, mn, e_list[f]) // p + 1
    if blocks * p ** d > 2 ** 63:  # key space rule: the frame is refused
        with pytest.raises(orc.OracleError) as ei:
            orc.compress_s(Xf, eb, "abs", p, log2_chunk)
        assert ei.value.status == orc.ERR_RANGE
        return
    r = orc.compress_s(Xf, eb, "abs", p, log2_chunk, streams=True)
    ids, cnts, rels, outl, slots = CP.streams_s_bruteforce(Xf, e_list, p, log2_chunk)
    assert list(r["ids"]) == ids and list(r["cnts"]) == cnts and list(r["rels"]) == rels
    assert r["K"] == len(outl) and list(r["pi"]) == slots
    h = CP.parse(r["bytes"])
    assert [s["values"] for s in h["streams"]] == [ids, cnts, rels]
    Y, q = orc.decompress(r["bytes"])
    check_bound(Xf, r, Y)


@pytest.mark.parametrize("seed", range(4))
def test_bruteforce_far_from_zero(orc, seed):
    """Eq. quantization holds for every real value: frames whose values sit
    2^33 bins or more away from zero (bounds far below the f32 spacing of the
    data, and negative offsets) are coded, and their streams equal the exact
    rational restatement."""
    rng = np.random.default_rng(300 + seed)
    n = int(rng.integers(2, 40))
    d = int(rng.integers(1, 4))
    p = int(2 ** rng.integers(0, 3))
    off = float(rng.choice([1.0e6, -3.0e7, 2.0e5]))
    eb = float(rng.choice([1e-5, 3e-6]))
    Xf = (off + rng.normal(size=(d, n)) * 0.5).astype(np.float32)
    e_list = [X.round_down_f32(eb)] * d
    assert max(abs(float(v)) for v in Xf.ravel()) >= 2 ** 32 * 2 * e_list[0]
    r = orc.compress_s(Xf, eb, "abs", p, 5, streams=True)
    ids, cnts, rels, outl, slots = CP.streams_s_bruteforce(Xf, e_list, p, 5)
    assert list(r["ids"]) == ids and list(r["cnts"]) == cnts and list(r["rels"]) == rels
    assert r["K"] == len(outl) and list(r["pi"]) == slots
    Y, q = orc.decompress(r["bytes"])
    check_bound(Xf, r, Y)
    # the bins are finer than the data's spacing: every value decodes exactly
    pi = r["pi"]
    assert np.array_equal(Y.view(np.uint32), Xf[:, pi].view(np.uint32))


def _frames():
    yield "uniform_clusters", synth.uniform_clusters(20000, 0), 1e-3, "abs", 8
    yield "md_fcc", synth.md_fcc(20000, 1, cells=20), 1e-4, "rel", 16
    yield "cosmology6", synth.cosmology(20000, 2), 1e-3, "rel", 4
    yield "cosmology6_p2", synth.cosmology(5000, 9), 1e-2, "rel", 2


@pytest.mark.parametrize("name,Xf,eb,mode,p", list(_frames()))
def test_roundtrip_invariants(orc, name, Xf, eb, mode, p):
    r = orc.compress_s(Xf, eb, mode, p, streams=True)
    d, n = Xf.shape
    ids, cnts, rels = r["ids"], r["cnts"], r["rels"]
    assert (ids[1:] >= 1).all()
    c = np.cumsum([(v >> 1) if v % 2 == 0 else -(v >> 1) - 1 for v in cnts.astype(np.int64)])
    assert (c >= 1).all() and c.sum() == n - r["K"]
    assert len(rels) == n - r["K"]
    assert sorted(r["pi"]) == list(range(n))
    Y, q = orc.decompress(r["bytes"])
    check_bound(Xf, r, Y)
    # decoded block particles sit at their bin centres
    h = CP.parse(r["bytes"])
    nb = n - r["K"]
    for f in range(d):
        fl = h["fields"][f]
        centres = orc.q2(q[f, :nb], float(fl["min"]), float(fl["e"]))
        assert np.array_equal(centres.view(np.uint32), Y[f, :nb].view(np.uint32))
    # the independent reader sees the same streams
    if n <= 5000:
        assert [s["values"] for s in h["streams"]] == [list(ids), list(cnts), list(rels)]
    # coder choice: never the larger of the two
    for s, vals in zip(h["streams"], (ids, cnts, rels)):
        if s["coder"] == 1:
            fixed, huff = CP.coder_sizes([int(v) for v in vals], h["log2_chunk"], s["lengths"])
            assert huff < fixed


def test_coder_choice_against_recomputed_costs(orc):
    """Both sizes recomputed from the oracle's Huffman lengths: the stream
    written is the smaller one, ties to fixed-length."""
    rng = np.random.default_rng(11)
    Xf = synth.uniform_clusters(30000, 4)
    r = orc.compress_s(Xf, 2e-3, "abs", 8, streams=True)
    h = CP.parse(r["bytes"])
    for s, vals in zip(h["streams"], (r["ids"], r["cnts"], r["rels"])):
        vals = [int(v) for v in vals]
        hist = np.zeros(4096, np.uint64)
        for v in vals:
            hist[min(v, 4095)] += 1
        ln = orc.huffman_lengths(hist)
        lengths = {k: int(ln[k]) for k in range(4096) if ln[k]}
        fixed, huff = CP.coder_sizes(vals, h["log2_chunk"], lengths)
        chosen = 1 if (huff is not None and huff < fixed) else 0
        assert s["coder"] == chosen
    del rng


def test_degenerate_frames(orc):
    # all particles identical: one block, one count, all relative deltas 0
    Xf = np.full((3, 3000), 0.37, np.float32)
    r = orc.compress_s(Xf, 1e-3, "abs", 8, streams=True)
    assert r["M"] == 1 and r["K"] == 0 and (r["rels"] == 0).all()
    assert len(r["bytes"]) < 400
    Y, _ = orc.decompress(r["bytes"])
    check_bound(Xf, r, Y)
    # one particle per block
    Xf = (np.arange(3 * 200, dtype=np.float32).reshape(3, 200) * 10.0).astype(np.float32)
    r = orc.compress_s(Xf, 0.5, "abs", 2, streams=True)
    assert r["M"] == 200
    # field with max == min (REL bound falls back to eb itself)
    Xf = np.stack([np.linspace(0, 1, 500, dtype=np.float32), np.full(500, 5.0, np.float32)])
    r = orc.compress_s(Xf, 1e-3, "rel", 4)
    Y, _ = orc.decompress(r["bytes"])
    check_bound(Xf, r, Y)
    # bound far below the f32 spacing: every centre rounds back to the value
    Xf = (1000.0 + np.random.default_rng(1).random((3, 400))).astype(np.float32)
    r = orc.compress_s(Xf, 1e-6, "abs", 4)
    Y, _ = orc.decompress(r["bytes"])
    assert r["K"] == 0 and np.array_equal(Y, Xf[:, r["pi"]])
    # bound comparable to the f32 spacing: the rounding of some centres misses
    # the bound and those particles are kept raw (outliers)
    r = orc.compress_s(Xf, 4e-5, "abs", 4)
    assert r["K"] > 0
    Y, _ = orc.decompress(r["bytes"])
    check_bound(Xf, r, Y)
    # empty and single-particle frames
    for n in (0, 1):
        Xf = np.ones((3, n), np.float32)
        r = orc.compress_s(Xf, 1e-3)
        Y, _ = orc.decompress(r["bytes"])
        assert Y.shape == (3, n)
    # D = 1 and D = 8
    for d in (1, 8):
        Xf = np.random.default_rng(d).random((d, 2000)).astype(np.float32)
        r = orc.compress_s(Xf, 0.05, "abs", 2)
        Y, _ = orc.decompress(r["bytes"])
        check_bound(Xf, r, Y)


def test_decoded_multiset_is_bin_centres(orc):
    """Without a stored permutation the decoded frame is the multiset of the
    particles' bin centres (plus raw outliers)."""
    Xf = synth.uniform_clusters(5000, 3)
    r = orc.compress_s(Xf, 1e-3, "abs", 8)
    Y, _ = orc.decompress(r["bytes"])
    h = CP.parse(r["bytes"])
    exp = []
    for f in range(3):
        fl = h["fields"][f]
        q = orc.q1(Xf[f], float(fl["min"]), float(fl["e"]))
        exp.append(orc.q2(q, float(fl["min"]), float(fl["e"])))
    exp = np.stack(exp)
    nb = 5000 - r["K"]
    a = sorted(map(tuple, Y[:, :nb].T.tolist()))
    pi = r["pi"][:nb]
    b = sorted(map(tuple, exp[:, pi].T.tolist()))
    assert a == b
