"""Pins of the oracle's LCP-T frames, the LCP-FSM reading and Algorithm 1.

* a static frame predicted from itself has only zero differences (closed
  form: every symbol 0, the stream collapses to a zero-width fixed code);
* a frame shifted by a whole number of bins in every particle (and so in its
  minimum) keeps every code, again all-zero differences;
* the round trip holds the bound on every particle through the slot map;
* the FSM follows its stated transitions on scripted sizes;
* Algorithm 1's anchor rule and the recursive decoding reproduce each frame
  within the bound.
"""
import numpy as np
import pytest

from oracle import hybrid
from paper_2411_00761_b300 import synth
from tests import container_py as CP


def test_static_frame_zero_differences(orc):
    Xf = synth.uniform_clusters(4000, 5)
    s = orc.compress_s(Xf, 1e-3, "abs", 8)
    t = orc.compress_t(Xf, 1e-3, "abs", s["q"], s["pi"])
    assert (t["syms"] == 0).all() and t["K"] == s["K"] * 0 + t["K"]
    h = CP.parse(t["bytes"])
    assert h["streams"][0]["coder"] == 0 and h["streams"][0]["width"] == 0
    Y, q = orc.decompress(t["bytes"], s["q"])
    assert np.array_equal(q, s["q"])


def test_whole_bin_shift_keeps_codes(orc):
    e = 0.125  # 2e = 0.25, exact; values on a coarse grid so shifts are exact
    rng = np.random.default_rng(2)
    Xf = (rng.integers(0, 4000, size=(3, 3000)) * 0.0625).astype(np.float32)
    s = orc.compress_s(Xf, e, "abs", 4)
    Xs = (Xf + np.float32(0.25 * 7)).astype(np.float32)
    t = orc.compress_t(Xs, e, "abs", s["q"], s["pi"])
    assert (t["syms"] == 0).all()


@pytest.mark.parametrize("d,mode", [(3, "abs"), (6, "rel")])
def test_temporal_roundtrip_bound(orc, d, mode):
    if d == 3:
        frames = list(synth.brownian_trajectory(6000, 3, 11))
    else:
        base = synth.cosmology(6000, 3)
        rng = np.random.default_rng(4)
        frames = [base, (base + rng.normal(0, 0.5, base.shape)).astype(np.float32)]
    s = orc.compress_s(frames[0], 1e-3, mode, 8)
    ref_q, pi = s["q"], s["pi"]
    for Xf in frames[1:]:
        t = orc.compress_t(Xf, 1e-3, mode, ref_q, pi)
        Y, q = orc.decompress(t["bytes"], ref_q)
        assert np.array_equal(q, t["q"])
        h = CP.parse(t["bytes"])
        assert len(h["patch_index"]) == t["K"]
        for f in range(d):
            err = np.abs(Xf[f, pi].astype(np.float64) - Y[f].astype(np.float64))
            assert err.max() <= float(h["fields"][f]["e"])
        ref_q = q
    # the independent reader agrees on the difference stream
    assert h["streams"][0]["values"] == [int(v) for v in t["syms"]]


def test_temporal_state_errors(orc):
    Xf = synth.uniform_clusters(100, 1)
    s = orc.compress_s(Xf, 1e-3, "abs", 8)
    with pytest.raises(orc.OracleError) as ei:
        orc.compress_t(Xf[:, :50], 1e-3, "abs", s["q"], s["pi"])
    assert ei.value.status == orc.ERR_STATE
    with pytest.raises(orc.OracleError) as ei:
        orc.decompress(orc.compress_t(Xf, 1e-3, "abs", s["q"], s["pi"])["bytes"], None)
    assert ei.value.status == orc.ERR_STATE


def test_fsm_transitions_scripted():
    f = hybrid.Fsm()
    assert f.plan(False) == "spatial"
    f.after_spatial(100)
    # S2: one frame coded spatially, the second tests LCP-T
    assert f.plan(True) == "spatial"
    assert f.plan(True) == "test"
    f.after_test(False, 100)        # S wins -> S4 (the paper's S2X -> S4X)
    assert f.state == 4
    assert [f.plan(True) for _ in range(4)] == ["spatial"] * 3 + ["test"]
    f.after_test(False, 90)
    assert f.state == 8 and f.s_est == 90
    for _ in range(7):
        assert f.plan(True) == "spatial"
    assert f.plan(True) == "test"
    f.after_test(False, 90)
    assert f.state == 16
    for _ in range(15):
        f.plan(True)
    assert f.plan(True) == "test"
    f.after_test(False, 90)
    assert f.state == 16             # capped
    for _ in range(15):
        f.plan(True)
    assert f.plan(True) == "test"
    f.after_test(True, None)         # T wins -> T, tests every frame
    assert f.state == "T" and f.plan(True) == "test"
    f.after_test(False, 95)          # T loses -> S2
    assert f.state == 2 and f.s_est == 95


def test_algorithm1_anchors_and_decoding(orc):
    n, nf, batch = 3000, 23, 5
    frames = list(synth.brownian_trajectory(n, nf, 21, sigma=0.02))
    enc = hybrid.encode_trajectory(frames, 1e-3, "abs", 8, batch=batch)
    heads = [orc.peek(b) for b, _ in enc]
    for t, (h, (_, m)) in enumerate(zip(heads, enc)):
        assert (h["method"] == 0) == (m == "S")
        assert bool(h["flags"] & hybrid.FLAG_FIRST_IN_BATCH) == (t % batch == 0)
        if m == "T":
            assert bool(h["flags"] & hybrid.FLAG_REF_ANCHOR) == (t % batch == 0)
    assert enc[0][1] == "S"
    assert any(m == "T" for _, m in enc)
    dec = hybrid.decode_trajectory([b for b, _ in enc])
    # slot maps: each S frame carries its own; T frames inherit their reference's
    pi_prev = pi_anchor = None
    for t, ((b, m), Xf, Y) in enumerate(zip(enc, frames, dec)):
        first = t % batch == 0
        if m == "S":
            pi = orc.compress_s(Xf, 1e-3, "abs", 8)["pi"]
            if first:
                pi_anchor = pi
        else:
            pi = pi_anchor if first else pi_prev
        pi_prev = pi
        err = np.abs(Xf[:, pi].astype(np.float64) - Y.astype(np.float64))
        assert err.max() <= float(np.float32(1e-3))


def test_block_size_choice_is_argmin(orc):
    Xf = synth.md_fcc(8000, 1, cells=13)
    best, sizes = hybrid.choose_block_size(Xf, 1e-4, "rel")
    assert sizes[best] == min(sizes.values())
    assert best == min(p for p in sizes if sizes[p] == sizes[best])
