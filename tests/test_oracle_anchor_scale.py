"""Anchor error-bound scaling in the oracle's Algorithm 1 (Sec. "Best
error-bound scale for anchor frames").

Re-quantization of reference codes across grids is checked against its
closed form on exactly representable grids and against the identity on an
unchanged grid; the scaled trajectory must decode with every frame inside its
own bound (eb, or eb / scale for a scaled anchor), and anchor_scale = 1 must
leave Algorithm 1 unchanged.
"""
import numpy as np
import pytest

import oracle
from oracle import hybrid
from paper_2411_00761_b300 import synth


def test_requantize_is_the_identity_on_the_same_grid():
    grid = [(-3.25, 0.0625, 4000), (0.0, 0.5, 77)]
    q = np.array([np.arange(0, 4001), np.arange(0, 4001) % 78])
    out = hybrid.requantize(q, grid, grid)
    assert np.array_equal(out, q)


def test_requantize_closed_form_on_a_finer_reference_grid():
    # reference bins of 2 * 0.125, frame bins of 2 * 0.625: centre (2q+1) / 8,
    # frame code floor(((2q+1) / 8) / 1.25) = floor((2q+1) / 10), clamped
    q = np.arange(0, 5000).reshape(1, -1)
    out = hybrid.requantize(q, [(0.0, 0.125, 4999)], [(0.0, 0.625, 300)])
    assert np.array_equal(out[0], np.minimum((2 * q[0] + 1) // 10, 300))
    # a frame grid starting above the reference centres clamps them to 0
    out = hybrid.requantize(q, [(0.0, 0.125, 4999)], [(10.0, 0.625, 300)])
    centre = (2 * q[0] + 1) / 8.0
    assert np.array_equal(out[0], np.clip(np.floor((centre - 10.0) / 1.25), 0, 300))


def frames16(sigma):
    return list(synth.brownian_trajectory(20011, 16, 3, sigma=sigma))


def test_scale_one_leaves_algorithm_1_unchanged():
    fr = frames16(0.02)
    assert hybrid.encode_trajectory(fr, 1e-3, "abs", 8, batch=4, anchor_scale=1) == \
        hybrid.encode_trajectory(fr, 1e-3, "abs", 8, batch=4)


@pytest.mark.parametrize("scale", [2, 5])
def test_scaled_anchors_decode_within_their_bounds(scale):
    eb = 1e-3
    fr = frames16(0.02)
    enc = hybrid.encode_trajectory(fr, eb, "abs", 8, batch=4, anchor_scale=scale)
    dec = hybrid.decode_trajectory([b for b, _ in enc])
    n_requant = n_scaled = 0
    for (buf, meth), X, Y in zip(enc, fr, dec):
        h = oracle.peek(buf)
        e = max(g[1] for g in hybrid.grid_of_container(buf))
        scaled = meth == "S" and e <= eb / scale
        n_scaled += scaled
        n_requant += bool(h["flags"] & hybrid.FLAG_REF_REQUANT)
        bound = eb / scale if scaled else eb
        # the decoded frame is in slot order: compare sorted values per field
        # (sorting keeps a per-element bound)
        for f in range(X.shape[0]):
            d = np.abs(np.sort(Y[f].astype(np.float64)) - np.sort(X[f].astype(np.float64)))
            assert d.max() <= bound, (meth, f, d.max(), bound)
    assert n_scaled >= 1 and n_requant >= 1
