"""Pins of the oracle's element rules against exact rationals.

Q1 (Eq. quantization), Q2 (its reverse, rounded once to f32) and Q3 (the
absolute bound of Eq. abs) are compared with Fraction restatements on random
values, on values placed at and next to bin edges, and on special cases.
"""
import numpy as np
import pytest

from tests import exact_ref as X


def _edge_values(m, e, ks, rng):
    """f32 values at and around the exact bin edges m + k*2e."""
    out = []
    for k in ks:
        edge = X.F(m) + k * 2 * X.F(e)
        r = X.rn32(edge)
        for v in (r, np.nextafter(r, np.float32(np.inf), dtype=np.float32),
                  np.nextafter(r, np.float32(-np.inf), dtype=np.float32)):
            if X.F(v) >= X.F(m):
                out.append(np.float32(v))
    return np.array(out, dtype=np.float32)


CASES = [
    # (min, eb, value scale)
    (0.0, 1e-3, 1.0),
    (-0.5, 3.7e-4, 1.0),
    (1000.0, 0.25, 50.0),
    (-2000.0, 3.6, 4000.0),
    (1.0e-6, 1e-3, 1.0),
    (-1.0, 0.1, 2.0),
    (0.0, 1e-7, 1e-3),       # bound near the f32 ulp of the values
    (123.456, 1e-5, 0.01),   # bound below the ulp: many outliers
]


@pytest.mark.parametrize("m,eb,scale", CASES)
def test_q1_q2_q3_random_and_edges(orc, m, eb, scale):
    rng = np.random.default_rng(abs(hash((m, eb))) % 2 ** 32)
    m = np.float32(m)
    e = X.round_down_f32(eb)
    vals = (m + rng.random(300) * scale).astype(np.float32)
    vals = vals[vals >= m]
    qmax = X.q1(vals.max(), m, e)
    ks = rng.integers(0, max(qmax, 1) + 1, size=60)
    vals = np.concatenate([vals, _edge_values(m, e, ks, rng), np.array([m], np.float32)])
    q = orc.q1(vals, float(m), float(e))
    qr = [X.q1(v, m, e) for v in vals]
    assert list(q) == qr
    xr = orc.q2(q, float(m), float(e))
    xr_ref = np.array([X.q2(int(k), m, e) for k in q], dtype=np.float32)
    assert np.array_equal(xr.view(np.uint32), xr_ref.view(np.uint32))
    v = orc.q3(vals, xr, float(e))
    v_ref = [X.q3(a, b, e) for a, b in zip(vals, xr)]
    assert list(v) == v_ref
    # where the guard passes the bound holds exactly
    for a, b, bad in zip(vals, xr, v):
        if not bad:
            assert abs(X.F(a) - X.F(b)) <= X.F(e)


def test_edges_are_half_open(orc):
    """q changes exactly at m + k*2e: the edge belongs to the upper bin."""
    m, e = np.float32(0.0), np.float32(0.25)  # 2e = 0.5, edges exact in f32
    vals = np.array([0.0, 0.49999997, 0.5, 0.99999994, 1.0, 1.5], np.float32)
    assert list(orc.q1(vals, 0.0, 0.25)) == [0, 0, 1, 1, 2, 3]
    # centres (2q+1) e + m
    assert list(orc.q2(np.array([0, 1, 2, 3]), 0.0, 0.25)) == [0.25, 0.75, 1.25, 1.75]


def test_reconstruction_rounding_is_single(orc):
    """x' = RN32 of the exact centre (no double rounding through f64)."""
    rng = np.random.default_rng(7)
    for _ in range(200):
        m = np.float32(rng.normal() * 100)
        e = X.round_down_f32(abs(rng.normal()) * 1e-3 + 1e-7)
        q = int(rng.integers(0, 2 ** 29))
        got = orc.q2(np.array([q]), float(m), float(e))[0]
        assert got.view(np.uint32) == X.q2(q, m, e).view(np.uint32)


def test_subnormal_and_signed_zero(orc):
    m = np.float32(-0.0)
    e = np.float32(1e-40)  # subnormal-scale values are handled exactly by Q1
    vals = np.array([0.0, 1e-45, 3e-40, 1e-39], np.float32)
    assert list(orc.q1(vals, float(m), float(e))) == [X.q1(v, m, e) for v in vals]
    # reconstruction of tiny centres: subnormal results are exact or RN
    q = np.array([0, 1, 2, 5])
    xr = orc.q2(q, float(m), float(e))
    ref = np.array([X.q2(int(k), m, e) for k in q], np.float32)
    assert np.array_equal(xr.view(np.uint32), ref.view(np.uint32))


def test_round_down(orc):
    rng = np.random.default_rng(3)
    for d in list(rng.random(200) * 10.0 ** rng.integers(-30, 30, 200)) + [1e-3, 0.1, 1.0, 2.5e-5]:
        assert np.float32(orc.round_down_f32(float(d))).view(np.uint32) == \
            X.round_down_f32(float(d)).view(np.uint32)


def test_plan_error_codes(orc):
    Xf = np.zeros((3, 10), np.float32)
    with pytest.raises(orc.OracleError) as ei:
        orc.compress_s(np.where(np.arange(30).reshape(3, 10) == 4, np.nan, Xf), 1e-3)
    assert ei.value.status == orc.ERR_NONFINITE
    with pytest.raises(orc.OracleError) as ei:
        orc.compress_s(Xf, -1.0)
    assert ei.value.status == orc.ERR_ARG
    with pytest.raises(orc.OracleError) as ei:
        orc.compress_s(Xf, 1e-3, p=3)
    assert ei.value.status == orc.ERR_ARG
    big = np.array([[0.0, 1.0e9]] * 3, np.float32)
    with pytest.raises(orc.OracleError) as ei:
        orc.compress_s(big, 1e-3)  # qmax >= 2^30
    assert ei.value.status == orc.ERR_RANGE
    wide = np.array([[0.0, 1.0e3]] * 8, np.float32)
    with pytest.raises(orc.OracleError) as ei:
        orc.compress_s(wide, 1e-4, p=2)  # key space above 2^63
    assert ei.value.status == orc.ERR_RANGE
