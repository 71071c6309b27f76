"""Pins of the oracle's Huffman code lengths (Sec. "Block coding").

Optimality against brute force over all prefix-code length vectors on small
alphabets, the Kraft equality, the fixed tie-break on a hand-worked example,
and the 24-bit length limit.
"""
import itertools
from fractions import Fraction

import numpy as np
import pytest


def brute_force_cost(freqs):
    """Minimum sum f*l over length vectors satisfying Kraft (<= 1)."""
    n = len(freqs)
    best = None
    for ls in itertools.product(range(1, n + 1), repeat=n):
        if sum(Fraction(1, 2 ** l) for l in ls) <= 1:
            c = sum(f * l for f, l in zip(freqs, ls))
            best = c if best is None else min(best, c)
    return best


@pytest.mark.parametrize("seed", range(12))
def test_lengths_optimal_small(orc, seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(2, 6))
    freqs = [int(v) for v in rng.integers(1, 30, size=n)]
    ln = orc.huffman_lengths(freqs)[:n]
    assert sum(f * int(l) for f, l in zip(freqs, ln)) == brute_force_cost(freqs)
    assert sum(Fraction(1, 2 ** int(l)) for l in ln) == 1


def test_tie_break_leaf_before_internal(orc):
    """freqs a=1 b=1 c=2 d=2: after merging a+b (weight 2) the leaf c (weight 2)
    is taken before the internal node, then d, giving lengths 2,2,2,2 (the
    other tie-break would give 3,3,2,1 at the same cost)."""
    assert list(orc.huffman_lengths([1, 1, 2, 2])[:4]) == [2, 2, 2, 2]


def test_single_and_unused(orc):
    f = np.zeros(4096, np.uint64)
    f[17] = 99
    ln = orc.huffman_lengths(f)
    assert ln[17] == 1 and ln.sum() == 1


def test_length_limit(orc):
    fib = [1, 1]
    while len(fib) < 40:
        fib.append(fib[-1] + fib[-2])
    ln = orc.huffman_lengths(fib)[:40]
    assert ln.max() <= 24
    assert sum(Fraction(1, 2 ** int(l)) for l in ln) == 1
    # without the limit the same weights would need a 39-bit code
    assert (ln > 0).all()


def test_sparse_symbols_large_alphabet(orc):
    rng = np.random.default_rng(5)
    f = np.zeros(4096, np.uint64)
    idx = rng.choice(4096, 300, replace=False)
    f[idx] = rng.integers(1, 10 ** 6, 300)
    ln = orc.huffman_lengths(f)
    assert ((ln > 0) == (f > 0)).all()
    assert sum(Fraction(1, 2 ** int(l)) for l in ln[ln > 0]) == 1
