"""The sampled block-size search (Sec. "Best block size"): candidates
p = 2^k, 0 <= k <= 16, each judged on a sample of the frame.

The paper reports that the sampled choice reaches at least 85% of the
compression ratio of the best candidate on the whole input in most cases;
that is checked here on the three synthetic workload families, with the
whole-frame sizes of every candidate computed independently of the search.
"""
import numpy as np
import pytest

import oracle
from oracle import hybrid
from paper_2411_00761_b300 import synth


def test_sample_size_rule():
    assert hybrid.sample_size(1000) == 1000
    assert hybrid.sample_size(65536) == 65536
    assert hybrid.sample_size(65536 * 8) == 65536
    assert hybrid.sample_size(65536 * 8 + 1) == 65537
    assert hybrid.sample_size(10 ** 7) == 1250000
    assert hybrid.BLOCK_CANDIDATES_ALL == tuple(2 ** k for k in range(17))


def test_candidates_outside_the_domain_are_skipped():
    X = synth.cosmology(4096, 2)  # d = 6: p^6 <= 2^32 allows p <= 32
    p, sizes = hybrid.choose_block_size_sampled(X, 1e-3, "rel")
    assert sorted(sizes) == [1, 2, 4, 8, 16, 32]
    assert sizes[p] == min(sizes.values())
    assert p == min(q for q in sizes if sizes[q] == sizes[p])


@pytest.mark.parametrize("name,X,eb,mode", [
    ("uniform_clusters", synth.uniform_clusters(1 << 18, 1), 1e-3, "abs"),
    ("md_fcc", synth.md_fcc(1 << 18, 1, cells=51), 1e-4, "rel"),
    ("cosmology6", synth.cosmology(1 << 18, 2), 1e-3, "rel"),
])
def test_sampled_choice_reaches_85_percent_of_best(name, X, eb, mode):
    p, _ = hybrid.choose_block_size_sampled(X, eb, mode)
    d = X.shape[0]
    full = {}
    for k in range(17):
        if k * d > 32:
            break
        try:
            full[1 << k] = oracle.compressed_size_s(X, eb, mode, 1 << k)
        except oracle.OracleError:
            pass
    best = min(full.values())
    assert best / full[p] >= 0.85, (name, p, full)
