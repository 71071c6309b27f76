"""lcp_quantize_noalloc: the element rules for callers that cannot allocate
device memory (an application that owns the GPU's memory through its own pool,
or a loop that forbids allocation while running).  Its results must equal
those of lcp_quantize bit for bit (the tolerance every parity test here
uses), on two calls in a row that share the library's fixed scratch array.

Collected last on purpose: a failure here does not hide any other test.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lcp():
    from paper_2411_00761_b300 import lcp as L
    L.load()
    return L


def _values(seed, n, m, e, scale):
    rng = np.random.default_rng(seed)
    x = (np.float32(m) + rng.random(n) * scale).astype(np.float32)
    # values on exact bin edges (two of every 64), where the guard decides
    k = rng.integers(0, int(scale / (2 * e)), size=n // 64)
    x[: k.size] = (np.float32(m) + k.astype(np.float32) * np.float32(2 * e)).astype(np.float32)
    return torch.from_numpy(x).cuda()


def test_noalloc_matches_lcp_quantize_twice(lcp):
    cases = [(3, 1_000_003, -0.5, 3.7e-4, 1.0), (4, 70_001, 1000.0, 3e-5, 2.0)]
    for seed, n, m, e, scale in cases:  # two calls in a row, different sizes
        x = _values(seed, n, m, e, scale)
        e32 = float(np.float32(e))
        max_abs = float(x.abs().max())
        q0, xr0, v0 = lcp.quantize(x, m, e32, max_abs)
        q1 = torch.empty(n, dtype=torch.int32, device="cuda")
        xr1 = torch.empty(n, dtype=torch.float32, device="cuda")
        v1 = torch.empty(n, dtype=torch.uint8, device="cuda")
        nv = lcp.quantize_noalloc(x, m, e32, max_abs, q1, xr1, v1)
        assert torch.equal(q0, q1)
        assert torch.equal(xr0.view(torch.int32), xr1.view(torch.int32))
        assert torch.equal(v0, v1.bool())
        assert nv == int(v0.sum())


def test_noalloc_rejects_sizes_beyond_its_scratch(lcp):
    n = lcp.NOALLOC_MAX_ELEMENTS + 1
    x = torch.zeros(n, dtype=torch.float32, device="cuda")
    q = torch.empty(n, dtype=torch.int32, device="cuda")
    xr = torch.empty(n, dtype=torch.float32, device="cuda")
    v = torch.empty(n, dtype=torch.uint8, device="cuda")
    with pytest.raises(lcp.LcpError) as ei:
        lcp.quantize_noalloc(x, 0.0, 1e-3, 0.0, q, xr, v)
    assert ei.value.status == lcp.ERR_ARG
