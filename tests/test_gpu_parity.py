"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Bit-exact throughout: quantization codes, reconstructed values and guard
decisions element by element; the container bytes of LCP-S and LCP-T frames;
the decoded particles; the slot permutation.  Sizes span several tiles,
partition buckets and a ragged tail; edge cases cover empty frames, a single
particle, all particles in one block, bounds near the f32 spacing (raw
outliers), one and eight fields, and buckets too large for shared memory.
"""
import numpy as np
import pytest
import torch

from paper_2411_00761_b300 import synth
from tests import exact_ref as X

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lcp():
    from paper_2411_00761_b300 import lcp as L
    return L


@pytest.fixture(scope="module")
def ctx(lcp):
    return lcp.Context(0)


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def gpu_bytes(res):
    return res["bytes"].cpu().numpy().tobytes()


# ---------------------------------------------------------------------------
# element rules
# ---------------------------------------------------------------------------
ELEM_CASES = [(0.0, 1e-3, 1.0), (-0.5, 3.7e-4, 1.0), (1000.0, 0.25, 50.0), (-2000.0, 3.6, 4000.0),
              (1.0e-6, 1e-3, 1.0), (0.0, 1e-7, 1e-3), (123.456, 1e-5, 0.01), (-3.0, 0.7, 6.0),
              (1.0e6, 1e-5, 1.0), (-3.0e7, 3e-6, 8.0)]  # the last two: |x| >= 2^32 * 2e


@pytest.mark.parametrize("m,eb,scale", ELEM_CASES)
def test_element_rules_bit_exact(lcp, orc, m, eb, scale):
    rng = np.random.default_rng(int(abs(m) * 1000 + eb * 1e7) % 2 ** 31)
    m = np.float32(m)
    e = np.float32(orc.round_down_f32(eb))
    vals = (m + rng.random(200000) * scale).astype(np.float32)
    # values at and next to exact bin edges
    ks = rng.integers(0, int(scale / (2 * float(e))) + 1, size=2000)
    edges = []
    for k in ks:
        r = X.rn32(X.F(m) + int(k) * 2 * X.F(e))
        edges += [r, np.nextafter(r, np.float32(np.inf), dtype=np.float32),
                  np.nextafter(r, np.float32(-np.inf), dtype=np.float32)]
    vals = np.concatenate([vals, np.array(edges, np.float32), np.array([m], np.float32)])
    vals = vals[vals >= m]
    q, xr, v = lcp.quantize(to_dev(vals), float(m), float(e))
    q_ref = orc.q1(vals, float(m), float(e))
    assert np.array_equal(q.cpu().numpy().astype(np.int64), q_ref)
    xr_ref = orc.q2(q_ref, float(m), float(e))
    assert np.array_equal(xr.cpu().numpy().view(np.uint32), xr_ref.view(np.uint32))
    v_ref = orc.q3(vals, xr_ref, float(e))
    assert np.array_equal(v.cpu().numpy(), v_ref)


# ---------------------------------------------------------------------------
# LCP-S frames
# ---------------------------------------------------------------------------
def frames_s():
    yield "uniform_clusters_ragged", synth.uniform_clusters((1 << 17) + 77, 0), 1e-3, "abs", 8
    yield "uniform_clusters_p2", synth.uniform_clusters(50001, 5), 1e-3, "abs", 2
    yield "md_fcc", synth.md_fcc(200003, 1, cells=40), 1e-4, "rel", 16
    yield "md_fcc_p32", synth.md_fcc(65536, 3, cells=30), 1e-4, "rel", 32
    yield "cosmology6", synth.cosmology(100000, 2), 1e-3, "rel", 4
    yield "cosmology6_p8", synth.cosmology(30011, 7), 1e-3, "rel", 8


def check_s(ctx, orc, Xf, eb, mode, p):
    o = orc.compress_s(Xf, eb, mode, p)
    # without the slot permutation (keys only) and with it (keys and indices)
    r0 = ctx.compress(to_dev(Xf), eb, mode, p)
    assert gpu_bytes(r0) == o["bytes"]
    r = ctx.compress(to_dev(Xf), eb, mode, p, perm=True)
    gb = gpu_bytes(r)
    assert len(gb) == len(o["bytes"])
    assert gb == o["bytes"]
    assert np.array_equal(r["perm"].cpu().numpy().astype(np.uint32), o["pi"])
    Y = ctx.decompress(r["bytes"]).cpu().numpy()
    Yo, _ = orc.decompress(o["bytes"])
    assert np.array_equal(Y.view(np.uint32), Yo.view(np.uint32))
    return r, o


@pytest.mark.parametrize("name,Xf,eb,mode,p", list(frames_s()))
def test_lcp_s_bytes_and_decode(ctx, orc, name, Xf, eb, mode, p):
    check_s(ctx, orc, Xf, eb, mode, p)


def test_lcp_s_decodes_oracle_containers_other_chunks(ctx, orc):
    Xf = synth.uniform_clusters(40000, 9)
    for lc in (5, 8, 10):
        o = orc.compress_s(Xf, 1e-3, "abs", 8, log2_chunk=lc)
        Y = ctx.decompress(to_dev(np.frombuffer(o["bytes"], np.uint8))).cpu().numpy()
        Yo, _ = orc.decompress(o["bytes"])
        assert np.array_equal(Y.view(np.uint32), Yo.view(np.uint32))


def test_degenerate_frames(ctx, orc):
    rng = np.random.default_rng(4)
    cases = [
        (np.full((3, 5000), 0.37, np.float32), 1e-3, "abs", 8),            # one block
        (np.zeros((3, 0), np.float32), 1e-3, "abs", 8),                    # empty
        (np.array([[0.5], [0.25], [0.125]], np.float32), 1e-3, "abs", 8),  # one particle
        ((1000.0 + rng.random((3, 20000))).astype(np.float32), 4e-5, "abs", 4),  # outliers
        ((1000.0 + rng.random((3, 3000))).astype(np.float32), 1e-6, "abs", 4),   # sub-ulp bound
        (rng.random((1, 70000)).astype(np.float32), 1e-4, "abs", 16),      # d = 1
        (rng.random((8, 30000)).astype(np.float32), 0.05, "abs", 2),       # d = 8
        (np.stack([np.linspace(0, 1, 9000, dtype=np.float32), np.full(9000, 5.0, np.float32)]),
         1e-3, "rel", 4),                                                  # constant field
    ]
    for Xf, eb, mode, p in cases:
        check_s(ctx, orc, Xf, eb, mode, p)


def test_large_bucket_global_path(ctx, orc):
    """Many distinct keys in one partition bucket: sorted in global memory."""
    rng = np.random.default_rng(8)
    n = 60000
    # all particles inside one block along the top axis, spread in the others
    Xf = np.stack([rng.random(n), rng.random(n), np.full(n, 0.5) + rng.random(n) * 1e-3])
    Xf = Xf.astype(np.float32)
    check_s(ctx, orc, Xf, 1e-3, "abs", 4)


def test_status_codes(ctx, lcp):
    Xn = np.zeros((3, 100), np.float32)
    Xn[1, 7] = np.nan
    with pytest.raises(lcp.LcpError) as ei:
        ctx.compress(to_dev(Xn), 1e-3)
    assert ei.value.status == lcp.ERR_NONFINITE
    with pytest.raises(lcp.LcpError) as ei:
        ctx.compress(to_dev(np.zeros((3, 10), np.float32)), 1e-3, p=3)
    assert ei.value.status == lcp.ERR_ARG
    big = np.array([[0.0, 1.0e9]] * 3, np.float32)
    with pytest.raises(lcp.LcpError) as ei:
        ctx.compress(to_dev(big), 1e-3)
    assert ei.value.status == lcp.ERR_RANGE
    wide = np.array([[0.0, 1.0e3]] * 8, np.float32)
    with pytest.raises(lcp.LcpError) as ei:
        ctx.compress(to_dev(wide), 1e-4, p=2)
    assert ei.value.status == lcp.ERR_RANGE
    # capacity
    Xf = synth.uniform_clusters(10000, 1)
    out = torch.empty(100, dtype=torch.uint8, device="cuda")
    with pytest.raises(lcp.LcpError) as ei:
        ctx.compress(to_dev(Xf), 1e-3, out=out)
    assert ei.value.status == lcp.ERR_CAPACITY
    # decompression into a buffer of a given number of values (no header read
    # by the caller): one value short is refused, the exact size decodes
    buf = ctx.compress(to_dev(Xf), 1e-3)["bytes"]
    short = torch.full((3 * 10000 - 1,), -7.0, dtype=torch.float32, device="cuda")
    with pytest.raises(lcp.LcpError) as ei:
        ctx.decompress(buf, out=short)
    assert ei.value.status == lcp.ERR_CAPACITY
    assert bool((short == -7.0).all())  # nothing written
    exact = torch.empty((3 * 10000,), dtype=torch.float32, device="cuda")
    y = ctx.decompress(buf, out=exact)
    assert tuple(y.shape) == (3, 10000)
    assert torch.equal(y, ctx.decompress(buf))
    # host-buffer entry points: the same container and the same frame
    Xh = torch.from_numpy(np.ascontiguousarray(Xf)).pin_memory()
    rh = ctx.compress_host(Xh, 1e-3)
    assert bytes(rh["bytes"].numpy()) == bytes(buf.cpu().numpy())
    yh = ctx.decompress_host(rh["bytes"].clone(), out=torch.empty(3 * 10000).pin_memory())
    assert torch.equal(yh, y.cpu())


def test_block_size_autotune_matches_oracle(ctx, orc):
    from oracle import hybrid
    Xf = synth.md_fcc(40000, 1, cells=25)
    best, sizes = hybrid.choose_block_size(Xf, 1e-4, "rel")
    r = ctx.compress(to_dev(Xf), 1e-4, "rel", p=0)
    assert r["size"] == sizes[best]
    assert gpu_bytes(r) == orc.compress_s(Xf, 1e-4, "rel", best)["bytes"]


@pytest.mark.parametrize("name,Xf,eb,mode,sample", [
    ("uniform_clusters", synth.uniform_clusters(150001, 3), 1e-3, "abs", 0),   # p = 1 .. 1024
    ("cosmology6", synth.cosmology(100003, 4), 1e-3, "rel", 0),                # p = 1 .. 32
    ("md_fcc_given_sample", synth.md_fcc(70001, 2, cells=28), 1e-4, "rel", 30011),
])
def test_choose_block_size_matches_oracle(ctx, orc, name, Xf, eb, mode, sample):
    from oracle import hybrid
    p_ref, sizes_ref = hybrid.choose_block_size_sampled(Xf, eb, mode, sample)
    p, sizes = ctx.choose_block_size(to_dev(Xf), eb, mode, sample)
    assert sizes == sizes_ref
    assert p == p_ref


def test_sort_paths(ctx, orc):
    """Sort units whose digit groups need every path of the unit sort:
    windows of 2..512 particles sorted by one warp (32- and 64-bit keys,
    with and without indices), windows too large for a warp (one digit
    group of identical keys), and units beyond shared memory."""
    rng = np.random.default_rng(12)
    # many identical particles (one key) among random ones
    a = np.concatenate([np.full((3, 3000), 0.4321, np.float32), rng.random((3, 2000))], axis=1)
    check_s(ctx, orc, a[:, rng.permutation(a.shape[1])].astype(np.float32), 1e-3, "abs", 8)
    # more identical particles than one shared-memory unit holds
    b = np.concatenate([np.full((3, 9000), 0.25, np.float32), rng.random((3, 3000))], axis=1)
    check_s(ctx, orc, b[:, rng.permutation(b.shape[1])].astype(np.float32), 1e-3, "abs", 8)
    # keys wider than 32 bits inside a unit (small frame, fine bound)
    check_s(ctx, orc, rng.random((3, 30000)).astype(np.float32), 1e-5, "abs", 4)
    # dense blocks of 200..500 particles: large windows
    cl = []
    for k in range(48):
        c = rng.random(3) * 0.9
        m = int(rng.integers(200, 500))
        cl.append(c[:, None] + rng.random((3, m)) * 0.015)
    c = np.concatenate(cl + [rng.random((3, 5000))], axis=1).astype(np.float32)
    check_s(ctx, orc, c[:, rng.permutation(c.shape[1])], 1e-3, "abs", 8)


# Field minima off the bin grid, from near zero to large offsets, and bin counts
# from ~10^2 to above 2^23, so that reconstruction (Eq. quantization, Q2) runs
# both its binary32 path (codes below 2^23) and its 64-bit path, in the LCP-S
# expand and in the LCP-T decode.
Q2_FRAMES = [
    ((1.0e6, -3.7e4, 2.5e-3), (100.0, 100.0, 100.0), 1e-3, "abs"),
    ((-0.75, 123.456, -9.9e3), (1.0, 1.0, 1.0), 3.3e-6, "abs"),
    ((0.0, 50.0, -100.0), (1.0, 1e-4, 1e-4), 2e-8, "abs"),  # 2.5e7 bins in the first field
    ((5.0e4, -5.0e4, 1.0), (1.0e4, 1.0e4, 1.0e4), 1e-4, "rel"),
    # minima 2^33 bins or more away from zero: Q2 on the exact wide path
    ((1.0e6, -3.0e7, 2.0e5), (1.0, 1.0, 1.0), 1e-5, "abs"),
]


@pytest.mark.parametrize("offs,scale,eb,mode", Q2_FRAMES)
def test_decode_q2_offsets_and_bounds(ctx, orc, lcp, offs, scale, eb, mode):
    rng = np.random.default_rng(11)
    sc = np.array(scale)[:, None]
    X0 = (rng.random((3, 20011)) * sc + np.array(offs)[:, None]).astype(np.float32)
    check_s(ctx, orc, X0, eb, mode, 8)
    X1 = (X0 + rng.normal(0.0, 1e-4, X0.shape) * sc).astype(np.float32)
    tr = lcp.Trajectory(ctx, batch=10, p=8)
    r0 = ctx.compress(to_dev(X0), eb, mode, traj=tr, method="spatial", perm=True)
    o0 = orc.compress_s(X0, eb, mode, 8, flags=1)
    assert gpu_bytes(r0) == o0["bytes"]
    r1 = ctx.compress(to_dev(X1), eb, mode, traj=tr, method="temporal")
    o1 = orc.compress_t(X1, eb, mode, o0["q"], o0["pi"])
    assert gpu_bytes(r1) == o1["bytes"]
    dt = lcp.Trajectory(ctx, batch=10, p=8)
    ctx.decompress(r0["bytes"], traj=dt)
    Y1 = ctx.decompress(r1["bytes"], traj=dt).cpu().numpy()
    Yo1, _ = orc.decompress(o1["bytes"], o0["q"])
    assert np.array_equal(Y1.view(np.uint32), Yo1.view(np.uint32))


# ---------------------------------------------------------------------------
# LCP-T and the hybrid (Algorithm 1 with the LCP-FSM)
# ---------------------------------------------------------------------------
def test_lcp_t_bytes_forced(ctx, orc, lcp):
    frames = list(synth.brownian_trajectory(30017, 3, 13))
    tr = lcp.Trajectory(ctx, batch=10, p=8)
    r0 = ctx.compress(to_dev(frames[0]), 1e-3, "abs", traj=tr, method="spatial", perm=True)
    o0 = orc.compress_s(frames[0], 1e-3, "abs", 8, flags=1)
    assert gpu_bytes(r0) == o0["bytes"]
    r1 = ctx.compress(to_dev(frames[1]), 1e-3, "abs", traj=tr, method="temporal")
    o1 = orc.compress_t(frames[1], 1e-3, "abs", o0["q"], o0["pi"])
    assert r1["method"] == "temporal"
    assert gpu_bytes(r1) == o1["bytes"]
    # decode side: S then T through a decoder trajectory
    dt = lcp.Trajectory(ctx, batch=10, p=8)
    Y0 = ctx.decompress(r0["bytes"], traj=dt).cpu().numpy()
    Y1 = ctx.decompress(r1["bytes"], traj=dt).cpu().numpy()
    Yo1, _ = orc.decompress(o1["bytes"], o0["q"])
    assert np.array_equal(Y1.view(np.uint32), Yo1.view(np.uint32))
    assert Y0.shape == frames[0].shape


def test_hybrid_trajectory_matches_oracle(ctx, orc, lcp):
    from oracle import hybrid
    n, nf, batch = 20011, 24, 5
    frames = list(synth.brownian_trajectory(n, nf, 21, sigma=0.02))
    enc = hybrid.encode_trajectory(frames, 1e-3, "abs", 8, batch=batch)
    tr = lcp.Trajectory(ctx, batch=batch, p=8)
    dt = lcp.Trajectory(ctx, batch=batch, p=8)
    dec_o = hybrid.decode_trajectory([b for b, _ in enc])
    for t, (Xf, (ob, om)) in enumerate(zip(frames, enc)):
        r = ctx.compress(to_dev(Xf), 1e-3, "abs", traj=tr, method="auto")
        assert r["method"] == {"S": "spatial", "T": "temporal"}[om], t
        assert gpu_bytes(r) == ob, t
        Y = ctx.decompress(r["bytes"], traj=dt).cpu().numpy()
        assert np.array_equal(Y.view(np.uint32), dec_o[t].view(np.uint32)), t


@pytest.mark.parametrize("scale", [2, 5])
def test_anchor_scaling_matches_oracle(ctx, orc, lcp, scale):
    """Anchors at eb / scale and value-space prediction from them (Sec. "Best
    error-bound scale for anchor frames"): containers byte-identical to the
    oracle's Algorithm 1, frames decoded bit-identical."""
    from oracle import hybrid
    frames = list(synth.brownian_trajectory(20011, 10, 3, sigma=0.02))
    enc = hybrid.encode_trajectory(frames, 1e-3, "abs", 8, batch=4, anchor_scale=scale)
    assert any(orc.peek(b)["flags"] & hybrid.FLAG_REF_REQUANT for b, _ in enc)
    tr = lcp.Trajectory(ctx, batch=4, p=8, anchor_scale=scale)
    got = []
    for X in frames:
        r = ctx.compress(to_dev(X), 1e-3, "abs", 8, method="auto", traj=tr)
        got.append(gpu_bytes(r))
    for t, (b, _) in enumerate(enc):
        assert got[t] == b, t
    dec = hybrid.decode_trajectory([b for b, _ in enc])
    dt = lcp.Trajectory(ctx, batch=4, p=8)
    for t, b in enumerate(got):
        Y = ctx.decompress(to_dev(np.frombuffer(b, np.uint8)), traj=dt).cpu().numpy()
        assert np.array_equal(Y.view(np.uint32), dec[t].view(np.uint32)), t


@pytest.mark.parametrize("scale", [1, 5])
def test_random_access_matches_oracle(ctx, orc, lcp, scale):
    """Random-access retrieval (Sec. "Spatial-Anchor-Frame-Based Batch
    Compression", recursive decompression) through lcp_decompress_frame and
    lcp_decompress_frames: every frame fetched alone, in a shuffled order, and
    every batch fetched at once equal the oracle's sequential decode of the
    whole stream bit for bit; frames the chain does not need may be absent,
    and a missing anchor is reported."""
    from oracle import hybrid
    batch = 4
    frames = list(synth.brownian_trajectory(20011, 17, 5, sigma=0.02))
    enc = hybrid.encode_trajectory(frames, 1e-3, "abs", 8, batch=batch, anchor_scale=scale)
    dec = hybrid.decode_trajectory([b for b, _ in enc])
    methods = [m for _, m in enc]
    # some batch opens with an LCP-T frame, so its anchor must be fetched
    assert any(methods[b0] == "T" for b0 in range(batch, len(frames), batch))
    bufs = [to_dev(np.frombuffer(b, np.uint8)) for b, _ in enc]
    dt = lcp.Trajectory(ctx, batch=batch, p=8)
    for t in np.random.default_rng(1).permutation(len(frames)):
        Y = ctx.decompress_frame(bufs, int(t), traj=dt).cpu().numpy()
        assert np.array_equal(ctx.decompress_frame(bufs, int(t), batch=batch).cpu().numpy().view(
            np.uint32), Y.view(np.uint32))
        assert np.array_equal(Y.view(np.uint32), dec[t].view(np.uint32)), t
    for b0 in range(0, len(frames), batch):
        last = min(b0 + batch - 1, len(frames) - 1)
        Ys = ctx.decompress_frames(bufs, b0, last, traj=dt)
        for k, Y in enumerate(Ys):
            assert np.array_equal(Y.cpu().numpy().view(np.uint32),
                                  dec[b0 + k].view(np.uint32)), (b0, k)
    # only the chain of frame t present (and the batch openings back to its
    # anchor, whose headers show which opening is the anchor)
    for t in range(len(frames)):
        b0 = t - t % batch
        s = max([i for i in range(b0, t + 1) if methods[i] == "S"], default=None)
        if s is None:
            a = max(i for i in range(0, b0, batch) if methods[i] == "S")
            need = [a] + list(range(a + batch, b0, batch)) + list(range(b0, t + 1))
        else:
            need = list(range(s, t + 1))
        part = [bufs[i] if i in need else None for i in range(t + 1)]
        Y = ctx.decompress_frame(part, t, traj=dt).cpu().numpy()
        assert np.array_equal(Y.view(np.uint32), dec[t].view(np.uint32)), t
        if need[0] < b0:  # without the anchor the chain cannot start
            part[need[0]] = None
            with pytest.raises(lcp.LcpError) as ei:
                ctx.decompress_frame(part, t, traj=dt)
            assert ei.value.status == lcp.ERR_STATE


def test_select_is_a_query(ctx, lcp):
    frames = list(synth.brownian_trajectory(5000, 4, 2))
    tr = lcp.Trajectory(ctx, batch=10, p=8)
    assert ctx.select(tr, to_dev(frames[0]), 1e-3)[0] == "spatial"
    ctx.compress(to_dev(frames[0]), 1e-3, traj=tr, method="auto")
    a = ctx.select(tr, to_dev(frames[1]), 1e-3)
    b = ctx.select(tr, to_dev(frames[1]), 1e-3)
    assert a == b
    r = ctx.compress(to_dev(frames[1]), 1e-3, traj=tr, method="auto")
    assert r["method"] == a[0]


def test_temporal_needs_reference(ctx, lcp):
    tr = lcp.Trajectory(ctx, batch=10, p=8)
    Xf = synth.uniform_clusters(1000, 1)
    with pytest.raises(lcp.LcpError) as ei:
        ctx.compress(to_dev(Xf), 1e-3, traj=tr, method="temporal")
    assert ei.value.status == lcp.ERR_STATE
    with pytest.raises(lcp.LcpError) as ei:
        ctx.compress(to_dev(Xf), 1e-3, method="temporal")
    assert ei.value.status == lcp.ERR_STATE


# ---------------------------------------------------------------------------
# full-size workloads in the bench's launch configuration
# ---------------------------------------------------------------------------
def test_full_size_plain_frame_bytes(ctx, orc):
    """2^20 particles, the plain LCP-S frame: the whole container."""
    Xf = synth.uniform_clusters(1 << 20, 0)
    check_s(ctx, orc, Xf, 1e-3, "abs", 8)


def test_bench_config_bytes_16M(ctx, orc):
    """The benchmarked configuration -- the cosmology-like 6-field frame, eb =
    1e-3 of each field's range, p = 8 -- at 2^24 particles: the whole
    container equals the oracle's byte for byte (with and without the slot
    permutation) and the decoded frame equals the oracle's decode bit for
    bit.  At this size dense halo buckets exceed 32K keys, so the multi-task
    level-2 split runs."""
    Xf = synth.cosmology(1 << 24, 2)
    r, o = check_s(ctx, orc, Xf, 1e-3, "rel", 8)
    assert o["M"] > 1 << 22


def test_bench_config_full_frame_64M(lcp, orc):
    """The benchmarked frame itself (2^26 particles x 6 fields, p = 8), in the
    bench's launch configuration (the schedule chosen by the autotuner, as the
    bench does): the container the bench times is decoded by the oracle, and
    every decoded value equals the GPU's decode bit for bit; the slot
    permutation is a permutation, every particle is within its bound, and on
    2^21 sampled slots the decoded code equals the oracle's own Q1 of the
    particle's value."""
    Xf = synth.cosmology(1 << 26, 2)
    d, n = Xf.shape
    Xd = to_dev(Xf)
    ctx = lcp.Context(0)
    sc = ctx.tune(Xd, 1e-3, "rel", 8, max_growth=0.01)
    ctx.set_schedule(sc["log2_chunk"], sc["bucket_delta"])
    r0 = ctx.compress(Xd, 1e-3, "rel", 8)  # the bench's call
    r = ctx.compress(Xd, 1e-3, "rel", 8, perm=True)
    assert torch.equal(r0["bytes"], r["bytes"])
    Y = ctx.decompress(r0["bytes"])
    buf = gpu_bytes(r0)
    Yo, qo = orc.decompress(buf)
    Yg = Y.cpu().numpy()
    assert np.array_equal(Yg.view(np.uint32), Yo.view(np.uint32))
    perm = r["perm"].long()
    assert torch.equal(torch.sort(perm).values, torch.arange(n, device="cuda"))
    hdr = np.frombuffer(buf[:48 + 16 * d], np.uint8)
    e = hdr[48:48 + 16 * d].view(np.float32).reshape(d, 4)[:, 1]
    m = hdr[48:48 + 16 * d].view(np.float32).reshape(d, 4)[:, 0]
    err = (Xd[:, perm].double() - Y.double()).abs().max(dim=1).values.cpu().numpy()
    assert (err <= e.astype(np.float64)).all()
    K = int(np.frombuffer(buf[24:32], np.uint64)[0])
    rng = np.random.default_rng(0)
    slots = np.sort(rng.choice(n - K, 1 << 21, replace=False))
    pi = perm.cpu().numpy()[slots]
    for f in range(d):
        q = orc.q1(Xf[f, pi], float(m[f]), float(e[f]))
        assert np.array_equal(q, qo[f, slots].astype(np.int64))


@pytest.mark.parametrize("lc", [5, 8, 9])
def test_schedule_chunks_match_oracle(lcp, orc, lc):
    """Chunks of 2^lc symbols (a schedule knob recorded in the container):
    LCP-S containers of the benchmarked configuration (2^22 particles) and an
    LCP-T frame equal the oracle's at the same chunk size byte for byte, and
    decode bit for bit."""
    ctx = lcp.Context(0)
    ctx.set_schedule(lc, 0)
    assert ctx.schedule()["log2_chunk"] == lc
    Xf = synth.cosmology(1 << 22, 2)
    o = orc.compress_s(Xf, 1e-3, "rel", 8, log2_chunk=lc)
    r = ctx.compress(to_dev(Xf), 1e-3, "rel", 8)
    assert gpu_bytes(r) == o["bytes"]
    Y = ctx.decompress(r["bytes"]).cpu().numpy()
    Yo, _ = orc.decompress(o["bytes"])
    assert np.array_equal(Y.view(np.uint32), Yo.view(np.uint32))
    frames = list(synth.brownian_trajectory(30011, 2, 5))
    tr = lcp.Trajectory(ctx, batch=10, p=8)
    r0 = ctx.compress(to_dev(frames[0]), 1e-3, "abs", traj=tr, method="spatial")
    o0 = orc.compress_s(frames[0], 1e-3, "abs", 8, log2_chunk=lc, flags=1)
    assert gpu_bytes(r0) == o0["bytes"]
    r1 = ctx.compress(to_dev(frames[1]), 1e-3, "abs", traj=tr, method="temporal")
    o1 = orc.compress_t(frames[1], 1e-3, "abs", o0["q"], o0["pi"], log2_chunk=lc)
    assert gpu_bytes(r1) == o1["bytes"]


def test_schedule_bucket_width_keeps_bytes(lcp, orc):
    """The width of the first sort partition changes no byte."""
    Xf = synth.cosmology(300007, 4)
    ref = orc.compress_s(Xf, 1e-3, "rel", 8)["bytes"]
    ctx = lcp.Context(0)
    for bd in (-4, -2, -1, 1):
        ctx.set_schedule(10, bd)
        assert gpu_bytes(ctx.compress(to_dev(Xf), 1e-3, "rel", 8)) == ref, bd
    with pytest.raises(lcp.LcpError):
        ctx.set_schedule(11, 0)
    with pytest.raises(lcp.LcpError):
        ctx.set_schedule(10, 2)


def test_full_size_md_sampled(ctx, orc, lcp):
    """The 16M-particle MD frame at the bench's p = 2: every decoded value is
    within the bound of its particle; on a sample of particles the decoded
    value equals the oracle's reconstruction of the oracle's code bit for
    bit; the decoded frame holds every particle once."""
    Xf, eb, mode, p = synth.md_fcc(1 << 24, 1), 1e-4, "rel", 2
    Xd = to_dev(Xf)
    r = ctx.compress(Xd, eb, mode, p, perm=True)
    Y = ctx.decompress(r["bytes"])
    perm = r["perm"].long()
    d, n = Xf.shape
    assert torch.equal(torch.sort(perm).values, torch.arange(n, device="cuda"))
    hdr = r["bytes"][:48 + 16 * d].cpu().numpy()
    e = hdr[48:48 + 16 * d].view(np.float32).reshape(d, 4)[:, 1]
    m = hdr[48:48 + 16 * d].view(np.float32).reshape(d, 4)[:, 0]
    err = (Xd[:, perm].double() - Y.double()).abs().max(dim=1).values.cpu().numpy()
    assert (err <= e.astype(np.float64)).all()
    rng = np.random.default_rng(0)
    slots = rng.choice(n, 20000, replace=False)
    pi = perm.cpu().numpy()[slots]
    Ys = Y[:, torch.from_numpy(slots).cuda()].cpu().numpy()
    K = int(np.frombuffer(r["bytes"][24:32].cpu().numpy().tobytes(), np.uint64)[0])
    for f in range(d):
        x = Xf[f, pi]
        q = orc.q1(x, float(m[f]), float(e[f]))
        xr = orc.q2(q, float(m[f]), float(e[f]))
        raw = slots >= n - K
        exp = np.where(raw, x, xr)
        assert np.array_equal(Ys[f].view(np.uint32), exp.view(np.uint32))
