"""The dictionary stage on the GPU (lcp_dict_compress / lcp_dict_decompress,
lcp_ctx_set_dict) against the oracle's LCPZ coder, byte for byte.

The stage is the last step of the encoding stage (Sec. "Block coding"; Zstd
in the paper, an LZ77-style coder here).  Inputs: empty and tiny strings, the
hand-worked chunks, runs, random bytes (every chunk stored), a ragged mix,
real containers of LCP-S and LCP-T frames, and a multi-hundred-chunk
container of a 2^24-particle frame.  The context option is checked end to
end: images in place of containers through every decompression entry point.
"""
import numpy as np
import pytest
import torch

from paper_2411_00761_b300 import synth

pytestmark = pytest.mark.gpu

CH = 1 << 16


@pytest.fixture(scope="module")
def lcp():
    from paper_2411_00761_b300 import lcp as L
    L.load()
    return L


def dev(b: bytes):
    t = torch.empty(max(len(b), 16), dtype=torch.uint8, device="cuda")
    if b:
        t[:len(b)] = torch.from_numpy(np.frombuffer(b, np.uint8).copy()).cuda()
    return t


def host(t) -> bytes:
    return t.cpu().numpy().tobytes()


def mixed(seed, parts=40):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(parts):
        k = int(rng.integers(1, 9000))
        kind = int(rng.integers(0, 3))
        if kind == 0:
            out.append(rng.integers(0, 256, k, dtype=np.uint8).tobytes())
        elif kind == 1:
            out.append(bytes([int(rng.integers(0, 256))]) * k)
        else:
            base = rng.integers(0, 4, int(rng.integers(1, 40)), dtype=np.uint8).tobytes()
            out.append((base * (k // len(base) + 1))[:k])
    return b"".join(out)


def cases(orc):
    X = synth.cosmology(1 << 16, 2)
    c_s = orc.compress_s(X, 1.0, "abs", 8)["bytes"]
    from oracle import hybrid
    frames = list(synth.brownian_trajectory(20011, 6, 7, sigma=0.02))
    enc = hybrid.encode_trajectory(frames, 1e-3, "abs", 8, batch=3)
    c_t = [b for b, m in enc if m == "T"][-1] if any(m == "T" for _, m in enc) else enc[-1][0]
    rng = np.random.default_rng(3)
    return {
        "empty": b"",
        "one": b"a",
        "three": b"abc",
        "four": b"abcd",
        "worked": b"abcabcabcabcX",
        "latest": b"abcd1abcd2abcd2",
        "inside": b"wxyzabcdwxyzabcdabcdE",
        "chunk_zeros": bytes(CH),
        "zeros_ragged": bytes(2 * CH + 100),
        "periodic": b"abcd" * (CH // 4) + b"xy",
        "random": rng.integers(0, 256, 3 * CH + 777, dtype=np.uint8).tobytes(),
        "mixed": mixed(9),
        "mixed2": mixed(10, 90),
        "lcp_s": c_s,
        "lcp_t": c_t,
    }


@pytest.fixture(scope="module")
def inputs(orc):
    return cases(orc)


@pytest.mark.parametrize("name", [
    "empty", "one", "three", "four", "worked", "latest", "inside", "chunk_zeros", "zeros_ragged",
    "periodic", "random", "mixed", "mixed2", "lcp_s", "lcp_t"])
def test_image_equals_oracle(lcp, orc, inputs, name):
    raw = inputs[name]
    ctx = lcp.Context(0)
    img = ctx.dict_compress(dev(raw), len(raw))
    want = orc.dict_compress(raw)
    assert host(img) == want
    back = ctx.dict_decompress(img)
    assert host(back)[:len(raw)] == raw and back.numel() == len(raw)
    # the oracle's image decodes the same on the GPU
    assert host(ctx.dict_decompress(dev(want), len(want))) == raw


def test_large_container_equals_oracle(lcp, orc):
    """A 2^24 x 6 cosmology-like container: hundreds of chunks, coded and
    stored ones, decoded back into a frame equal to the plain container's."""
    X = torch.from_numpy(synth.cosmology(1 << 24, 2)).cuda()
    ctx = lcp.Context(0)
    r = ctx.compress(X, 1.0, "abs", 8)
    raw = host(r["bytes"])
    img = ctx.dict_compress(r["bytes"], r["size"])
    want = orc.dict_compress(raw)
    assert host(img) == want
    assert len(want) < len(raw)
    back = ctx.dict_decompress(img)
    assert torch.equal(back, r["bytes"])
    Y0 = ctx.decompress(r["bytes"])
    Y1 = ctx.decompress(img)  # an image wherever a container is accepted
    assert torch.equal(Y0.view(torch.int32), Y1.view(torch.int32))


def test_context_option_end_to_end(lcp, orc):
    X = synth.cosmology(1 << 16, 2)
    ctx = lcp.Context(0)
    plain = host(ctx.compress(torch.from_numpy(X).cuda(), 1.0, "abs", 8)["bytes"])
    assert plain == orc.compress_s(X, 1.0, "abs", 8)["bytes"]
    ctx.set_dict(True)
    r = ctx.compress(torch.from_numpy(X).cuda(), 1.0, "abs", 8)
    img = orc.dict_compress(plain)
    assert len(img) < len(plain) and host(r["bytes"]) == img
    n, d, m, fl = ctx.peek(r["bytes"])
    assert (n, d, m) == (1 << 16, 6, "spatial")
    vals = orc.decompress(plain)[0]
    Y = ctx.decompress(r["bytes"]).cpu().numpy()
    assert np.array_equal(Y.view(np.uint32), vals.view(np.uint32))
    Yh = ctx.decompress_host(r["bytes"].cpu(), out=torch.empty(6 << 16, dtype=torch.float32))
    assert np.array_equal(Yh.numpy().view(np.uint32), vals.view(np.uint32))
    # a small random frame: the image is kept only when shorter
    R = np.random.default_rng(4).random((3, 300), dtype=np.float32)
    c = orc.compress_s(R, 1e-5, "abs", 2)["bytes"]
    img = orc.dict_compress(c)
    small = host(ctx.compress(torch.from_numpy(R).cuda(), 1e-5, "abs", 2)["bytes"])
    assert small == (img if len(img) < len(c) else c)


def test_trajectory_images_step_and_random_access(lcp, orc):
    """A trajectory compressed with the option on: every frame is the
    oracle's container or its image; the step decoder (images one by one)
    and random access through anchors and LCP-T chains equal the oracle."""
    from oracle import hybrid
    sizes = [20011, 3001]
    N, B = 8, 4
    frames = [list(synth.brownian_trajectory(n, N, 100 + k, sigma=0.02))
              for k, n in enumerate(sizes)]
    enc = [hybrid.encode_trajectory(fr, 1e-3, "abs", 8, batch=B) for fr in frames]
    dec = [hybrid.decode_trajectory([b for b, _ in e]) for e in enc]
    ctx = lcp.Context(0)
    ctx.set_dict(True)
    trs = [lcp.Trajectory(ctx, batch=B, p=8) for _ in sizes]
    bufs = [[], []]
    for t in range(N):
        for k in range(len(sizes)):
            r = ctx.compress(torch.from_numpy(frames[k][t]).cuda(), 1e-3, "abs", 8,
                             method="auto", traj=trs[k])
            c = enc[k][t][0]
            img = orc.dict_compress(c)
            assert host(r["bytes"]) == (img if len(img) < len(c) else c), (k, t)
            bufs[k].append(r["bytes"].clone())
    assert any(host(b)[:4] == b"LCPZ" for bb in bufs for b in bb)
    plain = lcp.Context(0)
    step = lcp.Step(plain, max_frames=4)
    dtr = [lcp.Trajectory(plain, batch=B, p=8) for _ in sizes]
    outs = [torch.empty((3, n), dtype=torch.float32, device="cuda") for n in sizes]
    for t in range(N):
        res = step.decompress([dict(buf=bufs[k][t], size=bufs[k][t].numel(), traj=dtr[k],
                                    out=outs[k]) for k in range(len(sizes))])
        for k in range(len(sizes)):
            assert res[k]["status"] == lcp.OK, (k, t)
            assert np.array_equal(outs[k].cpu().numpy().view(np.uint32),
                                  dec[k][t].view(np.uint32)), (k, t)
    step.close()
    for t in (N - 1, 2, 5):
        Y = plain.decompress_frame(bufs[0], t, batch=B)
        assert np.array_equal(Y.cpu().numpy().view(np.uint32), dec[0][t].view(np.uint32)), t


def test_status_codes(lcp, orc):
    ctx = lcp.Context(0)
    raw = b"abcabcabcabcX" * 100
    src = dev(raw)
    small = torch.empty(64, dtype=torch.uint8, device="cuda")
    with pytest.raises(lcp.LcpError) as ei:
        ctx.dict_compress(src, len(raw), out=small)
    assert ei.value.status == lcp.ERR_CAPACITY
    img = orc.dict_compress(raw)
    with pytest.raises(lcp.LcpError) as ei:
        ctx.dict_decompress(dev(img), len(img), out=torch.empty(100, dtype=torch.uint8,
                                                                device="cuda"))
    assert ei.value.status == lcp.ERR_CAPACITY
    # malformed images (the oracle rejects the same bytes): bad magic, offset
    # 0, offset beyond the output, copy past the chunk, size table and total
    one = orc.dict_compress(b"abcabcabcabcX")
    bad = []
    for at, v in [(3, ord("1")), (96 + 4, 0), (96 + 4, 4), (96, 0x3F), (80, 9), (80, 7),
                  (24, 96)]:
        b = bytearray(one)
        b[at] = v
        bad.append(bytes(b))
    for b in bad:
        with pytest.raises(orc.OracleError):
            orc.dict_decompress(b)
        with pytest.raises(lcp.LcpError) as ei:
            ctx.dict_decompress(dev(b), len(b))
        assert ei.value.status == lcp.ERR_FORMAT
        with pytest.raises(lcp.LcpError) as ei:
            ctx.decompress(dev(b), len(b), out=torch.empty((3, 16), dtype=torch.float32,
                                                            device="cuda"))
        assert ei.value.status == lcp.ERR_FORMAT
    # the context still works after the rejected images
    assert host(ctx.dict_compress(src, len(raw))) == orc.dict_compress(raw)
