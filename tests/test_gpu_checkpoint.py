"""Checkpoint and resume of a trajectory (lcp_traj_export / lcp_traj_import).

A trajectory restored from an image, on a fresh context, must code the
remaining frames into exactly the bytes the uninterrupted trajectory gives
(zero tolerance), and a restored decoder trajectory must decode the
remaining frames bit for bit as the uninterrupted one does.  Cut points
cover the middle, end and start of a batch; malformed images are rejected
on the host.
"""
import numpy as np
import pytest
import torch

from paper_2411_00761_b300 import synth

pytestmark = pytest.mark.gpu

N, STEPS, BATCH, EB, P = 30011, 12, 5, 1e-3, 8


@pytest.fixture(scope="module")
def lcp():
    from paper_2411_00761_b300 import lcp as L
    L.load()
    return L


@pytest.fixture(scope="module")
def frames():
    return list(synth.brownian_trajectory(N, STEPS, 21, sigma=0.02))


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def encode(lcp, ctx, tr, X):
    r = ctx.compress(dev(X), EB, "abs", P, method="auto", traj=tr)
    return r["bytes"].cpu().numpy().tobytes(), r["method"]


@pytest.fixture(scope="module")
def reference(lcp, frames):
    ctx = lcp.Context(0)
    tr = lcp.Trajectory(ctx, batch=BATCH, p=P)
    return [encode(lcp, ctx, tr, X) for X in frames]


@pytest.mark.parametrize("cut", [0, 3, 4, 5, 7])
def test_encoder_resumes_with_identical_bytes(lcp, frames, reference, cut):
    ctx = lcp.Context(0)
    tr = lcp.Trajectory(ctx, batch=BATCH, p=P)
    for t in range(cut + 1):
        assert encode(lcp, ctx, tr, frames[t]) == reference[t]
    image = tr.export()
    tr.close()
    ctx2 = lcp.Context(0)
    tr2 = lcp.Trajectory.restore(ctx2, image)
    for t in range(cut + 1, STEPS):
        assert encode(lcp, ctx2, tr2, frames[t]) == reference[t], t
    assert {m for _, m in reference} == {"spatial", "temporal"}


@pytest.mark.parametrize("cut", [2, 5, 8])
def test_decoder_resumes_bit_exact(lcp, reference, cut):
    ctx = lcp.Context(0)
    seq = lcp.Trajectory(ctx, batch=BATCH, p=P)
    ys = [ctx.decompress(dev(np.frombuffer(b, np.uint8)), traj=seq).cpu().numpy()
          for b, _ in reference]
    dt = lcp.Trajectory(ctx, batch=BATCH, p=P)
    for t in range(cut + 1):
        ctx.decompress(dev(np.frombuffer(reference[t][0], np.uint8)), traj=dt)
    dt2 = lcp.Trajectory.restore(lcp.Context(0), dt.export())
    for t in range(cut + 1, STEPS):
        y = dt2.ctx.decompress(dev(np.frombuffer(reference[t][0], np.uint8)), traj=dt2)
        assert np.array_equal(y.cpu().numpy().view(np.uint32), ys[t].view(np.uint32)), t


def test_malformed_images_are_rejected(lcp, frames):
    ctx = lcp.Context(0)
    fresh = lcp.Trajectory(ctx, batch=BATCH, p=P)
    img0 = fresh.export()
    assert len(img0) == 64
    lcp.Trajectory.restore(ctx, img0).close()
    tr = lcp.Trajectory(ctx, batch=BATCH, p=P)
    encode(lcp, ctx, tr, frames[0])
    img = tr.export()
    assert len(img) == 64 + 2 * (N * 3 * 4 + N * 4) + 2 * 3 * 80  # frames, grids
    for bad in (b"XXXX" + img[4:], img[:-4], img + b"\0"):
        with pytest.raises(lcp.LcpError) as ei:
            lcp.Trajectory.restore(ctx, bad)
        assert ei.value.status == lcp.ERR_FORMAT


# anchors written at eb / 5 (Sec. "Best error-bound scale for anchor frames"):
# a cut right after a scaled anchor, before the frame that predicts from it,
# must restore the anchor's grid and its scaled flag
SCALE = 5


@pytest.fixture(scope="module")
def scaled(lcp, frames):
    from oracle import hybrid
    enc = hybrid.encode_trajectory(frames, EB, "abs", P, batch=BATCH, anchor_scale=SCALE)
    ctx = lcp.Context(0)
    tr = lcp.Trajectory(ctx, batch=BATCH, p=P, anchor_scale=SCALE)
    got = [encode(lcp, ctx, tr, X) for X in frames]
    assert [b for b, _ in got] == [b for b, _ in enc]
    flags = [hybrid.oracle.peek(b)["flags"] for b, _ in enc]
    # frames predicted from a scaled anchor (re-quantized reference)
    req = [t for t, f in enumerate(flags) if f & hybrid.FLAG_REF_REQUANT]
    assert req, "no frame predicts from a scaled anchor"
    return got, enc, req


def test_encoder_resumes_after_scaled_anchor(lcp, frames, scaled):
    got, enc, req = scaled
    for t_req in req:
        cut = t_req - 1  # the scaled reference is the last frame coded before the cut
        ctx = lcp.Context(0)
        tr = lcp.Trajectory(ctx, batch=BATCH, p=P, anchor_scale=SCALE)
        for t in range(cut + 1):
            assert encode(lcp, ctx, tr, frames[t]) == got[t]
        tr2 = lcp.Trajectory.restore(lcp.Context(0), tr.export())
        for t in range(cut + 1, STEPS):
            assert encode(lcp, tr2.ctx, tr2, frames[t])[0] == enc[t][0], (t_req, t)


def test_decoder_resumes_after_scaled_anchor(lcp, scaled):
    from oracle import hybrid
    got, enc, req = scaled
    dec = hybrid.decode_trajectory([b for b, _ in enc])
    for t_req in req:
        cut = t_req - 1
        ctx = lcp.Context(0)
        dt = lcp.Trajectory(ctx, batch=BATCH, p=P)
        for t in range(cut + 1):
            ctx.decompress(dev(np.frombuffer(enc[t][0], np.uint8)), traj=dt)
        dt2 = lcp.Trajectory.restore(lcp.Context(0), dt.export())
        for t in range(cut + 1, STEPS):
            y = dt2.ctx.decompress(dev(np.frombuffer(enc[t][0], np.uint8)), traj=dt2)
            assert np.array_equal(y.cpu().numpy().view(np.uint32), dec[t].view(np.uint32)), \
                (t_req, t)
