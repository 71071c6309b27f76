"""Batched frames (lcp_compress_batch / lcp_decompress_batch).

Every frame's bytes must be identical whether it is compressed alone or in a
batch whose lanes run other frames at the same time (zero tolerance), and a
batched decode must give the frames a sequential decode gives.  One of the
trajectories is also checked against the oracle's Algorithm 1 directly.
"""
import numpy as np
import pytest
import torch

from paper_2411_00761_b300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lcp():
    from paper_2411_00761_b300 import lcp as L
    L.load()
    return L


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host_bytes(r):
    return r["bytes"].cpu().numpy().tobytes()


SIZES = [3001, 20011, 777, 65536, 12000]  # uneven trajectories
N_STEPS, BATCH, EB, P = 12, 5, 1e-3, 8


def trajectories():
    return [list(synth.brownian_trajectory(n, N_STEPS, 100 + k, sigma=0.02))
            for k, n in enumerate(SIZES)]


def test_batched_trajectories_equal_alone(lcp):
    frames = trajectories()
    # alone: one context, one trajectory per sequence, one frame per call
    ctx = lcp.Context(0)
    alone = []
    for tr_frames in frames:
        tr = lcp.Trajectory(ctx, batch=BATCH, p=P)
        seq = []
        for X in tr_frames:
            r = ctx.compress(dev(X), EB, "abs", P, method="auto", traj=tr)
            seq.append((host_bytes(r), r["method"]))
        alone.append(seq)
    # batched: three lanes, every time step's frames in one call
    lanes = lcp.Lanes(3)
    trs = [lcp.Trajectory(lanes.ctxs[0], batch=BATCH, p=P) for _ in SIZES]
    outs = [torch.empty(lcp.max_compressed_size(n, 3), dtype=torch.uint8, device="cuda")
            for n in SIZES]
    batched = [[] for _ in SIZES]
    for t in range(N_STEPS):
        Xs = [dev(frames[k][t]) for k in range(len(SIZES))]
        res = lanes.compress([dict(X=Xs[k], eb=EB, mode="abs", p=P, method="auto", traj=trs[k],
                                   out=outs[k]) for k in range(len(SIZES))])
        for k, r in enumerate(res):
            assert r["status"] == lcp.OK
            batched[k].append((host_bytes(r), r["method"]))
    for k in range(len(SIZES)):
        for t in range(N_STEPS):
            assert batched[k][t][1] == alone[k][t][1], (k, t)
            assert batched[k][t][0] == alone[k][t][0], (k, t)
    # both methods occurred (the FSM tested LCP-T somewhere)
    assert {m for seq in batched for _, m in seq} == {"spatial", "temporal"}


def test_batched_trajectory_matches_oracle(lcp, orc):
    from oracle import hybrid
    n = SIZES[1]
    frames = list(synth.brownian_trajectory(n, N_STEPS, 101, sigma=0.02))
    enc = hybrid.encode_trajectory(frames, EB, "abs", P, batch=BATCH)
    lanes = lcp.Lanes(2)
    tr = lcp.Trajectory(lanes.ctxs[0], batch=BATCH, p=P)
    out = torch.empty(lcp.max_compressed_size(n, 3), dtype=torch.uint8, device="cuda")
    out2 = torch.empty(lcp.max_compressed_size(1000, 3), dtype=torch.uint8, device="cuda")
    for t, X in enumerate(frames):
        side = dev(synth.uniform_clusters(1000, t))  # a stateless frame beside it
        res = lanes.compress([dict(X=dev(X), eb=EB, p=P, method="auto", traj=tr, out=out),
                              dict(X=side, eb=EB, p=P, method="spatial", traj=None, out=out2)])
        assert host_bytes(res[0]) == enc[t][0], t
        assert res[0]["method"] == {"S": "spatial", "T": "temporal"}[enc[t][1]], t
        assert host_bytes(res[1]) == orc.compress_s(synth.uniform_clusters(1000, t), EB, "abs",
                                                    P)["bytes"], t


def test_batched_decode_equals_sequential(lcp):
    frames = trajectories()
    lanes = lcp.Lanes(4)
    enc_trs = [lcp.Trajectory(lanes.ctxs[0], batch=BATCH, p=P) for _ in SIZES]
    dec_trs = [lcp.Trajectory(lanes.ctxs[0], batch=BATCH, p=P) for _ in SIZES]
    ctx = lcp.Context(0)
    seq_trs = [lcp.Trajectory(ctx, batch=BATCH, p=P) for _ in SIZES]
    outs = [torch.empty(lcp.max_compressed_size(n, 3), dtype=torch.uint8, device="cuda")
            for n in SIZES]
    Ys = [torch.empty((3, n), dtype=torch.float32, device="cuda") for n in SIZES]
    for t in range(N_STEPS):
        res = lanes.compress([dict(X=dev(frames[k][t]), eb=EB, p=P, method="auto",
                                   traj=enc_trs[k], out=outs[k]) for k in range(len(SIZES))])
        dres = lanes.decompress([dict(buf=outs[k], size=res[k]["size"], traj=dec_trs[k], out=Ys[k])
                                 for k in range(len(SIZES))])
        for k in range(len(SIZES)):
            assert dres[k]["status"] == lcp.OK and dres[k]["n"] == SIZES[k] and dres[k]["d"] == 3
            Y_seq = ctx.decompress(res[k]["bytes"], traj=seq_trs[k]).cpu().numpy()
            assert np.array_equal(Ys[k].cpu().numpy().view(np.uint32), Y_seq.view(np.uint32)), \
                (k, t)


def test_batch_reports_per_job_status(lcp):
    lanes = lcp.Lanes(2)
    X = dev(synth.uniform_clusters(5000, 1))
    out = torch.empty(lcp.max_compressed_size(5000, 3), dtype=torch.uint8, device="cuda")
    out_b = torch.empty_like(out)
    jobs = [dict(X=X, eb=EB, p=P, out=out), dict(X=X, eb=EB, p=3, out=out_b)]  # p not a power of 2
    with pytest.raises(lcp.LcpError) as ei:
        lanes.compress(jobs)
    assert ei.value.status == lcp.ERR_ARG
    # the valid job still completed with the bytes it has alone
    ctx = lcp.Context(0)
    alone = host_bytes(ctx.compress(X, EB, "abs", P))
    arr_ok = lanes.compress([dict(X=X, eb=EB, p=P, out=out)])
    assert host_bytes(arr_ok[0]) == alone


@pytest.mark.parametrize("scale,nlanes", [(1, 0), (5, 0), (1, 3)])
def test_step_decode_equals_oracle(lcp, orc, scale, nlanes):
    """lcp_decompress_step: every time step's frames decoded together (LCP-T
    frames in one persistent launch replayed as a CUDA graph, the others one
    by one) equal the oracle's sequential decode of each trajectory bit for
    bit; with anchor scaling the frames predicted from a scaled anchor take
    the one-by-one path.  The decoder state afterwards equals a sequential
    decoder's (checkpoint images compared).  With lanes, the frames the step
    does not fuse (the LCP-S anchors) are spread over them."""
    from oracle import hybrid
    frames = trajectories()
    enc = [hybrid.encode_trajectory(fr, EB, "abs", P, batch=BATCH, anchor_scale=scale)
           for fr in frames]
    dec = [hybrid.decode_trajectory([b for b, _ in e]) for e in enc]
    assert any(m == "T" for e in enc for _, m in e)
    ctx = lcp.Context(0)
    lanes = lcp.Lanes(nlanes) if nlanes else None
    step = lcp.Step(ctx, max_frames=len(SIZES), lanes=lanes)
    trs = [lcp.Trajectory(ctx, batch=BATCH, p=P) for _ in SIZES]
    seq = [lcp.Trajectory(ctx, batch=BATCH, p=P) for _ in SIZES]
    outs = [torch.empty((3, n), dtype=torch.float32, device="cuda") for n in SIZES]
    for t in range(N_STEPS):
        bufs = [dev(np.frombuffer(enc[k][t][0], np.uint8)) for k in range(len(SIZES))]
        res = step.decompress([dict(buf=bufs[k], size=bufs[k].numel(), traj=trs[k], out=outs[k])
                               for k in range(len(SIZES))])
        for k in range(len(SIZES)):
            assert res[k]["status"] == lcp.OK and res[k]["n"] == SIZES[k], (k, t)
            assert np.array_equal(outs[k].cpu().numpy().view(np.uint32),
                                  dec[k][t].view(np.uint32)), (k, t)
            ctx.decompress(bufs[k], traj=seq[k])
    for k in range(len(SIZES)):
        assert trs[k].export() == seq[k].export(), k
    step.close()
