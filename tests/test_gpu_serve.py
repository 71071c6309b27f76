"""The request loop (lcp_server_*).

A frame's container is identical whether it is compressed alone or served
among other producers' requests (zero tolerance); a served decompression of
any retained earlier frame (random access through its batch and anchor)
equals the oracle's sequential decode of the stream bit for bit; frames a
queued decompression needs survive eviction until it is served; admission
by the device-memory budget, per-request statuses and request-level faults
are host-side checks that leave the GPU and the server usable.
"""
import numpy as np
import pytest
import torch

from paper_2411_00761_b300 import synth

pytestmark = pytest.mark.gpu

BATCH, EB, P = 5, 1e-3, 8


@pytest.fixture(scope="module")
def lcp():
    from paper_2411_00761_b300 import lcp as L
    L.load()
    return L


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_served_frames_equal_alone_and_random_access_decode(lcp):
    sizes = [4001, 25013, 9000]
    n_frames = 13
    traj = [list(synth.brownian_trajectory(n, n_frames, 200 + k, sigma=0.02))
            for k, n in enumerate(sizes)]
    from oracle import hybrid
    # alone: containers, and the oracle's sequential decode of each stream
    ctx = lcp.Context(0)
    alone, decoded = [], []
    for k, frames in enumerate(traj):
        tr = lcp.Trajectory(ctx, batch=BATCH, p=P)
        cs = []
        for X in frames:
            r = ctx.compress(dev(X), EB, "abs", P, method="auto", traj=tr)
            cs.append(r["bytes"].cpu().numpy().tobytes())
        alone.append(cs)
        decoded.append(hybrid.decode_trajectory(cs))
    srv = lcp.Server(lanes=3, batch=BATCH)
    try:
        Xs = [[dev(X) for X in frames] for frames in traj]
        outs = [[torch.empty(lcp.max_compressed_size(n, 3), dtype=torch.uint8, device="cuda")
                 for _ in range(n_frames)] for n in sizes]
        tickets = []
        for t in range(n_frames):  # producers interleaved, every frame submitted at once
            for k in range(len(sizes)):
                tickets.append((k, t, srv.submit_compress(k, Xs[k][t], EB, "abs", P,
                                                          out=outs[k][t])))
        for k, t, tk in tickets:
            r = srv.wait(tk)
            assert r["status"] == lcp.OK and r["frame"] == t
            assert outs[k][t][: r["size"]].cpu().numpy().tobytes() == alone[k][t], (k, t)
            assert r["done_ms"] >= r["start_ms"] >= r["enqueue_ms"]
        # random access: every decodable frame, in a shuffled order
        rng = np.random.default_rng(0)
        reqs = []
        for k, n in enumerate(sizes):
            first, nxt = srv.frames(k)
            assert nxt == n_frames and first < nxt
            for f in rng.permutation(np.arange(first, nxt)):
                Y = torch.empty((3, n), dtype=torch.float32, device="cuda")
                reqs.append((k, int(f), Y, srv.submit_decompress(k, int(f), Y)))
        for k, f, Y, tk in reqs:
            r = srv.wait(tk)
            assert r["status"] == lcp.OK and r["frame"] == f
            assert np.array_equal(Y.cpu().numpy().view(np.uint32),
                                  decoded[k][f].view(np.uint32)), (k, f)
    finally:
        srv.close()


def test_pinned_frames_survive_eviction(lcp):
    """One lane, kept busy by a large frame of another producer while a
    producer queues compressions that will evict its oldest frames and then a
    decompression of its oldest frame: that frame and its chain are pinned at
    admission, so the request is served after the evictions and equals the
    oracle's decode; afterwards the frame is no longer retained."""
    from oracle import hybrid
    n, total = 3001, 4 * BATCH + 3
    frames = list(synth.brownian_trajectory(n, total, 77, sigma=0.02))
    big = dev(synth.uniform_clusters(1 << 22, 5))
    srv = lcp.Server(lanes=1, batch=BATCH)
    try:
        outs = [torch.empty(lcp.max_compressed_size(n, 3), dtype=torch.uint8, device="cuda")
                for _ in range(total)]
        sizes = []
        for t in range(2 * BATCH):
            r = srv.wait(srv.submit_compress(3, dev(frames[t]), EB, "abs", P, out=outs[t]))
            assert r["status"] == lcp.OK
            sizes.append(r["size"])
        first, _ = srv.frames(3)
        busy = srv.submit_compress(4, big, EB, "abs", P)  # the lane is taken
        comp_t = [srv.submit_compress(3, dev(frames[t]), EB, "abs", P, out=outs[t])
                  for t in range(2 * BATCH, total)]
        Y = torch.empty((3, n), dtype=torch.float32, device="cuda")
        dec_t = srv.submit_decompress(3, first, Y)  # pinned before any eviction
        assert srv.wait(busy)["status"] == lcp.OK
        for tk in comp_t:
            r = srv.wait(tk)
            assert r["status"] == lcp.OK
            sizes.append(r["size"])
        r = srv.wait(dec_t)
        assert r["status"] == lcp.OK and r["frame"] == first
        cs = [outs[t][:sizes[t]].cpu().numpy().tobytes() for t in range(total)]
        dec = hybrid.decode_trajectory(cs)
        assert np.array_equal(Y.cpu().numpy().view(np.uint32), dec[first].view(np.uint32))
        assert srv.frames(3)[0] > first  # evicted once the request let go of it
    finally:
        srv.close()


def test_admission_by_memory_budget(lcp):
    X = dev(synth.uniform_clusters(200000, 3))
    srv = lcp.Server(lanes=1, batch=BATCH, hbm_budget=16 << 20)  # 16 MiB
    try:
        # its reference state (~19 MB) and worst-case container (~14 MB) do not fit
        assert srv.submit_compress(0, X, EB, "abs", P) is None
    finally:
        srv.close()
    srv = lcp.Server(lanes=1, batch=BATCH, hbm_budget=8 << 30)
    try:
        t = srv.submit_compress(0, X, EB, "abs", P)
        assert t is not None and srv.wait(t)["status"] == lcp.OK
        assert 0 < srv.device_bytes() <= 8 << 30
    finally:
        srv.close()


def test_request_faults_are_reported_and_the_server_keeps_going(lcp):
    srv = lcp.Server(lanes=2, batch=BATCH)
    try:
        X = dev(synth.uniform_clusters(5000, 1))
        t = srv.submit_compress(7, X, EB, "abs", P)
        assert srv.wait(t)["status"] == lcp.OK
        # a frame of another shape for the same producer: refused at submission
        with pytest.raises(lcp.LcpError) as ei:
            srv.submit_compress(7, dev(synth.uniform_clusters(4000, 1)), EB, "abs", P)
        assert ei.value.status == lcp.ERR_STATE
        # a frame that was never coded: refused at submission
        Y = torch.empty((3, 5000), dtype=torch.float32, device="cuda")
        with pytest.raises(lcp.LcpError) as ei:
            srv.submit_decompress(7, 99, Y)
        assert ei.value.status == lcp.ERR_STATE
        # a non-finite input: reported, and the producer's next frame still codes
        Xbad = X.clone()
        Xbad[1, 17] = float("nan")
        assert srv.wait(srv.submit_compress(7, Xbad, EB, "abs", P))["status"] == lcp.ERR_NONFINITE
        t2 = srv.submit_compress(7, X, EB, "abs", P)
        r2 = srv.wait(t2)
        assert r2["status"] == lcp.OK and r2["frame"] == 1
        # a ticket is answered once
        with pytest.raises(lcp.LcpError):
            srv.wait(t2)
    finally:
        srv.close()
