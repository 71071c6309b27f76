"""The binary32 reconstruction rule of the decode kernels (codes below 2^23),
restated on the host in tests/q2_round_to_odd.c, equals the oracle's exact
Q2 (Eq. quantization) bit for bit: on random (m, e, q) over the whole
binary32 range of bounds and minima, and on values built to land exactly on
rounding ties.  The GPU parity tests check the kernels themselves on frames;
this checks the rule on far more inputs than frames reach."""
import ctypes as C
import shutil
import subprocess

import numpy as np
import pytest

import oracle


@pytest.fixture(scope="module")
def ro(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    import os
    src = os.path.join(os.path.dirname(__file__), "q2_round_to_odd.c")
    lib = str(tmp_path_factory.mktemp("q2ro") / "libq2ro.so")
    subprocess.check_call([cc, "-O1", "-frounding-math", "-fno-fast-math", "-ffp-contract=off",
                           "-shared", "-fPIC", "-o", lib, src, "-lm"])
    L = C.CDLL(lib)
    L.q2_ro_many.argtypes = [C.c_void_p, C.c_size_t, C.c_float, C.c_float, C.c_void_p,
                             C.c_void_p]
    return L


def run(ro, q, m, e):
    q = np.ascontiguousarray(q, dtype=np.int64)
    out = np.empty(q.size, dtype=np.float32)
    ok = np.empty(q.size, dtype=np.int32)
    ro.q2_ro_many(q.ctypes.data, q.size, C.c_float(m), C.c_float(e), out.ctypes.data,
                  ok.ctypes.data)
    return out, ok.astype(bool)


def test_random_bounds_and_minima(ro):
    rng = np.random.default_rng(2024)
    checked = 0
    for trial in range(1500):
        e = np.float32(np.ldexp(rng.uniform(1, 2), int(rng.integers(-100, 60))))
        kind = trial % 5
        if kind == 0:
            m = np.float32(0.0)
        elif kind == 1:
            m = np.float32(-rng.uniform(0, 1) * float(e) * float(rng.integers(1, 1 << 22)))
        elif kind == 2:
            m = np.float32(np.ldexp(rng.uniform(-2, 2), int(np.log2(float(e))) + int(rng.integers(-30, 40))))
        elif kind == 3:
            m = np.float32(np.ldexp(rng.uniform(-2, 2), int(rng.integers(-126, 100))))
        else:
            m = np.float32(-float(e) * float(rng.integers(0, 1 << 20)) * 2)  # on the grid
        if not np.isfinite(m):
            continue
        qmax = int(rng.choice([1000, 1 << 12, 1 << 16, (1 << 23) - 1]))
        q = rng.integers(0, qmax, size=200)
        q[:3] = [0, qmax - 1, qmax // 2]
        ref = oracle.q2(q, float(m), float(e))
        out, ok = run(ro, q, m, e)
        sel = ok & np.isfinite(ref)
        checked += int(sel.sum())
        assert np.array_equal(out[sel].view(np.uint32), ref[sel].view(np.uint32)), (m, e)
    assert checked > 250000


def test_exact_ties(ro):
    # m + (2q+1) e exactly halfway between two binary32 neighbours
    rng = np.random.default_rng(7)
    for trial in range(2000):
        E = int(rng.integers(-90, 60))
        if trial % 2:
            e = np.float32(np.ldexp(1.0, E))
        else:
            e = np.float32(np.ldexp(float(int(rng.integers(1 << 20, 1 << 21)) | 1), E - 20))
        m = np.float32(np.ldexp(float(int(rng.integers(-7, 8)) | 1), E - int(rng.integers(1, 4))))
        q = rng.integers(1 << 21, (1 << 23) - 1, size=64)
        ref = oracle.q2(q, float(m), float(e))
        out, ok = run(ro, q, m, e)
        assert ok.all()
        assert np.array_equal(out.view(np.uint32), ref.view(np.uint32)), (m, e)
