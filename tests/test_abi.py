"""The C-ABI library loads and exports every entry point include/lcp.h
declares (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "lcp.h")).read()
    return sorted(set(re.findall(r"LCP_API[^;(]*?\b(lcp_\w+)\s*\(", src)))


def test_header_declares_entry_points():
    names = declared()
    for must in ("lcp_compress", "lcp_decompress", "lcp_select", "lcp_ctx_create",
                 "lcp_traj_create", "lcp_quantize", "lcp_max_compressed_size"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_2411_00761_b300 import build
    lib_path = build.build()
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing
    # the binding knows every declared entry point
    from paper_2411_00761_b300 import lcp
    assert sorted(lcp.SIGNATURES) == declared()


def test_max_compressed_size_matches_oracle(orc):
    from paper_2411_00761_b300 import lcp
    for n, d in [(0, 1), (1, 3), (1000, 3), (12345, 6), (1 << 20, 8)]:
        assert lcp.max_compressed_size(n, d) == orc.max_compressed_size(n, d)


def test_binding_fails_loudly_without_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    from paper_2411_00761_b300 import lcp
    with pytest.raises(RuntimeError):
        lcp.Context(0)


def test_job_and_request_structs_match_the_header(tmp_path):
    """The binding's ctypes structs (batch jobs, server requests and
    responses) have the C layout: sizes and field offsets from the header
    compiled by gcc."""
    import subprocess
    from paper_2411_00761_b300 import lcp
    probe = tmp_path / "probe.c"
    structs = (("lcp_compress_job", lcp.CompressJob), ("lcp_decompress_job", lcp.DecompressJob),
               ("lcp_request", lcp.Request), ("lcp_response", lcp.Response))
    fields = {st: [f for f, _ in cls._fields_] for st, cls in structs}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "lcp.h"', "int main(void) {"]
    for st, fs in fields.items():
        lines.append(f'  printf("{st} %zu\\n", sizeof({st}));')
        for f in fs:
            lines.append(f'  printf("{st}.{f} %zu\\n", offsetof({st}, {f}));')
    lines += ["  return 0;", "}"]
    probe.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(probe), "-o", str(exe)],
                   check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                  check=True).stdout.splitlines())
    for st, cls in structs:
        assert int(got[st]) == ctypes.sizeof(cls), st
        for f, _ in cls._fields_:
            assert int(got[f"{st}.{f}"]) == getattr(cls, f).offset, (st, f)
