"""Resource guard for the kernels of the 512^3 hot path (CPU only: nvcc
cross-compiles for sm_103a).  ptxas reports each kernel's stack frame and
spills; a change that pushes a hot kernel's values into local memory shows up
here before any GPU run.  Bound: no spill in the row kernels and the n0 column
kernel; at most 16 bytes in the row-pair n1 kernel (its measured state, at
92 % of the copy bandwidth)."""
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1406_5597_gb300", "csrc")


def _nvcc():
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    return None


@pytest.fixture(scope="module")
def spills(tmp_path_factory):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc is not available")
    out = tmp_path_factory.mktemp("ptxas") / "inst_256_512.o"
    r = subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
                        "--expt-relaxed-constexpr", "-Xcompiler", "-fPIC", "-I" + os.path.join(ROOT, "include"),
                        "-I" + CSRC, "-Xptxas", "-v", "-c", os.path.join(CSRC, "inst_256_512.cu"), "-o", str(out)],
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    res, fn = {}, None
    for line in r.stderr.splitlines():
        m = re.search(r"Function properties for (\S+)", line)
        if m:
            fn = m.group(1)
            continue
        m = re.search(r"(\d+) bytes stack frame, (\d+) bytes spill stores, (\d+) bytes spill loads", line)
        if m and fn:
            res[fn] = (int(m.group(1)), int(m.group(2)), int(m.group(3)))
            fn = None
    assert res, "no ptxas report parsed"
    return res


def _find(spills, pattern):
    hits = {k: v for k, v in spills.items() if re.search(pattern, k)}
    assert hits, pattern
    return hits


def test_row_kernels_of_the_512_path_do_not_spill(spills):
    for pat in (r"row_r2c_warp_kernelILi256ELi16ELi4E", r"row_c2r_warp_kernelILi256ELi16ELi4E"):
        for k, (frame, st, ld) in _find(spills, pat).items():
            assert st == 0 and ld == 0, (k, st, ld)


def test_n0_column_kernel_does_not_spill(spills):
    # col_tma_kernel<512, 32, DIR, 16, 2, 0, PAIR = false, XB = true>, both directions
    hits = _find(spills, r"col_tma_kernelILi512ELi32EL[in]*1ELi16ELi2ELi0ELb0ELb1E")
    assert len(hits) == 2
    for k, (frame, st, ld) in hits.items():
        assert st == 0 and ld == 0, (k, st, ld)


def test_row_pair_column_kernel_spills_at_most_16_bytes(spills):
    hits = _find(spills, r"col_tma_kernelILi512ELi32EL[in]*1ELi16ELi2ELi2ELb1ELb1E")
    assert len(hits) == 2
    for k, (frame, st, ld) in hits.items():
        assert st <= 16 and ld <= 16, (k, st, ld)
