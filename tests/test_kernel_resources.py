"""Resource limits the fused launch shapes rely on, checked from the
compiler's report (nvcc -Xptxas -v; no GPU needed): the one-tile fused
kernels (1-D and 2-D tiles of up to 16 rows) must fit two blocks of 256
threads on an SM (at most 128 registers a thread), which grids of 153 to 304
tiles need to keep their tiles resident (at 130 registers the 1-D 2^18-cell
solve fell to the multi-tile loop and took 2.54 ms instead of 2.01 ms), and
the window kernel is launched two blocks per SM (128 registers, no spills)."""
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2411_00742_gb300", "csrc")


def _ptxas_report(unit):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    cmd = [nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-Xptxas", "-v",
           "-I", os.path.join(ROOT, "include"), "-I", CSRC, "-c", os.path.join(CSRC, unit), "-o", os.devnull]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    # entry name -> (registers, spill store bytes); an entry's report is its
    # "Function properties for <entry>" block and the "Used ... registers"
    # line after it (device functions have properties blocks of their own)
    out, entry, cur = {}, None, None
    for line in r.stderr.splitlines():
        m = re.search(r"Compiling entry function '(\S+)'", line)
        if m:
            entry = cur = m.group(1)
            out[entry] = [None, 0]
            continue
        m = re.search(r"Function properties for (\S+)", line)
        if m:
            cur = m.group(1)
            continue
        m = re.search(r"(\d+) bytes spill stores", line)
        if m and entry and cur == entry:
            out[entry][1] = int(m.group(1))
        m = re.search(r"Used (\d+) registers", line)
        if m and entry:
            out[entry][0] = int(m.group(1))
    return out


def test_one_tile_fused_kernels_fit_two_blocks_per_sm():
    rep = _ptxas_report("pbe_fused.cu")
    one_tile = {k: v for k, v in rep.items() if re.search(r"k_fusedILi[12]ELb1ELi16E", k)}
    assert len(one_tile) == 2, sorted(rep)
    for k, (regs, spill) in one_tile.items():
        assert regs is not None and regs <= 128, (k, regs)
        assert spill == 0, (k, spill)


def test_window_kernel_fits_two_blocks_per_sm_without_spills():
    rep = _ptxas_report("pbe_window.cu")
    win = {k: v for k, v in rep.items() if "k_fused_win" in k}
    assert len(win) == 3, sorted(rep)
    for k, (regs, spill) in win.items():
        assert regs is not None and regs <= 128, (k, regs)
        assert spill == 0, (k, spill)
