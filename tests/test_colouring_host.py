"""The conflict-free, colour-ordered assembly rules of the cell kernels
(first writer of every node, colours that share no node, boundary flags),
checked on the CPU over 1..13 cells per direction, p = 1..8, Dirichlet and
periodic: tests/colouring_check.cu includes the kernels' own host-callable
helpers, is compiled by nvcc for the host and run here (no GPU)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_colour_ordered_assembly_rules(tmp_path):
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if nvcc is None:
        pytest.skip("nvcc not found")
    exe = str(tmp_path / "colouring_check")
    src = os.path.join(ROOT, "tests", "colouring_check.cu")
    inc = ["-I", os.path.join(ROOT, "include"), "-I", os.path.join(ROOT, "paper_2208_07129_gb300", "csrc")]
    r = subprocess.run([nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-gencode", "arch=compute_103a,code=sm_103a",
                        *inc, src, "-o", exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    out = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0 and out.stdout.strip() == "ok", out.stdout + out.stderr
