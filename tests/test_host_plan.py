"""Host planning (csrc/plan.h) -- the split form's plain-FP32 integrals and the
ket lists of row batches with bra-ket symmetry -- compiled with the host
compiler and checked on seeded random classes."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_f32_tail_split(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path / "host_plan_check")
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", os.path.join(ROOT, "paper_2606_04316_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "host_plan_check.cpp"), "-o", exe], check=True, timeout=300)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stdout[-2000:]
