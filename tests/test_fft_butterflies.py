"""The register butterflies of the FFT convolution (radix 8, 16, 32 and their
pruned forms for zero-padded inputs, csrc/fft.cuh) compiled for the host and
checked against the DFT definition in double precision.  FP32 arithmetic on
unit-variance inputs: worst error per sqrt(N) well below 1e-6."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _cuda_include():
    for cand in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if cand and os.path.exists(os.path.join(cand, "include", "cuda_runtime.h")):
            return os.path.join(cand, "include")
    return None


def test_butterflies_match_dft(tmp_path):
    cxx = shutil.which("g++")
    inc = _cuda_include()
    if not cxx or not inc:
        pytest.skip("needs g++ and the CUDA headers")
    exe = tmp_path / "fft_butterflies"
    src = os.path.join(ROOT, "tests", "fft_butterflies_host.cpp")
    build = subprocess.run([cxx, "-std=c++17", "-O1", "-w", "-x", "c++", "-I", inc, "-I",
                            os.path.join(ROOT, "paper_1708_01663_gb300", "csrc"), "-I", os.path.join(ROOT, "include"),
                            src, "-o", str(exe)], capture_output=True, text=True)
    assert build.returncode == 0, build.stderr[-2000:]
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    rows = [line.split() for line in out if line.strip()]
    assert len(rows) == 9
    for name, direction, err in rows:
        assert float(err) < 1e-6, (name, direction, err)
