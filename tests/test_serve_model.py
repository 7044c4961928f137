"""The serving loop's host-side bookkeeping, checked on the CPU: the ring
allocator that holds queued requests' LLRs and unpolled results (contiguous
allocations, wrap-around, release in allocation order), and the admission
model that predicts a subframe's completion (it recovers a known latency
law, leaves stalls out, moves by a bounded step on one batch of outliers,
follows a lasting slowdown, keeps its margin below a sixth of the deadline,
and recovers from a start that begins with stalled completions).  The checks
are a small C++ program (tests/serve_model_check.cpp) built against the
library's own header with the host compiler."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1905_01141_gb300", "csrc")


def test_serve_model(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path / "serve_model_check")
    subprocess.run([cxx, "-std=c++17", "-O2", "-I", CSRC, "-o", exe,
                    os.path.join(HERE, "serve_model_check.cpp")], check=True)
    out = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stdout + out.stderr
    assert "0 failures" in out.stdout
