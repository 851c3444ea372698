"""Host logic of batching, on CPU: three cloths of different sizes (one pinned)
are prepared and merged exactly as dc_create_batch / dc_set_params_batch do, and
a C++ harness built from the library's host sources checks the layout
invariants (node maps, instance ranges, triangles, fronts and their levels,
supernodal panels)."""
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2106_05306_gb300", "csrc")
CUDA_INC = "/usr/local/cuda/include"


def test_batch_layout_invariants():
    cxx = shutil.which("g++")
    if cxx is None or not os.path.isdir(CUDA_INC):
        pytest.skip("needs g++ and the CUDA headers")
    srcs = [os.path.join(ROOT, "tests", "host", "merge_check.cpp")] + [
        os.path.join(CSRC, f) for f in ("dc_setup.cpp", "dc_frontal_setup.cpp", "dc_merge.cpp")]
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "merge_check")
        subprocess.check_call([cxx, "-std=c++17", "-O1", "-I", CSRC, "-I", os.path.join(ROOT, "include"),
                               "-I", CUDA_INC, *srcs, "-o", exe])
        out = subprocess.check_output([exe], timeout=120).decode()
    assert out.startswith("ok"), out
