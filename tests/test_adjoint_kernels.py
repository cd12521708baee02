"""CPU check of the generated expansion kernels (forward and reverse mode):
tests/adj_harness.cpp compiles the generated headers as host code with
T = double and checks every reverse-mode kernel against central finite
differences of its forward kernel, or against the dot-product identity."""
import os
import shutil
import subprocess
import tempfile

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")
def test_generated_adjoint_kernels():
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "adj_harness")
        subprocess.check_call(["g++", "-O1", "-std=c++17", "-o", exe, os.path.join(HERE, "adj_harness.cpp")])
        r = subprocess.run([exe], capture_output=True, text=True)
        assert r.returncode == 0, r.stdout + r.stderr
        assert r.stdout.startswith("OK")
