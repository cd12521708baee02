"""CPU check of the generated expansion kernels (forward and reverse mode):
tests/adj_harness.cpp compiles the generated headers as host code with
T = double and checks every reverse-mode kernel against central finite
differences of its forward kernel, or against the dot-product identity;
the packed FP32x2 kernels against the scalar FP32 ones bit for bit; and the
uniform-background terms against the oracle's expansion of a uniform cube."""
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))

pytestmark = pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    exe = str(tmp_path_factory.mktemp("harness") / "adj_harness")
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-o", exe, os.path.join(HERE, "adj_harness.cpp")])
    return exe


def test_generated_adjoint_kernels(harness):
    r = subprocess.run([harness], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.startswith("OK")


def test_background_terms_match_the_oracle_cube_expansion(harness):
    """The walk's generated order-4 and order-6 background terms of a unit
    cube of unit density (cube_bg_l4, cube_bg_l6 at q = 1) equal the order-4
    and order-6 terms of the oracle's multipole expansion of that cube
    (moments by or_cube_moments, Newtonian M2P by or_m2p_orders) outside its
    circumscribed sphere."""
    import oracle as O
    rng = np.random.default_rng(1)
    pts = rng.uniform(-3.0, 3.0, (60, 3))
    pts = pts[np.linalg.norm(pts, axis=1) > 1.0]
    r = subprocess.run([harness, "bg"], input="\n".join("%.17g %.17g %.17g" % tuple(p) for p in pts),
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    got = np.array([[float(v) for v in line.split()] for line in r.stdout.strip().split("\n")])
    assert got.shape == (len(pts), 6)
    M = O.cube_moments(1.0, 1.0, 6)
    for i, R in enumerate(pts):
        for k, l in enumerate((4, 6)):
            ref = O.m2p_orders(M, l, l, R, 0.0)
            assert np.abs(got[i, 3 * k:3 * k + 3] - ref).max() <= 1e-12 * np.abs(ref).max(), (l, R)
