"""CPU check of the generated expansion kernels (forward and reverse mode):
tests/adj_harness.cpp compiles the generated headers as host code with
T = double and checks every reverse-mode kernel against central finite
differences of its forward kernel, or against the dot-product identity;
the packed FP32x2 kernels against the scalar FP32 ones bit for bit; the forward
P2M, M2P and M2M kernels against the oracle; the image field's M2L and L2P
against the oracle's exact Ewald derivatives (convergence at their order);
and the uniform-background terms against the oracle's expansion of a uniform
cube."""
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
    assert got.shape == (len(pts), 8)
    M = O.cube_moments(1.0, 1.0, 6)
    for i, R in enumerate(pts):
        for k, l in enumerate((4, 6)):
            ref = O.m2p_orders(M, l, l, R, 0.0)
            assert np.abs(got[i, 3 * k:3 * k + 3] - ref).max() <= 1e-12 * np.abs(ref).max(), (l, R)
            pref = O.m2p_pot(M, l, l, R, 0.0)  # the potential forms
            # (scale: the term's size |a| |R|, as the angular factor can nearly vanish)
            assert abs(got[i, 6 + k] - pref) <= 1e-12 * max(abs(pref), np.abs(ref).max() * np.linalg.norm(R)), (l, R)


@pytest.mark.parametrize("p", [0, 1, 2, 3, 4])
def test_forward_expansion_kernels_match_the_oracle(harness, p):
    """The walk's generated forward kernels compiled as host FP64 code: P2M
    moments of a few particles, the M2P acceleration of their reduced
    moments (softened) and the M2M shift to a parent centre equal the
    oracle's p2m, m2p and m2m."""
    import oracle as O
    rng = np.random.default_rng(40 + p)
    for case in range(4):
        k = int(rng.integers(1, 12))
        d = rng.uniform(-0.5, 0.5, (k, 3))
        m = rng.uniform(0.5, 1.5, k)
        R = rng.uniform(-3.0, 3.0, 3)
        R *= (1.2 + 2.0 * rng.uniform()) / np.linalg.norm(R)
        eps = float(rng.choice([0.0, 0.01, 0.2]))
        sh = 0.25 * rng.choice([-1.0, 1.0], 3)
        inp = ("%d\n%d\n" % (p, k) + "\n".join("%.17g %.17g %.17g %.17g" % (m[i], *d[i]) for i in range(k))
               + "\n%.17g %.17g %.17g %.17g %.17g %.17g %.17g\n" % (*R, eps, *sh))
        r = subprocess.run([harness, "io"], input=inp, capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
        v = np.array([float(x) for x in r.stdout.split()])
        nm = O.nmom(p)
        assert len(v) == 2 * nm + 4
        Mo = O.p2m(d, m, np.zeros(3), p)
        ao = O.m2p(Mo, p, R, eps)
        Mpo = O.m2m(Mo, sh, np.zeros(3), p)
        po = O.m2p_pot(Mo, 0, p, R, eps)
        assert np.abs(v[:nm] - Mo).max() <= 1e-14 * np.abs(Mo).max()
        assert np.abs(v[nm:nm + 3] - ao).max() <= 1e-13 * np.abs(ao).max()
        assert np.abs(v[nm + 3:2 * nm + 3] - Mpo).max() <= 1e-14 * np.abs(Mpo).max()
        # the potential form (m2pot) from the same coefficients
        assert abs(v[-1] - po) <= 1e-13 * abs(po)


@pytest.mark.parametrize("pe", [1, 2, 3, 4, 5])
def test_image_field_expansion_converges_at_its_order(harness, pe):
    """The walk's generated image-field M2L and L2P, compiled as host FP64
    code, for a unit point source at offset delta from its cell centre and a
    sink at offset d from the expansion point, with the oracle's exact Ewald
    derivatives of phi~ at R0 = e - c*: the result is the Taylor expansion of
    -grad phi~(R0 + d - delta) to total order pe in the two offsets, so its
    error against the oracle's exact value falls as h^(pe+1) when both
    offsets scale with h.  A wrong coefficient of any order k <= pe would
    leave an error falling only as h^k."""
    import oracle as O
    R0 = np.array([0.3, 0.2, -0.25])
    u = np.array([0.6, -0.5, 0.62])
    w = np.array([-0.3, 0.8, 0.52])
    u /= np.linalg.norm(u)
    w /= np.linalg.norm(w)
    mi = O.multi_indices(pe)
    D = O.phitilde_mi(R0, pe + 1)
    errs, perrs = [], []
    for h in (0.08, 0.04, 0.02, 0.01):
        delta, d = h * u, 0.7 * h * w
        M = np.array([delta[0] ** n[0] * delta[1] ** n[1] * delta[2] ** n[2] for n in mi])
        inp = ("%d\n" % pe + "\n".join("%.17g" % v for v in M) + "\n" + "\n".join("%.17g" % v for v in D)
               + "\n%.17g %.17g %.17g\n" % tuple(d))
        r = subprocess.run([harness, "field"], input=inp, capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
        v = np.array([float(x) for x in r.stdout.split()])
        a = v[:3]
        exact = -O.phitilde_mi(R0 + d - delta, 1)[1:4]
        errs.append(np.linalg.norm(a - exact) / np.linalg.norm(exact))
        # the potential series (m2l0 + l2pot) against phi~ itself: the same
        # order (the order-(pe+1) moment term it lacks is the same at every sink)
        perrs.append(abs(v[3] - O.phitilde_mi(R0 + d - delta, 0)[0]))
    assert errs[2] <= 0.02 * 0.3 ** (pe - 1)
    for i in range(2):
        assert errs[i] / errs[i + 1] >= 0.8 * 2 ** (pe + 1), (pe, errs)
    # (the potential's two leading error orders nearly cancel at the larger
    # offsets for some pe: its rate is checked on the two smallest)
    assert perrs[2] / perrs[3] >= 0.75 * 2 ** (pe + 1), (pe, perrs)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_dual_form_kernels_match_the_oracle(harness, p):
    """The walk's generated derivative tensor of the softened kernel (by the
    Cartesian recurrence) against the oracle's Hermite-product form, and its
    generated cell-group M2L (one local coefficient at a time) followed by
    the L2P against the oracle's or_m2l / or_l2p, in FP64 on the host."""
    import oracle
    rng = np.random.default_rng(40 + p)
    for _ in range(6):
        c = rng.uniform(-0.1, 0.1, 3)
        pts = c + 0.05 * rng.standard_normal((12, 3))
        M = oracle.p2m(pts, rng.uniform(0.5, 1.5, 12), c, p)
        R = rng.uniform(0.4, 1.0, 3) * rng.choice([-1, 1], 3)
        eps = 10 ** rng.uniform(-3, -1)
        d = 0.1 * rng.standard_normal(3)
        inp = "%d\n%s\n%s\n%.17g\n%s\n" % (p, " ".join("%.17g" % v for v in M), " ".join("%.17g" % v for v in R),
                                          eps, " ".join("%.17g" % v for v in d))
        r = subprocess.run([harness, "dual"], input=inp, capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
        out = np.array([float(v) for v in r.stdout.split()])
        nd = oracle.nmom(p + 1)
        D, a = out[:nd], out[nd:]
        Dref = oracle.dtensor(R, eps, p + 1)
        order = np.array([sum(m) for m in oracle.multi_indices(p + 1)])
        for o in range(p + 2):
            sc = np.abs(Dref[order == o]).max()
            assert np.abs(D[order == o] - Dref[order == o]).max() <= 1e-13 * sc, (p, o)
        aref = oracle.l2p(oracle.m2l(M, p, R, eps), p, d)
        assert np.abs(a - aref).max() <= 1e-13 * np.abs(aref).max(), (p, a, aref)
