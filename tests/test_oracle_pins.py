"""Pins of the FP64 CPU oracle to facts outside itself (CPU only).

Each test checks the oracle against mathematics the paper's method rests on:
Ewald sums (alpha independence, symmetry zeros, the r -> 0 background limit,
the Madelung constant of the simple cubic lattice, harmonicity), exact
symmetry of direct summation (lattice, momentum), the multipole algebra
(M2M exactness, derivative tensors vs finite differences, one-particle
cells), convergence of the tree to direct summation, the integrator's
closed forms and linear growth, and the CIC loss gradient.
"""
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_1407_2600_gb300 import ics

RNG = np.random.default_rng(12345)


# ---- Ewald ---------------------------------------------------------------------
def test_ewald_alpha_independence():
    pts = RNG.uniform(-0.5, 0.5, (6, 3))
    for r in pts:
        a = [O.ewald_acc(r, O.ewald_cfg(al)) for al in (1.5, 2.0, 3.0)]
        scale = np.abs(a[1]).max()
        assert np.abs(a[0] - a[1]).max() <= 1e-12 * max(scale, 1.0)
        assert np.abs(a[2] - a[1]).max() <= 1e-12 * max(scale, 1.0)


def test_ewald_symmetry_zeros_and_parity():
    for r in ([0.5, 0, 0], [0.5, 0.5, 0], [0.5, 0.5, 0.5], [0, 0.5, 0.5]):
        assert np.abs(O.ewald_acc(np.array(r, float))).max() <= 1e-13
    r = np.array([0.21, -0.13, 0.34])
    a = O.ewald_acc(r)
    b = O.ewald_acc(r * np.array([-1, 1, 1]))
    assert abs(a[0] + b[0]) <= 1e-13 and abs(a[1] - b[1]) <= 1e-13 and abs(a[2] - b[2]) <= 1e-13
    c = O.ewald_acc(r[[1, 2, 0]])  # cubic symmetry: permuting axes permutes components
    assert np.abs(c - a[[1, 2, 0]]).max() <= 1e-12


def test_ewald_small_r_background_limit():
    # a_E - a_N -> +(4 pi / 3) r as r -> 0: the neutralising background's
    # repulsion; the lattice tidal term vanishes by cubic symmetry
    d = np.array([0.3, -0.5, 0.8])
    d /= np.linalg.norm(d)
    for h in (1e-2, 3e-3):
        r = h * d
        diff = O.ewald_acc(r) + r / h ** 3
        assert np.abs(diff / r - 4 * math.pi / 3).max() <= 5 * h ** 2 * 10


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _golden_lines(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]


def test_madelung_constant():
    # simple cubic lattice with neutralising background (literature value and
    # citation in tests/golden/madelung_simple_cubic.txt): the Coulomb-sign
    # regular part lim_{r->0} [psi(r) - 1/r] = -value, so for the oracle's
    # gravitational-sign potential lim_{r->0} [phi_E(r) + 1/r] = +value
    value = float(_golden_lines("madelung_simple_cubic.txt")[0][0])
    r = 1e-4 * np.array([1.0, 1.0, 1.0]) / math.sqrt(3.0)
    val = O.ewald_pot(r) + 1.0 / np.linalg.norm(r)
    assert abs(val - value) <= 1e-7


def test_oracle_matches_its_regression_fixture():
    """tests/golden/oracle_direct8.txt (written by make_oracle_fixture.py
    from the oracle alone): exact Ewald accelerations and the direct sum of
    eight particles are reproduced; a change here is a change of the
    oracle's arithmetic."""
    rows = _golden_lines("oracle_direct8.txt")
    ew = np.array([[float(v) for v in r[1:]] for r in rows if r[0] == "ewald"])
    for row in ew:
        a = O.ewald_acc(row[:3])
        assert np.abs(a - row[3:]).max() <= 1e-12 * np.abs(row[3:]).max()
    dr = np.array([[float(v) for v in r[1:]] for r in rows if r[0] == "direct"])
    acc = O.direct_forces(dr[:, 1:4], dr[:, 0], 0.02, table_n1=None)
    assert np.abs(acc - dr[:, 4:]).max() <= 1e-12 * np.abs(dr[:, 4:]).max()


def test_phitilde_consistency_and_harmonic():
    cfg = O.ewald_cfg()
    mi = O.multi_indices(5)
    idx = {m: i for i, m in enumerate(mi)}
    for r in RNG.uniform(-0.5, 0.5, (3, 3)):
        D = O.phitilde_mi(r, 5)
        # C~ = -grad phi~ equals a_E - a_N - (4 pi/3) r (independent code path)
        ae = O.ewald_acc(r)
        ct = ae + r / np.linalg.norm(r) ** 3 - 4 * math.pi / 3 * r
        assert np.abs(-D[1:4] - ct).max() <= 1e-11
        # phi~ is harmonic: every Laplacian-trace of its derivatives vanishes
        for m in mi:
            if sum(m) > 3:
                continue
            lap = sum(D[idx[tuple(m[k] + (2 if k == d else 0) for k in range(3))]] for d in range(3))
            assert abs(lap) <= 1e-8 * (1 + np.abs(D).max())
        # order-k derivatives are finite differences of order k-1
        h = 1e-5
        for d in range(3):
            e = np.zeros(3)
            e[d] = h
            Dp, Dm = O.phitilde_mi(r + e, 4), O.phitilde_mi(r - e, 4)
            for m in mi:
                if sum(m) > 4:
                    continue
                up = tuple(m[k] + (1 if k == d else 0) for k in range(3))
                fd = (Dp[idx[m]] - Dm[idx[m]]) / (2 * h)
                assert abs(fd - D[idx[up]]) <= 1e-5 * (1 + abs(D[idx[up]]))
        # the generic-order routine agrees with the explicit orders 0..3
        E = O.phitilde(r, cfg)
        assert np.abs(E[:4] - D[:4]).max() <= 1e-12 * (1 + np.abs(E).max())


# ---- O1 direct summation ------------------------------------------------------------
def test_direct_lattice_zero_and_momentum():
    q = ics.lattice(7)  # odd lattice: no pair sits exactly half a box apart
    a = O.direct_forces(q, None, 1.0 / 70, table_n1=None)
    assert np.abs(a).max() <= 1e-11
    x, eps = ics.config_small(3)
    a = O.direct_forces(x, None, eps, table_n1=64)
    assert np.abs(a.sum(axis=0)).max() <= 1e-13 * np.abs(a).sum(axis=0).max()


def test_direct_table_matches_exact_ewald():
    """The tricubic C~ table against the exact Ewald sum: its error falls as
    h^4 (about 16x per halving of the spacing) and is 3e-9 at the default
    128 intervals, six orders below the 1e-3 accuracy bar it is used to
    measure."""
    x, eps = ics.config_small(2)
    tg = ics.random_targets(len(x), 24, 2)
    a_ex = O.direct_forces(x, None, eps, targets=tg, table_n1=None)
    err = {}
    for n1 in (64, 128):
        a_tb = O.direct_forces(x, None, eps, targets=tg, table_n1=n1)
        err[n1] = (np.linalg.norm(a_ex - a_tb, axis=1) / np.linalg.norm(a_ex, axis=1)).max()
    assert err[128] <= 1e-8 and err[64] <= 1e-7, err
    assert err[64] >= 6 * err[128], err


def test_direct_pair_matches_definition():
    # two particles: a_1 = m_2 [a_E(r) - a_N(r*) + a_P(r*)]
    x = np.array([[0.1, 0.2, 0.3], [0.7, 0.25, 0.28]])
    eps = 0.02
    a = O.direct_forces(x, np.array([0.3, 0.7]), eps, table_n1=None)
    r = x[0] - x[1]
    rs = r - np.round(r)
    q = np.linalg.norm(rs)
    ref = 0.7 * (O.ewald_acc(r) + rs / q ** 3 - rs / (q * q + eps * eps) ** 1.5)
    assert np.abs(a[0] - ref).max() <= 1e-13
    assert np.abs(0.3 * a[0] + 0.7 * a[1]).max() <= 1e-13  # Newton's third law


def test_direct_plane_wave_linear_force():
    # small single-mode displacement on a lattice: force = 4 pi G rho psi up
    # to the lattice's discreteness correction, which falls as (k/k_Ny)^2
    ratios = []
    for ng in (8, 16):
        q = ics.lattice(ng)
        A = 1e-3 / ng
        x = q.copy()
        x[:, 0] += A * np.sin(2 * math.pi * q[:, 0])
        a = O.direct_forces(x, None, 1e-6, table_n1=64)
        pred = 4 * math.pi * A * np.sin(2 * math.pi * q[:, 0])
        i = int(np.argmax(np.abs(pred)))
        ratios.append(a[i, 0] / pred[i])
        assert np.abs(a[:, 1:]).max() <= 1e-5 * abs(pred[i])
    assert abs(ratios[1] - 1) <= 0.01
    assert 3.5 <= (ratios[0] - 1) / (ratios[1] - 1) <= 4.5


# ---- multipoles and tree ----------------------------------------------------------------
def test_m2m_exact():
    pts = RNG.uniform(0.1, 0.3, (40, 3))
    m = RNG.uniform(0.5, 1.5, 40)
    c, cp = np.array([0.2, 0.2, 0.2]), np.array([0.25, 0.15, 0.2])
    for p in range(5):
        direct = O.p2m(pts, m, cp, p)
        shifted = O.m2m(O.p2m(pts, m, c, p), c, cp, p)
        assert np.abs(direct - shifted).max() <= 1e-14 * np.abs(direct).max()


def test_dtensor_finite_differences():
    R = np.array([0.31, -0.22, 0.17])
    eps = 0.05
    mi = O.multi_indices(6)
    idx = {m: i for i, m in enumerate(mi)}
    D = O.dtensor(R, eps, 6)
    assert abs(D[0] - 1 / math.sqrt(R @ R + eps * eps)) <= 1e-15
    h = 1e-6
    for d in range(3):
        e = np.zeros(3)
        e[d] = h
        Dp, Dm = O.dtensor(R + e, eps, 5), O.dtensor(R - e, eps, 5)
        for m in mi:
            if sum(m) > 5:
                continue
            up = tuple(m[k] + (1 if k == d else 0) for k in range(3))
            fd = (Dp[idx[m]] - Dm[idx[m]]) / (2 * h)
            assert abs(fd - D[idx[up]]) <= 1e-6 * (1 + abs(D[idx[up]]))


def test_one_particle_cell_m2p_equals_p2p():
    c = np.array([0.5, 0.5, 0.5])
    y = np.array([[0.51, 0.49, 0.505]])  # one particle, (n, 3)
    x = np.array([0.8, 0.1, 0.6])
    eps = 0.01
    r = y[0] - x
    p2p = 0.7 * r / (r @ r + eps * eps) ** 1.5
    for p in (2, 4):
        M = O.p2m(y, np.array([0.7]), c, p)
        a = O.m2p(M, p, x - c, eps)
        # the expansion about c converges to the softened particle force
        assert np.abs(a - p2p).max() <= 5e-3 * np.abs(p2p).max() * (0.02 / 0.6) ** (p - 1)
    M = O.p2m(c[None, :], np.array([0.7]), c, 4)  # particle at the centre: exact
    assert np.abs(O.m2p(M, 4, x - c, eps) - 0.7 * (c - x) / ((c - x) @ (c - x) + eps * eps) ** 1.5).max() <= 1e-15


def _gauss_cube(s, k):
    """Gauss-Legendre nodes and weights (k per axis) on the cube [-s/2, s/2]^3."""
    t, w = np.polynomial.legendre.leggauss(k)
    t = 0.5 * s * t
    w = 0.5 * s * w
    X, Y, Z = np.meshgrid(t, t, t, indexing="ij")
    W = w[:, None, None] * w[None, :, None] * w[None, None, :]
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1), W.ravel()


def test_cube_moments_match_quadrature():
    """Moments of a uniform cube against Gauss-Legendre quadrature (exact for
    these polynomial degrees), for side and density not equal to 1."""
    s, rho = 0.37, 2.5
    y, w = _gauss_cube(s, 6)
    C_ = O.cube_moments(s, rho, 8)
    for t, (nx, ny, nz) in enumerate(O.multi_indices(8)):
        q = rho * np.sum(w * y[:, 0] ** nx * y[:, 1] ** ny * y[:, 2] ** nz)
        assert abs(C_[t] - q) <= 1e-14 * max(abs(q), rho * s ** 3 * (s / 2) ** (nx + ny + nz)), (nx, ny, nz)


def test_cube_expansion_converges_to_cube_field():
    """The Newtonian field of a uniform cube at an exterior point, by
    high-order quadrature, against its multipole series from the cube's
    moments: the error falls with every even order added (the odd orders
    vanish), so the background terms of the tree have the right sign and
    normalisation at each order."""
    s, rho = 0.25, 1.3
    y, w = _gauss_cube(s, 40)
    C_ = O.cube_moments(s, rho, 8)
    for R in (np.array([0.55, 0.21, 0.08]), np.array([0.4, 0.4, 0.35]), np.array([0.02, -0.61, 0.3])):
        d = y - R
        r = np.sqrt(np.sum(d * d, axis=1))
        exact = rho * np.sum((w / r ** 3)[:, None] * d, axis=0)
        errs = []
        for q in (0, 2, 4, 6, 8):
            a = O.m2p_orders(C_, 0, q, R, 0.0)
            errs.append(np.linalg.norm(a - exact) / np.linalg.norm(exact))
        # order 2 of a cube is isotropic and adds nothing to a Newtonian field
        assert abs(errs[1] - errs[0]) <= 1e-12
        assert errs[2] < 0.2 * errs[1] and errs[3] < 0.5 * errs[2] and errs[4] < 0.5 * errs[3], errs
        # the series converges outside the cube's circumscribed sphere
        assert errs[4] <= (math.sqrt(3.0) * s / 2 / np.linalg.norm(R)) ** 10, errs


def test_background_terms_cancel_a_lattice():
    """A perfect lattice feels no force.  The expansion error of the tree on
    it is the truncation error of each cell's uniform share, which the
    background terms remove: with them the residual force falls by more than
    an order of magnitude (a sign or factor error would not)."""
    ng = 16
    x = ics.lattice(ng)
    eps = 1.0 / (30 * ng)
    tg = ics.random_targets(len(x), 128, 5)
    scale = 4 * math.pi * 0.25 / ng  # force of a displacement of a quarter spacing
    res = {}
    for bg in (0, 4, 6):
        tp = O.tree_params(eps, 0.5, 2, n_direct=2, ewald=4, mac=0, ew_grid=4, bg=bg)
        res[bg] = np.median(np.linalg.norm(O.tree_forces(x, None, tp, targets=tg), axis=1)) / scale
    assert res[4] <= 0.1 * res[0] and res[6] <= 1.1 * res[4], res


def test_multistep_reduces_to_global_steps():
    """Block steps: with one rung (rmax = 0) the step is kdk_step; with every
    particle on the finest rung it is 2^rmax global steps on the tick grid;
    under a constant uniform field every particle's momentum changes by
    g K(a0, a1) whatever its rung (its kicks tile the step)."""
    rng = np.random.default_rng(3)
    x0 = rng.uniform(0, 1, (40, 3))
    p0 = rng.standard_normal((40, 3)) * 0.01
    force = lambda xx: -0.3 * (xx - 0.5)  # smooth position-dependent field
    g0 = force(x0)
    a0, a1 = 0.05, 0.07
    x1, p1, g1 = O.kdk_multistep(x0, p0, g0, np.zeros(40, int), a0, a1, 0, force)
    xr, pr, gr = O.kdk_step(x0, p0, g0, a0, a1, force)
    assert np.abs(x1 - xr).max() <= 1e-14 and np.abs(p1 - pr).max() <= 1e-14
    rmax = 2
    x1, p1, g1 = O.kdk_multistep(x0, p0, g0, np.full(40, rmax), a0, a1, rmax, force)
    xs, ps, gs = x0, p0, g0
    for k in range(1 << rmax):
        xs, ps, gs = O.kdk_step(xs, ps, gs, O.tick_a(a0, a1, rmax, 2 * k), O.tick_a(a0, a1, rmax, 2 * k + 2), force)
    assert np.abs(x1 - xs).max() <= 1e-14 and np.abs(p1 - ps).max() <= 1e-14
    gc = np.array([0.3, -0.2, 0.1])
    const = lambda xx: np.broadcast_to(gc, xx.shape).copy()
    rung = rng.integers(0, rmax + 1, 40)
    x1, p1, g1 = O.kdk_multistep(x0, p0, const(x0), rung, a0, a1, rmax, const)
    assert np.abs(p1 - (p0 + gc * O.kick_factor(a0, a1))).max() <= 1e-15
    # rung assignment: 4^r >= q at the smallest r, capped
    g = np.array([[1.0, 0, 0], [4.0, 0, 0], [4.001, 0, 0], [1e6, 0, 0]], dtype=np.float32)
    c = 1.0 / ((0.5 ** 2) * O.H0 ** 2 * 1.0)
    # q = |g| dlna^2 / (eta^2 H0^2 eps) with dlna = 1, eta = 0.5, eps = 1
    r = O.assign_rungs(g, 1.0, 0.5, 1.0, 5)
    q = np.array([1.0, 4.0, 4.001, 1e6]) * c
    want = [min(5, int(np.ceil(np.log(v) / np.log(4.0) - 1e-12))) if v > 1 else 0 for v in q]
    assert list(r) == want, (list(r), want)


def test_tree_topology_invariants():
    x, _ = ics.config_haloes(16, seed=4, n_halo=3, nmin=100, nmax=400)
    key, lev, st, ct = O.tree_cells(x, n_leaf=8)
    n = len(x)
    assert ct[0] == n and lev[0] == 0
    # cells of one level are disjoint and sorted; a cell's count equals its prefix range
    okeys = O.morton_keys(x)[O.sort_perm(O.morton_keys(x))]
    for c in range(0, len(key), 7):
        l = int(lev[c])
        pre = int(key[c]) ^ (1 << (3 * l))
        span = okeys[st[c]:st[c] + ct[c]] >> np.uint64(3 * (21 - l)) if l > 0 else np.zeros(ct[c], np.uint64)
        assert np.all(span == np.uint64(pre))
    # leaves: no cell may have a child if it has <= n_leaf particles
    for l in range(int(lev.max())):
        par = (lev == l) & (ct <= 8)
        kids = lev == l + 1
        pk = set((key[par] ^ np.uint64(0)).tolist())
        kp = set(((key[kids] >> np.uint64(3))).tolist())
        assert not (pk & kp)


def test_tree_converges_to_direct():
    x, eps = ics.config_small(1)
    ad = O.direct_forces(x, None, eps, table_n1=64)

    def med(th, p):
        at = O.tree_forces(x, None, O.tree_params(eps, th, p, ewald=4))
        return np.median(np.linalg.norm(at - ad, axis=1) / np.linalg.norm(ad, axis=1))

    # with no cell accepted only the image-field expansion remains
    assert med(1e-3, 2) <= 1e-4
    # truncation error of an order-p expansion falls at least like theta^(p+1)
    assert med(0.6, 2) / med(0.3, 2) >= 2 ** 3
    assert med(0.9, 4) / med(0.45, 4) >= 2 ** 5


def test_face_distance_mac_meets_quadrupole_bar():
    """Opening distance measured from the cell faces (mac = 1): at theta 0.5
    with quadrupole moments the small box meets median <= 1e-3 and 99th
    percentile <= 1e-2 against the direct Ewald sum, where the centre
    distance (mac = 0) does not; the face test opens at least as much."""
    x, eps = ics.config_small(1)
    ad = O.direct_forces(x, None, eps, table_n1=64)
    out = {}
    for mac in (0, 1):
        at, st = O.tree_forces(x, None, O.tree_params(eps, 0.5, 2, ewald=4, mac=mac), return_stats=True)
        r = np.linalg.norm(at - ad, axis=1) / np.linalg.norm(ad, axis=1)
        out[mac] = (np.median(r), np.percentile(r, 99), st["p2p"] + st["m2p"])
    assert out[1][0] <= 1e-3 and out[1][1] <= 1e-2, out[1]
    assert out[0][0] > 1e-3, out[0]
    assert out[1][2] >= out[0][2]


def test_face_distance_mac_at_scale_setting():
    """The 512^3 scale workload's setting (P ~ k^-1.5, rms displacement 0.25
    spacing, theta 0.7, hexadecapole, opening distance from the cell faces,
    uniform-background terms, accepted cells of <= 8 particles summed
    directly, groups inside level-4 cells) on a 64^3 box of the same
    spectrum: median error against the direct Ewald sum <= 1e-3 (1.9e-4
    here), where the distance from the cell centre gives more (2.9e-3 here).
    The centre test's error grows with the particle number on this
    near-uniform box (3.4e-3, 7.7e-3, 2.1e-2, 4.7e-2 at 64^3 to 512^3 over
    256 targets); the face test's grows more slowly (2.1e-4 to 1.05e-3) and
    with the background terms stays at 3.7e-4 at 512^3 (2.5e-4 at 128^3,
    3.2e-4 at 256^3).  Those sizes take the direct sum minutes to an hour,
    so only the 64^3 case is a test."""
    q, psi = ics.zeldovich_particles(64, -1.5, 0.25, 3)
    x = np.mod(q + psi, 1.0)
    x[x >= 1.0] = 0.0
    eps = 1.0 / (30 * 64)
    tg = ics.random_targets(len(x), 128, 5)
    ad = O.direct_forces(x, None, eps, targets=tg, table_n1=128)
    med = {}
    for mac, bg in ((0, 0), (1, 6)):
        at = O.tree_forces(x, None, O.tree_params(eps, 0.7, 4, n_direct=8, ewald=4, ew_grid=5, mac=mac, bg=bg),
                           targets=tg)
        med[mac, bg] = np.median(np.linalg.norm(at - ad, axis=1) / np.linalg.norm(ad, axis=1))
    assert med[1, 6] <= 1e-3, med
    assert med[0, 0] > 1e-3, med


def test_image_field_order_convergence():
    x, eps = ics.config_small(6)
    ad = O.direct_forces(x, None, eps, table_n1=64)
    med = []
    for pe in (1, 2, 4):
        at = O.tree_forces(x, None, O.tree_params(eps, 1e-3, 2, ewald=pe))
        med.append(np.median(np.linalg.norm(at - ad, axis=1) / np.linalg.norm(ad, axis=1)))
    assert med[0] > med[1] > med[2]


def test_image_field_converges_at_every_order():
    """With negligible softening and no cell accepted (theta -> 0) the tree
    differs from the exact direct Ewald sum only by the image field's local
    expansion: its error falls by about ten per order p_E = 2..5 on an 8^3
    box (3.8e-4, 3.0e-5, 2.2e-6, 2.1e-7), so a wrong term of any order
    would stall it."""
    q, psi = ics.zeldovich_particles(8, -2.0, 0.25, 6)
    x = np.mod(q + psi, 1.0)
    eps = 1e-6
    ad = O.direct_forces(x, None, eps, table_n1=None)
    med = []
    for pe in (2, 3, 4, 5):
        at = O.tree_forces(x, None, O.tree_params(eps, 1e-3, 2, ewald=pe))
        med.append(np.median(np.linalg.norm(at - ad, axis=1) / np.linalg.norm(ad, axis=1)))
    for k in range(3):
        assert med[k + 1] <= med[k] / 5, med
    assert med[3] <= 1e-6, med


# ---- O3 integrator ---------------------------------------------------------------
def test_kick_drift_factors_quadrature():
    from scipy.integrate import quad
    a0, a1 = 0.05, 0.2
    H = lambda a: O.H0 * a ** -1.5
    k = quad(lambda a: 1.0 / (a * a * H(a)), a0, a1, epsabs=0, epsrel=2e-14)[0]
    d = quad(lambda a: 1.0 / (a ** 3 * H(a)), a0, a1, epsabs=0, epsrel=2e-14)[0]
    assert abs(O.kick_factor(a0, a1) - k) <= 1e-13 * k
    assert abs(O.drift_factor(a0, a1) - d) <= 1e-13 * d


def test_linear_growth_second_order():
    # with the linear-theory force g = 4 pi (x - q) the growing mode is D = a
    q = np.full((1, 3), 0.5)
    psi = np.array([[1e-3, -2e-3, 5e-4]])
    errs = []
    for S in (8, 16):
        a0, a1 = 0.05, 0.1
        x, p = O.zeldovich_state(q, psi, a0)
        force = lambda xx: 4 * math.pi * (xx - 0.5)
        g = force(x)
        al = a0 * np.exp(np.arange(S + 1) * math.log(a1 / a0) / S)
        for k in range(S):
            x, p, g = O.kdk_step(x, p, g, al[k], al[k + 1], force)
        errs.append(np.abs((x - 0.5) / psi / a1 - 1).max())
    assert errs[1] <= 1e-3
    assert 3.5 <= errs[0] / errs[1] <= 4.5


# ---- CIC loss and the direct adjoint ---------------------------------------------------------
def test_cic_loss_and_gradient():
    ng = 8
    q = ics.lattice(ng)
    L, g = O.cic_loss(q, None, ng)  # particles at cell centres: delta = 0
    assert L <= 1e-20 and np.abs(g).max() <= 1e-12
    x = np.mod(q + 0.03 * RNG.standard_normal(q.shape), 1.0)
    L, g = O.cic_loss(x, None, ng)
    h = 1e-7
    for i in (0, 17, 300):
        for d in range(3):
            xp, xm = x.copy(), x.copy()
            xp[i, d] += h
            xm[i, d] -= h
            fd = (O.cic_loss(xp, None, ng)[0] - O.cic_loss(xm, None, ng)[0]) / (2 * h)
            assert abs(fd - g[i, d]) <= 1e-5 * (1 + abs(g[i, d]))


def test_direct_vjp_dot_product():
    x = np.mod(ics.lattice(4) + 0.02 * RNG.standard_normal((64, 3)), 1.0)
    eps = 0.02
    v = RNG.standard_normal(x.shape)
    w = RNG.standard_normal(x.shape)
    h = 1e-6
    jv = (O.direct_forces(x + h * v, None, eps, table_n1=64) -
          O.direct_forces(x - h * v, None, eps, table_n1=64)) / (2 * h)
    jtw = O.direct_vjp(x, w, None, eps, n1=64)
    assert abs(np.sum(jv * w) - np.sum(v * jtw)) <= 1e-4 * abs(np.sum(jv * w))


# ---- keys and sort, by hand -------------------------------------------------------------
def test_morton_keys_hand_computed():
    """Keys of hand-placed points, worked out by hand (no call to the oracle
    to get them) in the layout the tree rests on: q_d = floor(x_d 2^21) mod
    2^21, and bit b of q_x, q_y, q_z goes to key bit 3b, 3b+1, 3b+2.  A
    swapped axis, an interleave off by one or a quantisation that rounds
    instead of flooring fails one of these."""
    u = 2.0 ** -21
    cases = [
        ((0.5, 0.0, 0.0), 1 << 60),                    # q_x = 2^20: bit 20 -> key bit 60
        ((0.0, 0.5, 0.0), 1 << 61),                    # q_y = 2^20 -> key bit 61
        ((0.0, 0.0, 0.5), 1 << 62),                    # q_z = 2^20 -> key bit 62
        ((u, 0.0, 0.0), 1),                            # q_x = 1
        ((0.0, 3 * u, 0.0), 0b10010),                  # q_y = 0b11: key bits 1 and 4
        ((0.75, 0.25, 0.125), (1 << 60) | (1 << 58) | (1 << 57) | (1 << 56)),
        # q_x = floor(3 - 2^-39) = 2 (bit 1 -> key bit 3); q_z = 0b101 (key bits 2, 8)
        ((3 * u - 2.0 ** -60, 0.0, 5 * u), 8 + 4 + 256),
        ((1.0, 0.0, 0.0), 0),                          # x = 1 wraps to 0
        ((-u, 0.0, 0.0), 0x1249249249249249),          # q_x = 2^21 - 1: every x bit
        ((0.0, 1.0 - u, 0.0), 0x2492492492492492),     # q_y = 2^21 - 1: every y bit
        ((0.0, 0.0, 1.0 - 0.5 * u), 0x4924924924924924),  # q_z = floor(2^21 - 1/2)
        ((1.0 - u, 1.0 - u, 1.0 - u), 0x7FFFFFFFFFFFFFFF),
        ((2.25, -0.75, 0.0), (1 << 57) | (1 << 58)),   # wrapped: 0.25 and 0.25
    ]
    pts = np.array([c[0] for c in cases], dtype=np.float64)
    want = np.array([c[1] for c in cases], dtype=np.uint64)
    got = O.morton_keys(pts)
    assert np.array_equal(got, want), [(i, hex(int(g)), hex(int(w))) for i, (g, w) in enumerate(zip(got, want))
                                      if g != w]


def test_sort_perm_hand_computed():
    """Stable key order of a hand-written key list: equal keys keep their
    input order."""
    keys = np.array([5, 3, 5, 1, 3, 0x7FFFFFFFFFFFFFFF, 0, 3], dtype=np.uint64)
    assert O.sort_perm(keys).tolist() == [6, 3, 1, 4, 7, 0, 2, 5]


# ---- the reverse mode of a KDK trajectory -------------------------------------------------
def test_adjoint_kdk_matches_central_differences():
    """adjoint_kdk over three KDK steps of the direct Ewald forces against
    FP64 central differences of the same trajectory (kdk_step driven by
    direct_forces with the exact Ewald sum, g(x0) recomputed from x0).  The
    functional is F = <w_x, x_S> + <w_p, p_S>, so its cotangents are
    (w_x, w_p); <lam_x0, v> + <lam_p0, u> must equal dF along (v, u).  Which
    state each force VJP uses and where K1, K2 and D enter all change the
    result by far more than the 1e-6 allowed."""
    rng = np.random.default_rng(77)
    q = ics.lattice(3)                                  # 27 particles at (i + 1/2)/3
    psi = 0.04 * rng.standard_normal(q.shape)
    a_list = [0.1, 0.15, 0.22, 0.3]
    eps = 0.05
    x0, p0 = O.zeldovich_state(q, psi, a_list[0])
    force = lambda x: O.direct_forces(x, None, eps, table_n1=None)

    def run(x, p):
        xs, ps = [x], [p]
        g = force(x)
        for k in range(len(a_list) - 1):
            x, p, g = O.kdk_step(x, p, g, a_list[k], a_list[k + 1], force)
            xs.append(x)
            ps.append(p)
        return xs, ps

    xs, ps = run(x0, p0)
    wx = rng.standard_normal(q.shape)
    wp = rng.standard_normal(q.shape)
    lx0, lp0 = O.adjoint_kdk(xs, ps, a_list, wx, wp, None, eps, n1=None)
    h = 1e-6
    for _ in range(3):
        v = rng.standard_normal(q.shape)
        u = rng.standard_normal(q.shape)
        xp, pp = run(x0 + h * v, p0 + h * u)
        xm, pm = run(x0 - h * v, p0 - h * u)
        # unwrapped final positions: no particle crosses the box edge here
        fd = (np.sum(wx * (xp[-1] - xm[-1])) + np.sum(wp * (pp[-1] - pm[-1]))) / (2 * h)
        ad = np.sum(lx0 * v) + np.sum(lp0 * u)
        assert abs(fd - ad) <= 1e-6 * abs(ad), (fd, ad)
    # the chaining matters: reversing with the VJPs at swapped states is far off
    assert np.abs(lx0 - O.adjoint_kdk(xs[::-1][:1] + xs[1:], ps, a_list, wx, wp, None, eps,
                                      n1=None)[0]).max() > 1e-4 * np.abs(lx0).max()


# ---- Dehnen's K1 softening kernel --------------------------------------------------------
def _k1_density(x):
    """The K1 kernel's density for eps = 1, written from its definition: the
    quadratic kernel 1 - x^2 times (5 - 9 x^2), normalised to unit mass."""
    return 105.0 / (64.0 * math.pi) * (1.0 - x * x) * (5.0 - 9.0 * x * x)


def test_k1_kernel_mass_second_moment_and_newtonian_exterior():
    """The oracle's K1 pair factor against quadrature of the kernel's density:
    the enclosed mass M(x) = int_0^x 4 pi s^2 rho ds equals x^3 f(x) (Gauss's
    law, eps = 1) at every radius, the total mass is 1, the second moment
    int 4 pi s^4 rho ds vanishes (what makes the kernel compensating), the
    field is exactly Newtonian from eps on, and the force is continuous with a
    continuous slope at eps."""
    xg, wg = np.polynomial.legendre.leggauss(40)
    for x in (0.1, 0.3, 0.5, 0.77, 0.95, 1.0):
        s = 0.5 * x * (xg + 1.0)
        m = 0.5 * x * np.sum(wg * 4.0 * math.pi * s * s * _k1_density(s))
        assert abs(m - x ** 3 * O.soft_factor(x * x, 1.0, 1)) <= 1e-13, x
    s = 0.5 * (xg + 1.0)
    assert abs(0.5 * np.sum(wg * 4.0 * math.pi * s ** 2 * _k1_density(s)) - 1.0) <= 1e-13
    assert abs(0.5 * np.sum(wg * 4.0 * math.pi * s ** 4 * _k1_density(s))) <= 1e-13
    eps = 0.02
    for r in (eps, 1.5 * eps, 0.3):
        assert O.soft_factor(r * r, eps, 1) == 1.0 / (r * r * r)
    h = 1e-6
    g = lambda r: r * O.soft_factor(r * r, eps, 1)  # force magnitude per unit mass
    assert abs(g(eps * (1 - h)) - g(eps)) <= 3 * h * g(eps)  # continuous: changes at first order in h
    slope_in = (g(eps) - g(eps * (1 - h))) / (eps * h)
    slope_out = (g(eps * (1 + h)) - g(eps)) / (eps * h)
    assert abs(slope_in - slope_out) <= 1e-4 * abs(slope_out)


def test_k1_direct_sum_is_newtonian_beyond_eps_and_tree_converges():
    """With K1 softening the direct Ewald sum of particles farther apart than
    eps equals the unsoftened one (Plummer with negligible eps); and the tree
    with K1 pairs and Newtonian expansions converges to the K1 direct sum as
    theta -> 0."""
    rng = np.random.default_rng(5)
    x = np.array([[0.2, 0.3, 0.4], [0.45, 0.31, 0.38], [0.8, 0.1, 0.9]])
    a1 = O.direct_forces(x, None, 0.05, table_n1=None, kernel=1)
    a0 = O.direct_forces(x, None, 1e-9, table_n1=None, kernel=0)
    assert np.abs(a1 - a0).max() <= 1e-12 * np.abs(a0).max()
    x, eps = ics.config_small(4)
    eps = 4 * eps  # enough pairs inside eps to matter
    ad = O.direct_forces(x, None, eps, table_n1=128, kernel=1)
    ap = O.direct_forces(x, None, eps, table_n1=128, kernel=0)
    assert np.median(np.linalg.norm(ad - ap, axis=1) / np.linalg.norm(ad, axis=1)) > 1e-4  # the kernels differ
    at = O.tree_forces(x, None, O.tree_params(eps, 1e-3, 2, ewald=5, kernel=1))
    rel = np.linalg.norm(at - ad, axis=1) / np.linalg.norm(ad, axis=1)
    assert np.median(rel) <= 1e-4, np.median(rel)


# ---- the dual (cell-group) form -----------------------------------------------------------
def test_m2l_at_the_expansion_point_is_m2p_and_converges_at_its_order():
    """The local expansion of a cell's field about z, evaluated at z, is the
    cell's M2P there (same derivative orders); for a point mass at the cell
    centre it is the Taylor series of the softened force to order p in the
    offset d, so its error falls as |d|^(p+1)."""
    rng = np.random.default_rng(9)
    c = np.array([0.3, 0.5, 0.45])
    pts = c + 0.02 * rng.standard_normal((40, 3))
    m = rng.uniform(0.5, 1.5, 40)
    z = np.array([0.62, 0.41, 0.5])
    eps = 0.003
    for p in range(5):
        M = O.p2m(pts, m, c, p)
        L = O.m2l(M, p, z - c, eps)
        a = O.l2p(L, p, np.zeros(3))
        ref = O.m2p(M, p, z - c, eps)
        assert np.abs(a - ref).max() <= 1e-13 * np.abs(ref).max(), p
    M = np.zeros(O.nmom(4))
    M[0] = 1.0
    u = rng.standard_normal(3)
    u /= np.linalg.norm(u)
    for p in (2, 4):
        Mp = M[:O.nmom(p)]
        L = O.m2l(Mp, p, z - c, eps)
        errs = []
        for h in (0.02, 0.01):
            x = z + h * u
            r = c - x
            exact = r / (r @ r + eps * eps) ** 1.5
            errs.append(np.linalg.norm(O.l2p(L, p, x - z) - exact))
        assert 2 ** (p + 1) * 0.8 <= errs[0] / errs[1] <= 2 ** (p + 1) * 1.25, (p, errs)


def test_dual_tree_accuracy_and_work():
    """The dual form on a clustered box (48^3 Zel'dovich + NFW haloes, theta
    0.6, hexadecapole): cell-group local expansions replace most M2P
    interactions (fewer than half remain), the force error against the
    direct Ewald sum stays within 25 % of the M2P tree's, and the dual tree
    converges to the direct sum as theta falls."""
    import bench
    x, _, eps = bench.workload(3, 48)
    tg = ics.random_targets(len(x), 128, 5)
    ad = O.direct_forces(x, None, eps, targets=tg, table_n1=128)
    med = {}
    for dual in (0, 1):
        a, st = O.tree_forces(x, None, O.tree_params(eps, 0.6, 4, n_direct=8, ewald=4, ew_grid=5, dual=dual),
                              targets=tg, return_stats=True)
        med[dual] = np.median(np.linalg.norm(a - ad, axis=1) / np.linalg.norm(ad, axis=1))
        if dual:
            m2p_dual, m2l = st["m2p"], st["m2l"]
        else:
            m2p_plain = st["m2p"]
    assert m2l > 0 and m2p_dual < 0.5 * m2p_plain, (m2p_dual, m2p_plain, m2l)
    assert med[1] <= 1.25 * med[0], med
    errs = []
    for th in (0.4, 0.2):
        a = O.tree_forces(x, None, O.tree_params(eps, th, 4, n_direct=8, ewald=5, ew_grid=5, dual=1), targets=tg)
        errs.append(np.median(np.linalg.norm(a - ad, axis=1) / np.linalg.norm(ad, axis=1)))
    assert errs[1] < errs[0] < med[1], (errs, med)


# ---- potentials ---------------------------------------------------------------------------
def test_soft_pot_from_the_densities_and_the_force():
    """The softened pair potentials against their definitions elsewhere: the
    K1 potential is the potential of its density by quadrature,
    phi(r) = -M(r)/r - int_r^eps 4 pi s rho(s) ds (eps = 1), so phi(0) =
    -105/32; both kernels give -1/r beyond the support (Plummer
    asymptotically), and each potential's radial slope is r times the pair
    factor of the force (finite differences)."""
    xg, wg = np.polynomial.legendre.leggauss(40)
    for r in (1e-9, 0.2, 0.5, 0.8, 0.99):
        s = 0.5 * r * (xg + 1.0)
        mass = 0.5 * r * np.sum(wg * 4.0 * math.pi * s * s * _k1_density(s))
        s = r + 0.5 * (1.0 - r) * (xg + 1.0)
        outer = 0.5 * (1.0 - r) * np.sum(wg * 4.0 * math.pi * s * _k1_density(s))
        assert abs(O.soft_pot(r * r, 1.0, 1) - (-mass / r - outer)) <= 1e-12, r
    assert abs(O.soft_pot(0.0, 1.0, 1) + 105.0 / 32.0) <= 1e-14
    eps = 0.02
    for r in (eps, 2 * eps, 0.3):
        assert O.soft_pot(r * r, eps, 1) == -1.0 / r
    assert abs(O.soft_pot(1.0, 1e-4, 0) + 1.0) <= 1e-8
    h = 1e-6
    for k in (0, 1):
        for r in (0.3 * eps, 0.9 * eps, 1.7 * eps):
            slope = (O.soft_pot((r + h * eps) ** 2, eps, k) - O.soft_pot((r - h * eps) ** 2, eps, k)) / (2 * h * eps)
            assert abs(slope - r * O.soft_factor(r * r, eps, k)) <= 1e-7 * abs(slope), (k, r)


def _lattice(k):
    g = (np.arange(k) + 0.5) / k
    return np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)


def test_direct_pot_madelung_lattice_and_two_particles():
    """The direct potential of a simple cubic lattice of k^3 equal masses
    (total mass 1) is the single-particle periodic potential of a box of side
    1/k: phi = m k xi with xi the Madelung constant of the golden fixture
    (exact Ewald sum and the tricubic phi~ table).  For two particles with
    negligible softening it is m_2 phi_E(r_12) + m_1 xi, phi_E the Ewald
    potential (zero-mean convention) evaluated by its own routine."""
    xi = float(_golden_lines("madelung_simple_cubic.txt")[0][0])
    for k in (4, 5):
        x = _lattice(k)
        n = len(x)
        want = xi * k / n
        assert np.abs(O.direct_pot(x, None, 1e-9, table_n1=None) - want).max() <= 1e-9 * want
        assert np.abs(O.direct_pot(x, None, 1e-9, table_n1=128) - want).max() <= 1e-7 * want
    x = np.array([[0.1, 0.2, 0.3], [0.55, 0.05, 0.9]])
    m = np.array([0.7, 1.9])
    pot = O.direct_pot(x, m, 0.0, table_n1=None)
    r = x[0] - x[1]
    assert abs(pot[0] - (m[1] * O.ewald_pot(r) + m[0] * xi)) <= 1e-9
    assert abs(pot[1] - (m[0] * O.ewald_pot(-r) + m[1] * xi)) <= 1e-9


def test_direct_pot_gradient_is_minus_the_direct_force():
    """phi_i depends on x_i only through its pairs (its own images and the
    background give a constant), so -d phi_i / d x_i is the direct sum's
    acceleration (central differences, exact Ewald sums, Plummer and K1)."""
    rng = np.random.default_rng(21)
    x = rng.random((10, 3))
    m = rng.uniform(0.5, 1.5, 10)
    h = 1e-5
    for kern, eps in ((0, 0.01), (1, 0.3)):
        acc = O.direct_forces(x, m, eps, table_n1=None, kernel=kern)
        for i in (0, 3, 7):
            for d in range(3):
                xp, xm = x.copy(), x.copy()
                xp[i, d] += h
                xm[i, d] -= h
                fd = -(O.direct_pot(xp, m, eps, targets=[i], table_n1=None, kernel=kern)[0] -
                       O.direct_pot(xm, m, eps, targets=[i], table_n1=None, kernel=kern)[0]) / (2 * h)
                assert abs(fd - acc[i, d]) <= 1e-6 * np.abs(acc[i]).max(), (kern, i, d, fd, acc[i, d])


def test_tree_pot_converges_to_direct_and_its_gradient_is_its_force():
    """The tree's potential converges to the direct one as theta falls
    (order 4), with and without K1 and the dual form; and at a massless probe
    (which moves no moment) minus the central-difference gradient of the
    tree's potential is the tree's own acceleration whenever the opening
    decisions are the same at both ends: the expansions, the image field's
    series and the background term are each the gradient of their potential
    form, so a dropped or mis-signed term of either shows here."""
    rng = np.random.default_rng(22)
    x = rng.random((1200, 3))
    eps = 1e-3
    pd = O.direct_pot(x, None, eps, table_n1=128)
    rms = np.sqrt(np.mean(pd ** 2))
    errs = []
    for th in (0.6, 0.4, 0.25):
        _, p = O.tree_forces(x, None, O.tree_params(eps, th, 4, ewald=4), return_pot=True)
        errs.append(np.median(np.abs(p - pd)) / rms)
    assert errs[0] > errs[1] > errs[2] and errs[2] <= 2e-5, errs
    for extra in ({"kernel": 1}, {"dual": 1}, {"mac": 1, "bg": 6}):
        pk = O.direct_pot(x, None, eps, table_n1=128, kernel=extra.get("kernel", 0))
        _, p = O.tree_forces(x, None, O.tree_params(eps, 0.25, 4, ewald=4, **extra), return_pot=True)
        assert np.median(np.abs(p - pk)) / rms <= 5e-5, extra
    # massless probe
    m = np.full(len(x) + 1, 1.0 / len(x))
    m[-1] = 0.0
    y = np.array([0.437, 0.611, 0.282])
    h = 1e-6
    checked = 0
    for prm in (O.tree_params(eps, 0.6, 4, ewald=4), O.tree_params(eps, 0.5, 2, ewald=3, mac=1, bg=4),
                O.tree_params(eps, 0.6, 3, ewald=5, kernel=1)):
        a0, _ = O.tree_forces(np.vstack([x, y]), m, prm, targets=[len(x)], return_pot=True)
        for d in range(3):
            e = np.zeros(3)
            e[d] = h
            _, pp, sp = O.tree_forces(np.vstack([x, y + e]), m, prm, targets=[len(x)], return_pot=True,
                                      return_stats=True)
            _, pm, sm = O.tree_forces(np.vstack([x, y - e]), m, prm, targets=[len(x)], return_pot=True,
                                      return_stats=True)
            if sp != sm:
                continue
            fd = -(pp[0] - pm[0]) / (2 * h)
            assert abs(fd - a0[0, d]) <= 1e-6 * np.abs(a0[0]).max(), (d, fd, a0[0, d])
            checked += 1
    assert checked >= 6


def test_tree_pot_rejects_a_first_order_image_field():
    """The background's potential needs the level-l_E cells' second moments,
    which an order-1 image field does not carry."""
    x = np.random.default_rng(2).random((100, 3))
    with pytest.raises(ValueError):
        O.tree_forces(x, None, O.tree_params(1e-3, 0.5, 2, ewald=1), return_pot=True)
    O.tree_forces(x, None, O.tree_params(1e-3, 0.5, 2, ewald=1))  # forces alone are fine


# ---- periodic images by near replicas and a far-lattice expansion ---------------------------
def test_lattice_tensor_symmetries_and_laplacian():
    """The far-lattice potential Phi_F (images beyond |n|_inf <= 2, with the
    background) is even and cubic-symmetric, and away from its images it
    satisfies Laplace's equation with the background's source:
    sum_d T_(m + 2 e_d) = -4 pi for m = 0 and 0 for |m| >= 1 (checked to the
    accuracy the Ewald sums' order-8 derivatives carry)."""
    import itertools
    T = O.lattice_tensor(8, 2)
    mi = O.multi_indices(8)
    idx = {m: i for i, m in enumerate(mi)}
    scale = np.abs(T).max()
    for i, m in enumerate(mi):
        if sum(m) % 2:
            assert abs(T[i]) <= 1e-12 * scale, m
        for pm in itertools.permutations(range(3)):
            assert abs(T[i] - T[idx[tuple(m[k] for k in pm)]]) <= 1e-9 * scale
    for m in mi:
        if sum(m) > 6:
            continue
        terms = [T[idx[tuple(m[k] + (2 if k == d else 0) for k in range(3))]] for d in range(3)]
        want = -4.0 * math.pi if sum(m) == 0 else 0.0
        assert abs(sum(terms) - want) <= 1e-5 * max(1.0, max(abs(t) for t in terms)), m


def test_near_replicas_and_far_lattice_match_the_ewald_sum():
    """With every near-replica pair summed directly (theta so small that no
    cell is accepted), the only approximation left is the order-8 far-lattice
    expansion: against the exact Ewald sum at negligible softening the
    forces agree to a median of 1e-6 with two shells of replicas (the
    paper's periodic scheme is stated to reach one part in 1e7), about a
    hundred times better than with one shell; the potential agrees as well;
    and as theta falls the replica tree converges to the same sum."""
    rng = np.random.default_rng(31)
    x = rng.random((200, 3))
    ad = O.direct_forces(x, None, 1e-7, table_n1=None)
    na = np.linalg.norm(ad, axis=1)
    med = {}
    for W in (1, 2):
        at = O.tree_forces(x, None, O.tree_params(1e-7, 0.02, 4, ewald=0, replicas=W, n_direct=16))
        med[W] = np.median(np.linalg.norm(at - ad, axis=1) / na)
    assert med[2] <= 1e-6 and med[1] >= 100 * med[2], med
    pd = O.direct_pot(x, None, 1e-7, table_n1=None)
    _, pt = O.tree_forces(x, None, O.tree_params(1e-7, 0.02, 4, ewald=0, replicas=2, n_direct=16),
                          return_pot=True)
    assert np.median(np.abs(pt - pd)) <= 1e-6 * np.sqrt(np.mean(pd ** 2))
    errs = []
    for th in (0.6, 0.4, 0.25):
        at = O.tree_forces(x, None, O.tree_params(1e-7, th, 4, ewald=0, replicas=2, n_direct=4))
        errs.append(np.median(np.linalg.norm(at - ad, axis=1) / na))
    assert errs[0] > errs[1] > errs[2], errs
    with pytest.raises(ValueError):
        O.tree_forces(x, None, O.tree_params(1e-7, 0.5, 2, ewald=4, replicas=2))
