"""GPU reverse mode against the FP64 CPU oracle: the CIC loss, the force VJP
and the KDK adjoint against central finite differences of the oracle tree
(same method definition, FP64), the differentiable trajectory against finite
differences of the oracle trajectory, and against the direct-sum adjoint.

Finite differences keep the perturbed coordinate inside one key quantum
(2^-21 box) so that the tree's discrete decisions do not change; components
whose runs change the oracle's interaction counts are skipped."""
import math

import numpy as np
import pytest

import oracle
from paper_1407_2600_gb300 import ics

pytestmark = pytest.mark.gpu
Q = 2.0 ** -21


def _t(x, dev, dtype=None):
    import torch
    return torch.tensor(np.ascontiguousarray(x.T), dtype=dtype or torch.float64, device=dev)


def _safe(v, h):
    return math.floor((v + h) / Q) == math.floor(v / Q) == math.floor((v - h) / Q)


def test_cic_loss_matches_oracle(cuda):
    import paper_1407_2600_gb300.nbody as nb
    x, _ = ics.config_small(3)
    L, g = nb.cic_loss(_t(x, cuda), 16)
    Lo, go = oracle.cic_loss(x, None, 16)
    assert abs(float(L) - Lo) <= 1e-12 * Lo
    assert np.abs(g.cpu().numpy().T - go).max() <= 1e-10 * np.abs(go).max()


def _prm(eps, theta, order, flags=0):
    import paper_1407_2600_gb300.nbody as nb
    return nb.params(eps=eps, theta=theta, order=order, n_direct=2 if order <= 2 else 4, flags=flags)


@pytest.mark.parametrize("theta,order,bg", [(0.5, 4, False), (0.6, 2, False), (0.5, 4, True), (0.5, 2, True)])
def test_force_vjp_vs_finite_differences(cuda, theta, order, bg):
    """With bg the uniform-background terms are on (their sink-side
    derivative is part of the product)."""
    import torch
    import paper_1407_2600_gb300.nbody as nb
    x, eps = ics.config_haloes(16, seed=4, n_halo=2, nmin=200, nmax=400)
    n = len(x)
    rng = np.random.default_rng(11)
    lam = rng.standard_normal((n, 3))
    tree = nb.Tree(_prm(eps, theta, order, nb.NBODY_FLAG_BACKGROUND if bg else 0), _t(x, cuda))
    mu = tree.forces_vjp(_t(lam.astype(np.float32), cuda, torch.float32)).cpu().numpy().T
    tree.close()
    op = oracle.tree_params(eps, theta, order, n_direct=2 if order <= 2 else 4, ewald=4,
                            bg={2: 4, 4: 6}[order] if bg else 0)
    lam32 = lam.astype(np.float32).astype(np.float64)
    h = 5e-9
    rms = np.sqrt(np.mean(mu ** 2))
    checked = 0
    for _ in range(60):
        j, d = int(rng.integers(n)), int(rng.integers(3))
        if not _safe(x[j, d], h):
            continue
        xp, xm = x.copy(), x.copy()
        xp[j, d] += h
        xm[j, d] -= h
        ap, sp = oracle.tree_forces(xp, None, op, return_stats=True)
        am, sm = oracle.tree_forces(xm, None, op, return_stats=True)
        if sp != sm:
            continue
        fd = (np.sum(lam32 * ap) - np.sum(lam32 * am)) / (2 * h)
        assert abs(mu[j, d] - fd) <= 2e-4 * max(abs(fd), rms), (j, d, mu[j, d], fd, rms)
        checked += 1
        if checked >= 16:
            break
    assert checked >= 8


def test_kdk_adjoint_vs_finite_differences(cuda):
    import torch
    import paper_1407_2600_gb300.nbody as nb
    q, psi = ics.zeldovich_particles(16, -2.0, 0.25, 21)
    a0, a1 = 0.05, 0.06
    x0, p0 = oracle.zeldovich_state(q, psi / a0, a0)
    p0 = p0.astype(np.float32).astype(np.float64)
    eps = 1.0 / 480
    n = len(x0)
    rng = np.random.default_rng(5)
    lx1 = rng.standard_normal((n, 3))
    lp1 = rng.standard_normal((n, 3)).astype(np.float32).astype(np.float64)
    tree = nb.Tree(_prm(eps, 0.5, 4), _t(x0, cuda))
    lx0, lp0 = tree.kdk_adjoint(_t(x0, cuda), _t(p0, cuda, torch.float32), a0, a1, _t(lx1, cuda),
                                _t(lp1, cuda, torch.float32))
    lx0 = lx0.cpu().numpy().T
    lp0 = lp0.cpu().numpy().T.astype(np.float64)
    tree.close()
    op = oracle.tree_params(eps, 0.5, 4, ewald=4)

    def f(x, p):
        force = lambda xx: oracle.tree_forces(xx, None, op)
        x1, p1, _ = oracle.kdk_step(x, p, force(x), a0, a1, force)
        d = np.mod(x1 - x0 + 0.5, 1.0) - 0.5  # unwrap against a fixed reference
        return np.sum(lx1 * d) + np.sum(lp1 * p1)

    h = 5e-9
    rmsx, rmsp = np.sqrt(np.mean(lx0 ** 2)), np.sqrt(np.mean(lp0 ** 2))
    checked = 0
    for _ in range(40):
        j, d = int(rng.integers(n)), int(rng.integers(3))
        if not _safe(x0[j, d], h) or not (1e-3 < x0[j, d] < 1 - 1e-3):
            continue
        xp, xm = x0.copy(), x0.copy()
        xp[j, d] += h
        xm[j, d] -= h
        fdx = (f(xp, p0) - f(xm, p0)) / (2 * h)
        pp, pm = p0.copy(), p0.copy()
        hp = 1e-7
        pp[j, d] += hp
        pm[j, d] -= hp
        fdp = (f(x0, pp) - f(x0, pm)) / (2 * hp)
        assert abs(lx0[j, d] - fdx) <= 5e-4 * max(abs(fdx), rmsx), (j, d, lx0[j, d], fdx)
        assert abs(lp0[j, d] - fdp) <= 5e-4 * max(abs(fdp), rmsp), (j, d, lp0[j, d], fdp)
        checked += 1
        if checked >= 6:
            break
    assert checked >= 3


def test_trajectory_gradient_vs_finite_differences(cuda):
    """d(CIC delta^2 after 4 KDK steps)/d psi against FD of the oracle trajectory."""
    import torch
    import paper_1407_2600_gb300.nbody as nb
    from paper_1407_2600_gb300.autograd import trajectory_loss
    q, psi = ics.zeldovich_particles(16, -2.0, 0.25, 33)
    a_init, a_end, S = 0.05, 0.1, 4
    psi = psi / a_init
    a_list = [a_init * (a_end / a_init) ** (k / S) for k in range(S + 1)]
    eps = 1.0 / 480
    prm = _prm(eps, 0.5, 4)
    psi_t = _t(psi, cuda).requires_grad_(True)
    L = trajectory_loss(psi_t, _t(q, cuda), prm, a_list, 16, every=2)
    L.backward()
    g = psi_t.grad.cpu().numpy().T
    op = oracle.tree_params(eps, 0.5, 4, ewald=4)
    force = lambda xx: oracle.tree_forces(xx, None, op)

    def loss(ps):
        # FP64 momenta: the psi perturbation moves p by about one FP32 quantum
        x, p = oracle.zeldovich_state(q, ps, a_init)
        gcur = force(x)
        for k in range(S):
            x, p, gcur = oracle.kdk_step(x, p, gcur, a_list[k], a_list[k + 1], force)
        return oracle.cic_loss(x, None, 16)[0]

    assert abs(float(L) - loss(psi)) <= 1e-4 * abs(loss(psi))
    rng = np.random.default_rng(8)
    rms = np.sqrt(np.mean(g ** 2))
    checked = 0
    for _ in range(30):
        j, d = int(rng.integers(len(q))), int(rng.integers(3))
        h = 2e-8  # in psi units; the position moves by a_init h
        pp, pm = psi.copy(), psi.copy()
        pp[j, d] += h
        pm[j, d] -= h
        fd = (loss(pp) - loss(pm)) / (2 * h)
        if abs(g[j, d] - fd) > 1e-3 * max(abs(fd), rms):
            # a key quantum or CIC cell crossed by the perturbation: redraw
            x0 = np.mod(q + a_init * psi, 1.0)
            if not _safe(x0[j, d], a_init * h):
                continue
        assert abs(g[j, d] - fd) <= 1e-3 * max(abs(fd), rms), (j, d, g[j, d], fd, rms)
        checked += 1
        if checked >= 5:
            break
    assert checked >= 3


def test_trajectory_gradient_vs_direct_sum_adjoint(cuda):
    """The tree adjoint against the FP64 direct-sum adjoint (O1 dynamics) at
    16^3 on the differentiable-trajectory schedule (16 KDK steps from a =
    0.05 to 0.2, checkpoints every 4); they differ by the tree's force error,
    so the bound is the tree's accuracy."""
    import torch
    import paper_1407_2600_gb300.nbody as nb
    from paper_1407_2600_gb300.autograd import trajectory_loss
    q, psi = ics.zeldovich_particles(16, -2.0, 0.25, 44)
    a_init, a_end, S = 0.05, 0.2, 16
    psi = psi / a_init
    a_list = [a_init * (a_end / a_init) ** (k / S) for k in range(S + 1)]
    eps = 1.0 / 480
    psi_t = _t(psi, cuda).requires_grad_(True)
    L = trajectory_loss(psi_t, _t(q, cuda), _prm(eps, 0.4, 4), a_list, 16, every=4)
    L.backward()
    g = psi_t.grad.cpu().numpy().T
    force = lambda xx: oracle.direct_forces(xx, None, eps, table_n1=64)
    x, p = oracle.zeldovich_state(q, psi, a_init)
    xs, ps = [x], [p]
    gcur = force(x)
    for k in range(S):
        x, p, gcur = oracle.kdk_step(x, p, gcur, a_list[k], a_list[k + 1], force)
        xs.append(x)
        ps.append(p)
    _, gx = oracle.cic_loss(x, None, 16)
    lx, lp = oracle.adjoint_kdk(xs, ps, a_list, gx, np.zeros_like(gx), None, eps, n1=64)
    gd = a_init * lx + oracle.H0 * a_init ** 1.5 * lp
    rel = np.linalg.norm(g - gd, axis=1) / np.linalg.norm(gd, axis=1)
    print("tree vs direct-sum adjoint gradient: median %.2e p90 %.2e" % (np.median(rel), np.percentile(rel, 90)))
    assert np.median(rel) <= 5e-3, np.median(rel)


def _trajectory_states(nb, tree, x, p, a_list):
    """States (x, p, g(x)) of a short trajectory stepped by nbody_kdk_step."""
    acc = tree.forces()
    states = [(x.clone(), p.clone(), acc.clone())]
    for k in range(len(a_list) - 1):
        tree.kdk_step(p, acc, a_list[k], a_list[k + 1])
        states.append((x.clone(), p.clone(), acc.clone()))
    return states


def test_kdk_adjoint_chain_reuses_and_matches_unchained(cuda):
    """A reverse sweep of nbody_kdk_adjoint_acc calls reuses each previous
    call's product (every call after the first), and gives the results of
    unchained calls (a fresh tree per step) up to the reverse walk's atomic
    summation order; nbody_kdk_adjoint (g(x0) recomputed) agrees too."""
    import torch
    import paper_1407_2600_gb300.nbody as nb
    q, psi = ics.zeldovich_particles(16, -2.0, 0.25, 9)
    a_list = [0.05 * 1.1 ** k for k in range(5)]
    x0, p0 = oracle.zeldovich_state(q, psi / a_list[0], a_list[0])
    prm = _prm(1.0 / 480, 0.5, 4)
    x = _t(x0, cuda)
    p = _t(p0, cuda, torch.float32)
    tree = nb.Tree(prm, x)
    states = _trajectory_states(nb, tree, x, p, a_list)
    rng = np.random.default_rng(2)
    n = len(q)
    lx_end = _t(rng.standard_normal((n, 3)), cuda)
    lp_end = _t(rng.standard_normal((n, 3)), cuda, torch.float32)

    tree.timing(reset=True)
    lx, lp = lx_end.clone(), lp_end.clone()
    for k in range(len(a_list) - 2, -1, -1):
        xs, ps, gs = states[k]
        lx, lp = tree.kdk_adjoint(xs, ps, a_list[k], a_list[k + 1], lx, lp, acc0=gs)
    tm = tree.timing(reset=True)
    assert tm["adjoint_steps"] == len(a_list) - 1
    assert tm["adjoint_reused"] == len(a_list) - 2

    ux, up = lx_end.clone(), lp_end.clone()
    for k in range(len(a_list) - 2, -1, -1):
        xs, ps, _ = states[k]
        fresh = nb.Tree(prm, xs.clone())
        ux, up = fresh.kdk_adjoint(xs, ps, a_list[k], a_list[k + 1], ux, up)
        assert fresh.timing(reset=True)["adjoint_reused"] == 0
        fresh.close()
    tree.close()
    for a, b in ((lx, ux), (lp.double(), up.double())):
        a, b = a.cpu().numpy(), b.cpu().numpy()
        rms = np.sqrt(np.mean(b ** 2))
        assert np.abs(a - b).max() <= 1e-5 * rms, np.abs(a - b).max() / rms


def test_batched_force_vjp_matches_single_boxes(cuda):
    """The force VJP of a batched tree (three uneven boxes in one forest)
    equals, box by box, the VJP of each box on its own."""
    import torch
    import paper_1407_2600_gb300.nbody as nb
    boxes = [ics.config_small(21)[0], ics.config_haloes(12, seed=6, n_halo=2, nmin=40, nmax=200)[0],
             np.random.default_rng(8).uniform(0, 1, (777, 3))]
    eps = [1.0 / 480, 1.0 / 360, 2e-3]
    off = np.cumsum([0] + [len(b) for b in boxes])
    rng = np.random.default_rng(4)
    lam = rng.standard_normal((off[-1], 3)).astype(np.float32)
    prm = _prm(1e-3, 0.55, 4)
    tree = nb.Tree(prm, _t(np.concatenate(boxes), cuda), offsets=off.tolist(), eps=eps)
    mu = tree.forces_vjp(_t(lam, cuda, torch.float32)).cpu().numpy().T
    tree.close()
    for b, xb in enumerate(boxes):
        t1 = nb.Tree(_prm(eps[b], 0.55, 4), _t(xb, cuda))
        m1 = t1.forces_vjp(_t(lam[off[b]:off[b + 1]], cuda, torch.float32)).cpu().numpy().T
        t1.close()
        got = mu[off[b]:off[b + 1]]
        rms = np.sqrt(np.mean(m1 ** 2))
        assert np.abs(got - m1).max() <= 1e-5 * rms, (b, np.abs(got - m1).max() / rms)


def test_zeldovich_state_and_its_transpose(cuda):
    """The trajectory's starting state x = q + a psi (wrapped), p = H0
    a^(3/2) psi through the C ABI against the oracle's zeldovich_state, and
    the transpose dpsi = a lam_x + H0 a^(3/2) lam_p against the same linear
    map applied on the host (positions bit for bit, FP32 momenta within an
    ulp, the transpose to FP64 rounding)."""
    import torch
    import paper_1407_2600_gb300.nbody as nb
    rng = np.random.default_rng(21)
    q = ics.lattice(12)
    psi = 0.3 * rng.standard_normal(q.shape)  # large enough to cross the box edge
    a = 0.07
    x, p = nb.zeldovich_state(_t(q, cuda), _t(psi, cuda), a)
    xo, po = oracle.zeldovich_state(q, psi, a)
    assert np.array_equal(x.cpu().numpy().T, xo)
    assert np.abs(p.cpu().numpy().T - po).max() <= 2 * np.spacing(np.float32(np.abs(po).max()))
    lx = rng.standard_normal(q.shape)
    lp = rng.standard_normal(q.shape).astype(np.float32)
    d = nb.zeldovich_vjp(a, _t(lx, cuda), _t(lp, cuda, torch.float32)).cpu().numpy().T
    ref = a * lx + oracle.H0 * a ** 1.5 * lp.astype(np.float64)
    assert np.abs(d - ref).max() <= 1e-14 * np.abs(ref).max()
