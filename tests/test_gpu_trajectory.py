"""The differentiable-trajectory workload at full size: 64^3 particles, 16
KDK steps from a = 0.05 to 0.2 (uniform in ln a), CIC delta^2 loss on a 64^3
grid, gradient with respect to the initial Zel'dovich displacement by the
checkpointed reverse sweep (checkpoints every 4 steps, FP32 interactions,
FP64 positions).

Checked against FP64 central finite differences (h = 1e-6 box units of the
displacement) of the same method run in FP64 on the GPU (`precision` FP64,
`nbody_forces64`, the KDK and the loss in FP64) on 32 seeded components;
a component whose +h or -h trajectory takes other discrete tree decisions
than the unperturbed one (the walks' decision checksums differ) or ends
with a particle in another CIC cell is redrawn.  Tolerance 1e-4 relative,
per component against max(|FD|, rms of the gradient)."""
import math

import numpy as np
import pytest

from paper_1407_2600_gb300 import ics

pytestmark = pytest.mark.gpu
H0 = math.sqrt(8.0 * math.pi / 3.0)
NG = 64
A0, A1, S = 0.05, 0.2, 16
THETA, ORDER = 0.5, 4


def _a_list():
    return [A0 * (A1 / A0) ** (k / S) for k in range(S + 1)]


def _fp64_loss(nb, torch, q, psi, prm64, a_list):
    """FP64 forward of the same method: returns (loss, interaction counts and
    the walks' decision checksum summed over the trajectory)."""
    x = torch.remainder(q + a_list[0] * psi, 1.0)
    x[x >= 1.0] = 0.0
    p = H0 * a_list[0] ** 1.5 * psi
    tree = nb.Tree(prm64, x)
    g = tree.forces64()
    for k in range(S):
        a0, a1 = a_list[k], a_list[k + 1]
        ah = math.sqrt(a0 * a1)
        k1 = 2.0 / H0 * (math.sqrt(ah) - math.sqrt(a0))
        k2 = 2.0 / H0 * (math.sqrt(a1) - math.sqrt(ah))
        d = 2.0 / H0 * (1.0 / math.sqrt(a0) - 1.0 / math.sqrt(a1))
        p = p + k1 * g
        x = x + d * p
        x = x - torch.floor(x)
        x[x >= 1.0] = 0.0
        tree.pos = x
        tree.rebuild()
        g = tree.forces64()
        p = p + k2 * g
    loss, _ = nb.cic_loss(x, NG, grad=False)
    tm = tree.timing(reset=True)
    tree.close()
    # the lower CIC cell of every particle (cell-centred grid): the loss is
    # smooth only while none of them changes
    cic = torch.floor(x * NG - 0.5).to(torch.int32)
    return float(loss), (tm["p2p"], tm["m2p"], tm["decision_hash"]), cic


def test_config5_gradient_vs_fp64_finite_differences(cuda):
    import torch
    import paper_1407_2600_gb300.nbody as nb
    from paper_1407_2600_gb300.autograd import trajectory_loss
    q, disp = ics.zeldovich_particles(NG, -2.0, 0.25, 5)
    psi = disp / A0  # displacement per unit a: x = q + a psi
    qt = torch.tensor(np.ascontiguousarray(q.T), dtype=torch.float64, device=cuda)
    eps = 1.0 / (30.0 * NG)
    prm = nb.params(eps=eps, theta=THETA, order=ORDER, n_direct=4)
    prm64 = nb.params(eps=eps, theta=THETA, order=ORDER, n_direct=4, precision=1)
    a_list = _a_list()
    psi_t = torch.tensor(np.ascontiguousarray(psi.T), dtype=torch.float64, device=cuda).requires_grad_(True)
    loss = trajectory_loss(psi_t, qt, prm, a_list, NG, every=4)
    loss.backward()
    g = psi_t.grad.cpu().numpy().T
    base = psi_t.detach()
    l64, c0, k0 = _fp64_loss(nb, torch, qt, base, prm64, a_list)
    assert abs(float(loss.detach()) - l64) <= 1e-4 * abs(l64), (float(loss.detach()), l64)
    rms = np.sqrt(np.mean(g ** 2))
    rng = np.random.default_rng(12)
    h = 1e-6 / A0  # 1e-6 box units of displacement at a = 0.05
    checked, worst, redrawn = 0, 0.0, 0
    for _ in range(80):
        j, d = int(rng.integers(len(q))), int(rng.integers(3))
        pp, pm = base.clone(), base.clone()
        pp[d, j] += h
        pm[d, j] -= h
        lp, cp, kp = _fp64_loss(nb, torch, qt, pp, prm64, a_list)
        lm, cm, km = _fp64_loss(nb, torch, qt, pm, prm64, a_list)
        if cp != c0 or cm != c0 or not (torch.equal(kp, k0) and torch.equal(km, k0)):
            # a perturbed run took other tree decisions, or moved a particle
            # into another CIC cell, than the linearised one
            redrawn += 1
            continue
        fd = (lp - lm) / (2 * h)
        err = abs(g[j, d] - fd) / max(abs(fd), rms)
        worst = max(worst, err)
        assert err <= 1e-4, (j, d, g[j, d], fd, rms)
        checked += 1
        if checked >= 32:
            break
    print("config 5: %d components (%d redrawn), worst relative difference %.2e" % (checked, redrawn, worst))
    assert checked >= 24
