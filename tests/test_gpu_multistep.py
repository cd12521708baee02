"""Block steps (the hierarchical form of the symplectic integrator cited in
Sec. 2.1): rung assignment bit for bit against the oracle, accelerations of
an active subset equal to the full evaluation's, and a block step against
the oracle's block step with the oracle tree."""
import math

import numpy as np
import pytest

import oracle
from paper_1407_2600_gb300 import ics

pytestmark = pytest.mark.gpu

A0, A1 = 0.05, 0.06
ETA, RMAX = 1.0, 3


def _state(dev):
    import torch
    x, eps = ics.config_haloes(16, seed=6, n_halo=2, nmin=300, nmax=600)
    rng = np.random.default_rng(8)
    p = rng.standard_normal(x.shape) * 0.02
    pos = torch.tensor(np.ascontiguousarray(x.T), dtype=torch.float64, device=dev)
    mom = torch.tensor(np.ascontiguousarray(p.T), dtype=torch.float32, device=dev)
    return x, p, eps, pos, mom


def _tree(eps, pos):
    import paper_1407_2600_gb300.nbody as nb
    return nb.Tree(nb.params(eps=eps, theta=0.5, order=4), pos)


def test_assign_rungs_bitexact(cuda):
    x, p, eps, pos, mom = _state(cuda)
    tree = _tree(eps, pos)
    acc = tree.forces()
    dlna = math.log(A1 / A0)
    rung = tree.assign_rungs(acc, ETA, dlna, RMAX).cpu().numpy().astype(np.int64)
    ref = oracle.assign_rungs(acc.cpu().numpy().T, eps, ETA, dlna, RMAX)
    assert np.array_equal(rung, ref)
    assert len(np.unique(rung)) >= 3, np.bincount(rung)
    tree.close()


def test_forces_active_subset(cuda):
    import torch
    x, p, eps, pos, mom = _state(cuda)
    tree = _tree(eps, pos)
    full = tree.forces()
    rng = np.random.default_rng(2)
    r = rng.integers(0, 4, len(x))
    rung = torch.tensor(r, dtype=torch.int8, device=cuda)
    for rmin in (0, 2, 3):
        acc = torch.full_like(full, 7.0)
        tree.forces_active(rung, rmin, acc)
        on = torch.tensor(r >= rmin, device=cuda)
        assert torch.equal(acc[:, on], full[:, on])
        assert bool((acc[:, ~on] == 7.0).all())
    tree.close()


def test_block_step_vs_oracle(cuda):
    import torch
    x, p, eps, pos, mom = _state(cuda)
    tree = _tree(eps, pos)
    acc = tree.forces()
    dlna = math.log(A1 / A0)
    rung = tree.assign_rungs(acc, ETA, dlna, RMAX)
    r = rung.cpu().numpy().astype(np.int64)
    op = oracle.tree_params(eps, 0.5, 4, ewald=4)
    force = lambda xx: oracle.tree_forces(xx, None, op)
    g0 = force(x)
    p32 = mom.cpu().numpy().T.astype(np.float64)
    x1, p1, g1 = oracle.kdk_multistep(x, p32, g0, r, A0, A1, RMAX, force)
    tree.kdk_multistep(mom, acc, rung, A0, A1, RMAX)
    torch.cuda.synchronize()
    xg = tree.pos.cpu().numpy().T
    dx = np.mod(xg - x1 + 0.5, 1.0) - 0.5
    step = np.abs(np.mod(x1 - x + 0.5, 1.0) - 0.5).max()
    assert np.max(np.abs(dx)) <= 1e-5 * step + 1e-13, (np.max(np.abs(dx)), step)
    pg = mom.cpu().numpy().T.astype(np.float64)
    assert np.max(np.abs(pg - p1)) <= 1e-5 * np.abs(p1).max()
    ag = acc.cpu().numpy().T.astype(np.float64)
    rel = np.linalg.norm(ag - g1, axis=1) / np.linalg.norm(g1, axis=1)
    assert np.median(rel) <= 1e-5
    tree.close()


def test_block_step_one_rung_is_the_global_step(cuda):
    import torch
    x, p, eps, pos, mom = _state(cuda)
    t1 = _tree(eps, pos.clone())
    a1 = t1.forces()
    m1 = mom.clone()
    t1.kdk_step(m1, a1, A0, A1)
    t2 = _tree(eps, pos.clone())
    a2 = t2.forces()
    m2 = mom.clone()
    rung = torch.zeros(len(x), dtype=torch.int8, device=cuda)
    t2.kdk_multistep(m2, a2, rung, A0, A1, 0)
    torch.cuda.synchronize()
    # the same step; only the half-step expansion factor is formed differently
    assert torch.allclose(t1.pos, t2.pos, rtol=0, atol=1e-12)
    assert torch.allclose(m1, m2, rtol=1e-6, atol=1e-9)
    t1.close()
    t2.close()
