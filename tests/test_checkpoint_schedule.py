"""The checkpointed reverse sweep of the differentiable trajectory (host
logic of paper_1407_2600_gb300.autograd), on the CPU with a stand-in tree.

forward_steps keeps the state every `every` steps; reverse_steps recomputes
each segment from its checkpoint and reverses its steps last first.  The
stand-in tree implements the same calls (rebuild, forces, kdk_step,
kdk_adjoint) for a smooth nonlinear force in torch FP64, with the step's
exact vector-Jacobian product from torch.autograd, so that the sweep's
result can be compared with autograd through the whole uncheckpointed
trajectory: a segment boundary off by one step, a state taken from the
wrong end of a step or a checkpoint reused after it was advanced all change
the gradient.  No GPU is involved."""
import math

import pytest
import torch

from paper_1407_2600_gb300.autograd import forward_steps, reverse_steps

H0 = math.sqrt(8.0 * math.pi / 3.0)


def _force(x):
    # nonlinear and coupled, so the adjoint of each step depends on its state
    return -0.7 * torch.sin(2 * math.pi * x) + 0.2 * torch.roll(torch.cos(2 * math.pi * x), 1, dims=1)


def _step(x, p, a0, a1):
    """KDK in the EdS factors of the library's step, g(x0) recomputed."""
    ah = math.sqrt(a0 * a1)
    k1 = 2.0 / H0 * (math.sqrt(ah) - math.sqrt(a0))
    k2 = 2.0 / H0 * (math.sqrt(a1) - math.sqrt(ah))
    d = 2.0 / H0 * (1.0 / math.sqrt(a0) - 1.0 / math.sqrt(a1))
    p = p + k1 * _force(x)
    x = x + d * p
    p = p + k2 * _force(x)
    return x, p


class StandInTree:
    """The calls reverse_steps and forward_steps make, on CPU tensors."""

    def __init__(self, pos):
        self.pos = pos
        self.calls = {"rebuild": 0, "forces": 0, "kdk_step": 0, "kdk_adjoint": 0}

    def rebuild(self):
        self.calls["rebuild"] += 1

    def forces(self):
        self.calls["forces"] += 1
        return _force(self.pos)

    def kdk_step(self, p, acc, a0, a1):
        self.calls["kdk_step"] += 1
        assert torch.equal(acc, _force(self.pos)), "acc must hold g(x) at the step's start"
        x1, p1 = _step(self.pos, p, a0, a1)
        self.pos.copy_(x1)
        p.copy_(p1)
        acc.copy_(_force(x1))

    def kdk_adjoint(self, x0, p0, a0, a1, lx, lp, acc0=None):
        self.calls["kdk_adjoint"] += 1
        assert acc0 is not None and torch.equal(acc0, _force(x0)), "acc0 must be g(x0)"
        x0 = x0.clone().requires_grad_(True)
        p0 = p0.clone().requires_grad_(True)
        x1, p1 = _step(x0, p0, a0, a1)
        gx, gp = torch.autograd.grad((x1, p1), (x0, p0), (lx, lp))
        return gx.detach(), gp.detach()


@pytest.mark.parametrize("S,every", [(1, 4), (4, 4), (5, 4), (8, 4), (9, 2), (7, 1), (6, 10), (16, 4)])
def test_reverse_sweep_matches_autograd(S, every):
    g = torch.Generator().manual_seed(100 * S + every)
    n = 37
    x0 = torch.rand((3, n), dtype=torch.float64, generator=g)
    p0 = 0.05 * torch.randn((3, n), dtype=torch.float64, generator=g)
    wx = torch.randn((3, n), dtype=torch.float64, generator=g)
    wp = torch.randn((3, n), dtype=torch.float64, generator=g)
    a_list = [0.05 * 4.0 ** (k / S) for k in range(S + 1)]

    # reference: autograd through the whole trajectory, no checkpoints
    xr = x0.clone().requires_grad_(True)
    pr = p0.clone().requires_grad_(True)
    x, p = xr, pr
    for k in range(S):
        x, p = _step(x, p, a_list[k], a_list[k + 1])
    loss = (x * wx).sum() + (p * wp).sum()
    gx_ref, gp_ref = torch.autograd.grad(loss, (xr, pr))

    # the checkpointed forward and reverse sweep
    x = x0.clone()
    p = p0.clone()
    tree = StandInTree(x)
    acc = tree.forces()
    ckpt = forward_steps(tree, x, p, acc, a_list, every)
    assert sorted(ckpt) == [k for k in range(0, S, every)]
    assert torch.allclose(x, _run(x0, p0, a_list)[0], rtol=0, atol=1e-13)  # stepped in place
    gx, gp = reverse_steps(tree, ckpt, a_list, wx.clone(), wp.clone())
    assert torch.allclose(gx, gx_ref, rtol=1e-12, atol=1e-12)
    assert torch.allclose(gp, gp_ref, rtol=1e-12, atol=1e-12)
    # every step is reversed once; the recompute repeats each segment's steps
    # but its last (its end state is the next segment's checkpoint)
    nseg = len(ckpt)
    assert tree.calls["kdk_adjoint"] == S
    assert tree.calls["kdk_step"] == S + (S - nseg)
    assert tree.calls["rebuild"] == nseg


def _run(x, p, a_list):
    for k in range(len(a_list) - 1):
        x, p = _step(x, p, a_list[k], a_list[k + 1])
    return x, p
