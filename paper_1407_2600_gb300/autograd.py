"""Differentiable KDK trajectories (torch.autograd.Function over the C ABI).

forward: Zel'dovich initial state from the displacement field psi
(x = q + a0 psi wrapped, p = H0 a0^(3/2) psi), S kick-drift-kick steps with
nbody_kdk_step, the CIC delta^2 loss with nbody_cic_loss.  The state (x, p)
is checkpointed every `every` steps.
backward: for each segment, last first, the states are recomputed from its
checkpoint and the steps are reversed with nbody_kdk_adjoint_acc (chained:
each call reuses the previous call's reverse product at its end state); the
loss's gradient with respect to psi is a0 lam_x0 + H0 a0^(3/2) lam_p0.

All arithmetic of the path runs in the CUDA library (the initial-state map
and its transpose too: nbody_zeldovich_state, nbody_zeldovich_vjp); torch
supplies device memory, the stream and the autograd plumbing.
"""
from __future__ import annotations

import torch

from . import nbody as nb

def zeldovich_state(q, psi, a):
    return nb.zeldovich_state(q, psi, a)


def forward_steps(tree, x, p, acc, a_list, every):
    """S = len(a_list) - 1 KDK steps of (x, p) in place (acc holds g(x) on
    entry and on exit); returns the checkpoints {step: (x, p)} taken every
    `every` steps (step 0 included)."""
    ckpt = {0: (x.clone(), p.clone())}
    S = len(a_list) - 1
    for k in range(S):
        tree.kdk_step(p, acc, a_list[k], a_list[k + 1])
        if (k + 1) % every == 0 and k + 1 < S:
            ckpt[k + 1] = (x.clone(), p.clone())
    return ckpt


def reverse_steps(tree, ckpt, a_list, lx, lp):
    """Reverse sweep over the steps of forward_steps: for each segment, last
    first, the states (and their accelerations) are recomputed from its
    checkpoint with nbody_kdk_step, then the steps are reversed with
    nbody_kdk_adjoint_acc.  Consecutive calls chain (each reuses the previous
    call's product at its x1), so a step costs one recomputed step plus one
    tree build, moment pass and reverse walk.  Returns (lam_x0, lam_p0)."""
    S = len(a_list) - 1
    starts = sorted(ckpt.keys())
    for si in range(len(starts) - 1, -1, -1):
        c = starts[si]
        end = starts[si + 1] if si + 1 < len(starts) else S
        xs, ps = ckpt[c][0].clone(), ckpt[c][1].clone()
        tree.pos = xs
        tree.rebuild()
        acc = tree.forces()
        states = [(xs.clone(), ps.clone(), acc.clone())]
        for k in range(c, end - 1):
            tree.kdk_step(ps, acc, a_list[k], a_list[k + 1])
            states.append((xs.clone(), ps.clone(), acc.clone()))
        for k in range(end - 1, c - 1, -1):
            x0, p0, g0 = states[k - c]
            lx, lp = tree.kdk_adjoint(x0, p0, a_list[k], a_list[k + 1], lx, lp, acc0=g0)
    return lx, lp


class Trajectory(torch.autograd.Function):
    @staticmethod
    def forward(ctx, psi, q, prm, a_list, ng, every):
        x, p = zeldovich_state(q, psi.detach(), a_list[0])
        tree = nb.Tree(prm, x)
        acc = tree.forces()
        ckpt = forward_steps(tree, x, p, acc, a_list, every)
        loss, gx = nb.cic_loss(x, ng)
        ctx.tree = tree
        ctx.ckpt = ckpt
        ctx.gx = gx
        ctx.a_list = list(a_list)
        return loss

    @staticmethod
    def backward(ctx, gL):
        tree = ctx.tree
        a = ctx.a_list
        lx = (ctx.gx * gL).contiguous()
        lp = torch.zeros_like(ctx.ckpt[0][1])
        lx, lp = reverse_steps(tree, ctx.ckpt, a, lx, lp)
        dpsi = nb.zeldovich_vjp(a[0], lx, lp)
        tree.close()
        return dpsi, None, None, None, None, None


def trajectory_loss(psi, q, prm, a_list, ng, every=4):
    """CIC delta^2 loss after len(a_list)-1 KDK steps from Zel'dovich ICs;
    differentiable with respect to psi ((3, n) float64 CUDA tensor)."""
    return Trajectory.apply(psi, q, prm, a_list, ng, every)
