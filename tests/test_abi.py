"""CPU checks of the boundary: the C-ABI library loads and exports every
symbol include/nbody.h declares; the generated kernel header is current."""
import os
import re
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "nbody.h")).read()
    return sorted(set(re.findall(r"\b(nbody_[a-z_0-9]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    from paper_1407_2600_gb300 import build as B
    B.build()
    import paper_1407_2600_gb300.nbody as nb
    lib = nb.lib()
    names = _declared()
    assert len(names) >= 10
    for s in names:
        assert hasattr(lib, s), s
    assert sorted(nb.SYMBOLS) == names


def test_defaults_and_strerror():
    import paper_1407_2600_gb300.nbody as nb
    p = nb.nbody_default_params()
    assert p.order == 4 and p.n_group == 32 and p.ewald_order == 4 and p.lmax == 21
    for code in range(0, -7, -1):
        assert nb.nbody_strerror(code) != "unknown error"


def test_invalid_arguments_are_rejected_without_gpu_work():
    import paper_1407_2600_gb300.nbody as nb
    p = nb.nbody_default_params()
    rc, h = nb.nbody_build_tree(p, 0, 0, None)
    assert rc == nb.NBODY_EINVAL and not h
    p.eps = 0.0
    rc, h = nb.nbody_build_tree(p, 10, 1, None)
    assert rc == nb.NBODY_EINVAL and not h
    p = nb.nbody_default_params()
    p.n_direct = p.n_leaf + 1
    rc, h = nb.nbody_build_tree(p, 10, 1, None)
    assert rc == nb.NBODY_EINVAL
    assert nb.nbody_forces(None, 0) == nb.NBODY_EINVAL
    assert nb.nbody_forces64(None, 0) == nb.NBODY_EINVAL
    assert nb.nbody_kdk_adjoint_acc(None, 0, 0, 0, 0.1, 0.2, 0, 0, 0, 0) == nb.NBODY_EINVAL
    assert nb.nbody_reserve(None, 1000, 100) == nb.NBODY_EINVAL
    assert nb.nbody_autotune(None) == nb.NBODY_EINVAL
    assert nb.nbody_assign_rungs(None, 0, 1.0, 0.1, 3, 0) == nb.NBODY_EINVAL
    assert nb.nbody_forces_active(None, 0, 0, 0) == nb.NBODY_EINVAL
    assert nb.nbody_kdk_multistep(None, 0, 0, 0, 0, 0.1, 0.2, 2) == nb.NBODY_EINVAL
    # flags: a walk variant beyond the table is rejected before any work
    p = nb.nbody_default_params()
    p.flags = nb.NBODY_FLAG_WALK_VARIANT(4)
    rc, h = nb.nbody_build_tree(p, 10, 1, None)
    assert rc == nb.NBODY_EINVAL and not h
    # background terms need a spare coefficient slot: not at orders 1 and 3
    for order in (1, 3):
        p = nb.nbody_default_params()
        p.order = order
        p.flags = nb.NBODY_FLAG_BACKGROUND
        rc, h = nb.nbody_build_tree(p, 10, 1, None)
        assert rc == nb.NBODY_EINVAL and not h


def test_generated_kernel_header_is_current():
    gen = os.path.join(ROOT, "paper_1407_2600_gb300", "csrc", "gen_m2p.py")
    r = subprocess.run([sys.executable, gen, "--check"])
    assert r.returncode == 0


def test_reduced_m2p_matches_oracle_dtensor_form():
    """The walk's reduced-coefficient M2P is algebraically the oracle's
    Hermite-form contraction; check the generator's tables numerically."""
    import math
    import numpy as np
    sys.path.insert(0, os.path.join(ROOT, "paper_1407_2600_gb300", "csrc"))
    import gen_m2p as G
    import oracle as O
    rng = np.random.default_rng(3)
    for p in range(5):
        sl, contrib = G.contributions(p)
        M = rng.standard_normal(O.nmom(p))
        # stored coefficients are a! B_{j,a}; monomials are R^a / a!
        fa = lambda a: math.factorial(a[0]) * math.factorial(a[1]) * math.factorial(a[2])
        B = np.array([fa(sl[t][1]) * sum(c * M[i] for i, c in cs) for t, cs in enumerate(contrib)])
        R = rng.standard_normal(3) * 0.5
        eps = 0.05
        s = R @ R + eps ** 2
        F = [((-1) ** j) * math.prod(range(1, 2 * j, 2)) * s ** (-0.5 - j) for j in range(p + 2)]
        mu = lambda a: R[0] ** a[0] * R[1] ** a[1] * R[2] ** a[2] / fa(a)
        S = np.zeros(p + 1)
        Gd = np.zeros((p + 1, 3))
        for t, (j, a) in enumerate(sl):
            S[j] += B[t] * mu(a)
            for d in range(3):
                if a[d] > 0:
                    aa = list(a)
                    aa[d] -= 1
                    Gd[j, d] += B[t] * mu(aa)
        acc = sum(R * F[j + 1] * S[j] + F[j] * Gd[j] for j in range(p + 1))
        ref = O.m2p(M, p, R, eps)
        assert np.abs(acc - ref).max() <= 1e-13 * np.abs(ref).max()


def test_more_invalid_arguments_are_rejected_without_gpu_work():
    """Host-side fault injection: out-of-range parameters, malformed box
    offsets, sizes beyond the limits and NULL handles or pointers are
    rejected with NBODY_EINVAL (NBODY_ERANGE for the allocation-free sort's
    size limit) before any CUDA call, so these run on a machine without a GPU.
    The device address 1 stands in for a buffer that is never touched."""
    import paper_1407_2600_gb300.nbody as nb
    EINVAL = nb.NBODY_EINVAL
    # every parameter outside its documented range
    bad = [("theta", 0.0), ("theta", -0.5), ("eps", -1e-3), ("order", 5), ("order", -1), ("n_leaf", 0),
           ("n_leaf", 65), ("n_group", 0), ("n_group", 33), ("n_direct", -1), ("lmax", 1), ("lmax", 22),
           ("ewald_order", 6), ("ewald_grid", 3), ("ewald_grid", 9), ("ewald_level", 0), ("precision", 2),
           ("box_len", -1.0), ("box_len", float("nan")), ("box_len", float("inf")), ("flags", 64),
           ("flags", 1 << 12)]
    for name, value in bad:
        p = nb.nbody_default_params()
        setattr(p, name, value)
        rc, h = nb.nbody_build_tree(p, 10, 1, None)
        assert rc == EINVAL and not h, (name, value, rc)
    # combinations the dual form does not take: order 0, FP64, background terms
    for name, value in (("order", 0), ("precision", 1), ("flags", nb.NBODY_FLAG_DUAL | nb.NBODY_FLAG_BACKGROUND)):
        p = nb.nbody_default_params()
        p.flags = nb.NBODY_FLAG_DUAL
        setattr(p, name, value if name != "flags" else value)
        rc, h = nb.nbody_build_tree(p, 10, 1, None)
        assert rc == nb.NBODY_ENOTSUP and not h, (name, value, rc)
    p = nb.nbody_default_params()
    # sizes: no particles, or at least 2^30 of them
    for n in (0, -5, 1 << 30):
        rc, h = nb.nbody_build_tree(p, n, 1, None)
        assert rc == EINVAL and not h, n
    # box offsets: an empty box, a first offset other than 0, no box, a
    # non-positive softening
    for off, eps in (([0, 5, 5], None), ([1, 5, 9], None), ([0], None), ([0, 4, 8], [1e-3, 0.0])):
        rc, h = nb.nbody_build_tree_batched(p, off, eps, 1, None)
        assert rc == EINVAL and not h, (off, eps)
    rc, h = nb.nbody_build_tree_batched(p, [0, 4, 8], None, 0, None)  # NULL positions
    assert rc == EINVAL and not h
    # build-and-evaluate: NULL accelerations, a non-positive box length
    rc, h = nb.nbody_forces_batched(p, [0, 4, 8], None, None, 1, None, 0)
    assert rc == EINVAL and not h
    for ln in ([1.0, 0.0], [250.0, -1.0], [float("nan"), 1.0]):
        rc, h = nb.nbody_forces_batched(p, [0, 4, 8], ln, None, 1, None, 1)
        assert rc == EINVAL and not h, ln
    # NULL tree handles
    assert nb.nbody_tree_count(None, 0) == EINVAL
    assert nb.nbody_tree_export(None, 0, 1) == EINVAL
    assert nb.nbody_check(None) == EINVAL
    assert nb.nbody_forces_vjp(None, 1, 1) == EINVAL
    assert nb.nbody_kdk_step(None, 1, 1, 1, 0.1, 0.2) == EINVAL
    assert nb.nbody_kdk_adjoint(None, 1, 1, 0.1, 0.2, 1, 1, 1, 1) == EINVAL
    assert nb.nbody_timing_read(None, nb.Timing(), 0) == EINVAL
    assert nb.nbody_tree_lookup(None, 1, 1, 1) == EINVAL
    nb.nbody_tree_free(None)  # freeing nothing is allowed
    # the CIC loss: grid sizes outside 2..1024, no particles, NULL pointers
    for n, ng, pos in ((10, 1, 1), (10, 1025, 1), (0, 8, 1), (10, 8, 0)):
        assert nb.nbody_cic_loss(pos, None, n, ng, 1, 1, None) == EINVAL, (n, ng, pos)
    # the allocation-free sort: no particles or NULL outputs, and its size limit
    assert nb.nbody_sort_keys_noalloc(1, 0, 1, 1) == EINVAL
    assert nb.nbody_sort_keys_noalloc(1, 16, 0, 1) == EINVAL
    assert nb.nbody_sort_keys_noalloc(1, (1 << 20) + 1, 1, 1) == nb.NBODY_ERANGE


def test_replicas_need_no_image_field():
    """The near-replica scheme replaces the image field: with ewald_order > 0
    the parameters are rejected before any CUDA call."""
    import paper_1407_2600_gb300.nbody as nb
    p = nb.nbody_default_params()
    p.flags = nb.NBODY_FLAG_REPLICAS
    rc, h = nb.nbody_build_tree(p, 10, 1, None)
    assert rc == nb.NBODY_EINVAL and not h
    p.ewald_order = 0
    p.ewald_grid = 9
    rc, h = nb.nbody_build_tree(p, 10, 1, None)
    assert rc == nb.NBODY_EINVAL and not h
