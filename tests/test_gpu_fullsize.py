"""Full-size parity on the benchmark workload (128^3 Zel'dovich + 64 NFW
haloes): keys, sort and tree topology exactly against the oracle, forces on
a seeded sample of particles against the oracle tree and the direct Ewald sum."""
import numpy as np
import pytest

import oracle
from paper_1407_2600_gb300 import ics

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cfg2():
    x, eps = ics.config_haloes(128, seed=1)
    return x, eps


def _tree(x, dev, **kw):
    import torch
    import paper_1407_2600_gb300.nbody as nb
    pos = torch.tensor(np.ascontiguousarray(x.T), dtype=torch.float64, device=dev)
    return nb.Tree(nb.params(**kw), pos)


def test_fullsize_sort_and_topology(cuda, cfg2):
    x, eps = cfg2
    tree = _tree(x, cuda, eps=eps)
    keys = tree.export("sorted_keys").cpu().numpy().view(np.uint64)
    perm = tree.export("perm").cpu().numpy().astype(np.int64)
    ck = tree.export("cell_keys").cpu().numpy().view(np.uint64)
    lev = tree.export("cell_level").cpu().numpy()
    rng_ = tree.export("cell_range").cpu().numpy()
    tree.close()
    okeys = oracle.morton_keys(x)
    operm = oracle.sort_perm(okeys)
    assert np.array_equal(keys, okeys[operm]), "sorted keys differ"
    assert np.array_equal(perm, operm), "permutation differs"
    okey, olev, ost, oct_ = oracle.tree_cells(x, n_leaf=16)
    assert len(ck) == len(okey), (len(ck), len(okey))
    assert np.array_equal(lev, olev)
    assert np.array_equal(ck, okey)
    assert np.array_equal(rng_[:, 0], ost) and np.array_equal(rng_[:, 1], oct_)


def _forces(x, dev, **kw):
    import torch
    tree = _tree(x, dev, **kw)
    acc, st = tree.forces(stats=True)
    torch.cuda.synchronize()
    a = acc.cpu().numpy().T.astype(np.float64)
    tree.close()
    return a, st


def _rel(a, b):
    return np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)


@pytest.mark.parametrize("theta,order,grid,nd,dual", [(0.6, 4, 5, 8, 0), (0.6, 4, 5, 8, 1), (0.5, 2, 6, 2, 0)])
def test_fullsize_forces_vs_oracle_tree(cuda, cfg2, theta, order, grid, nd, dual):
    """The first two cases are the benchmark's setting in its two walk forms."""
    import paper_1407_2600_gb300.nbody as nb
    x, eps = cfg2
    a, st = _forces(x, cuda, eps=eps, theta=theta, order=order, n_direct=nd, ewald_grid=grid,
                    flags=nb.NBODY_FLAG_DUAL if dual else 0)
    assert np.isfinite(a).all()
    tg = ics.random_targets(len(x), 1024, 3)
    ref = oracle.tree_forces(x, None, oracle.tree_params(eps, theta, order, n_direct=nd, ewald=4, ew_grid=grid,
                                                         dual=dual), targets=tg)
    rel = _rel(a[tg], ref)
    assert np.median(rel) <= 1e-5 and np.percentile(rel, 99) <= 1e-4, (np.median(rel), np.percentile(rel, 99))


@pytest.fixture(scope="module")
def cfg2_direct(cfg2):
    x, eps = cfg2
    tg = ics.random_targets(len(x), 256, 5)
    return tg, oracle.direct_forces(x, None, eps, targets=tg, table_n1=128)


def test_fullsize_error_vs_direct_ewald(cuda, cfg2, cfg2_direct):
    """The benchmark setting's force error against FP64 direct summation, in
    both walk forms: the metric's bar is the median (<= 1e-3); the 99th
    percentile is printed (on the configuration's 4096-particle subset the
    oracle gives 1.2e-2 for the M2P form and 1.3e-2 for the dual form, so a
    256-particle sample does not bound it).  At theta 0.5 both are met."""
    import paper_1407_2600_gb300.nbody as nb
    x, eps = cfg2
    tg, ad = cfg2_direct
    for name, fl in (("M2P", 0), ("dual", nb.NBODY_FLAG_DUAL)):
        a, _ = _forces(x, cuda, eps=eps, theta=0.6, order=4, n_direct=8, ewald_grid=5, flags=fl)
        rel = _rel(a[tg], ad)
        print("theta=0.6 p=4 %s (benchmark setting): median %.3e p99 %.3e" % (name, np.median(rel),
                                                                             np.percentile(rel, 99)))
        assert np.median(rel) <= 1e-3
    a, _ = _forces(x, cuda, eps=eps, theta=0.5, order=4, n_direct=4, ewald_grid=6)
    rel = _rel(a[tg], ad)
    print("theta=0.5 p=4: median %.3e p99 %.3e" % (np.median(rel), np.percentile(rel, 99)))
    assert np.median(rel) <= 1e-3 and np.percentile(rel, 99) <= 1e-2


def test_batched_uneven_boxes_vs_direct_and_tree(cuda):
    """Three uneven boxes of the batched workload (48^3, 64^3, 80^3) in one
    build at the benchmark's setting (theta 0.5, quadrupole, face-distance
    opening test, uniform-background terms, accepted cells of <= 16
    particles summed directly): per box, sampled forces against the oracle
    tree (median <= 1e-5) and against the direct Ewald sum at the accuracy
    bar (median <= 1e-3, 99th percentile <= 1e-2).  Without the background
    terms and with the tuned direct-sum threshold of 2 these near-uniform
    boxes (rms displacement 0.25 spacing) sit at 1-2.5e-3."""
    import torch
    import paper_1407_2600_gb300.nbody as nb
    x, p, off, eps = ics.config_batched(7, sizes=(48, 64, 80))
    pos = torch.tensor(np.ascontiguousarray(x.T), dtype=torch.float64, device=cuda)
    prm = nb.params(eps=eps[0], theta=0.5, order=2, n_direct=16, ewald_grid=4,
                    flags=nb.NBODY_FLAG_MAC_EDGE | nb.NBODY_FLAG_BACKGROUND)
    tree = nb.Tree(prm, pos, offsets=off.tolist(), eps=eps)
    acc = tree.forces().cpu().numpy().T.astype(np.float64)
    tree.close()
    for b in range(3):
        xb = x[off[b]:off[b + 1]]
        tg = ics.random_targets(len(xb), 256, 50 + b)
        ad = oracle.direct_forces(xb, None, eps[b], targets=tg, table_n1=128)
        at = oracle.tree_forces(xb, None, oracle.tree_params(eps[b], 0.5, 2, n_direct=16, ewald=4, mac=1,
                                                             ew_grid=4, bg=4), targets=tg)
        a = acc[off[b] + tg]
        rd = np.linalg.norm(a - ad, axis=1) / np.linalg.norm(ad, axis=1)
        rt = np.linalg.norm(a - at, axis=1) / np.linalg.norm(at, axis=1)
        print("box %d: median %.3e p99 %.3e vs direct Ewald" % (b, np.median(rd), np.percentile(rd, 99)))
        assert np.median(rd) <= 1e-3 and np.percentile(rd, 99) <= 1e-2, (b, np.median(rd), np.percentile(rd, 99))
        assert np.median(rt) <= 1e-5, (b, np.median(rt))


def _scale_flags(nb):
    """The scale workload's flags: face-distance opening test and the
    uniform-background terms."""
    return nb.NBODY_FLAG_MAC_EDGE | nb.NBODY_FLAG_BACKGROUND


def test_scale_setting_vs_oracle(cuda):
    """The 512^3 scale workload's setting on a 64^3 box of the same spectrum
    (P ~ k^-1.5, rms displacement 0.25 spacing): theta 0.7 with the opening
    distance from the cell faces and the uniform-background terms,
    hexadecapole, accepted cells of <= 8 particles summed directly, groups
    inside level-4 cells.  Sampled forces match the oracle tree (median <=
    1e-5, 99th percentile <= 1e-4) and the direct Ewald sum (median <= 1e-3)."""
    import paper_1407_2600_gb300.nbody as nb
    q, psi = ics.zeldovich_particles(64, -1.5, 0.25, 3)
    x = np.mod(q + psi, 1.0)
    x[x >= 1.0] = 0.0
    eps = 1.0 / (30 * 64)
    a, _ = _forces(x, cuda, eps=eps, theta=0.7, order=4, n_direct=8, ewald_grid=5, flags=_scale_flags(nb))
    assert np.isfinite(a).all()
    tg = ics.random_targets(len(x), 1024, 3)
    at = oracle.tree_forces(x, None, oracle.tree_params(eps, 0.7, 4, n_direct=8, ewald=4, ew_grid=5, mac=1,
                                                        bg=6), targets=tg)
    rt = _rel(a[tg], at)
    assert np.median(rt) <= 1e-5 and np.percentile(rt, 99) <= 1e-4, (np.median(rt), np.percentile(rt, 99))
    td = tg[:256]
    ad = oracle.direct_forces(x, None, eps, targets=td, table_n1=128)
    rd = _rel(a[td], ad)
    print("scale setting at 64^3: median %.3e p99 %.3e vs direct Ewald" % (np.median(rd), np.percentile(rd, 99)))
    assert np.median(rd) <= 1e-3
