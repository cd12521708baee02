"""Steps on reserved capacities and captured in a CUDA graph (the batched
realisations, Sec. 2.1): builds that keep their counts on the device give
bit-identical trees and forces, a captured sequence of KDK steps replays to
the same state as the same steps called one by one, its final forces match
the oracle tree, capacities that are too small are reported as
NBODY_EOVERFLOW without touching memory past the buffers, and the walk tile
autotuner keeps the fastest of its candidates without changing the method."""
import math

import numpy as np
import pytest

import oracle
from paper_1407_2600_gb300 import ics

pytestmark = pytest.mark.gpu

SIZES = (16, 16, 24, 24, 32)


def _setup(dev, flags=0, seed=3):
    import torch
    import paper_1407_2600_gb300.nbody as nb
    x, p, off, eps = ics.config_batched(seed, sizes=SIZES)
    pos = torch.tensor(np.ascontiguousarray(x.T), dtype=torch.float64, device=dev)
    mom = torch.tensor(np.ascontiguousarray(p.T), dtype=torch.float32, device=dev)
    prm = nb.params(eps=eps[0], theta=0.5, order=2, n_direct=2, ewald_grid=4,
                    flags=nb.NBODY_FLAG_MAC_EDGE | flags)
    tree = nb.Tree(prm, pos, offsets=off.tolist(), eps=eps)
    return tree, pos, mom, off, eps


def test_reserved_capacity_builds_match_exact(cuda):
    import torch
    tree, pos, mom, off, eps = _setup(cuda)
    acc0, st0 = tree.forces(stats=True)
    keys0 = tree.export("cell_keys").clone()
    groups0 = tree.export("groups").clone()
    mc, mg = tree.reserve(0.25)
    assert mc > st0["ncells"] and mg > st0["ngroups"]
    acc1, st1 = tree.forces(stats=True)
    assert st1["ncells"] == st0["ncells"] and st1["ngroups"] == st0["ngroups"]
    assert st1["decision_hash"] == st0["decision_hash"]
    assert torch.equal(tree.export("cell_keys"), keys0)
    assert torch.equal(tree.export("groups"), groups0)
    assert torch.equal(acc1, acc0)
    # back to counts read per build
    tree.reserve(-1)
    acc2 = tree.forces()
    assert torch.equal(acc2, acc0)
    tree.close()


def test_graph_captured_kdk_steps_match_eager_and_oracle(cuda):
    import torch
    import paper_1407_2600_gb300.nbody as nb
    steps, a0, dlna = 3, 0.02, 0.1
    a_list = [a0 * math.exp(dlna * k) for k in range(steps + 1)]
    # eager reference: counts read back per build
    te, pe, me, off, eps = _setup(cuda)
    ae = te.forces()
    for k in range(steps):
        te.kdk_step(me, ae, a_list[k], a_list[k + 1])
    torch.cuda.synchronize()
    # reserved capacities, asynchronous calls, captured
    tg, pg, mg, _, _ = _setup(cuda, flags=nb.NBODY_FLAG_ASYNC)
    ag = tg.forces()
    tg.reserve(0.25)
    tg.forces(ag)           # sizes the evaluation buffers on the reserved capacities
    x_init, p_init, g_init = pg.clone(), mg.clone(), ag.clone()
    torch.cuda.synchronize()
    tg.check()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        for k in range(steps):
            tg.kdk_step(mg, ag, a_list[k], a_list[k + 1])
    # capture records the steps without running them
    assert torch.equal(pg, x_init) and torch.equal(mg, p_init)
    graph.replay()
    torch.cuda.synchronize()
    tg.check()
    assert torch.equal(pg, pe) and torch.equal(mg, me) and torch.equal(ag, ae)
    # a second replay from the restored initial state gives the same state again
    pg.copy_(x_init)
    mg.copy_(p_init)
    ag.copy_(g_init)
    graph.replay()
    torch.cuda.synchronize()
    tg.check()
    assert torch.equal(pg, pe) and torch.equal(mg, me) and torch.equal(ag, ae)
    # the replayed forces at the final positions against the oracle tree
    x = pg.cpu().numpy().T
    acc = ag.cpu().numpy().T.astype(np.float64)
    for b in (0, len(SIZES) - 1):
        xb = x[off[b]:off[b + 1]]
        tgt = ics.random_targets(len(xb), 128, 90 + b)
        at = oracle.tree_forces(xb, None, oracle.tree_params(eps[b], 0.5, 2, n_direct=2, ewald=4, mac=1,
                                                             ew_grid=4), targets=tgt)
        a = acc[off[b] + tgt]
        rt = np.linalg.norm(a - at, axis=1) / np.linalg.norm(at, axis=1)
        assert np.median(rt) <= 1e-5, (b, np.median(rt))
    del graph
    te.close()
    tg.close()


def test_capacity_overflow_is_reported_and_recovers(cuda):
    import torch
    import paper_1407_2600_gb300.nbody as nb
    tree, pos, mom, off, eps = _setup(cuda)
    acc0, st = tree.forces(stats=True)
    nc, ng = st["ncells"], st["ngroups"]
    for mc, mg in ((nc // 2, ng + 64), (nc + 64, ng // 2), (nc - 1, ng)):
        with pytest.raises(nb.NbodyError) as ei:
            tree.reserve(max_cells=mc, max_groups=mg)
        assert ei.value.code == nb.NBODY_EOVERFLOW
        # the overflowed build evaluates nothing and reports it again
        acc = torch.zeros_like(acc0)
        with pytest.raises(nb.NbodyError) as ei:
            tree.forces(acc)
        assert ei.value.code == nb.NBODY_EOVERFLOW
    # exact capacities fit
    tree.reserve(max_cells=nc, max_groups=ng)
    assert torch.equal(tree.forces(), acc0)
    tree.close()


def test_autotune_picks_a_candidate_and_keeps_the_method(cuda):
    """The tile autotuner times every (sinks per group, direct-sum threshold)
    candidate, keeps the fastest, and the tuned tree gives the forces of a
    tree built with those sizes, which match the oracle with them."""
    import torch
    import paper_1407_2600_gb300.nbody as nb
    tree, pos, mom, off, eps = _setup(cuda)
    res = tree.autotune()
    cands = res["candidates"]
    assert len(cands) == 12
    best = min(cands, key=lambda c: c["ms"])
    assert (res["n_group"], res["n_direct"]) == (best["n_group"], best["n_direct"])
    acc = tree.forces()
    prm = nb.params(eps=eps[0], theta=0.5, order=2, n_direct=res["n_direct"], n_group=res["n_group"],
                    ewald_grid=4, flags=nb.NBODY_FLAG_MAC_EDGE)
    fresh = nb.Tree(prm, pos, offsets=off.tolist(), eps=eps)
    assert torch.equal(fresh.forces(), acc)
    fresh.close()
    x = pos.cpu().numpy().T
    a = acc.cpu().numpy().T.astype(np.float64)
    b = len(SIZES) - 1
    xb = x[off[b]:off[b + 1]]
    tgt = ics.random_targets(len(xb), 128, 77)
    at = oracle.tree_forces(xb, None, oracle.tree_params(eps[b], 0.5, 2, n_direct=res["n_direct"],
                                                         n_group=res["n_group"], ewald=4, mac=1, ew_grid=4),
                            targets=tgt)
    rt = np.linalg.norm(a[off[b] + tgt] - at, axis=1) / np.linalg.norm(at, axis=1)
    assert np.median(rt) <= 1e-5, np.median(rt)
    tree.close()



def test_fullsize_96_boxes_captured_force_vs_oracle(cuda):
    """The full batched workload in the benchmark's launch configuration: 96
    boxes (32 x 48^3 + 32 x 64^3 + 32 x 80^3 = 28,311,552 particles) in one
    build and one walk, on capacities reserved at 1.1x the counts, the
    rebuild and force evaluation captured in a CUDA graph and replayed.  The
    replayed forces equal the uncaptured ones bit for bit, and sampled
    particles of one box of each size match the oracle tree of that box."""
    import torch
    import paper_1407_2600_gb300.nbody as nb
    x, p, off, eps = ics.config_batched(1)
    assert off[-1] == 32 * (48 ** 3 + 64 ** 3 + 80 ** 3)
    pos = torch.tensor(np.ascontiguousarray(x.T), dtype=torch.float64, device=cuda)
    prm = nb.params(eps=eps[0], theta=0.5, order=2, n_direct=16, ewald_grid=4,
                    flags=nb.NBODY_FLAG_ASYNC | nb.NBODY_FLAG_MAC_EDGE | nb.NBODY_FLAG_BACKGROUND)
    tree = nb.Tree(prm, pos, offsets=off.tolist(), eps=eps)
    acc_e = tree.forces()
    torch.cuda.synchronize()
    tree.check()
    tree.reserve(0.1)
    acc = torch.zeros_like(acc_e)
    tree.forces(acc)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        tree.rebuild()
        tree.forces(acc)
    acc.zero_()
    graph.replay()
    torch.cuda.synchronize()
    tree.check()
    assert torch.equal(acc, acc_e)
    a = acc.cpu().numpy().T.astype(np.float64)
    del graph
    tree.close()
    for b in (0, 40, 95):
        xb = x[off[b]:off[b + 1]]
        tgt = ics.random_targets(len(xb), 256, 300 + b)
        at = oracle.tree_forces(xb, None, oracle.tree_params(eps[b], 0.5, 2, n_direct=16, ewald=4, mac=1,
                                                             ew_grid=4, bg=4), targets=tgt)
        rt = np.linalg.norm(a[off[b] + tgt] - at, axis=1) / np.linalg.norm(at, axis=1)
        assert np.median(rt) <= 1e-5, (b, np.median(rt))
