"""GPU parity of the potential (nbody_forces' pot_dev) against the FP64 CPU
oracle's tree potential, through the C ABI.

The potential crosses zero (zero-mean periodic convention), so errors are
measured per particle against the root-mean-square potential of the sample:
|phi_gpu - phi_oracle| / rms(phi_oracle), with the tree-parity bars of the
forces (median <= 1e-5, 99th percentile <= 1e-4) in the mixed-precision mode,
and the FP32 rounding of output and masses in the all-FP64 mode."""
import numpy as np
import pytest

import oracle
from paper_1407_2600_gb300 import ics

pytestmark = pytest.mark.gpu


def _nb():
    import paper_1407_2600_gb300.nbody as nb
    return nb


def _pos(x, dev):
    import torch
    return torch.tensor(np.ascontiguousarray(x.T), dtype=torch.float64, device=dev)


def _gpu(x, dev, **kw):
    import torch
    nb = _nb()
    tree = nb.Tree(nb.params(**kw), _pos(x, dev))
    acc, pot, st = tree.forces(pot=True, stats=True)
    torch.cuda.synchronize()
    out = acc.cpu().numpy().T.astype(np.float64), pot.cpu().numpy().astype(np.float64), st
    tree.close()
    return out


def _err(p, ref):
    e = np.abs(p - ref) / np.sqrt(np.mean(ref ** 2))
    return np.median(e), np.percentile(e, 99)


def _clustered(seed=7):
    x, eps = ics.config_small(seed)
    x = np.concatenate([x, np.mod(0.3 + 0.01 * np.random.default_rng(3).standard_normal((800, 3)), 1.0)])
    return x, eps


CASES = [
    # (name, extra GPU flags, extra oracle parameters, order, theta)
    ("plain_p4", 0, {}, 4, 0.5),
    ("plain_p2", 0, {}, 2, 0.6),
    ("k1_p4", "K1", {"kernel": 1}, 4, 0.5),
    ("edge_bg_p4", "MAC_EDGE|BACKGROUND", {"mac": 1, "bg": 6}, 4, 0.7),
    ("edge_bg_p2", "MAC_EDGE|BACKGROUND", {"mac": 1, "bg": 4}, 2, 0.5),
    ("dual_p4", "DUAL", {"dual": 1}, 4, 0.5),
]


def _flags(nb, spec):
    if not spec:
        return 0
    f = 0
    for name in spec.split("|"):
        f |= getattr(nb, "NBODY_FLAG_" + name)
    return f


@pytest.mark.parametrize("name,flags,extra,order,theta", CASES)
def test_potential_vs_oracle_tree(cuda, name, flags, extra, order, theta):
    """The same method on both sides (identical opening decisions), so the
    differences are FP32 rounding; the accelerations returned with the
    potential are the oracle tree's too (with the dual form, the dual
    form's)."""
    nb = _nb()
    x, eps = _clustered()
    if extra.get("kernel") == 1:
        eps = 4 * eps
    a, p, st = _gpu(x, cuda, eps=eps, theta=theta, order=order, n_direct=4, flags=_flags(nb, flags))
    ra, rp = oracle.tree_forces(x, None, oracle.tree_params(eps, theta, order, n_direct=4, ewald=4, **extra),
                                return_pot=True)
    assert np.isfinite(p).all()
    med, p99 = _err(p, rp)
    assert med <= 1e-5 and p99 <= 1e-4, (med, p99)
    rel = np.linalg.norm(a - ra, axis=1) / np.linalg.norm(ra, axis=1)
    assert np.median(rel) <= 1e-5 and np.percentile(rel, 99) <= 1e-4, (np.median(rel), np.percentile(rel, 99))


def test_potential_fp64_mode_and_no_images(cuda):
    """All-FP64 interactions match the oracle to the rounding of the FP32
    output (2^-24 of each value) and of the FP32 particle mass 1/n (every
    term carries the same mass, so it scales the whole potential), plus
    1e-10 of the rms (periodic, and with the image field off, where the
    potential is the walk's alone)."""
    x, eps = _clustered(8)
    n = len(x)
    dm = abs(float(np.float32(1.0 / n)) * n - 1.0)
    for ew in (4, 0):
        _, p, _ = _gpu(x, cuda, eps=eps, theta=0.5, order=4, n_direct=4, precision=1, ewald_order=ew)
        _, rp = oracle.tree_forces(x, None, oracle.tree_params(eps, 0.5, 4, n_direct=4, ewald=ew),
                                   return_pot=True)
        bound = (2.0 ** -24 + dm) * np.abs(rp) + 1e-10 * np.sqrt(np.mean(rp ** 2))
        assert np.all(np.abs(p - rp) <= bound), (ew, np.max(np.abs(p - rp) / bound))


def test_potential_accelerations_equal_the_force_path(cuda):
    """Asking for the potential leaves the accelerations as nbody_forces
    gives them without it (to FP32 summation order: the potential variant
    of the walk is the scalar one)."""
    import torch
    nb = _nb()
    x, eps = _clustered(9)
    tree = nb.Tree(nb.params(eps=eps, theta=0.6, order=4), _pos(x, cuda))
    a0 = tree.forces().cpu().numpy().T.astype(np.float64)
    a1, p = tree.forces(pot=True)
    torch.cuda.synchronize()
    a1 = a1.cpu().numpy().T.astype(np.float64)
    a2 = tree.forces().cpu().numpy().T.astype(np.float64)
    tree.close()
    assert np.array_equal(a0, a2)
    rel = np.linalg.norm(a1 - a0, axis=1) / np.linalg.norm(a0, axis=1)
    assert np.median(rel) <= 1e-6 and rel.max() <= 1e-4, (np.median(rel), rel.max())


def test_potential_box_length_and_lattice(cuda):
    """With a box of side L the potential comes back as G m / L (exactly, L a
    power of two); a simple cubic lattice's potential is the Madelung value
    m k xi everywhere (xi from the golden fixture; the oracle tree with the
    background terms is within 4e-7 of it), and the order-1 image field is
    refused.  On the lattice the potential (2.8e-3) is the small remainder
    of terms summing to about 2.4 in magnitude, so FP32 rounding bounds the
    agreement in absolute terms: 1e-5 (G M / L), a few hundred terms of
    relative rounding 6e-8."""
    import os
    import torch
    nb = _nb()
    x, eps = ics.config_small(2)
    _, p1, _ = _gpu(x, cuda, eps=eps, theta=0.5, order=2)
    _, pL, _ = _gpu(x * 64.0, cuda, eps=eps * 64.0, theta=0.5, order=2, box_len=64.0)
    assert np.array_equal(pL * 64.0, p1)
    k = 32
    g = (np.arange(k) + 0.5) / k
    lat = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "madelung_simple_cubic.txt")) as f:
        xi = float([ln for ln in f if ln.strip() and not ln.startswith("#")][0])
    want = xi * k / len(lat)
    _, p, _ = _gpu(lat, cuda, eps=1e-6, theta=0.5, order=4, flags=nb.NBODY_FLAG_MAC_EDGE | nb.NBODY_FLAG_BACKGROUND)
    tg = ics.random_targets(len(lat), 64, 4)
    _, rp = oracle.tree_forces(lat, None, oracle.tree_params(1e-6, 0.5, 4, ewald=4, mac=1, bg=6), targets=tg,
                               return_pot=True)
    assert np.abs(p[tg] - rp).max() <= 1e-5, np.abs(p[tg] - rp).max()
    assert np.abs(p - want).max() <= 1e-5, np.abs(p - want).max()
    tree = nb.Tree(nb.params(eps=eps, theta=0.5, order=2, ewald_order=1), _pos(x, cuda))
    acc = torch.empty((3, len(x)), dtype=torch.float32, device=cuda)
    pot = torch.empty(len(x), dtype=torch.float32, device=cuda)
    assert nb.nbody_forces(tree.handle, acc.data_ptr(), pot.data_ptr(), None, nb._stream()) == nb.NBODY_ENOTSUP
    tree.close()


def test_potential_fullsize_sampled(cuda):
    """The benchmark workload (128^3 Zel'dovich + 64 NFW haloes) at its
    setting: the potential of 512 seeded targets against the oracle tree's."""
    x, eps = ics.config_haloes(128, seed=1)
    _, p, _ = _gpu(x, cuda, eps=eps, theta=0.6, order=4, n_direct=8, ewald_grid=5)
    assert np.isfinite(p).all()
    tg = ics.random_targets(len(x), 512, 11)
    _, rp = oracle.tree_forces(x, None, oracle.tree_params(eps, 0.6, 4, n_direct=8, ewald=4, ew_grid=5),
                               targets=tg, return_pot=True)
    med, p99 = _err(p[tg], rp)
    assert med <= 1e-5 and p99 <= 1e-4, (med, p99)
