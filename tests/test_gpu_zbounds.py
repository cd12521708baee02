"""Every path of the library run through its bounds-checked debug build.

The debug library (libnbody_dbg.so, compiled with -DNB_DEBUG_BOUNDS) checks
each index that a kernel derives from data (sorted ranks, cell and group
indices read from the tree, stack entries, particle indices of leaves, run
heads, table nodes, scatter targets of the permutation) before it is used.
A failed check records (site, index) in its translation unit's fault word and
the access is skipped, so a bad index is reported instead of being read or
written.  This file builds that library, runs small cases of every path
through it in a child process (the sort, the allocation-free sort, the tree
build, the upward pass, both walk forms, the uniform-background terms, K1
softening, the near replicas, the potential, the FP64 mode, batched boxes, a
KDK step and the reverse mode), and checks that no check fired and that the
results equal those of the product library.  It is the bounds evidence that
does not rely on a stray access happening to break a parity test."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_1407_2600_gb300 import ics

pytestmark = pytest.mark.gpu

UNITS = ("sort", "build", "upward", "walk", "periodic", "adjoint")


def run_cases(dev: str, after=None) -> dict:
    """Small cases of every path; arrays keyed by case (the library is the
    one paper_1407_2600_gb300.nbody loads).  after(name), when given, runs
    after each case (the child reads the fault words there)."""
    import torch
    import paper_1407_2600_gb300.nbody as nb

    def t(a, dtype=torch.float64):
        return torch.tensor(np.ascontiguousarray(a.T), dtype=dtype, device=dev)

    x, eps = ics.config_haloes(16, seed=5, n_halo=3, nmin=100, nmax=600)
    n = len(x)
    out = {}

    def done(name):
        torch.cuda.synchronize()
        if after is not None:
            after(name)

    settings = {
        "m2p": dict(theta=0.6, order=4),
        "dual": dict(theta=0.6, order=4, flags=nb.NBODY_FLAG_DUAL),
        "bg_face": dict(theta=0.5, order=4, n_direct=4, flags=nb.NBODY_FLAG_MAC_EDGE | nb.NBODY_FLAG_BACKGROUND),
        "k1": dict(theta=0.5, order=2, flags=nb.NBODY_FLAG_K1),
        "replicas": dict(theta=0.5, order=4, ewald_order=0, flags=nb.NBODY_FLAG_REPLICAS),
        "fp64": dict(theta=0.5, order=4, precision=1),
    }
    for name, kw in settings.items():
        tree = nb.Tree(nb.params(eps=eps, **kw), t(x))
        if name == "fp64":
            out[name] = tree.forces64().cpu().numpy()
        else:
            out[name] = tree.forces().cpu().numpy()
        tree.close()
        done(name)
    # the potential beside the forces
    tree = nb.Tree(nb.params(eps=eps, theta=0.5, order=4), t(x))
    acc, pot = tree.forces(pot=True)
    out["pot_acc"] = acc.cpu().numpy()
    out["pot"] = pot.cpu().numpy()
    tree.close()
    done("pot")
    # one KDK step, then the reverse mode of the force
    tree = nb.Tree(nb.params(eps=eps, theta=0.5, order=4), t(x))
    acc = tree.forces()
    mom = torch.zeros((3, n), dtype=torch.float32, device=dev)
    tree.kdk_step(mom, acc, 0.05, 0.06)
    out["kdk_pos"] = tree.pos.cpu().numpy()
    done("kdk")
    lam = np.random.default_rng(3).standard_normal((n, 3)).astype(np.float32)
    out["vjp"] = tree.forces_vjp(t(lam, torch.float32)).cpu().numpy()
    tree.close()
    done("vjp")
    # batched boxes of uneven sizes
    boxes = [ics.config_small(7)[0], np.random.default_rng(8).uniform(0, 1, (999, 3))]
    off = np.cumsum([0] + [len(b) for b in boxes])
    tree = nb.Tree(nb.params(eps=1e-3, theta=0.5, order=2), t(np.concatenate(boxes)), offsets=off.tolist(),
                   eps=[1.0 / 480, 2e-3])
    out["batched"] = tree.forces().cpu().numpy()
    tree.close()
    done("batched")
    # the allocation-free sort
    keys = torch.empty(n, dtype=torch.int64, device=dev)
    perm = torch.empty(n, dtype=torch.int32, device=dev)
    pos = t(x)
    rc = nb.nbody_sort_keys_noalloc(pos.data_ptr(), n, keys.data_ptr(), perm.data_ptr(), nb._stream())
    assert rc == nb.NBODY_OK, nb.nbody_strerror(rc)
    out["noalloc_perm"] = perm.cpu().numpy()
    done("noalloc")
    return out


_CHILD = r"""
import importlib.util, json, sys, ctypes
import numpy as np
sys.path.insert(0, sys.argv[1])
spec = importlib.util.spec_from_file_location("zbounds", sys.argv[2])
m = importlib.util.module_from_spec(spec)
spec.loader.exec_module(m)
import paper_1407_2600_gb300.nbody as nb
L = nb.lib()
faults = {}
def after(name):
    for u in m.UNITS:
        f = getattr(L, "nbody_dbg_fault_" + u)
        f.argtypes = [ctypes.POINTER(ctypes.c_ulonglong), ctypes.c_int]
        v = ctypes.c_ulonglong(0)
        rc = f(ctypes.byref(v), 1)
        if rc or v.value:
            faults.setdefault(name, {})[u] = [int(rc), int(v.value)]
    print("CASE " + name + " " + json.dumps(faults.get(name, {})), flush=True)
try:
    out = m.run_cases("cuda:0", after)
    np.savez(sys.argv[3], **out)
finally:
    print("FAULTS " + json.dumps(faults), flush=True)
"""


def test_debug_bounds_build_every_path(cuda, tmp_path):
    from paper_1407_2600_gb300 import build as libbuild
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    dbg = libbuild.build(debug_bounds=True)
    npz = str(tmp_path / "dbg.npz")
    env = dict(os.environ, NBODY_LIBRARY=dbg)
    r = subprocess.run([sys.executable, "-c", _CHILD, root, os.path.abspath(__file__), npz], env=env,
                       capture_output=True, text=True, timeout=900)
    lines = [s for s in r.stdout.splitlines() if s.startswith("FAULTS ")]
    faults = json.loads(lines[-1][len("FAULTS "):]) if lines else {}
    # a nonzero word is (site << 48) | index of the first failed check
    failed = ["case %s, unit %s: rc %d, site %d, index %d" % (case, u, rc, word >> 48, word & ((1 << 48) - 1))
              for case, units in faults.items() for u, (rc, word) in units.items() if rc or word]
    assert not failed, failed
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    got = dict(np.load(npz))
    ref = run_cases(str(cuda))
    assert set(got) == set(ref)
    for k in ref:
        if ref[k].dtype.kind in "iu":
            assert np.array_equal(got[k], ref[k]), k  # integer work: bit-exact
        else:
            # the same arithmetic; only code placement differs between the builds
            scale = np.max(np.abs(ref[k])) + 1e-300
            assert np.max(np.abs(got[k] - ref[k])) <= 1e-6 * scale, (k, np.max(np.abs(got[k] - ref[k])) / scale)
