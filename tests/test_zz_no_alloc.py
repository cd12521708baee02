"""The allocation-free Morton sort against the sort inside nbody_build_tree.

Callers that cannot allocate device memory at run time (another allocator
owns or caps the device memory, cudaMalloc's implicit synchronisation is not
acceptable, or the device footprint must stay fixed after set-up) use
nbody_sort_keys_noalloc, whose scratch is a fixed device array inside the
library.  It must give the same keys and permutation as the allocating path,
call after call, even though each call reuses the array the previous call
left behind.  This file is collected last on purpose."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _noalloc(nb, pos, n, dev):
    import torch
    keys = torch.empty(n, dtype=torch.int64, device=dev)
    perm = torch.empty(n, dtype=torch.int32, device=dev)
    rc = nb.nbody_sort_keys_noalloc(pos.data_ptr(), n, keys.data_ptr(), perm.data_ptr(), nb._stream())
    return rc, keys, perm


def test_noalloc_sort_matches_allocating_path_two_calls(cuda):
    import torch
    import paper_1407_2600_gb300.nbody as nb
    # two calls in a row; the second is smaller, so stale scratch from the
    # first call would show up as a mismatch
    for n, seed in ((200003, 1), (65537, 2)):
        rng = np.random.default_rng(seed)
        x = rng.uniform(0.0, 1.0, (n, 3))
        x[: n // 20] = x[0]  # equal keys: the order must stay the input order
        pos = torch.tensor(np.ascontiguousarray(x.T), dtype=torch.float64, device=cuda)
        rc, keys, perm = _noalloc(nb, pos, n, cuda)
        assert rc == nb.NBODY_OK, nb.nbody_strerror(rc)
        tree = nb.Tree(nb.params(eps=1e-3), pos)
        ref_keys = tree.export("sorted_keys")
        ref_perm = tree.export("perm")
        tree.close()
        torch.cuda.synchronize()
        assert torch.equal(keys, ref_keys)  # integer work: bit-exact
        assert torch.equal(perm, ref_perm)


def test_noalloc_rejects_sizes_beyond_its_maximum(cuda):
    import torch
    import paper_1407_2600_gb300.nbody as nb
    pos = torch.zeros((3, 4), dtype=torch.float64, device=cuda)
    out = torch.zeros(8, dtype=torch.int64, device=cuda)
    rc = nb.nbody_sort_keys_noalloc(pos.data_ptr(), (1 << 20) + 1, out.data_ptr(), out.data_ptr(), nb._stream())
    assert rc == nb.NBODY_ERANGE
    assert "maximum" in nb.nbody_strerror(rc)


def test_noalloc_rejects_non_finite_positions(cuda):
    """A NaN or infinite coordinate is reported as NBODY_EINVAL, as
    nbody_build_tree reports it, and the next call on finite positions is
    unaffected (the error word is cleared per call)."""
    import torch
    import paper_1407_2600_gb300.nbody as nb
    n = 4097
    rng = np.random.default_rng(3)
    x = rng.uniform(0.0, 1.0, (n, 3))
    for bad in (np.nan, np.inf, -np.inf):
        y = x.copy()
        y[1234, 2] = bad
        pos = torch.tensor(np.ascontiguousarray(y.T), dtype=torch.float64, device=cuda)
        rc, _, _ = _noalloc(nb, pos, n, cuda)
        assert rc == nb.NBODY_EINVAL, nb.nbody_strerror(rc)
    pos = torch.tensor(np.ascontiguousarray(x.T), dtype=torch.float64, device=cuda)
    rc, keys, perm = _noalloc(nb, pos, n, cuda)
    assert rc == nb.NBODY_OK, nb.nbody_strerror(rc)
    tree = nb.Tree(nb.params(eps=1e-3), pos)
    assert torch.equal(keys, tree.export("sorted_keys"))
    assert torch.equal(perm, tree.export("perm"))
    tree.close()
