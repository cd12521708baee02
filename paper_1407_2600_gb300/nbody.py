"""Thin Python binding of the C ABI in include/nbody.h (argument marshalling only).

Every function here forwards to the entry point of the same name in
``libnbody.so``; the ``*_t`` helpers accept torch CUDA tensors and pass their
device pointers and the current stream.  All computation happens in the CUDA
library; there is no fallback.  Loading fails loudly when the library has not
been built (``python -m paper_1407_2600_gb300.build`` or ``__graft_entry__.build()``).
"""
from __future__ import annotations

import ctypes as C
import math
import os
from dataclasses import dataclass, field

HERE = os.path.dirname(os.path.abspath(__file__))
# NBODY_LIBRARY names another build of the same library (the tests' bounds-
# checked debug build); by default the product library beside this file
LIB_PATH = os.environ.get("NBODY_LIBRARY") or os.path.join(HERE, "libnbody.so")

NBODY_OK = 0
NBODY_EINVAL = -1
NBODY_ENOMEM = -2
NBODY_ECUDA = -3
NBODY_EOVERFLOW = -4
NBODY_ETIMEOUT = -5
NBODY_ENOTSUP = -6
NBODY_ERANGE = -7
NBODY_MIXED = 0
NBODY_FP64 = 1
NBODY_FLAG_ASYNC = 1
NBODY_FLAG_MAC_EDGE = 2
NBODY_FLAG_BACKGROUND = 4
NBODY_FLAG_K1 = 8
NBODY_FLAG_DUAL = 16
NBODY_FLAG_REPLICAS = 32


def NBODY_FLAG_WALK_VARIANT(v: int) -> int:
    """flags bits selecting walk launch variant v instead of the autotuned one"""
    return (v + 1) << 8
EXPORT = {"sorted_keys": 1, "perm": 2, "cell_keys": 3, "cell_range": 4, "cell_level": 5,
          "moments": 6, "groups": 7, "image_table": 8}

# every symbol include/nbody.h declares
SYMBOLS = ["nbody_default_params", "nbody_build_tree", "nbody_build_tree_batched", "nbody_forces_batched",
           "nbody_forces", "nbody_forces64",
           "nbody_kdk_step", "nbody_assign_rungs", "nbody_forces_active", "nbody_kdk_multistep", "nbody_kdk_adjoint", "nbody_kdk_adjoint_acc", "nbody_forces_vjp", "nbody_tree_count",
           "nbody_tree_export", "nbody_tree_lookup", "nbody_reserve", "nbody_autotune", "nbody_check",
           "nbody_tree_free",
           "nbody_strerror", "nbody_timing_read", "nbody_sort_keys_noalloc", "nbody_cic_loss",
           "nbody_zeldovich_state", "nbody_zeldovich_vjp"]


class Params(C.Structure):
    _fields_ = [("eps", C.c_double), ("theta", C.c_double), ("order", C.c_int), ("n_leaf", C.c_int),
                ("n_group", C.c_int), ("n_direct", C.c_int), ("lmax", C.c_int),
                ("ewald_order", C.c_int), ("ewald_level", C.c_int), ("ewald_grid", C.c_int),
                ("precision", C.c_int), ("flags", C.c_int), ("box_len", C.c_double)]


class Stats(C.Structure):
    _fields_ = [("p2p", C.c_double), ("m2p", C.c_double), ("m2l", C.c_double),
                ("ncells", C.c_int64), ("ngroups", C.c_int64), ("max_level", C.c_int32),
                ("nbox", C.c_int32), ("ms_sort", C.c_float), ("ms_build", C.c_float),
                ("ms_upward", C.c_float), ("ms_walk", C.c_float), ("ms_periodic", C.c_float),
                ("decision_hash", C.c_uint64)]

    def asdict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Timing(C.Structure):
    _fields_ = [("builds", C.c_int64), ("evaluations", C.c_int64), ("launches", C.c_int64),
                ("p2p", C.c_double), ("m2p", C.c_double), ("m2l", C.c_double),
                ("ms_sort", C.c_double), ("ms_build", C.c_double), ("ms_upward", C.c_double),
                ("ms_walk", C.c_double), ("ms_periodic", C.c_double),
                ("adjoint_steps", C.c_int64), ("adjoint_reused", C.c_int64),
                ("decision_hash", C.c_uint64), ("walk_variant", C.c_int64), ("walk_tune_ms", C.c_double * 8),
                ("m2l_dual", C.c_double)]

    def asdict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["walk_tune_ms"] = list(self.walk_tune_ms)
        return d


class Tune(C.Structure):
    _fields_ = [("ncand", C.c_int32), ("n_group", C.c_int32 * 12), ("n_direct", C.c_int32 * 12),
                ("ms", C.c_double * 12), ("best", C.c_int32)]

    def asdict(self):
        k = self.ncand
        return {"candidates": [{"n_group": self.n_group[i], "n_direct": self.n_direct[i], "ms": self.ms[i]}
                               for i in range(k)],
                "n_group": self.n_group[self.best] if self.best >= 0 else None,
                "n_direct": self.n_direct[self.best] if self.best >= 0 else None}


class NbodyError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__("%s failed: %s (%d)" % (where, nbody_strerror(code), code))


_LIB = None
_vp = C.c_void_p


def lib():
    """Load libnbody.so; raises if it is missing (no CPU fallback exists)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libnbody.so is not built: run __graft_entry__.build() "
                               "(the CUDA library is required; there is no fallback)")
        L = C.CDLL(LIB_PATH)
        L.nbody_default_params.argtypes = [C.POINTER(Params)]
        L.nbody_default_params.restype = None
        L.nbody_build_tree.argtypes = [C.POINTER(Params), C.c_int64, _vp, _vp, C.POINTER(_vp), _vp]
        L.nbody_build_tree_batched.argtypes = [C.POINTER(Params), C.c_int, C.POINTER(C.c_int64),
                                               C.POINTER(C.c_double), _vp, _vp, C.POINTER(_vp), _vp]
        L.nbody_forces_batched.argtypes = [C.POINTER(Params), C.c_int, C.POINTER(C.c_int64),
                                           C.POINTER(C.c_double), C.POINTER(C.c_double), _vp, _vp, _vp,
                                           C.POINTER(_vp), _vp]
        L.nbody_forces.argtypes = [_vp, _vp, _vp, C.POINTER(Stats), _vp]
        L.nbody_forces64.argtypes = [_vp, _vp, _vp]
        L.nbody_kdk_step.argtypes = [_vp, _vp, _vp, _vp, C.c_double, C.c_double, _vp]
        L.nbody_assign_rungs.argtypes = [_vp, _vp, C.c_double, C.c_double, C.c_int, _vp, _vp]
        L.nbody_forces_active.argtypes = [_vp, _vp, C.c_int, _vp, _vp]
        L.nbody_kdk_multistep.argtypes = [_vp, _vp, _vp, _vp, _vp, C.c_double, C.c_double, C.c_int, _vp]
        L.nbody_kdk_adjoint.argtypes = [_vp, _vp, _vp, C.c_double, C.c_double, _vp, _vp, _vp, _vp, _vp]
        L.nbody_kdk_adjoint_acc.argtypes = [_vp, _vp, _vp, _vp, C.c_double, C.c_double, _vp, _vp, _vp, _vp,
                                            _vp]
        L.nbody_forces_vjp.argtypes = [_vp, _vp, _vp, _vp]
        L.nbody_tree_count.argtypes = [_vp, C.c_int]
        L.nbody_tree_count.restype = C.c_int64
        L.nbody_tree_export.argtypes = [_vp, C.c_int, _vp, _vp]
        L.nbody_tree_lookup.argtypes = [_vp, _vp, C.c_int64, _vp, _vp]
        L.nbody_reserve.argtypes = [_vp, C.c_int64, C.c_int64, _vp]
        L.nbody_autotune.argtypes = [_vp, C.POINTER(Tune), _vp]
        L.nbody_check.argtypes = [_vp, _vp]
        L.nbody_tree_free.argtypes = [_vp]
        L.nbody_tree_free.restype = None
        L.nbody_timing_read.argtypes = [_vp, C.POINTER(Timing), C.c_int]
        L.nbody_sort_keys_noalloc.argtypes = [_vp, C.c_int64, _vp, _vp, _vp]
        L.nbody_cic_loss.argtypes = [_vp, _vp, C.c_int64, C.c_int, _vp, _vp, _vp, _vp]
        L.nbody_zeldovich_state.argtypes = [C.c_int64, _vp, _vp, C.c_double, _vp, _vp, _vp]
        L.nbody_zeldovich_vjp.argtypes = [C.c_int64, C.c_double, _vp, _vp, _vp, _vp]
        L.nbody_strerror.argtypes = [C.c_int]
        L.nbody_strerror.restype = C.c_char_p
        _LIB = L
    return _LIB


def _check(rc, where):
    if rc != NBODY_OK:
        raise NbodyError(rc, where)


# ---- the C entry points, same names -------------------------------------------
def nbody_default_params() -> Params:
    p = Params()
    lib().nbody_default_params(C.byref(p))
    return p


def nbody_build_tree(params: Params, n: int, pos_dev: int, mass_dev: int | None, tree=None,
                     stream: int | None = None):
    h = _vp(tree)
    rc = lib().nbody_build_tree(C.byref(params), n, pos_dev, mass_dev, C.byref(h), stream)
    return rc, h.value


def nbody_build_tree_batched(params: Params, offsets, eps, pos_dev: int, mass_dev: int | None,
                             tree=None, stream: int | None = None):
    nbox = len(offsets) - 1
    off = (C.c_int64 * (nbox + 1))(*[int(v) for v in offsets])
    ep = None if eps is None else (C.c_double * nbox)(*[float(v) for v in eps])
    h = _vp(tree)
    rc = lib().nbody_build_tree_batched(C.byref(params), nbox, off, ep, pos_dev, mass_dev,
                                        C.byref(h), stream)
    return rc, h.value


def nbody_forces_batched(params: Params, offsets, box_len, eps, pos_dev: int, mass_dev: int | None, acc_dev: int,
                         tree=None, stream: int | None = None):
    nbox = len(offsets) - 1
    off = (C.c_int64 * (nbox + 1))(*[int(v) for v in offsets])
    ln = None if box_len is None else (C.c_double * nbox)(*[float(v) for v in box_len])
    ep = None if eps is None else (C.c_double * nbox)(*[float(v) for v in eps])
    h = _vp(tree)
    rc = lib().nbody_forces_batched(C.byref(params), nbox, off, ln, ep, pos_dev, mass_dev, acc_dev, C.byref(h),
                                    stream)
    return rc, h.value


def nbody_forces(tree: int, acc_dev: int, pot_dev: int | None = None, stats: Stats | None = None,
                 stream: int | None = None) -> int:
    return lib().nbody_forces(tree, acc_dev, pot_dev, C.byref(stats) if stats is not None else None, stream)


def nbody_forces64(tree: int, acc_dev: int, stream: int | None = None) -> int:
    return lib().nbody_forces64(tree, acc_dev, stream)


def nbody_kdk_step(tree: int, pos_dev: int, mom_dev: int, acc_dev: int, a0: float, a1: float,
                   stream: int | None = None) -> int:
    return lib().nbody_kdk_step(tree, pos_dev, mom_dev, acc_dev, a0, a1, stream)


def nbody_assign_rungs(tree: int, acc_dev: int, eta: float, dlna: float, rmax: int, rung_dev: int,
                       stream: int | None = None) -> int:
    return lib().nbody_assign_rungs(tree, acc_dev, eta, dlna, rmax, rung_dev, stream)


def nbody_forces_active(tree: int, rung_dev: int, rmin: int, acc_dev: int, stream: int | None = None) -> int:
    return lib().nbody_forces_active(tree, rung_dev, rmin, acc_dev, stream)


def nbody_kdk_multistep(tree: int, pos_dev: int, mom_dev: int, acc_dev: int, rung_dev: int, a0: float, a1: float,
                        rmax: int, stream: int | None = None) -> int:
    return lib().nbody_kdk_multistep(tree, pos_dev, mom_dev, acc_dev, rung_dev, a0, a1, rmax, stream)


def nbody_kdk_adjoint(tree: int, pos0_dev: int, mom0_dev: int, a0: float, a1: float,
                      lam_pos1_dev: int, lam_mom1_dev: int, lam_pos0_dev: int, lam_mom0_dev: int,
                      stream: int | None = None) -> int:
    return lib().nbody_kdk_adjoint(tree, pos0_dev, mom0_dev, a0, a1, lam_pos1_dev, lam_mom1_dev,
                                   lam_pos0_dev, lam_mom0_dev, stream)


def nbody_kdk_adjoint_acc(tree: int, pos0_dev: int, mom0_dev: int, acc0_dev: int, a0: float, a1: float,
                          lam_pos1_dev: int, lam_mom1_dev: int, lam_pos0_dev: int, lam_mom0_dev: int,
                          stream: int | None = None) -> int:
    return lib().nbody_kdk_adjoint_acc(tree, pos0_dev, mom0_dev, acc0_dev, a0, a1, lam_pos1_dev, lam_mom1_dev,
                                       lam_pos0_dev, lam_mom0_dev, stream)


def nbody_forces_vjp(tree: int, lam_dev: int, out_dev: int, stream: int | None = None) -> int:
    return lib().nbody_forces_vjp(tree, lam_dev, out_dev, stream)


def nbody_tree_count(tree: int, what: int) -> int:
    return lib().nbody_tree_count(tree, what)


def nbody_tree_export(tree: int, what: int, dst_dev: int, stream: int | None = None) -> int:
    return lib().nbody_tree_export(tree, what, dst_dev, stream)


def nbody_tree_lookup(tree: int, keys_dev: int, nkeys: int, idx_dev: int, stream: int | None = None) -> int:
    return lib().nbody_tree_lookup(tree, keys_dev, nkeys, idx_dev, stream)


def nbody_reserve(tree: int, max_cells: int, max_groups: int, stream: int | None = None) -> int:
    return lib().nbody_reserve(tree, max_cells, max_groups, stream)


def nbody_autotune(tree: int, out: Tune | None = None, stream: int | None = None) -> int:
    return lib().nbody_autotune(tree, C.byref(out) if out is not None else None, stream)


def nbody_check(tree: int, stream: int | None = None) -> int:
    return lib().nbody_check(tree, stream)


def nbody_tree_free(tree: int) -> None:
    if tree:
        lib().nbody_tree_free(tree)


def nbody_timing_read(tree: int, out: Timing, reset: int) -> int:
    return lib().nbody_timing_read(tree, C.byref(out), reset)


def nbody_sort_keys_noalloc(pos_dev: int, n: int, keys_out_dev: int, perm_out_dev: int,
                            stream: int | None = None) -> int:
    return lib().nbody_sort_keys_noalloc(pos_dev, n, keys_out_dev, perm_out_dev, stream)


def nbody_cic_loss(pos_dev: int, mass_dev: int | None, n: int, ng: int, grid_dev: int, loss_dev: int,
                   grad_dev: int | None, stream: int | None = None) -> int:
    return lib().nbody_cic_loss(pos_dev, mass_dev, n, ng, grid_dev, loss_dev, grad_dev, stream)


def nbody_strerror(code: int) -> str:
    return lib().nbody_strerror(code).decode()


# ---- torch-tensor conveniences (marshalling only) ------------------------------------
def _stream():
    import torch
    return torch.cuda.current_stream().cuda_stream


def params(**kw) -> Params:
    p = nbody_default_params()
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


class Tree:
    """Owns one nbody_tree handle built from torch CUDA tensors (SoA (3, n))."""

    def __init__(self, prm: Params, pos, mass=None, offsets=None, eps=None):
        import torch
        if not pos.is_cuda or pos.dtype != torch.float64 or pos.dim() != 2 or pos.shape[0] != 3:
            raise ValueError("pos must be a CUDA float64 tensor of shape (3, n)")
        self.params = prm
        self.pos = pos.contiguous()
        self.mass = None if mass is None else mass.contiguous().float()
        self.n = pos.shape[1]
        self.offsets = offsets
        self.eps = eps
        self.handle = None
        self.rebuild()

    def rebuild(self):
        mp = None if self.mass is None else self.mass.data_ptr()
        if self.offsets is None:
            rc, h = nbody_build_tree(self.params, self.n, self.pos.data_ptr(), mp, self.handle, _stream())
        else:
            rc, h = nbody_build_tree_batched(self.params, self.offsets, self.eps, self.pos.data_ptr(), mp,
                                             self.handle, _stream())
        if h:
            self.handle = h
        _check(rc, "nbody_build_tree")

    def forces(self, acc=None, stats=False, pot=None):
        """(3, n) float32 accelerations; with pot=True (or an (n,) float32
        tensor to fill) also the potential: returns (acc, pot[, stats])."""
        import torch
        if acc is None:
            acc = torch.empty((3, self.n), dtype=torch.float32, device=self.pos.device)
        if pot is True:
            pot = torch.empty(self.n, dtype=torch.float32, device=self.pos.device)
        st = Stats() if stats else None
        _check(nbody_forces(self.handle, acc.data_ptr(), None if pot is None else pot.data_ptr(), st, _stream()),
               "nbody_forces")
        out = (acc,) if pot is None else (acc, pot)
        if stats:
            out = out + (st.asdict(),)
        return out[0] if len(out) == 1 else out

    def forces64(self, acc=None):
        """(3, n) float64 accelerations (nbody_forces64)."""
        import torch
        if acc is None:
            acc = torch.empty((3, self.n), dtype=torch.float64, device=self.pos.device)
        _check(nbody_forces64(self.handle, acc.data_ptr(), _stream()), "nbody_forces64")
        return acc

    def kdk_step(self, mom, acc, a0, a1):
        _check(nbody_kdk_step(self.handle, self.pos.data_ptr(), mom.data_ptr(), acc.data_ptr(), a0, a1,
                              _stream()), "nbody_kdk_step")

    def assign_rungs(self, acc, eta, dlna, rmax):
        """(n,) int8 rungs from (3, n) FP32 accelerations (nbody_assign_rungs)."""
        import torch
        rung = torch.empty(self.n, dtype=torch.int8, device=self.pos.device)
        _check(nbody_assign_rungs(self.handle, acc.data_ptr(), eta, dlna, rmax, rung.data_ptr(), _stream()),
               "nbody_assign_rungs")
        return rung

    def forces_active(self, rung, rmin, acc):
        """Accelerations of the particles with rung >= rmin written into acc."""
        _check(nbody_forces_active(self.handle, rung.data_ptr(), rmin, acc.data_ptr(), _stream()),
               "nbody_forces_active")
        return acc

    def kdk_multistep(self, mom, acc, rung, a0, a1, rmax):
        _check(nbody_kdk_multistep(self.handle, self.pos.data_ptr(), mom.data_ptr(), acc.data_ptr(),
                                   rung.data_ptr(), a0, a1, rmax, _stream()), "nbody_kdk_multistep")

    def forces_vjp(self, lam, out=None):
        """(d acc / d pos)^T lam for the tree as last built (lam: (3, n) float32)."""
        import torch
        if out is None:
            out = torch.empty((3, self.n), dtype=torch.float64, device=self.pos.device)
        lam = lam.contiguous().float()
        _check(nbody_forces_vjp(self.handle, lam.data_ptr(), out.data_ptr(), _stream()), "nbody_forces_vjp")
        return out

    def kdk_adjoint(self, pos0, mom0, a0, a1, lam_pos1, lam_mom1, acc0=None):
        """Cotangents of (pos0, mom0) of one KDK step given those of its outputs.
        With acc0 (g(x0) as nbody_forces / nbody_kdk_step returned it) the walk
        at x0 is skipped (nbody_kdk_adjoint_acc)."""
        import torch
        dev = self.pos.device
        # keep every converted input alive until the call has been issued
        x0 = pos0.contiguous()
        p0 = mom0.contiguous()
        lx1 = lam_pos1.to(torch.float64).contiguous()
        lp1 = lam_mom1.to(torch.float32).contiguous()
        lx0 = torch.empty((3, self.n), dtype=torch.float64, device=dev)
        lp0 = torch.empty((3, self.n), dtype=torch.float32, device=dev)
        if acc0 is None:
            _check(nbody_kdk_adjoint(self.handle, x0.data_ptr(), p0.data_ptr(), a0, a1, lx1.data_ptr(),
                                     lp1.data_ptr(), lx0.data_ptr(), lp0.data_ptr(), _stream()),
                   "nbody_kdk_adjoint")
        else:
            g0 = acc0.contiguous()
            _check(nbody_kdk_adjoint_acc(self.handle, x0.data_ptr(), p0.data_ptr(), g0.data_ptr(), a0, a1,
                                         lx1.data_ptr(), lp1.data_ptr(), lx0.data_ptr(), lp0.data_ptr(),
                                         _stream()), "nbody_kdk_adjoint_acc")
        return lx0, lp0

    def reserve(self, slack: float = 0.25, max_cells: int | None = None, max_groups: int | None = None):
        """Fix the cell and group capacities (nbody_reserve) at the given
        counts, or at the last build's counts times (1 + slack); slack < 0
        returns to counts read back per build.  Returns (max_cells, max_groups)."""
        if slack < 0:
            _check(nbody_reserve(self.handle, 0, 0, _stream()), "nbody_reserve")
            return 0, 0
        nc = nbody_tree_count(self.handle, EXPORT["cell_keys"])
        ng = nbody_tree_count(self.handle, EXPORT["groups"])
        if nc < 0 or ng < 0:
            _check(int(min(nc, ng)), "nbody_tree_count")
        mc = int(max_cells) if max_cells is not None else int(math.ceil(nc * (1.0 + slack))) + 64
        mg = int(max_groups) if max_groups is not None else int(math.ceil(ng * (1.0 + slack))) + 64
        _check(nbody_reserve(self.handle, mc, mg, _stream()), "nbody_reserve")
        return mc, mg

    def autotune(self):
        """Pick the walk tile sizes (sinks per group, direct-sum threshold) by
        timing (nbody_autotune); the tree's parameters and tree are updated.
        Returns the timings and the choice."""
        t = Tune()
        _check(nbody_autotune(self.handle, t, _stream()), "nbody_autotune")
        d = t.asdict()
        self.params.n_group = d["n_group"]
        self.params.n_direct = d["n_direct"]
        return d

    def check(self):
        """Status of the calls made since the last read (nbody_check)."""
        _check(nbody_check(self.handle, _stream()), "nbody_check")

    def timing(self, reset=True):
        t = Timing()
        _check(nbody_timing_read(self.handle, t, 1 if reset else 0), "nbody_timing_read")
        return t.asdict()

    def export(self, what: str):
        import torch
        code = EXPORT[what]
        cnt = nbody_tree_count(self.handle, code)
        if cnt < 0:
            _check(int(cnt), "nbody_tree_count")
        if what in ("sorted_keys", "cell_keys"):
            t = torch.empty(cnt, dtype=torch.int64, device=self.pos.device)
        elif what == "perm":
            t = torch.empty(cnt, dtype=torch.int32, device=self.pos.device)
        elif what in ("cell_range", "groups"):
            t = torch.empty((cnt, 2), dtype=torch.int32, device=self.pos.device)
        elif what == "cell_level":
            t = torch.empty(cnt, dtype=torch.int32, device=self.pos.device)
        elif what == "image_table":
            t = torch.empty(cnt, dtype=torch.float64, device=self.pos.device)
        else:
            o = self.params.order
            t = torch.empty((cnt, (o + 1) * (o + 2) * (o + 3) // 6), dtype=torch.float64, device=self.pos.device)
        _check(nbody_tree_export(self.handle, code, t.data_ptr(), _stream()), "nbody_tree_export")
        return t

    def lookup(self, keys):
        import torch
        out = torch.empty(keys.shape[0], dtype=torch.int32, device=keys.device)
        _check(nbody_tree_lookup(self.handle, keys.data_ptr(), keys.shape[0], out.data_ptr(), _stream()),
               "nbody_tree_lookup")
        return out

    def close(self):
        if self.handle:
            nbody_tree_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def nbody_zeldovich_state(n: int, q_dev: int, psi_dev: int, a: float, pos_dev: int, mom_dev: int,
                          stream: int | None = None) -> int:
    return lib().nbody_zeldovich_state(n, q_dev, psi_dev, a, pos_dev, mom_dev, stream)


def nbody_zeldovich_vjp(n: int, a: float, lam_pos_dev: int, lam_mom_dev: int, dpsi_dev: int,
                        stream: int | None = None) -> int:
    return lib().nbody_zeldovich_vjp(n, a, lam_pos_dev, lam_mom_dev, dpsi_dev, stream)


def zeldovich_state(q, psi, a):
    """(x, p) = (q + a psi wrapped, H0 a^(3/2) psi) from (3, n) FP64 CUDA tensors."""
    import torch
    q, psi = q.contiguous(), psi.contiguous()
    x = torch.empty_like(q)
    p = torch.empty(q.shape, dtype=torch.float32, device=q.device)
    _check(nbody_zeldovich_state(q.shape[1], q.data_ptr(), psi.data_ptr(), a, x.data_ptr(), p.data_ptr(),
                                 _stream()), "nbody_zeldovich_state")
    return x, p


def zeldovich_vjp(a, lam_x, lam_p):
    """a lam_x + H0 a^(3/2) lam_p as a (3, n) FP64 CUDA tensor."""
    import torch
    lx, lp = lam_x.contiguous(), lam_p.contiguous().float()
    out = torch.empty(lx.shape, dtype=torch.float64, device=lx.device)
    _check(nbody_zeldovich_vjp(lx.shape[1], a, lx.data_ptr(), lp.data_ptr(), out.data_ptr(), _stream()),
           "nbody_zeldovich_vjp")
    return out


def cic_loss(pos, ng, mass=None, grad=True):
    """CIC delta^2 loss of positions pos ((3, n) float64 CUDA tensor); returns
    (loss tensor of shape (), dL/dpos or None)."""
    import torch
    n = pos.shape[1]
    grid = torch.empty(ng ** 3, dtype=torch.float64, device=pos.device)
    loss = torch.empty((), dtype=torch.float64, device=pos.device)
    g = torch.empty((3, n), dtype=torch.float64, device=pos.device) if grad else None
    m = None if mass is None else mass.contiguous().float()
    x = pos.contiguous()
    _check(nbody_cic_loss(x.data_ptr(), None if m is None else m.data_ptr(), n, ng, grid.data_ptr(),
                          loss.data_ptr(), None if g is None else g.data_ptr(), _stream()), "nbody_cic_loss")
    return loss, g
