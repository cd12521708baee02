"""Plain FP64 CPU oracle for the periodic treecode force path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import this package.  It
shares no code with the CUDA library in ``paper_1407_2600_gb300``; the only
module both sides use is the seeded input generator
``paper_1407_2600_gb300.ics``, which holds none of the method's arithmetic.

Contents (each function cites the passage it follows):

* ``direct_forces``  O1, FP64 direct sum with Ewald images (Plummer or
  Dehnen K1 softening, ``soft_factor``).
* ``tree_forces``    O2, FP64 CPU treecode with the same method definition as
  the GPU path (Sec. 2.1: keys, key-implied tree, multipoles, MAC, groups).
* ``kick_factor`` / ``drift_factor`` / ``kdk_step``  O3, comoving leapfrog in an
  Einstein-de Sitter background (Sec. 2.1 cites a symplectic integrator);
  ``assign_rungs`` / ``kdk_multistep``  its block-step (hierarchical) form.
* ``cic_loss``       CIC density contrast and sum of squares, with gradient.
* ``direct_vjp`` / ``adjoint_kdk``  O4, exact reverse mode of O1 + O3.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None
_LOCK = threading.Lock()
_SOURCES = ["ewald.c", "direct.c", "tree.c"]


def lib_path() -> str:
    return os.path.join(_HERE, "liboracle.so")


def build(force: bool = False) -> str:
    """Compile the oracle's C sources with gcc (OpenMP, -O2, no -march)."""
    out = lib_path()
    srcs = [os.path.join(_HERE, s) for s in _SOURCES] + [os.path.join(_HERE, "oracle.h")]
    if not force and os.path.exists(out):
        mt = os.path.getmtime(out)
        if all(os.path.getmtime(s) <= mt for s in srcs):
            return out
    tmp = out + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=gnu11", "-o", tmp] + [
        os.path.join(_HERE, s) for s in _SOURCES] + ["-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, out)
    return out


class TreeParams(C.Structure):
    _fields_ = [("eps", C.c_double), ("theta", C.c_double), ("order", C.c_int),
                ("n_leaf", C.c_int), ("n_group", C.c_int), ("n_direct", C.c_int),
                ("lmax", C.c_int), ("ewald", C.c_int), ("ew_level", C.c_int),
                ("ew_grid", C.c_int), ("mac", C.c_int), ("bg", C.c_int), ("kernel", C.c_int),
                ("dual", C.c_int), ("replicas", C.c_int)]


class EwaldCfg(C.Structure):
    _fields_ = [("alpha", C.c_double), ("rcut", C.c_double), ("h2max", C.c_int)]


_dp = C.POINTER(C.c_double)
_i64p = C.POINTER(C.c_int64)


def _lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            L = C.CDLL(build())
            L.or_ewald_acc.argtypes = [_dp, C.POINTER(EwaldCfg), _dp]
            L.or_ewald_pot.argtypes = [_dp, C.POINTER(EwaldCfg)]
            L.or_ewald_pot.restype = C.c_double
            L.or_phitilde.argtypes = [_dp, C.POINTER(EwaldCfg), _dp]
            L.or_phitilde_mi.argtypes = [_dp, C.POINTER(EwaldCfg), C.c_int, _dp]
            L.or_phitilde_lattice.argtypes = [C.c_int, C.c_int, _dp]
            L.or_phitilde_lattice_get.argtypes = [_dp, C.c_int, C.c_int, _i64p, _dp]
            L.or_ctilde_table_build.argtypes = [C.c_int, _dp]
            L.or_ctilde_table_eval.argtypes = [_dp, C.c_int, _dp, _dp]
            L.or_ctilde_grad_table_build.argtypes = [C.c_int, _dp]
            L.or_ctilde_grad_table_eval.argtypes = [_dp, C.c_int, _dp, _dp]
            L.or_direct_forces.argtypes = [C.c_int64, _dp, _dp, C.c_double, C.c_int64, _i64p,
                                           _dp, C.c_int, _dp]
            L.or_direct_forces_k.argtypes = [C.c_int64, _dp, _dp, C.c_double, C.c_int, C.c_int64, _i64p,
                                             _dp, C.c_int, _dp]
            L.or_soft_factor.argtypes = [C.c_double, C.c_double, C.c_int]
            L.or_soft_pot.argtypes = [C.c_double, C.c_double, C.c_int]
            L.or_soft_pot.restype = C.c_double
            L.or_direct_pot.argtypes = [C.c_int64, _dp, _dp, C.c_double, C.c_int, C.c_int64, _i64p,
                                        _dp, C.c_int, _dp]
            L.or_phitilde_table_build.argtypes = [C.c_int, _dp]
            L.or_phitilde_table_eval.argtypes = [_dp, C.c_int, _dp, _dp]
            L.or_tree_forces_pot.argtypes = [C.c_int64, _dp, _dp, C.POINTER(TreeParams), _dp,
                                             C.c_int64, _i64p, _dp, _dp, _dp]
            L.or_soft_factor.restype = C.c_double
            L.or_direct_vjp.argtypes = [C.c_int64, _dp, _dp, C.c_double, _dp, C.c_int, _dp, _dp]
            L.or_tree_forces.argtypes = [C.c_int64, _dp, _dp, C.POINTER(TreeParams), _dp,
                                         C.c_int64, _i64p, _dp, _dp]
            L.or_tree_cells.argtypes = [C.c_int64, _dp, C.c_int, C.c_int, C.c_int64,
                                        C.POINTER(C.c_uint64), C.POINTER(C.c_int32), _i64p, _i64p]
            L.or_tree_cells.restype = C.c_int64
            L.or_morton_keys.argtypes = [C.c_int64, _dp, C.POINTER(C.c_uint64)]
            L.or_sort_perm.argtypes = [C.c_int64, C.POINTER(C.c_uint64), _i64p]
            L.or_nmom.argtypes = [C.c_int]
            L.or_p2m.argtypes = [C.c_int64, _dp, _dp, _dp, C.c_int, _dp]
            L.or_m2m.argtypes = [_dp, _dp, _dp, C.c_int, _dp]
            L.or_dtensor.argtypes = [_dp, C.c_double, C.c_int, _dp]
            L.or_m2p.argtypes = [_dp, C.c_int, _dp, C.c_double, _dp]
            L.or_m2p_orders.argtypes = [_dp, C.c_int, C.c_int, _dp, C.c_double, _dp]
            L.or_m2p_pot_orders.argtypes = [_dp, C.c_int, C.c_int, _dp, C.c_double]
            L.or_m2p_pot_orders.restype = C.c_double
            L.or_cube_moments.argtypes = [C.c_double, C.c_double, C.c_int, _dp]
            L.or_m2l.argtypes = [_dp, C.c_int, _dp, C.c_double, _dp]
            L.or_lattice_tensor.argtypes = [C.c_int, C.c_int, _dp]
            L.or_l2p.argtypes = [_dp, C.c_int, _dp, _dp]
            _LIB = L
    return _LIB


def _d(a):
    return a.ctypes.data_as(_dp)


def _soa(pos):
    """(n, 3) array (one row per particle) -> contiguous FP64 SoA (3, n).
    Only the (n, 3) layout is accepted, so that n = 3 is unambiguous."""
    p = np.asarray(pos, dtype=np.float64)
    if p.ndim != 2 or p.shape[1] != 3:
        raise ValueError("positions must have shape (n, 3)")
    return np.ascontiguousarray(p.T)


def ewald_cfg(alpha=2.0, rcut=None, h2max=None) -> EwaldCfg:
    if rcut is None:
        rcut = 6.0 / alpha
    if h2max is None:
        h2max = int(math.ceil((6.0 * alpha / math.pi) ** 2))
    return EwaldCfg(alpha, rcut, h2max)


def ewald_acc(r, cfg: EwaldCfg | None = None) -> np.ndarray:
    """a_E(r): periodic acceleration from a unit source with background."""
    cfg = cfg or ewald_cfg()
    r = np.ascontiguousarray(r, dtype=np.float64)
    out = np.zeros(3)
    _lib().or_ewald_acc(_d(r), C.byref(cfg), _d(out))
    return out


def ewald_pot(r, cfg: EwaldCfg | None = None) -> float:
    cfg = cfg or ewald_cfg()
    r = np.ascontiguousarray(r, dtype=np.float64)
    return float(_lib().or_ewald_pot(_d(r), C.byref(cfg)))


def phitilde(r, cfg: EwaldCfg | None = None) -> np.ndarray:
    """phi~ and its derivatives of orders 1..3 (20 values)."""
    cfg = cfg or ewald_cfg()
    r = np.ascontiguousarray(r, dtype=np.float64)
    out = np.zeros(20)
    _lib().or_phitilde(_d(r), C.byref(cfg), _d(out))
    return out


_TABLE_CACHE: dict = {}


def phitilde_mi(r, P, cfg: EwaldCfg | None = None) -> np.ndarray:
    """All derivatives d^m phi~ with |m| <= P in multi-index order."""
    cfg = cfg or ewald_cfg()
    r = np.ascontiguousarray(r, dtype=np.float64)
    out = np.zeros(nmom(P))
    _lib().or_phitilde_mi(_d(r), C.byref(cfg), P, _d(out))
    return out


def phitilde_lattice(lg: int, P: int) -> np.ndarray:
    """Exact phi~ derivatives (|m| <= P) on the lattice 2^-lg over [0, 1/2 + h]^3 (cached)."""
    key = ("lat", lg, P)
    if key not in _TABLE_CACHE:
        m = (1 << (lg - 1)) + 2
        tab = np.zeros(m ** 3 * nmom(P))
        _lib().or_phitilde_lattice(lg, P, _d(tab))
        _TABLE_CACHE[key] = tab
    return _TABLE_CACHE[key]


def phitilde_lattice_get(tab, lg, P, ir) -> np.ndarray:
    ir = np.ascontiguousarray(ir, dtype=np.int64)
    out = np.zeros(nmom(P))
    _lib().or_phitilde_lattice_get(_d(tab), lg, P, ir.ctypes.data_as(_i64p), _d(out))
    return out


def ctilde_table(n1: int = 128) -> np.ndarray:
    """Tricubic table of C~ (3 per node), nodes -h..1/2+2h (cached)."""
    key = ("c3", n1)
    if key not in _TABLE_CACHE:
        tab = np.zeros((n1 + 4) ** 3 * 3)
        _lib().or_ctilde_table_build(n1, _d(tab))
        _TABLE_CACHE[key] = tab
    return _TABLE_CACHE[key]


def ctilde_table_eval(tab, n1, r) -> np.ndarray:
    r = np.ascontiguousarray(r, dtype=np.float64)
    out = np.zeros(3)
    _lib().or_ctilde_table_eval(_d(tab), n1, _d(r), _d(out))
    return out


def ctilde_grad_table(n1: int = 64) -> np.ndarray:
    key = ("g6", n1)
    if key not in _TABLE_CACHE:
        tab = np.zeros((n1 + 4) ** 3 * 6)
        _lib().or_ctilde_grad_table_build(n1, _d(tab))
        _TABLE_CACHE[key] = tab
    return _TABLE_CACHE[key]


def soft_factor(r2, eps, kernel=0) -> float:
    """f(r) of the pair acceleration m (x_j - x_i) f: kernel 0 Plummer, 1 Dehnen K1."""
    return float(_lib().or_soft_factor(float(r2), float(eps), int(kernel)))


def direct_forces(pos, mass=None, eps=0.0, targets=None, table_n1: int | None = 128, kernel: int = 0):
    """O1: a_i = sum_j m_j [a_E(r_ij) - a_N(r*_ij) + a_S(r*_ij)] (FP64), a_S the
    softened pair force of ``kernel`` (0 Plummer, 1 Dehnen K1).

    ``table_n1=None`` evaluates the exact Ewald sum for every pair (slow);
    otherwise C~ comes from the tricubic table with ``table_n1`` intervals.
    Returns (ntarget, 3)."""
    P = _soa(pos)
    n = P.shape[1]
    m = None if mass is None else np.ascontiguousarray(mass, dtype=np.float64)
    tg = None if targets is None else np.ascontiguousarray(targets, dtype=np.int64)
    nt = n if tg is None else len(tg)
    acc = np.zeros(3 * nt)
    tab = None if table_n1 is None else ctilde_table(table_n1)
    rc = _lib().or_direct_forces_k(n, _d(P), None if m is None else _d(m), eps, kernel, nt,
                                   None if tg is None else tg.ctypes.data_as(_i64p),
                                   None if tab is None else _d(tab), table_n1 or 0, _d(acc))
    if rc != 0:
        raise ValueError("or_direct_forces_k rejected its parameters (%d)" % rc)
    return acc.reshape(3, nt).T.copy()


def soft_pot(r2, eps, kernel=0) -> float:
    """Softened pair potential of unit masses (Plummer or K1)."""
    return _lib().or_soft_pot(float(r2), float(eps), int(kernel))


def phitilde_table(n1: int = 128) -> np.ndarray:
    """Tricubic table of phi~ itself (one value per node)."""
    tab = np.zeros((n1 + 4) ** 3)
    rc = _lib().or_phitilde_table_build(n1, _d(tab))
    if rc != 0:
        raise ValueError("or_phitilde_table_build failed (%d)" % rc)
    return tab


def direct_pot(pos, mass=None, eps=0.0, targets=None, table_n1: int | None = 128, kernel: int = 0):
    """O1's potential: the zero-mean Ewald potential of every other particle
    (nearest image softened) plus each particle's own images and the
    background; ``table_n1=None`` evaluates phi~ by the exact Ewald sum."""
    P = _soa(pos)
    n = P.shape[1]
    m = None if mass is None else np.ascontiguousarray(mass, dtype=np.float64)
    tg = None if targets is None else np.ascontiguousarray(targets, dtype=np.int64)
    nt = n if tg is None else len(tg)
    out = np.zeros(nt)
    tab = None if table_n1 is None else phitilde_table(table_n1)
    rc = _lib().or_direct_pot(n, _d(P), None if m is None else _d(m), eps, kernel, nt,
                              None if tg is None else tg.ctypes.data_as(_i64p),
                              None if tab is None else _d(tab), table_n1 or 0, _d(out))
    if rc != 0:
        raise ValueError("or_direct_pot rejected its parameters (%d)" % rc)
    return out


def direct_vjp(pos, lam, mass=None, eps=0.0, n1: int | None = 64):
    """(d a / d x)^T lam for O1 (all particles); lam and result are (n,3).
    ``n1=None`` takes grad C~ from the exact Ewald sum for every pair (slow);
    otherwise from the tricubic table with ``n1`` intervals."""
    P = _soa(pos)
    n = P.shape[1]
    m = None if mass is None else np.ascontiguousarray(mass, dtype=np.float64)
    L = _soa(lam)
    out = np.zeros(3 * n)
    tab = None if n1 is None else ctilde_grad_table(n1)
    _lib().or_direct_vjp(n, _d(P), None if m is None else _d(m), eps, None if tab is None else _d(tab),
                         n1 or 0, _d(L), _d(out))
    return out.reshape(3, n).T.copy()


def tree_params(eps, theta, order, n_leaf=16, n_group=32, n_direct=None, lmax=21, ewald=4,
                ew_level=3, ew_grid=6, mac=0, bg=0, kernel=0, dual=0, replicas=0) -> TreeParams:
    """mac 0: the opening test measures d from the cell centre to the group
    box; mac 1: from the cell's faces (box to box).  bg = q > order adds the
    orders order+1..q of each expanded cell's uniform background share.
    kernel 0: Plummer softening; 1: Dehnen K1 for direct pairs, Newtonian
    cell expansions.  dual 1: well-separated cell-group pairs through a local
    expansion of the group (or_m2l / or_l2p).  replicas W = 1 or 2 (with
    ewald 0): periodic images by the (2W+1)^3 near replicas walked
    explicitly and an order-8 far-lattice expansion about the box centre."""
    if n_direct is None:
        n_direct = 2 if order <= 2 else 4
    return TreeParams(eps, theta, order, n_leaf, n_group, n_direct, lmax, ewald, ew_level,
                      ew_grid, mac, bg, kernel, dual, replicas)


def tree_forces(pos, mass=None, params: TreeParams | None = None, targets=None,
                return_stats=False, return_pot=False):
    """O2: FP64 CPU treecode; returns (ntarget, 3) accelerations, then (with
    return_pot) the (ntarget,) potential, then (with return_stats) the
    interaction counts."""
    P = _soa(pos)
    n = P.shape[1]
    m = None if mass is None else np.ascontiguousarray(mass, dtype=np.float64)
    tg = None if targets is None else np.ascontiguousarray(targets, dtype=np.int64)
    nt = n if tg is None else len(tg)
    acc = np.zeros(3 * nt)
    pot = np.zeros(nt) if return_pot else None
    st = np.zeros(7)
    tab = phitilde_lattice(params.ew_grid, params.ewald + 1) if params.ewald > 0 else None
    rc = _lib().or_tree_forces_pot(n, _d(P), None if m is None else _d(m), C.byref(params),
                                   None if tab is None else _d(tab), nt,
                                   None if tg is None else tg.ctypes.data_as(_i64p), _d(acc),
                                   None if pot is None else _d(pot), _d(st))
    if rc != 0:
        raise ValueError("or_tree_forces rejected its parameters (%d)" % rc)
    out = [acc.reshape(3, nt).T.copy()]
    if return_pot:
        out.append(pot)
    if return_stats:
        out.append({"p2p": st[0], "m2p": st[1], "ewald": st[2], "cells": st[3], "groups": st[4],
                    "sinks": st[5], "m2l": st[6]})
    return out[0] if len(out) == 1 else tuple(out)


def tree_cells(pos, n_leaf=16, lmax=21):
    """Oracle tree topology: (keys, level, start, count) in (level, key) order."""
    P = _soa(pos)
    n = P.shape[1]
    cap = max(1024, 4 * n)
    while True:
        key = np.zeros(cap, np.uint64)
        lev = np.zeros(cap, np.int32)
        st = np.zeros(cap, np.int64)
        ct = np.zeros(cap, np.int64)
        nc = _lib().or_tree_cells(n, _d(P), n_leaf, lmax, cap,
                                  key.ctypes.data_as(C.POINTER(C.c_uint64)),
                                  lev.ctypes.data_as(C.POINTER(C.c_int32)),
                                  st.ctypes.data_as(_i64p), ct.ctypes.data_as(_i64p))
        if nc >= 0:
            return key[:nc], lev[:nc], st[:nc], ct[:nc]
        cap = -nc


def morton_keys(pos) -> np.ndarray:
    P = _soa(pos)
    n = P.shape[1]
    k = np.zeros(n, np.uint64)
    _lib().or_morton_keys(n, _d(P), k.ctypes.data_as(C.POINTER(C.c_uint64)))
    return k


def sort_perm(keys) -> np.ndarray:
    k = np.ascontiguousarray(keys, dtype=np.uint64)
    perm = np.zeros(len(k), np.int64)
    _lib().or_sort_perm(len(k), k.ctypes.data_as(C.POINTER(C.c_uint64)), perm.ctypes.data_as(_i64p))
    return perm


def nmom(p: int) -> int:
    return int(_lib().or_nmom(p))


def p2m(pos, mass, c, p):
    P = _soa(pos)
    n = P.shape[1]
    m = np.ascontiguousarray(mass, dtype=np.float64)
    c = np.ascontiguousarray(c, dtype=np.float64)
    M = np.zeros(nmom(p))
    _lib().or_p2m(n, _d(P), _d(m), _d(c), p, _d(M))
    return M


def m2m(M, c, cp, p):
    M = np.ascontiguousarray(M, dtype=np.float64)
    c = np.ascontiguousarray(c, dtype=np.float64)
    cp = np.ascontiguousarray(cp, dtype=np.float64)
    out = np.zeros(nmom(p))
    _lib().or_m2m(_d(M), _d(c), _d(cp), p, _d(out))
    return out


def dtensor(R, eps, pmax):
    R = np.ascontiguousarray(R, dtype=np.float64)
    D = np.zeros(nmom(pmax))
    _lib().or_dtensor(_d(R), eps, pmax, _d(D))
    return D


def m2p(M, p, R, eps):
    M = np.ascontiguousarray(M, dtype=np.float64)
    R = np.ascontiguousarray(R, dtype=np.float64)
    a = np.zeros(3)
    _lib().or_m2p(_d(M), p, _d(R), eps, _d(a))
    return a


def m2p_orders(M, pmin, pmax, R, eps):
    """Acceleration from the orders pmin..pmax of the moments M only."""
    M = np.ascontiguousarray(M, dtype=np.float64)
    R = np.ascontiguousarray(R, dtype=np.float64)
    a = np.zeros(3)
    _lib().or_m2p_orders(_d(M), pmin, pmax, _d(R), eps, _d(a))
    return a


def lattice_tensor(P: int = 8, W: int = 2) -> np.ndarray:
    """d^m Phi_F(0), |m| <= P: the far-lattice potential (the images beyond
    |n|_inf <= W, with the uniform background)."""
    T = np.zeros(nmom(P))
    _lib().or_lattice_tensor(P, W, _d(T))
    return T


def m2p_pot(M, pmin, pmax, R, eps) -> float:
    """Psi of the orders pmin..pmax of moments M at R (a = grad Psi)."""
    Mv = np.ascontiguousarray(M, dtype=np.float64)
    Rv = np.ascontiguousarray(R, dtype=np.float64)
    return _lib().or_m2p_pot_orders(_d(Mv), pmin, pmax, _d(Rv), eps)


def m2l(M, p, R, eps):
    """Local expansion coefficients (nmom(p + 1), index 0 unused) about z of a
    cell's field, R = z - c (the dual form's cell-group interaction)."""
    M = np.ascontiguousarray(M, dtype=np.float64)
    R = np.ascontiguousarray(R, dtype=np.float64)
    L = np.zeros(nmom(p + 1))
    _lib().or_m2l(_d(M), p, _d(R), eps, _d(L))
    return L


def l2p(L, p, d):
    L = np.ascontiguousarray(L, dtype=np.float64)
    d = np.ascontiguousarray(d, dtype=np.float64)
    a = np.zeros(3)
    _lib().or_l2p(_d(L), p, _d(d), _d(a))
    return a


def cube_moments(s, rho, p):
    """Moments (|n| <= p) about its centre of a cube of side s, density rho."""
    C_ = np.zeros(nmom(p))
    _lib().or_cube_moments(s, rho, p, _d(C_))
    return C_


def multi_indices(p):
    """Multi-indices |n| <= p in the oracle's storage order."""
    out = []
    for o in range(p + 1):
        for nx in range(o, -1, -1):
            for ny in range(o - nx, -1, -1):
                out.append((nx, ny, o - nx - ny))
    return out


# ---- O3: comoving KDK leapfrog, Einstein-de Sitter ---------------------------
# Canonical momentum p = a^2 dx/dt; dx/dt = p/a^2, dp/dt = g/a with g the
# comoving peculiar acceleration (G rho_bar = 1 in box units).  H(a) = H0 a^-3/2
# with H0^2 = 8 pi G rho_bar / 3.  Sec. 2.1 names a symplectic integrator
# (Quinn et al. 1997); the global-step kick-drift-kick form is the reading used.
H0 = math.sqrt(8.0 * math.pi / 3.0)


def kick_factor(a0: float, a1: float) -> float:
    """int dt / a from a0 to a1 = (2/H0)(sqrt(a1) - sqrt(a0))."""
    return 2.0 / H0 * (math.sqrt(a1) - math.sqrt(a0))


def drift_factor(a0: float, a1: float) -> float:
    """int dt / a^2 from a0 to a1 = (2/H0)(a0^-1/2 - a1^-1/2)."""
    return 2.0 / H0 * (1.0 / math.sqrt(a0) - 1.0 / math.sqrt(a1))


def kdk_step(x, p, g0, a0, a1, force):
    """One KDK step: p += K(a0,a_h) g0; x += D(a0,a1) p (wrapped); g1 = force(x);
    p += K(a_h,a1) g1 with a_h = sqrt(a0 a1).  Arrays are (n,3)."""
    ah = math.sqrt(a0 * a1)
    p = p + kick_factor(a0, ah) * g0
    x = np.mod(x + drift_factor(a0, a1) * p, 1.0)
    g1 = force(x)
    p = p + kick_factor(ah, a1) * g1
    return x, p, g1


# Hierarchical (block) steps: Sec. 2.1 cites the adaptive symplectic
# integrator of Quinn et al. (1997), whose particles take power-of-two
# fractions of the global step.  Reading used here: a global step in ln a is
# cut into T = 2^rmax ticks; a particle on rung r takes steps of S = 2^(rmax-r)
# ticks in kick-drift-kick form: at the tick where its step starts it is
# kicked over the first half of that step, every tick all particles drift,
# and at the tick where its step ends its acceleration is recomputed at the
# new positions and it is kicked over the second half.  Rungs are fixed for
# the global step.  With rmax = 0 this is kdk_step.
def assign_rungs(g32, eps, eta, dlna, rmax):
    """Rung of each particle: the smallest r in [0, rmax] with
    (dlna / 2^r)^2 <= eta^2 H0^2 eps / |g|, i.e. 4^r >= q with
    q = |g| dlna^2 / (eta^2 H0^2 eps) (rmax if none): the step in ln a at
    which a particle moves about eta^2 eps under its acceleration.  g32 (n,3)
    are the accelerations as float32 values; |g| and q are formed in FP64 in
    the order written.  eps may be per particle."""
    g = np.asarray(g32, dtype=np.float32).astype(np.float64)
    s = np.sqrt((g[:, 0] * g[:, 0] + g[:, 1] * g[:, 1]) + g[:, 2] * g[:, 2])
    eps = np.broadcast_to(np.asarray(eps, dtype=np.float64), s.shape)
    c = (dlna * dlna) / ((eta * eta) * (H0 * H0) * eps)
    q = s * c
    r = np.zeros(len(s), dtype=np.int64)
    f = np.ones(len(s))
    for _ in range(rmax):
        up = f < q
        r[up] += 1
        f = np.where(up, f * 4.0, f)
    return r


def tick_a(a0, a1, rmax, j2):
    """Expansion factor at half-tick j2 (tick j2/2) of the step a0 -> a1."""
    T = 1 << rmax
    L = math.log(a1 / a0)
    return a0 * math.exp(L * j2 / (2 * T))


def kdk_multistep(x, p, g, rung, a0, a1, rmax, force):
    """One global step a0 -> a1 with block steps (see above).  x, p, g (n,3);
    rung (n,) in [0, rmax]; force(x) -> (n,3).  Returns x, p, g with g the
    accelerations at each particle's last force evaluation."""
    T = 1 << rmax
    rung = np.asarray(rung, dtype=np.int64)
    S = np.left_shift(1, rmax - rung)
    x, p, g = x.copy(), p.copy(), g.copy()
    for k in range(T):
        start = (k % S) == 0
        for r in range(rmax + 1):
            sel = start & (rung == r)
            if sel.any():
                st = 1 << (rmax - r)
                p[sel] += kick_factor(tick_a(a0, a1, rmax, 2 * k), tick_a(a0, a1, rmax, 2 * k + st)) * g[sel]
        x = np.mod(x + drift_factor(tick_a(a0, a1, rmax, 2 * k), tick_a(a0, a1, rmax, 2 * k + 2)) * p, 1.0)
        end = ((k + 1) % S) == 0
        if end.any():
            gn = force(x)
            g[end] = gn[end]
            for r in range(rmax + 1):
                sel = end & (rung == r)
                if sel.any():
                    st = 1 << (rmax - r)
                    p[sel] += kick_factor(tick_a(a0, a1, rmax, 2 * (k + 1) - st),
                                          tick_a(a0, a1, rmax, 2 * (k + 1))) * g[sel]
    return x, p, g


def zeldovich_state(q, psi, a):
    """x = q + a psi (wrapped), p = H0 a^(3/2) psi (growing mode, D = a)."""
    x = np.mod(q + a * psi, 1.0)
    p = H0 * a ** 1.5 * psi
    return x, p


# ---- CIC density and loss ------------------------------------------------------
def cic_weights(x, ng):
    """Cell-centred CIC: grid cell c has centre (c + 1/2)/ng."""
    u = x * ng - 0.5
    i0 = np.floor(u).astype(np.int64)
    f = u - i0
    return i0, f


def cic_loss(x, mass, ng):
    """L = sum_c delta_c^2, delta = rho/rho_bar - 1, rho from CIC; returns (L, dL/dx)."""
    x = np.asarray(x, dtype=np.float64)
    n = x.shape[0]
    m = np.full(n, 1.0 / n) if mass is None else np.asarray(mass, dtype=np.float64)
    i0, f = cic_weights(x, ng)
    rho = np.zeros((ng, ng, ng))
    corners = [(dx, dy, dz) for dx in (0, 1) for dy in (0, 1) for dz in (0, 1)]
    w = []
    for dx, dy, dz in corners:
        wx = f[:, 0] if dx else 1.0 - f[:, 0]
        wy = f[:, 1] if dy else 1.0 - f[:, 1]
        wz = f[:, 2] if dz else 1.0 - f[:, 2]
        idx = ((i0[:, 0] + dx) % ng, (i0[:, 1] + dy) % ng, (i0[:, 2] + dz) % ng)
        w.append((idx, wx, wy, wz, dx, dy, dz))
        np.add.at(rho, idx, m * wx * wy * wz * ng ** 3)
    delta = rho - 1.0
    L = float(np.sum(delta * delta))
    grad = np.zeros((n, 3))
    for idx, wx, wy, wz, dx, dy, dz in w:
        g = 2.0 * delta[idx] * m * ng ** 3
        sx = ng if dx else -ng
        sy = ng if dy else -ng
        sz = ng if dz else -ng
        grad[:, 0] += g * sx * wy * wz
        grad[:, 1] += g * wx * sy * wz
        grad[:, 2] += g * wx * wy * sz
    return L, grad


# ---- O4: exact reverse mode of O1 dynamics ----------------------------------------
def adjoint_kdk(x_list, p_list, a_list, lam_x, lam_p, mass, eps, n1=64):
    """Reverse a KDK trajectory of O1 forces.

    ``x_list[k], p_list[k]`` are the states at ``a_list[k]`` (k = 0..S); each
    step recomputes nothing (states given).  The force at step start is a
    function of x_k, so every step contributes two force VJPs.  Returns the
    cotangents (lam_x0, lam_p0).  ``n1`` is passed to ``direct_vjp``
    (None: exact Ewald derivatives)."""
    S = len(a_list) - 1
    lx = np.array(lam_x, dtype=np.float64)
    lp = np.array(lam_p, dtype=np.float64)
    for k in range(S - 1, -1, -1):
        a0, a1 = a_list[k], a_list[k + 1]
        ah = math.sqrt(a0 * a1)
        K1, K2, D = kick_factor(a0, ah), kick_factor(ah, a1), drift_factor(a0, a1)
        # forward: ph = p0 + K1 g(x0); x1 = x0 + D ph; p1 = ph + K2 g(x1)
        lg1 = K2 * lp
        lx1 = lx + direct_vjp(x_list[k + 1], lg1, mass, eps, n1)
        lph = lp + D * lx1
        lg0 = K1 * lph
        lx = lx1 + direct_vjp(x_list[k], lg0, mass, eps, n1)
        lp = lph
    return lx, lp
