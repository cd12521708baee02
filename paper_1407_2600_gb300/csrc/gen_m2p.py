"""Generate m2p_gen.cuh: straight-line multipole-to-particle code.

The acceleration of a cell with moments M_n (about its geometric centre) at
R = x - c is the truncated expansion of Sec. 2.1's multipole method,

    a_i = sum_{|n|<=p} C_n d^{n+e_i} g(R),  C_n = (-1)^|n| M_n / n!,
    g(R) = (|R|^2 + eps^2)^(-1/2).

With s = |R|^2 + eps^2 and F_j = (-1)^j (2j-1)!! s^(-1/2-j), the Hermite form
d^n g = sum_k h(n,k) R^(n-2k) F_{|n|-|k|},
h(n,k) = prod_d n_d! / (k_d! (n_d - 2k_d)! 2^k_d), regroups the potential as

    phi(R) = sum_j F_j S_j(R),   S_j(R) = sum_a B_{j,a} R^a,
    B_{j,a} = sum_{n - 2k = a, |n| - |k| = j} C_n h(n,k),

so that, with d_i F_j = R_i F_{j+1},

    a_i = d_i phi = R_i sum_j F_{j+1} S_j + sum_j F_j d_i S_j.

The per-cell coefficients are stored as a! B_{j,a} with the divided monomials
mu_a = R^a / a!, so that d_i mu_a = mu_{a - e_i} exactly and the gradient sums
need no integer factors (every term is one fused multiply-add).  They are
formed once in the upward pass (FP64) and stored in the walk's precision;
each M2P then costs a few hundred flops.
Run ``python gen_m2p.py`` to regenerate; a CPU test checks that the committed
header equals this script's output.
"""
from __future__ import annotations

import math
import os
import re
import sys
from itertools import product


def multi(p):
    out = []
    for o in range(p + 1):
        for nx in range(o, -1, -1):
            for ny in range(o - nx, -1, -1):
                out.append((nx, ny, o - nx - ny))
    return out


def hcoef(n, k):
    c = 1.0
    for d in range(3):
        c *= math.factorial(n[d]) / (math.factorial(k[d]) * math.factorial(n[d] - 2 * k[d]) * 2 ** k[d])
    return c


def slots(p):
    """(j, a) pairs of the reduced expansion, in storage order."""
    out = []
    for j in range(p + 1):
        for a in multi(p):
            s = sum(a)
            if s <= j and 2 * j - s <= p:
                out.append((j, a))
    return out


def contributions(p):
    """For each slot: list of (moment index, coefficient multiplying M_n)."""
    mi = {m: i for i, m in enumerate(multi(p))}
    sl = slots(p)
    idx = {s: i for i, s in enumerate(sl)}
    contrib = [[] for _ in sl]
    for n in multi(p):
        on = sum(n)
        sign = -1.0 if on % 2 else 1.0
        nf = math.factorial(n[0]) * math.factorial(n[1]) * math.factorial(n[2])
        for k in product(*(range(n[d] // 2 + 1) for d in range(3))):
            a = tuple(n[d] - 2 * k[d] for d in range(3))
            j = on - sum(k)
            contrib[idx[(j, a)]].append((mi[n], sign / nf * hcoef(n, k)))
    return sl, contrib


def flop_count(p):
    """Flops of one M2P as the walk runs it (FMA = 2, rsqrt = 1): the scaled
    separation R = (x - c) 2^level as 3 FMA, eps^2 scaled per cell (0), and
    the generated expansion."""
    mon = multi(p)
    fl = 6            # R: 3 FMA
    fl += 6           # s = eps2 + Rx^2 + Ry^2 + Rz^2: 3 FMA
    fl += 1           # rsqrt
    fl += 1           # inv_s = F0*F0
    fl += 2 * (p + 1)  # F_j chain: c_j = k*inv_s, F_j = F_{j-1}*c_j
    fl += 3 * max(p - 1, 0)  # R_d / k for k = 2..p
    fl += len(mon) - 1  # divided monomials
    sl = slots(p)
    for (j, a) in sl:
        fl += 2  # S_j FMA
        fl += 2 * sum(1 for d in range(3) if a[d] > 0)  # G_{j,d} FMA
    fl += 1 + 2 * p  # t = sum_j F_{j+1} S_j
    fl += 3 * 2 * (p + 1)  # a_i += R_i t + sum_{j>=1} F_j G_ji
    return fl


def emit_m2p(p):
    mon = multi(p)
    mi = {m: i for i, m in enumerate(mon)}
    sl = slots(p)
    L = []
    L.append("// REF: the reciprocal square root refined (near-uniform boxes), else the")
    L.append("// hardware approximation alone")
    L.append("template <typename T, bool REF = true>")
    L.append("__device__ __forceinline__ void m2p_p%d(const T* __restrict__ B, T Rx, T Ry, T Rz, T eps2," % p)
    L.append("                                     T& ax, T& ay, T& az) {")
    L.append("  const T s = fma(Rx, Rx, fma(Ry, Ry, fma(Rz, Rz, eps2)));")
    L.append("  const T F0 = REF ? nbody_rsqrt(s) : nbody_rsqrt_pair(s);")
    L.append("  const T is = F0 * F0;")
    for j in range(1, p + 2):
        L.append("  const T F%d = F%d * (T(%d) * is);" % (j, j - 1, -(2 * j - 1)))
    for d, R in enumerate(("Rx", "Ry", "Rz")):
        for k in range(2, p + 1):
            L.append("  const T %s_%d = %s * T(%.17g);" % (R, k, R, 1.0 / k))
    L.append("  const T m0 = T(1);")
    for i, m in enumerate(mon):
        if i == 0:
            continue
        for d in range(3):
            if m[d] > 0:
                par = list(m)
                par[d] -= 1
                pi = mi[tuple(par)]
                R = ("Rx", "Ry", "Rz")[d]
                fac = R if m[d] == 1 else "%s_%d" % (R, m[d])
                L.append("  const T m%d = %s;" % (i, fac if pi == 0 else "m%d * %s" % (pi, fac)))
                break
    for j in range(p + 1):
        L.append("  T S%d = T(0), G%dx = T(0), G%dy = T(0), G%dz = T(0);" % (j, j, j, j))
    for t, (j, a) in enumerate(sl):
        ai = mi[a]
        L.append("  { const T b = B[%d];" % t)
        L.append("    S%d = fma(b, m%d, S%d);" % (j, ai, j))
        for d, ax in enumerate("xyz"):
            if a[d] > 0:
                par = list(a)
                par[d] -= 1
                L.append("    G%d%s = fma(b, m%d, G%d%s);" % (j, ax, mi[tuple(par)], j, ax))
        L.append("  }")
    # a = R sum_j F_{j+1} S_j + sum_{j>=1} F_j G_j  (G_0 = 0)
    L.append("  T t = F1 * S0;")
    for j in range(1, p + 1):
        L.append("  t = fma(F%d, S%d, t);" % (j + 1, j))
    for c in "xyz":
        e = "a%s" % c
        for j in range(p, 0, -1):
            e = "fma(F%d, G%d%s, %s)" % (j, j, c, e)
        L.append("  a%s = fma(R%s, t, %s);" % (c, c, e))
    L.append("}")
    return "\n".join(L)


def emit_m2pot(p):
    """The expansion's potential form phi(R) = sum_j F_j S_j(R) (the walk's
    potential is -phi), from the same stored coefficients as m2p_p<p>."""
    mon = multi(p)
    mi = {m: i for i, m in enumerate(mon)}
    sl = slots(p)
    L = []
    L.append("template <typename T>")
    L.append("__device__ __forceinline__ T m2pot_p%d(const T* __restrict__ B, T Rx, T Ry, T Rz, T eps2) {" % p)
    L.append("  const T s = fma(Rx, Rx, fma(Ry, Ry, fma(Rz, Rz, eps2)));")
    L.append("  const T F0 = nbody_rsqrt(s);")
    L.append("  const T is = F0 * F0;")
    for j in range(1, p + 1):
        L.append("  const T F%d = F%d * (T(%d) * is);" % (j, j - 1, -(2 * j - 1)))
    for d, R in enumerate(("Rx", "Ry", "Rz")):
        for k in range(2, p + 1):
            L.append("  const T %s_%d = %s * T(%.17g);" % (R, k, R, 1.0 / k))
    for i, m in enumerate(mon):
        if i == 0:
            continue
        for d in range(3):
            if m[d] > 0:
                par = list(m)
                par[d] -= 1
                pi = mi[tuple(par)]
                R = ("Rx", "Ry", "Rz")[d]
                fac = R if m[d] == 1 else "%s_%d" % (R, m[d])
                L.append("  const T m%d = %s;" % (i, fac if pi == 0 else "m%d * %s" % (pi, fac)))
                break
    for j in range(p + 1):
        L.append("  T S%d = T(0);" % j)
    for t, (j, a) in enumerate(sl):
        ai = mi[a]
        L.append("  S%d = %s;" % (j, "S%d + B[%d]" % (j, t) if ai == 0 else "fma(B[%d], m%d, S%d)" % (t, ai, j)))
    e = "F0 * S0"
    for j in range(1, p + 1):
        e = "fma(F%d, S%d, %s)" % (j, j, e)
    L.append("  return %s;" % e)
    L.append("}")
    return "\n".join(L)


def emit_m2p2(p):
    """The M2P of two cells at once for one sink, in packed FP32 pairs (the
    .x and .y halves are the two cells; B holds the two cells' coefficients
    interleaved).  Every half performs the operations of m2p_p<p> in the
    same order, so each cell's result equals the scalar one bit for bit."""
    mon = multi(p)
    mi = {m: i for i, m in enumerate(mon)}
    sl = slots(p)
    L = []
    L.append("template <bool REF = true>")
    L.append("__device__ __forceinline__ void m2p2_p%d(const float2* __restrict__ B, float2 Rx, float2 Ry, float2 Rz," % p)
    L.append("                                       float2 eps2, float2& ax, float2& ay, float2& az) {")
    L.append("  const float2 s = __ffma2_rn(Rx, Rx, __ffma2_rn(Ry, Ry, __ffma2_rn(Rz, Rz, eps2)));")
    L.append("  const float2 F0 = REF ? make_float2(nbody_rsqrt(s.x), nbody_rsqrt(s.y))")
    L.append("                        : make_float2(nbody_rsqrt_pair(s.x), nbody_rsqrt_pair(s.y));")
    L.append("  const float2 is = __fmul2_rn(F0, F0);")
    for j in range(1, p + 2):
        c = -(2 * j - 1)
        L.append("  const float2 F%d = __fmul2_rn(F%d, __fmul2_rn(make_float2(%d.0f, %d.0f), is));" % (j, j - 1, c, c))
    for d, R in enumerate(("Rx", "Ry", "Rz")):
        for k in range(2, p + 1):
            c = "%.9gf" % (1.0 / k)
            L.append("  const float2 %s_%d = __fmul2_rn(%s, make_float2(%s, %s));" % (R, k, R, c, c))
    for i, m in enumerate(mon):
        if i == 0:
            continue
        for d in range(3):
            if m[d] > 0:
                par = list(m)
                par[d] -= 1
                pi = mi[tuple(par)]
                R = ("Rx", "Ry", "Rz")[d]
                fac = R if m[d] == 1 else "%s_%d" % (R, m[d])
                L.append("  const float2 m%d = %s;" % (i, fac if pi == 0 else "__fmul2_rn(m%d, %s)" % (pi, fac)))
                break
    started = set()

    def acc(name, b, mono):
        if name not in started:  # first term: the accumulator starts from zero
            started.add(name)
            return "    %s = %s;" % (name, b if mono == 0 else "__fmul2_rn(%s, m%d)" % (b, mono))
        if mono == 0:
            return "    %s = __fadd2_rn(%s, %s);" % (name, b, name)
        return "    %s = __ffma2_rn(%s, m%d, %s);" % (name, b, mono, name)

    names = []
    for j in range(p + 1):
        names += ["S%d" % j] + ["G%d%s" % (j, c) for c in "xyz"]
    used = set()
    for (j, a) in sl:
        used.add("S%d" % j)
        for d, c in enumerate("xyz"):
            if a[d] > 0:
                used.add("G%d%s" % (j, c))
    L.append("  float2 %s;" % ", ".join(n for n in names if n in used))
    for t, (j, a) in enumerate(sl):
        ai = mi[a]
        L.append("  { const float2 b = B[%d];" % t)
        L.append(acc("S%d" % j, "b", ai))
        for d, c in enumerate("xyz"):
            if a[d] > 0:
                par = list(a)
                par[d] -= 1
                L.append(acc("G%d%s" % (j, c), "b", mi[tuple(par)]))
        L.append("  }")
    L.append("  float2 t = __fmul2_rn(F1, S0);")
    for j in range(1, p + 1):
        L.append("  t = __ffma2_rn(F%d, S%d, t);" % (j + 1, j))
    for c in "xyz":
        e = "a%s" % c
        for j in range(p, 0, -1):
            e = "__ffma2_rn(F%d, G%d%s, %s)" % (j, j, c, e)
        L.append("  a%s = __ffma2_rn(R%s, t, %s);" % (c, c, e))
    L.append("}")
    return "\n".join(L)


def emit_reduce(p):
    """FP64 moments (multi-index order) -> stored coefficients a! B_{j,a}."""
    sl, contrib = contributions(p)
    L = []
    L.append("__device__ __forceinline__ void reduce_moments_p%d(const double* __restrict__ M, double* __restrict__ B) {" % p)
    for t, cs in enumerate(contrib):
        a = sl[t][1]
        af = math.factorial(a[0]) * math.factorial(a[1]) * math.factorial(a[2])
        terms = " + ".join("%.17g * M[%d]" % (c * af, i) for i, c in cs)
        L.append("  B[%d] = %s;" % (t, terms))
    L.append("}")
    return "\n".join(L)


def emit_m2l(pe, with_m2l=True):
    """Image-field local expansion about the expansion point e:
    L_m += sum_n (-1)^|n|/n! M_n d^{m+n} phi~(R0), 1 <= |m| <= pe+1, |m|+|n| <= pe+1
    (m2l_pe), and its evaluation (l2p_pe); with_m2l False emits the latter only."""
    P = pe + 1
    mP = multi(P)
    mi = {m: i for i, m in enumerate(mP)}
    me = multi(pe)
    L = []
    L.append("template <typename T>")
    L.append("__device__ __forceinline__ void m2l_pe%d(const T* __restrict__ M, const T* __restrict__ D, T* __restrict__ Lc) {" % pe)
    L.append("  // Lc[t-1] accumulates L_m for multi-index t >= 1 (orders 1..%d)" % P)
    for t, m in enumerate(mP):
        if t == 0:
            continue
        terms = []
        for u, n in enumerate(me):
            if sum(m) + sum(n) > P:
                continue
            c = (-1.0 if sum(n) % 2 else 1.0) / (math.factorial(n[0]) * math.factorial(n[1]) * math.factorial(n[2]))
            k = mi[(m[0] + n[0], m[1] + n[1], m[2] + n[2])]
            terms.append((u, c, k))
        expr = "Lc[%d]" % (t - 1)
        for u, c, k in terms:
            if c == 1.0:
                expr = "fma(M[%d], D[%d], %s)" % (u, k, expr)
            elif c == -1.0:
                expr = "fma(-M[%d], D[%d], %s)" % (u, k, expr)
            else:
                expr = "fma(M[%d] * T(%.17g), D[%d], %s)" % (u, c, k, expr)
        L.append("  Lc[%d] = %s;" % (t - 1, expr))
    L.append("}")
    if not with_m2l:
        L = []
    # L2P
    L.append("template <typename T>")
    L.append("__device__ __forceinline__ void l2p_pe%d(const T* __restrict__ Lc, T dx, T dy, T dz, T& ax, T& ay, T& az) {" % pe)
    L.append("  // a_k -= sum_{|n|<=%d} d^n/n! L_{n+e_k}" % pe)
    mon = me
    mmi = {m: i for i, m in enumerate(mon)}
    L.append("  const T q0 = T(1);")
    for i, m in enumerate(mon):
        if i == 0:
            continue
        for d in range(3):
            if m[d] > 0:
                par = list(m)
                par[d] -= 1
                pi = mmi[tuple(par)]
                L.append("  const T q%d = q%d * (%s * T(%.17g));" % (i, pi, "dxdydz"[2 * d:2 * d + 2], 1.0 / m[d]))
                break
    for k, ax in enumerate("xyz"):
        terms = []
        for i, n in enumerate(mon):
            nn = list(n)
            nn[k] += 1
            terms.append((i, mi[tuple(nn)] - 1))
        expr = "a%s" % ax
        for i, li in terms:
            expr = "fma(-q%d, Lc[%d], %s)" % (i, li, expr)
        L.append("  a%s = %s;" % (ax, expr))
    L.append("}")
    return "\n".join(L)


def emit_dtensor(P):
    """D[t] = d^t g(R) for |t| <= P, g = (|R|^2 + eps^2)^-1/2, by the
    Cartesian recurrence on the radial ladder g_j = ((1/r) d/dr)^j g:
    T^(j)_(n + e_a) = R_a T^(j+1)_n + n_a T^(j+1)_(n - e_a), T^(j)_0 = g_j."""
    mP = multi(P)
    mi = {m: i for i, m in enumerate(mP)}
    L = []
    L.append("template <typename T>")
    L.append("__device__ __forceinline__ void dtensor_p%d(T Rx, T Ry, T Rz, T eps2, T* __restrict__ D) {" % P)
    L.append("  const T s = fma(Rx, Rx, fma(Ry, Ry, fma(Rz, Rz, eps2)));")
    L.append("  const T g0_0 = nbody_rsqrt(s);")
    L.append("  const T is = g0_0 * g0_0;")
    for j in range(1, P + 1):
        L.append("  const T g%d_0 = g%d_0 * (T(%d) * is);" % (j, j - 1, -(2 * j - 1)))
    R = "RxRyRz"
    for t, n in enumerate(mP):
        if t == 0:
            continue
        o = sum(n)
        a = next(d for d in range(3) if n[d] > 0)
        m1 = list(n)
        m1[a] -= 1
        d1 = mi[tuple(m1)]
        d2 = None
        if n[a] >= 2:
            m2 = list(m1)
            m2[a] -= 1
            d2 = mi[tuple(m2)]
        for j in range(P - o + 1):
            e = "%s * g%d_%d" % (R[2 * a:2 * a + 2], j + 1, d1)
            if d2 is not None:
                e = "fma(T(%d), g%d_%d, %s)" % (n[a] - 1, j + 1, d2, e)
            L.append("  const T g%d_%d = %s;" % (j, t, e))
    for t in range(len(mP)):
        L.append("  D[%d] = g0_%d;" % (t, t))
    L.append("}")
    return "\n".join(L)


def emit_m2l_red(p):
    """The dual form's cell-group M2L, one local coefficient at a time:
    v_t = sum_n (-1)^|n|/n! M_n D_(t+n), 1 <= |t|, |t| + |n| <= p + 1, each
    handed to red(t - 1, |t|, v_t) as soon as it is formed (so that only
    the moments, the derivatives and one coefficient are live).  M is read
    through M[u] (an accessor)."""
    P = p + 1
    mP = multi(P)
    mi = {m: i for i, m in enumerate(mP)}
    me = multi(p)
    L = []
    L.append("template <typename T, typename MA, typename Red>")
    L.append("__device__ __forceinline__ void m2l_red_p%d(const MA& M, const T* __restrict__ D, Red&& red) {" % p)
    for t, m in enumerate(mP):
        if t == 0:
            continue
        expr = None
        for u, n in enumerate(me):
            if sum(m) + sum(n) > P:
                continue
            c = (-1.0 if sum(n) % 2 else 1.0) / (math.factorial(n[0]) * math.factorial(n[1]) * math.factorial(n[2]))
            k = mi[(m[0] + n[0], m[1] + n[1], m[2] + n[2])]
            mm = "M[%d]" % u if c == 1.0 else ("(-M[%d])" % u if c == -1.0 else "(M[%d] * T(%.17g))" % (u, c))
            expr = "%s * D[%d]" % (mm, k) if expr is None else "fma(%s, D[%d], %s)" % (mm, k, expr)
        L.append("  red(%d, %d, %s);" % (t - 1, sum(m), expr))
    L.append("}")
    return "\n".join(L)


def _code_flops(code):
    """Flops of generated straight-line code: FMA = 2, a product = 1, rsqrt = 1."""
    return 2 * code.count("fma(") + len(re.findall(r" \* ", code)) + code.count("nbody_rsqrt(")


def upward_flop_counts(p):
    """FP64 flops of the upward pass as generated (FMA = 2, product = 1,
    addition = 1): per particle (P2M, plus the three coordinate differences
    from the leaf centre), per daughter (its M2M shift into the parent, the
    three centre differences being exact integer conversions), and per cell
    (the power-of-two scalings of its moments and coefficients and the
    reduction to the walk's coefficients)."""
    def count(code):
        return (2 * code.count("fma(") + len(re.findall(r" \* ", code)) + code.count("+=") +
                len(re.findall(r" \+ ", code)))
    nm, nb = len(multi(p)), len(slots(p))
    return {"p2m_per_particle": count(emit_p2m(p)) + 3, "m2m_per_daughter": count(emit_m2m(p)),
            "per_cell": count(emit_reduce(p)) + nm + nb}


def m2l_dual_flop_count(p):
    """Flops of one cell-group expansion of the dual form at order p: the
    softened derivative tensor to order p + 1 (with its negation), the
    generated contraction, and per local coefficient one product taking it to
    the group's unit and one addition joining it to the group's sum."""
    nl = len(multi(p + 1)) - 1
    return _code_flops(emit_dtensor(p + 1)) + len(multi(p + 1)) + _code_flops(emit_m2l_red(p)) + 2 * nl


def l2p_flop_count(p):
    """Flops of the group's local expansion evaluated at one sink (the
    image-field L2P of order p, the offset to the group's unit, the unit
    factor and the sum into the acceleration)."""
    code = emit_m2l(p)
    code = code[code.index("l2p_pe"):]
    return _code_flops(code) + 3 * 2 + 3 + 3 * 4


def emit_p2m(p):
    """M_n += m (x - c)^n for |n| <= p (FP64)."""
    mon = multi(p)
    mi = {m: i for i, m in enumerate(mon)}
    L = ["__device__ __forceinline__ void p2m_acc_p%d(double m, double dx, double dy, double dz, double* __restrict__ M) {" % p]
    L.append("  const double q0 = m;")
    L.append("  M[0] += q0;")
    for i, mm in enumerate(mon):
        if i == 0:
            continue
        for d in range(3):
            if mm[d] > 0:
                par = list(mm)
                par[d] -= 1
                L.append("  const double q%d = q%d * %s;" % (i, mi[tuple(par)], "dxdydz"[2 * d:2 * d + 2]))
                break
        L.append("  M[%d] += q%d;" % (i, i))
    L.append("}")
    return "\n".join(L)


def emit_m2m(p):
    """Mp_n += sum_{k <= n} C(n,k) s^(n-k) Mc_k, s = c_child - c_parent (FP64)."""
    mon = multi(p)
    mi = {m: i for i, m in enumerate(mon)}
    L = ["__device__ __forceinline__ void m2m_acc_p%d(const double* __restrict__ Mc, double sx, double sy, double sz, double* __restrict__ Mp) {" % p]
    L.append("  const double w0 = 1.0;")
    for i, mm in enumerate(mon):
        if i == 0:
            continue
        for d in range(3):
            if mm[d] > 0:
                par = list(mm)
                par[d] -= 1
                L.append("  const double w%d = w%d * %s;" % (i, mi[tuple(par)], "sxsysz"[2 * d:2 * d + 2]))
                break
    for t, n in enumerate(mon):
        expr = "Mp[%d]" % t
        for k in product(*(range(n[d] + 1) for d in range(3))):
            b = math.comb(n[0], k[0]) * math.comb(n[1], k[1]) * math.comb(n[2], k[2])
            w = mi[(n[0] - k[0], n[1] - k[1], n[2] - k[2])]
            if b == 1:
                expr = "fma(w%d, Mc[%d], %s)" % (w, mi[k], expr)
            else:
                expr = "fma(w%d * %d.0, Mc[%d], %s)" % (w, b, mi[k], expr)
        L.append("  Mp[%d] = %s;" % (t, expr))
    L.append("}")
    return "\n".join(L)


# ---- uniform-background terms of an expanded cell ------------------------------------
# A cell used through its expansion also gets the orders p < l <= l_bg of the
# field of a cube of the mean density filling it (Newtonian kernel): the higher
# moments of its uniform share, whose truncation dominates the expansion error
# of near-uniform states.  In the cell's length unit (side 1) and for unit
# density, the order-l potential term of the expansion is
#     psi_l(R) = sum_{|n|=l} (c_n / n!) d^n (1/r),  c_n = prod_d m(n_d),
#     m(k) = 1 / ((k+1) 2^k) for even k, 0 for odd k,
# and the Hermite form of d^n (1/r) (eps = 0) makes r^(2l+1) psi_l = h(X, Y, Z)
# a polynomial in X = Rx^2, Y = Ry^2, Z = Rz^2.  The field term is
#     a_i = d_i psi_l = R_i w_i(X, Y, Z) / r^(2l+3),  w_i = 2 r^2 dh/dX_i - (2l+1) h,
# scaled by q = rho h_cell (rho the mean density, h_cell the cell's side).
def _padd(a, b, f=1):
    from fractions import Fraction
    out = dict(a)
    for k, v in b.items():
        out[k] = out.get(k, Fraction(0)) + f * v
    return {k: v for k, v in out.items() if v != 0}


def _pmul(a, b):
    from fractions import Fraction
    out = {}
    for ka, va in a.items():
        for kb, vb in b.items():
            k = (ka[0] + kb[0], ka[1] + kb[1], ka[2] + kb[2])
            out[k] = out.get(k, Fraction(0)) + va * vb
    return {k: v for k, v in out.items() if v != 0}


def _pdiff(a, d):
    out = {}
    for k, v in a.items():
        if k[d] > 0:
            kk = list(k)
            kk[d] -= 1
            out[tuple(kk)] = out.get(tuple(kk), 0) + v * k[d]
    return {k: v for k, v in out.items() if v != 0}


def bg_flop_count(l):
    """Flops (FMA = 2, multiply = 1, rsqrt = 1) of the order-l background term
    as emitted by emit_bg; the walk adds it to an M2P whose scaled separation
    it reuses, so these are the term's whole extra cost per M2P."""
    import re
    body = "\n".join(emit_bg(l).split("\n")[2:-1])
    return 2 * body.count("fma(") + len(re.findall(r" \* ", body)) + body.count("nbody_rsqrt(")


def bg_order(p):
    """order of the background term added at expansion order p (0 = none)"""
    return {0: 4, 2: 4, 4: 6}.get(p, 0)


def bg_poly(l):
    """h(X, Y, Z) = r^(2l+1) psi_l(R) as {(a, b, c): Fraction} for X^a Y^b Z^c"""
    from fractions import Fraction

    def mom(k):
        return Fraction(0) if k % 2 else Fraction(1, (k + 1) * 2 ** k)

    def dfact(j):  # (2j-1)!!
        v = 1
        for t in range(1, 2 * j, 2):
            v *= t
        return v

    r2 = {(1, 0, 0): Fraction(1), (0, 1, 0): Fraction(1), (0, 0, 1): Fraction(1)}
    h = {}
    for n in multi(l):
        if sum(n) != l:
            continue
        cn = mom(n[0]) * mom(n[1]) * mom(n[2])
        if cn == 0:
            continue
        nf = math.factorial(n[0]) * math.factorial(n[1]) * math.factorial(n[2])
        for k in product(*(range(n[d] // 2 + 1) for d in range(3))):
            K = sum(k)
            j = l - K
            hc = Fraction(1)
            for d in range(3):
                hc *= Fraction(math.factorial(n[d]),
                               math.factorial(k[d]) * math.factorial(n[d] - 2 * k[d]) * 2 ** k[d])
            coef = cn / nf * hc * (-1) ** j * dfact(j)
            term = {((n[0] - 2 * k[0]) // 2, (n[1] - 2 * k[1]) // 2, (n[2] - 2 * k[2]) // 2): coef}
            for _ in range(K):
                term = _pmul(term, r2)
            h = _padd(h, term)
    return h


def _bg_parts(l):
    h = bg_poly(l)
    r2 = {(1, 0, 0): 1, (0, 1, 0): 1, (0, 0, 1): 1}
    w = [_padd(_pmul({k: 2 * v for k, v in _pdiff(h, d).items()}, r2), h, -(2 * l + 1)) for d in range(3)]
    return h, w


def _emit_poly(L, name, poly, mono_name):
    """name = sum_k c_k mono_k in the fma subset (first term assigns)"""
    first = True
    for k in sorted(poly):
        c = "T(%.17g)" % float(poly[k])
        mn = mono_name(k)
        if first:
            L.append("  T %s = %s;" % (name, c if mn is None else "%s * %s" % (c, mn)))
            first = False
        else:
            L.append("  %s = fma(%s, %s, %s);" % (name, c, "T(1)" if mn is None else mn, name))
    if first:
        L.append("  T %s = T(0);" % name)


def _emit_monomials(L, polys):
    """declare every monomial X^a Y^b Z^c (degree >= 2) the polynomials use"""
    need = set()
    for p in polys:
        need |= set(p)
    names = {(0, 0, 0): None, (1, 0, 0): "X", (0, 1, 0): "Y", (0, 0, 1): "Z"}
    for k in sorted(need, key=lambda k: (sum(k), k)):
        if k in names:
            continue
        # build from a lower monomial times X, Y or Z
        for d, v in enumerate("XYZ"):
            if k[d] > 0:
                par = list(k)
                par[d] -= 1
                par = tuple(par)
                if par not in names:
                    raise ValueError("monomial %s needs %s" % (k, par))
                nm = "X%dY%dZ%d" % k
                L.append("  const T %s = %s * %s;" % (nm, names[par], v) if names[par] else "  const T %s = %s;" % (nm, v))
                names[k] = nm
                break
    return lambda k: names[k]


def _close_monomials(polys):
    """all lower monomials needed to build the ones the polynomials use"""
    need = set()
    for p in polys:
        for k in p:
            stack = [k]
            while stack:
                m = stack.pop()
                if m in need:
                    continue
                need.add(m)
                for d in range(3):
                    if m[d] > 0:
                        par = list(m)
                        par[d] -= 1
                        stack.append(tuple(par))
                        break
    return [{k: 1 for k in need}]


def emit_bg(l):
    h, w = _bg_parts(l)
    L = ["template <typename T>",
         "__device__ __forceinline__ void cube_bg_l%d(T q, T Rx, T Ry, T Rz, T& ax, T& ay, T& az) {" % l,
         "  const T X = Rx * Rx, Y = Ry * Ry, Z = Rz * Rz;",
         "  const T r2 = fma(Rx, Rx, fma(Ry, Ry, Z));",
         "  const T ir = nbody_rsqrt(r2);",
         "  const T ir2 = ir * ir;"]
    # u = q / r^(2l+3)
    e = "ir"
    for _ in range(l + 1):
        e = "%s * ir2" % e if e != "ir" else "ir * ir2"
    L.append("  const T u = q * %s;" % " * ".join(["ir"] + ["ir2"] * (l + 1)))
    mono = _emit_monomials(L, _close_monomials(w))
    for d in range(3):
        _emit_poly(L, "w%d" % d, w[d], mono)
    for d, (R, a) in enumerate((("Rx", "ax"), ("Ry", "ay"), ("Rz", "az"))):
        L.append("  %s = fma(%s * u, w%d, %s);" % (a, R, d, a))
    L.append("}")
    return "\n".join(L)


def emit_bgpot(l):
    """The background term's potential form q h / r^(2l+1) (its gradient is
    cube_bg_l<l>'s acceleration)."""
    h, _ = _bg_parts(l)
    L = ["template <typename T>",
         "__device__ __forceinline__ T cube_bgpot_l%d(T q, T Rx, T Ry, T Rz) {" % l,
         "  const T X = Rx * Rx, Y = Ry * Ry, Z = Rz * Rz;",
         "  const T r2 = fma(Rx, Rx, fma(Ry, Ry, Z));",
         "  const T ir = nbody_rsqrt(r2);",
         "  const T ir2 = ir * ir;"]
    mono = _emit_monomials(L, _close_monomials([h]))
    _emit_poly(L, "hv", h, mono)
    L.append("  return q * hv * (%s);" % " * ".join(["ir"] + ["ir2"] * l))
    L.append("}")
    return "\n".join(L)


def emit_m2l0(p):
    """m2l0_p<p>(M, D) = sum_{|n| <= p} (-1)^|n|/n! M_n D_n (the local
    expansion's constant term from moments to order p)."""
    me = multi(p)
    L = ["template <typename T>",
         "__device__ __forceinline__ T m2l0_p%d(const T* __restrict__ M, const T* __restrict__ D) {" % p,
         "  T v = T(0);"]
    for u, n in enumerate(me):
        c = (-1.0 if sum(n) % 2 else 1.0) / (math.factorial(n[0]) * math.factorial(n[1]) * math.factorial(n[2]))
        L.append("  v = fma(M[%d] * T(%.17g), D[%d], v);" % (u, c, u))
    L.append("  return v;")
    L.append("}")
    return "\n".join(L)


def emit_l2pot(pe):
    """Image-field potential: L_0 = sum_n (-1)^|n|/n! M_n d^n phi~(R0) per
    cell (m2l0_pe), and the series L_0 + sum_{1 <= |m| <= pe+1} d^m/m! L_m
    at offset d from the expansion point (l2pot_pe), whose gradient is minus
    l2p_pe's acceleration."""
    me = multi(pe)
    L = ["template <typename T>",
         "__device__ __forceinline__ T m2l0_pe%d(const T* __restrict__ M, const T* __restrict__ D) {" % pe]
    e = "T(0)"
    for u, n in enumerate(me):
        c = (-1.0 if sum(n) % 2 else 1.0) / (math.factorial(n[0]) * math.factorial(n[1]) * math.factorial(n[2]))
        e = "fma(M[%d] * T(%.17g), D[%d], %s)" % (u, c, u, e) if c not in (1.0, -1.0) else \
            "fma(%sM[%d], D[%d], %s)" % ("-" if c < 0 else "", u, u, e)
    L.append("  return %s;" % e)
    L.append("}")
    mP = multi(pe + 1)
    mmi = {m: i for i, m in enumerate(mP)}
    L.append("template <typename T>")
    L.append("__device__ __forceinline__ T l2pot_pe%d(T L0, const T* __restrict__ Lc, T dx, T dy, T dz) {" % pe)
    L.append("  const T q0 = T(1);")
    for i, m in enumerate(mP):
        if i == 0:
            continue
        for d in range(3):
            if m[d] > 0:
                par = list(m)
                par[d] -= 1
                L.append("  const T q%d = q%d * (%s * T(%.17g));" % (i, mmi[tuple(par)], "dxdydz"[2 * d:2 * d + 2],
                                                                    1.0 / m[d]))
                break
    e = "L0"
    for i in range(1, len(mP)):
        e = "fma(q%d, Lc[%d], %s)" % (i, i - 1, e)
    L.append("  return %s;" % e)
    L.append("}")
    return "\n".join(L)


def emit_bg_hvp(l):
    """o += J lam, J_ij = d a_i / d R_j of the background term:
    (J lam)_i = u [w_i lam_i + R_i sum_j 2 R_j (dw_i/dX_j) lam_j - (2l+3) R_i w_i (R.lam) / r^2]."""
    h, w = _bg_parts(l)
    D = [[_pdiff(w[i], j) for j in range(3)] for i in range(3)]
    L = ["template <typename T>",
         "__device__ __forceinline__ void cube_bg_hvp_l%d(T q, T Rx, T Ry, T Rz, T lx, T ly, T lz, T& ox, T& oy," % l,
         "                                             T& oz) {",
         "  const T X = Rx * Rx, Y = Ry * Ry, Z = Rz * Rz;",
         "  const T r2 = fma(Rx, Rx, fma(Ry, Ry, Z));",
         "  const T ir = nbody_rsqrt(r2);",
         "  const T ir2 = ir * ir;"]
    L.append("  const T u = q * %s;" % " * ".join(["ir"] + ["ir2"] * (l + 1)))
    mono = _emit_monomials(L, _close_monomials(w + [D[i][j] for i in range(3) for j in range(3)]))
    for d in range(3):
        _emit_poly(L, "w%d" % d, w[d], mono)
    for i in range(3):
        for j in range(3):
            _emit_poly(L, "d%d%d" % (i, j), D[i][j], mono)
    L.append("  const T t0 = T(2) * Rx * lx, t1 = T(2) * Ry * ly, t2 = T(2) * Rz * lz;")
    L.append("  const T rl = fma(Rx, lx, fma(Ry, ly, Rz * lz)) * (T(%d) * ir2);" % (-(2 * l + 3)))
    for i, (R, lv, o) in enumerate((("Rx", "lx", "ox"), ("Ry", "ly", "oy"), ("Rz", "lz", "oz"))):
        L.append("  const T s%d = fma(d%d0, t0, fma(d%d1, t1, d%d2 * t2));" % (i, i, i, i))
        L.append("  %s = fma(u, fma(w%d, %s, %s * fma(w%d, rl, s%d)), %s);" % (o, i, lv, R, i, i, o))
    L.append("}")
    return "\n".join(L)


def generate():
    out = []
    out.append("// Generated by gen_m2p.py -- do not edit by hand.")
    out.append("// Reduced-coefficient multipole-to-particle kernels, orders 0..4.")
    out.append("#pragma once")
    out.append("")
    for p in range(5):
        out.append("constexpr int kNB%d = %d;  // reduced coefficients at order %d" % (p, len(slots(p)), p))
        out.append("constexpr int kM2PFlops%d = %d;  // flops per M2P (FMA = 2, rsqrt = 1)" % (p, flop_count(p)))
    out.append("")
    for p in range(5):
        out.append(emit_m2p(p))
        out.append("")
        out.append(emit_m2pot(p))
        out.append("")
        out.append(emit_m2p2(p))
        out.append("")
        out.append(emit_reduce(p))
        out.append("")
    for p in range(6):
        out.append(emit_p2m(p))
        out.append("")
        out.append(emit_m2m(p))
        out.append("")
    for pe in range(1, 6):
        out.append("constexpr int kNL%d = %d;  // local coefficients, image-field order %d" % (pe, len(multi(pe + 1)) - 1, pe))
        out.append(emit_m2l(pe))
        out.append("")
        out.append(emit_l2pot(pe))
        out.append("")
    # the far lattice of the near-replica scheme: its evaluation at order 7
    # (coefficients to order 8) and the constant term from order-8 moments
    out.append("constexpr int kNL7 = %d;  // far-lattice local coefficients (orders 1..8)" % (len(multi(8)) - 1))
    out.append(emit_m2l(7, with_m2l=False))
    out.append("")
    out.append("\n".join(emit_l2pot(7).split("\n")[emit_l2pot(7).split("\n").index("template <typename T>", 1):]))
    out.append("")
    out.append(emit_m2l0(8))
    out.append("")
    for p in range(1, 5):
        out.append(emit_dtensor(p + 1))
        out.append("")
        out.append(emit_m2l_red(p))
        out.append("")
    out.append("__device__ __forceinline__ float2 nbody_rsqrt2(float2 s) {")
    out.append("  return make_float2(nbody_rsqrt(s.x), nbody_rsqrt(s.y));")
    out.append("}")
    out.append("")
    for l in (4, 6):
        out.append(emit_bg(l))
        out.append("")
        out.append(emit_bgpot(l))
        out.append("")
        out.append(pack(emit_bg(l), "cube_bg_l%d" % l, "cube_bg2_l%d" % l))
        out.append("")
    return "\n".join(out) + "\n"




# ---- reverse-mode (adjoint) kernels -------------------------------------------------
def emit_m2p_adj_self(p):
    """J lam with J = dA/dR (symmetric) of the reduced M2P A(R) = sum_j (R F_{j+1} S_j + F_j G_j):
    (J lam)_k = sum_j [F_{j+1} S_j lam_k + R_k F_{j+2} S_j (R.lam) + R_k F_{j+1} (G_j.lam)
                       + F_{j+1} G_{j,k} (R.lam) + F_j (H_j lam)_k],
    (H_j lam)_k = sum_a B_{j,a} Lmu_{a-e_k},  Lmu_c = sum_l lam_l mu_{c-e_l}."""
    mon = multi(p)
    mi = {m: i for i, m in enumerate(mon)}
    sl = slots(p)
    L = ["template <typename T>",
         "__device__ __forceinline__ void m2p_adj_self_p%d(const T* __restrict__ B, T Rx, T Ry, T Rz, T eps2," % p,
         "                                          T lx, T ly, T lz, T& ox, T& oy, T& oz) {",
         "  const T s = fma(Rx, Rx, fma(Ry, Ry, fma(Rz, Rz, eps2)));",
         "  const T F0 = nbody_rsqrt(s);",
         "  const T is = F0 * F0;"]
    for j in range(1, p + 3):
        L.append("  const T F%d = F%d * (T(%d) * is);" % (j, j - 1, -(2 * j - 1)))
    for d, R in enumerate(("Rx", "Ry", "Rz")):
        for k in range(2, p + 1):
            L.append("  const T %s_%d = %s * T(%.17g);" % (R, k, R, 1.0 / k))
    L.append("  const T m0 = T(1);")
    for i, m in enumerate(mon):
        if i == 0:
            continue
        for d in range(3):
            if m[d] > 0:
                par = list(m)
                par[d] -= 1
                pi = mi[tuple(par)]
                R = ("Rx", "Ry", "Rz")[d]
                fac = R if m[d] == 1 else "%s_%d" % (R, m[d])
                L.append("  const T m%d = %s;" % (i, fac if pi == 0 else "m%d * %s" % (pi, fac)))
                break
    # Lmu_c for |c| <= p-1
    lam = ("lx", "ly", "lz")
    # q_c = sum_l lam_l mu_{c-e_l}, so that (H_j lam)_k = sum_a B_{j,a} q_{a-e_k}
    for i, c in enumerate(mon):
        if sum(c) > p - 1 or sum(c) == 0:
            continue
        first = True
        for d in range(3):
            if c[d] > 0:
                cc = list(c)
                cc[d] -= 1
                mk = mi[tuple(cc)]
                if first:
                    L.append("  T q%d = %s;" % (i, lam[d] if mk == 0 else "%s * m%d" % (lam[d], mk)))
                    first = False
                else:
                    L.append("  q%d = fma(%s, m%d, q%d);" % (i, lam[d], mk, i))
    # accumulators start at their first term; terms of the unit monomial are
    # plain additions; G_0 and H_0 vanish and are not formed
    started = set()

    def acc(name, mono, qv=False):
        src = ("q%d" if qv else "m%d") % mono
        if name not in started:
            started.add(name)
            return "    %s = %s;" % (name, "b" if (mono == 0 and not qv) else "b * %s" % src)
        if mono == 0 and not qv:
            return "    %s += b;" % name
        return "    %s = fma(b, %s, %s);" % (name, src, name)

    body = []
    for t, (j, a) in enumerate(sl):
        body.append((t, j, a))
    # declare every accumulator up front (first terms assign)
    decl = []
    for (t, j, a) in body:
        for nm in ["S%d" % j] + ["G%d%s" % (j, c) for d, c in enumerate("xyz") if a[d] > 0] + \
                  ["H%d%s" % (j, c) for d, c in enumerate("xyz") if a[d] > 0 and sum(a) > 1]:
            if nm not in decl:
                decl.append(nm)
    L.append("  T %s;" % ", ".join(decl))
    for (t, j, a) in body:
        L.append("  { const T b = B[%d];" % t)
        L.append(acc("S%d" % j, mi[a]))
        for d, ax in enumerate("xyz"):
            if a[d] > 0:
                par = list(a)
                par[d] -= 1
                L.append(acc("G%d%s" % (j, ax), mi[tuple(par)]))
                if sum(par) > 0:
                    L.append(acc("H%d%s" % (j, ax), mi[tuple(par)], qv=True))
        L.append("  }")
    L.append("  const T rl = fma(Rx, lx, fma(Ry, ly, Rz * lz));")
    L.append("  T ax = ox, ay = oy, az = oz;")
    for j in range(p + 1):
        hasG = ("G%dx" % j) in decl
        hasH = ("H%dx" % j) in decl
        L.append("  { const T a1 = F%d * S%d;  // F_{j+1} S_j" % (j + 1, j))
        if hasG:
            L.append("    const T gl = fma(G%dx, lx, fma(G%dy, ly, G%dz * lz));" % (j, j, j))
            L.append("    const T c1 = fma(F%d * S%d, rl, F%d * gl);  // R_k coefficient" % (j + 2, j, j + 1))
            L.append("    const T c2 = F%d * rl;  // G_{j,k} coefficient" % (j + 1))
        else:
            L.append("    const T c1 = F%d * S%d * rl;  // R_k coefficient" % (j + 2, j))
        for ax, Rv, lv in (("x", "Rx", "lx"), ("y", "Ry", "ly"), ("z", "Rz", "lz")):
            e = "a%s" % ax
            if hasH:
                e = "fma(F%d, H%d%s, %s)" % (j, j, ax, e)
            if hasG:
                e = "fma(c2, G%d%s, %s)" % (j, ax, e)
            L.append("    a%s = fma(a1, %s, fma(%s, c1, %s));" % (ax, lv, Rv, e))
        L.append("  }")
    L.append("  ox = ax;")
    L.append("  oy = ay;")
    L.append("  oz = az;")
    L.append("}")
    return "\n".join(L)


def emit_m2p_adj_src(p):
    """nu_n += sum_l lam_l d^{n+e_l} g(R), |n| <= p, via nu_n = (lam.R) E_n + sum_d n_d lam_d E_{n-e_d},
    E_m = d^m F_1 = sum_k h(m,k) R^(m-2k) F_{1+|m|-|k|}."""
    mon = multi(p)
    mi = {m: i for i, m in enumerate(mon)}
    L = ["template <typename T>",
         "__device__ __forceinline__ void m2p_adj_src_p%d(T Rx, T Ry, T Rz, T eps2, T lx, T ly, T lz," % p,
         "                                         T* __restrict__ nu) {",
         "  const T s = fma(Rx, Rx, fma(Ry, Ry, fma(Rz, Rz, eps2)));",
         "  const T F0 = nbody_rsqrt(s);",
         "  const T is = F0 * F0;"]
    for j in range(1, p + 2):
        L.append("  const T F%d = F%d * (T(%d) * is);" % (j, j - 1, -(2 * j - 1)))
    L.append("  const T r0 = T(1);")
    for i, m in enumerate(mon):
        if i == 0:
            continue
        for d in range(3):
            if m[d] > 0:
                par = list(m)
                par[d] -= 1
                pi = mi[tuple(par)]
                R = ("Rx", "Ry", "Rz")[d]
                L.append("  const T r%d = %s;" % (i, R if pi == 0 else "r%d * %s" % (pi, R)))
                break
    # E_m
    for i, m in enumerate(mon):
        byj = {}
        for k in product(*(range(m[d] // 2 + 1) for d in range(3))):
            a = tuple(m[d] - 2 * k[d] for d in range(3))
            j = 1 + sum(m) - sum(k)
            byj.setdefault(j, []).append((hcoef(m, k), mi[a]))
        parts = []
        for j, terms in sorted(byj.items()):
            expr = None
            for c, ai in terms:
                if expr is None:
                    expr = "r%d * T(%.17g)" % (ai, c) if c != 1.0 else "r%d" % ai
                else:
                    expr = "fma(r%d, T(%.17g), %s)" % (ai, c, expr)
            parts.append((j, expr))
        e = None
        for j, expr in parts:
            e = "F%d * (%s)" % (j, expr) if e is None else "fma(F%d, %s, %s)" % (j, expr, e)
        L.append("  const T E%d = %s;" % (i, e))
    L.append("  const T rl = fma(Rx, lx, fma(Ry, ly, Rz * lz));")
    lam = ("lx", "ly", "lz")
    for i, n in enumerate(mon):
        expr = "fma(rl, E%d, nu[%d])" % (i, i)
        for d in range(3):
            if n[d] > 0:
                nn = list(n)
                nn[d] -= 1
                fac = lam[d] if n[d] == 1 else "(%s * T(%d))" % (lam[d], n[d])
                expr = "fma(%s, E%d, %s)" % (fac, mi[tuple(nn)], expr)
        L.append("  nu[%d] = %s;" % (i, expr))
    L.append("}")
    return "\n".join(L)


def emit_m2m_adj(p):
    """nuc_k += sum_{n >= k} C(n,k) s^(n-k) nup_n (transpose of the M2M shift), FP64."""
    mon = multi(p)
    mi = {m: i for i, m in enumerate(mon)}
    L = ["__device__ __forceinline__ void m2m_adj_acc_p%d(const double* __restrict__ nup, double sx, double sy, double sz, double* __restrict__ nuc) {" % p,
         "  const double w0 = 1.0;"]
    for i, mm in enumerate(mon):
        if i == 0:
            continue
        for d in range(3):
            if mm[d] > 0:
                par = list(mm)
                par[d] -= 1
                L.append("  const double w%d = w%d * %s;" % (i, mi[tuple(par)], "sxsysz"[2 * d:2 * d + 2]))
                break
    for kk, k in enumerate(mon):
        expr = "nuc[%d]" % kk
        for n in mon:
            if all(n[d] >= k[d] for d in range(3)):
                b = math.comb(n[0], k[0]) * math.comb(n[1], k[1]) * math.comb(n[2], k[2])
                w = mi[(n[0] - k[0], n[1] - k[1], n[2] - k[2])]
                expr = ("fma(w%d, nup[%d], %s)" % (w, mi[n], expr)) if b == 1 else \
                       ("fma(w%d * %d.0, nup[%d], %s)" % (w, b, mi[n], expr))
        L.append("  nuc[%d] = %s;" % (kk, expr))
    L.append("}")
    return "\n".join(L)


def emit_p2m_adj(p):
    """g += m sum_n nu_n grad (d^n) (transpose of P2M), FP64."""
    mon = multi(p)
    mi = {m: i for i, m in enumerate(mon)}
    L = ["__device__ __forceinline__ void p2m_adj_p%d(double m, double dx, double dy, double dz, const double* __restrict__ nu, double& gx, double& gy, double& gz) {" % p,
         "  const double q0 = 1.0;"]
    for i, mm in enumerate(mon):
        if i == 0 or sum(mm) > p - 1:
            continue
        for d in range(3):
            if mm[d] > 0:
                par = list(mm)
                par[d] -= 1
                L.append("  const double q%d = q%d * %s;" % (i, mi[tuple(par)], "dxdydz"[2 * d:2 * d + 2]))
                break
    for d, gv in enumerate(("gx", "gy", "gz")):
        expr = "0.0"
        for i, n in enumerate(mon):
            if n[d] == 0:
                continue
            nn = list(n)
            nn[d] -= 1
            c = n[d]
            expr = ("fma(nu[%d], q%d, %s)" % (i, mi[tuple(nn)], expr)) if c == 1 else \
                   ("fma(nu[%d] * %d.0, q%d, %s)" % (i, c, mi[tuple(nn)], expr))
        L.append("  %s = fma(m, %s, %s);" % (gv, expr, gv))
    L.append("}")
    return "\n".join(L)


def emit_field_adj(pe):
    """Image-field reverse kernels: Hessian-vector of the local expansion, the
    cotangent of its coefficients, and the transposed M2L."""
    P = pe + 1
    mP = multi(P)
    miP = {m: i for i, m in enumerate(mP)}
    me = multi(pe)
    L = []
    # (a) hess: o_k -= sum_l lam_l sum_{|c| <= pe-1} d^c/c! L_{c+e_k+e_l}
    L.append("template <typename T>")
    L.append("__device__ __forceinline__ void l2p_hess_pe%d(const T* __restrict__ Lc, T dx, T dy, T dz, T lx, T ly, T lz, T& ox, T& oy, T& oz) {" % pe)
    mc = [c for c in me if sum(c) <= pe - 1]
    mci = {c: i for i, c in enumerate(me)}
    L.append("  const T q0 = T(1);")
    for i, m in enumerate(me):
        if i == 0 or sum(m) > pe - 1:
            continue
        for d in range(3):
            if m[d] > 0:
                par = list(m)
                par[d] -= 1
                L.append("  const T q%d = q%d * (%s * T(%.17g));" % (i, mci[tuple(par)], "dxdydz"[2 * d:2 * d + 2], 1.0 / m[d]))
                break
    lam = ("lx", "ly", "lz")
    for k, ov in enumerate(("ox", "oy", "oz")):
        expr = ov
        for l in range(3):
            for c in mc:
                t = list(c)
                t[k] += 1
                t[l] += 1
                expr = "fma(-%s * q%d, Lc[%d], %s)" % (lam[l], mci[c], miP[tuple(t)] - 1, expr)
        L.append("  %s = %s;" % (ov, expr))
    L.append("}")
    # (b) cotangent of L: Lbar_m -= sum_{l: m_l>=1} lam_l d^{m-e_l}/(m-e_l)!
    L.append("template <typename T>")
    L.append("__device__ __forceinline__ void l2p_adj_pe%d(T dx, T dy, T dz, T lx, T ly, T lz, T* __restrict__ Lbar) {" % pe)
    L.append("  const T q0 = T(1);")
    for i, m in enumerate(me):
        if i == 0:
            continue
        for d in range(3):
            if m[d] > 0:
                par = list(m)
                par[d] -= 1
                L.append("  const T q%d = q%d * (%s * T(%.17g));" % (i, mci[tuple(par)], "dxdydz"[2 * d:2 * d + 2], 1.0 / m[d]))
                break
    for t, m in enumerate(mP):
        if t == 0:
            continue
        expr = "Lbar[%d]" % (t - 1)
        for l in range(3):
            if m[l] >= 1:
                c = list(m)
                c[l] -= 1
                if sum(c) <= pe:
                    expr = "fma(-%s, q%d, %s)" % (lam[l], mci[tuple(c)], expr)
        L.append("  Lbar[%d] = %s;" % (t - 1, expr))
    L.append("}")
    # (c) transposed M2L: nu_n += (-1)^|n|/n! sum_m Lbar_m D_{m+n}
    L.append("template <typename T>")
    L.append("__device__ __forceinline__ void m2l_adj_pe%d(const T* __restrict__ Lbar, const T* __restrict__ D, T* __restrict__ nu) {" % pe)
    for u, n in enumerate(me):
        c = (-1.0 if sum(n) % 2 else 1.0) / (math.factorial(n[0]) * math.factorial(n[1]) * math.factorial(n[2]))
        expr = None
        for t, m in enumerate(mP):
            if t == 0 or sum(m) + sum(n) > P:
                continue
            k = miP[(m[0] + n[0], m[1] + n[1], m[2] + n[2])]
            expr = ("Lbar[%d] * D[%d]" % (t - 1, k)) if expr is None else ("fma(Lbar[%d], D[%d], %s)" % (t - 1, k, expr))
        L.append("  nu[%d] = fma(T(%.17g), %s, nu[%d]);" % (u, c, expr, u))
    L.append("}")
    return "\n".join(L)


# ---- packed FP32 pairs from the scalar emitters -----------------------------------
# The scalar emitters above write a small C subset: declarations and
# assignments of T values built from fma(a, b, c), products a * b, constants
# T(c), nbody_rsqrt(x), names and B[i] / nu[i] elements.  pack() rewrites such
# a function for float2 operands, one pair instruction per scalar operation in
# the same order, so each half of the result is bitwise the scalar FP32 one.
def _flit(v):
    """a float literal for the value of the decimal string v"""
    t = "%.9g" % float(v)
    if not any(ch in t for ch in ".en"):
        t += ".0"
    return t + "f"


def _tokens(src):
    import re
    tok = re.compile(r"\s*(?:([A-Za-z_][A-Za-z0-9_]*)|([0-9][0-9.eE+\-]*)|(\+=|[()\[\],*=;{}+\-]))")
    out, pos = [], 0
    while pos < len(src):
        m = tok.match(src, pos)
        if not m or m.end() == pos:
            if src[pos:].strip() == "":
                break
            raise ValueError("cannot tokenize: %r" % src[pos:])
        out.append(m.group(1) or m.group(2) or m.group(3))
        pos = m.end()
    return out


class _P:
    def __init__(self, toks):
        self.t, self.i = toks, 0

    def peek(self):
        return self.t[self.i] if self.i < len(self.t) else None

    def take(self, want=None):
        v = self.t[self.i]
        if want is not None and v != want:
            raise ValueError("expected %s got %s" % (want, v))
        self.i += 1
        return v

    def expr(self):
        e = self.unary()
        while self.peek() == "*":
            self.take()
            e = "__fmul2_rn(%s, %s)" % (e, self.unary())
        return e

    def unary(self):
        if self.peek() == "-":
            self.take()
            return "__fmul2_rn(make_float2(-1.0f, -1.0f), %s)" % self.unary()
        return self.primary()

    def number(self):
        sign = ""
        if self.peek() == "-":
            self.take()
            sign = "-"
        return sign + _flit(self.take())

    def primary(self):
        v = self.take()
        if v == "fma":
            self.take("(")
            a = self.expr()
            self.take(",")
            b = self.expr()
            self.take(",")
            c = self.expr()
            self.take(")")
            return "__ffma2_rn(%s, %s, %s)" % (a, b, c)
        if v == "T":
            self.take("(")
            c = self.number()
            self.take(")")
            return "make_float2(%s, %s)" % (c, c)
        if v == "nbody_rsqrt":
            self.take("(")
            a = self.expr()
            self.take(")")
            return "nbody_rsqrt2(%s)" % a
        if v == "(":
            e = self.expr()
            self.take(")")
            return e
        if self.peek() == "[":
            self.take("[")
            k = self.take()
            self.take("]")
            return "%s[%s]" % (v, k)
        if v[0].isdigit():
            c = _flit(v)
            return "make_float2(%s, %s)" % (c, c)
        return v


def _pack_decls(toks):
    """T a = e, b, ...  ->  float2 a = e', b, ..."""
    P = _P(toks)
    parts = []
    while P.peek() is not None:
        name = P.take()
        if P.peek() == "=":
            P.take("=")
            parts.append("%s = %s" % (name, P.expr()))
        else:
            parts.append(name)
        if P.peek() == ",":
            P.take()
    return ", ".join(parts)


def pack(code, name_from, name_to):
    out = []
    lines = code.split("\n")
    i = 0
    while lines[i].startswith("template"):
        i += 1
    sig = []
    while True:
        sig.append(lines[i])
        if lines[i].rstrip().endswith("{"):
            break
        i += 1
    sig = " ".join(x.strip() for x in sig)
    sig = sig.replace(name_from, name_to).replace("const T*", "const float2*").replace("T*", "float2*")
    sig = sig.replace("T&", "float2&").replace("(T ", "(float2 ").replace(", T ", ", float2 ")
    out.append(sig)
    for ln in lines[i + 1:]:
        body = ln.split("//")[0].rstrip()
        ind = body[: len(body) - len(body.lstrip())]
        st = body.strip()
        if st in ("", "}"):
            out.append(body)
            continue
        pre = ""
        if st.startswith("{ "):
            pre, st = "{ ", st[2:]
        assert st.endswith(";"), st
        st = st[:-1]
        if st.startswith("const T "):
            out.append("%s%sconst float2 %s;" % (ind, pre, _pack_decls(_tokens(st[len("const T "):]))))
        elif st.startswith("T "):
            out.append("%s%sfloat2 %s;" % (ind, pre, _pack_decls(_tokens(st[2:]))))
        elif "+=" in st:
            lhs, rhs = st.split("+=")
            out.append("%s%s%s = __fadd2_rn(%s, %s);" % (ind, pre, lhs.strip(), lhs.strip(), _P(_tokens(rhs)).expr()))
        else:
            lhs, rhs = st.split("=", 1)
            out.append("%s%s%s = %s;" % (ind, pre, lhs.strip(), _P(_tokens(rhs)).expr()))
    return "\n".join(out)


def generate_adjoint():
    out = ["// Generated by gen_m2p.py -- do not edit by hand.",
           "// Reverse-mode (adjoint) kernels of the M2P, M2M, P2M and image-field expansions.",
           "#pragma once", ""]
    for l in (4, 6):
        out.append(emit_bg_hvp(l))
        out.append("")
    for p in range(5):
        out.append(emit_m2p_adj_self(p))
        out.append("")
        out.append(pack(emit_m2p_adj_self(p), "m2p_adj_self_p%d" % p, "m2p2_adj_self_p%d" % p))
        out.append("")
        out.append(emit_m2p_adj_src(p))
        out.append("")
        out.append(emit_m2m_adj(p))
        out.append("")
        out.append(emit_p2m_adj(p))
        out.append("")
    for pe in range(1, 6):
        out.append(emit_field_adj(pe))
        out.append("")
    return "\n".join(out) + "\n"


if __name__ == "__main__":
    here = os.path.dirname(os.path.abspath(__file__))
    outputs = {os.path.join(here, "m2p_gen.cuh"): generate(),
               os.path.join(here, "adj_gen.cuh"): generate_adjoint()}
    if len(sys.argv) > 1 and sys.argv[1] == "--check":
        sys.exit(0 if all(os.path.exists(k) and open(k).read() == v for k, v in outputs.items()) else 1)
    for k, v in outputs.items():
        with open(k, "w") as f:
            f.write(v)
