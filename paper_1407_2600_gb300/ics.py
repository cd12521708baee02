"""Seeded synthetic inputs (shared by the oracle tests and the CUDA path).

This module holds none of the force method's arithmetic: it only draws the
particle distributions the workloads are defined on.  Everything is FP64,
seeded, in box units (unit periodic cube).

* Zel'dovich displacements: white noise from ``numpy.random.Generator(PCG64(seed))``
  on an ng^3 grid, FFT, multiplication by sqrt(P(k)) with P(k) ~ k^n, a
  spherical cut at the grid Nyquist |k| <= pi ng (Nyquist planes zeroed),
  psi_k = i k delta_k / k^2, inverse FFT, rescaled so that the rms of |psi|
  equals the requested fraction of the grid spacing.
* NFW haloes: counts log-uniform in [nmin, nmax], concentration uniform in
  [cmin, cmax], r200 from 200 times the mean density, radii by inverting the
  enclosed-mass profile ln(1+x) - x/(1+x) for x <= c, isotropic directions,
  centres uniform; halo particles replace distinct random grid particles so
  that N is unchanged.
"""
from __future__ import annotations

import math

import numpy as np


def lattice(ng: int) -> np.ndarray:
    """Grid points q = (i + 1/2)/ng, (ng^3, 3), x fastest-varying last."""
    g = (np.arange(ng, dtype=np.float64) + 0.5) / ng
    qx, qy, qz = np.meshgrid(g, g, g, indexing="ij")
    return np.stack([qx.ravel(), qy.ravel(), qz.ravel()], axis=1)


def zeldovich_displacement(ng: int, n_index: float, rms_spacing: float, seed: int) -> np.ndarray:
    """Displacement field psi (ng^3, 3) in box units with rms |psi| =
    rms_spacing / ng; power spectrum P(k) ~ k^n_index."""
    rng = np.random.Generator(np.random.PCG64(seed))
    white = rng.standard_normal((ng, ng, ng))
    dk = np.fft.rfftn(white)
    kx = np.fft.fftfreq(ng, d=1.0 / ng) * 2.0 * math.pi
    kz = np.fft.rfftfreq(ng, d=1.0 / ng) * 2.0 * math.pi
    KX, KY, KZ = np.meshgrid(kx, kx, kz, indexing="ij")
    k2 = KX ** 2 + KY ** 2 + KZ ** 2
    kk = np.sqrt(k2)
    kny = math.pi * ng
    amp = np.zeros_like(kk)
    ok = (kk > 0) & (kk <= kny)
    amp[ok] = kk[ok] ** (n_index / 2.0)
    # zero the Nyquist planes
    nyq = ng // 2 if ng % 2 == 0 else None
    if nyq is not None:
        amp[nyq, :, :] = 0.0
        amp[:, nyq, :] = 0.0
        amp[:, :, -1] = 0.0
    dk = dk * amp
    k2s = np.where(k2 > 0, k2, 1.0)
    psi = []
    for K in (KX, KY, KZ):
        comp = np.fft.irfftn(1j * K * dk / k2s, s=(ng, ng, ng), axes=(0, 1, 2))
        psi.append(comp.ravel())
    psi = np.stack(psi, axis=1)
    rms = math.sqrt(np.mean(np.sum(psi * psi, axis=1)))
    if rms > 0:
        psi *= (rms_spacing / ng) / rms
    return psi


def zeldovich_particles(ng: int, n_index: float, rms_spacing: float, seed: int):
    """Lagrangian grid q and displacement psi, both (ng^3, 3)."""
    return lattice(ng), zeldovich_displacement(ng, n_index, rms_spacing, seed)


def lpt2_displacement(psi1: np.ndarray, ng: int) -> np.ndarray:
    """Second-order Lagrangian displacement of a first-order field.

    psi1 (ng^3, 3) on the lattice of `lattice` is the Zel'dovich displacement
    -grad phi1.  Returns psi2 = grad phi2 (ng^3, 3), where phi2 solves
    lap phi2 = sum over i < j of (phi1_ii phi1_jj - phi1_ij^2), all derivatives
    spectral (first derivatives without the Nyquist component; the Nyquist
    planes of phi2 zeroed, as those of the first-order field are).  In an
    Einstein-de Sitter background the second-order positions and momenta
    (p = a^2 dx/dt) at linear growth factor D (D = 1 where psi1 is given) are
    x = q + D psi1 - (3/7) D^2 psi2 and p = H0 a^(1/2) D (psi1 - (6/7) D psi2);
    see lpt2_state."""
    k1 = np.fft.fftfreq(ng, d=1.0 / ng) * 2.0 * math.pi
    kd = k1.copy()
    if ng % 2 == 0:
        kd[ng // 2] = 0.0
    K = np.meshgrid(kd, kd, kd, indexing="ij")
    P = [np.fft.fftn(psi1[:, d].reshape(ng, ng, ng)) for d in range(3)]
    # phi1_ij = -d_j psi1_i, symmetrised (psi1 is a gradient field)
    phi = {}
    for i in range(3):
        for j in range(i, 3):
            phi[i, j] = np.real(np.fft.ifftn(-0.5j * (K[j] * P[i] + K[i] * P[j])))
    src = (phi[0, 0] * phi[1, 1] + phi[0, 0] * phi[2, 2] + phi[1, 1] * phi[2, 2]
           - phi[0, 1] ** 2 - phi[0, 2] ** 2 - phi[1, 2] ** 2)
    Q = np.meshgrid(k1, k1, k1, indexing="ij")
    k2 = Q[0] ** 2 + Q[1] ** 2 + Q[2] ** 2
    phi2 = -np.fft.fftn(src) / np.where(k2 > 0, k2, 1.0)
    phi2[k2 == 0] = 0.0
    if ng % 2 == 0:  # Nyquist planes zeroed, as in the first-order field
        phi2[ng // 2, :, :] = 0.0
        phi2[:, ng // 2, :] = 0.0
        phi2[:, :, ng // 2] = 0.0
    return np.stack([np.real(np.fft.ifftn(1j * K[d] * phi2)).ravel() for d in range(3)], axis=1)


def lpt2_state(q: np.ndarray, psi1: np.ndarray, psi2: np.ndarray, growth: float, a: float):
    """Second-order positions (wrapped to [0,1)) and momenta p = a^2 dx/dt at
    expansion factor a with linear growth factor `growth` in Einstein-de
    Sitter (D proportional to a, second-order growth -(3/7) D^2)."""
    h0 = math.sqrt(8.0 * math.pi / 3.0)
    x = np.mod(q + growth * psi1 - (3.0 / 7.0) * growth ** 2 * psi2, 1.0)
    x[x >= 1.0] = 0.0
    p = h0 * math.sqrt(a) * growth * (psi1 - (6.0 / 7.0) * growth * psi2)
    return x, p


def nfw_radii(rng, count: int, c: float, r200: float) -> np.ndarray:
    """Radii drawn from the NFW enclosed-mass profile truncated at r200."""
    def mu(x):
        return np.log1p(x) - x / (1.0 + x)

    u = rng.uniform(0.0, 1.0, count) * mu(c)
    lo = np.zeros(count)
    hi = np.full(count, c)
    for _ in range(80):  # bisection of mu(x) = u on [0, c]
        mid = 0.5 * (lo + hi)
        f = mu(mid) - u
        lo = np.where(f < 0, mid, lo)
        hi = np.where(f < 0, hi, mid)
    return 0.5 * (lo + hi) * (r200 / c)


def add_nfw_haloes(x: np.ndarray, n_halo: int, nmin: int, nmax: int, cmin: float, cmax: float,
                   seed: int):
    """Replace random distinct particles of x (n,3) by NFW haloes.

    Returns (x_new, halo_member_index, halo_table) where halo_table rows are
    (count, concentration, r200, cx, cy, cz)."""
    n = x.shape[0]
    rng = np.random.Generator(np.random.PCG64(seed))
    counts = np.exp(rng.uniform(math.log(nmin), math.log(nmax), n_halo)).astype(np.int64)
    total = int(counts.sum())
    if total > n:
        raise ValueError("haloes need more particles than exist")
    conc = rng.uniform(cmin, cmax, n_halo)
    centres = rng.uniform(0.0, 1.0, (n_halo, 3))
    chosen = rng.permutation(n)[:total]
    xn = x.copy()
    table = []
    off = 0
    for h in range(n_halo):
        cnt = int(counts[h])
        # mean density of the box is n particles per unit volume
        r200 = (3.0 * cnt / (4.0 * math.pi * 200.0 * n)) ** (1.0 / 3.0)
        r = nfw_radii(rng, cnt, conc[h], r200)
        v = rng.standard_normal((cnt, 3))
        v /= np.linalg.norm(v, axis=1, keepdims=True)
        xn[chosen[off:off + cnt]] = np.mod(centres[h] + r[:, None] * v, 1.0)
        table.append((cnt, conc[h], r200, *centres[h]))
        off += cnt
    return xn, chosen, np.array(table)


def config_small(seed: int = 1):
    """16^3 particles, P(k) ~ k^-2, rms displacement 0.25 spacing;
    eps = spacing/30; positions (n,3) in [0,1)."""
    ng = 16
    q, psi = zeldovich_particles(ng, -2.0, 0.25, seed)
    x = np.mod(q + psi, 1.0)
    return x, 1.0 / (30.0 * ng)


def config_haloes(ng: int = 128, seed: int = 1, n_halo: int = 64, rms: float = 0.6,
                  nmin: int = 2000, nmax: int = 50000):
    """ng^3 particles, P(k) ~ k^-2, rms displacement `rms` spacing, plus
    `n_halo` NFW haloes (nmin..nmax particles, log-uniform; c in [5,15])
    replacing random grid particles; eps = spacing/30."""
    q, psi = zeldovich_particles(ng, -2.0, rms, seed)
    x = np.mod(q + psi, 1.0)
    if n_halo > 0:
        x, _, _ = add_nfw_haloes(x, n_halo, nmin, nmax, 5.0, 15.0, seed + 1000)
    return x, 1.0 / (30.0 * ng)


def config_batched(seed: int = 1, sizes=(48,) * 32 + (64,) * 32 + (80,) * 32, rms: float = 0.25,
                   a: float = 0.02):
    """Independent periodic boxes of uneven sizes (default: 32 of 48^3, 32 of
    64^3, 32 of 80^3 particles), each with its own seeded Zel'dovich field
    (P(k) ~ k^-2, rms displacement `rms` spacing) at expansion factor a.
    Returns the concatenated positions (N, 3) and growing-mode momenta
    p = H0 a^(1/2) psi (N, 3), the box offsets (nbox + 1) and the per-box
    softening eps = spacing/30."""
    h0 = np.sqrt(8.0 * np.pi / 3.0)
    xs, ps, eps = [], [], []
    for b, ng in enumerate(sizes):
        q, psi = zeldovich_particles(ng, -2.0, rms, seed * 1000 + b)
        xs.append(np.mod(q + psi, 1.0))
        ps.append(h0 * np.sqrt(a) * psi)
        eps.append(1.0 / (30.0 * ng))
    off = np.cumsum([0] + [len(x) for x in xs])
    return np.concatenate(xs), np.concatenate(ps), off, eps


def zeldovich_device(ng: int, n_index: float, rms_spacing: float, seed: int, a: float, device):
    """The Zel'dovich recipe of zeldovich_displacement for large grids,
    generated on a CUDA device with torch (white noise from a seeded torch
    generator, so a different realisation than the numpy one).  Returns
    positions (3, ng^3) float64 wrapped to [0, 1) and growing-mode momenta
    p = H0 a^(1/2) psi (3, ng^3) float32, particle order as lattice()."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    white = torch.randn((ng, ng, ng), dtype=torch.float64, device=device, generator=g)
    dk = torch.fft.rfftn(white)
    del white
    kx = torch.fft.fftfreq(ng, d=1.0 / ng, dtype=torch.float64, device=device) * 2.0 * math.pi
    kz = torch.fft.rfftfreq(ng, d=1.0 / ng, dtype=torch.float64, device=device) * 2.0 * math.pi
    k2 = kx.view(-1, 1, 1) ** 2 + kx.view(1, -1, 1) ** 2 + kz.view(1, 1, -1) ** 2
    kk = torch.sqrt(k2)
    amp = torch.where((kk > 0) & (kk <= math.pi * ng), kk.clamp_min(1e-300) ** (n_index / 2.0),
                      torch.zeros_like(kk))
    del kk
    if ng % 2 == 0:
        amp[ng // 2, :, :] = 0.0
        amp[:, ng // 2, :] = 0.0
        amp[:, :, -1] = 0.0
    dk = dk * amp / torch.where(k2 > 0, k2, torch.ones_like(k2))
    del amp, k2
    psi = torch.empty((3, ng ** 3), dtype=torch.float64, device=device)
    shapes = ((-1, 1, 1), (1, -1, 1), (1, 1, -1))
    for d in range(3):
        kd = (kx if d < 2 else kz).view(*shapes[d])
        psi[d] = torch.fft.irfftn(1j * kd * dk, s=(ng, ng, ng)).reshape(-1)
    del dk
    rms = float(torch.sqrt(torch.mean(torch.sum(psi * psi, dim=0))))
    if rms > 0:
        psi *= (rms_spacing / ng) / rms
    q = (torch.arange(ng, dtype=torch.float64, device=device) + 0.5) / ng
    pos = torch.empty_like(psi)
    pos[0] = q.view(-1, 1, 1).expand(ng, ng, ng).reshape(-1)
    pos[1] = q.view(1, -1, 1).expand(ng, ng, ng).reshape(-1)
    pos[2] = q.view(1, 1, -1).expand(ng, ng, ng).reshape(-1)
    pos = torch.remainder(pos + psi, 1.0)
    pos[pos >= 1.0] = 0.0
    h0 = math.sqrt(8.0 * math.pi / 3.0)
    mom = (h0 * math.sqrt(a) * psi).float()
    return pos.contiguous(), mom.contiguous()


def random_targets(n: int, k: int, seed: int) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed + 7))
    return np.sort(rng.choice(n, size=min(k, n), replace=False)).astype(np.int64)
