"""The seeded synthetic inputs (paper_1407_2600_gb300.ics) against the recipe
they are stated to follow: Zel'dovich displacements that are the gradient of
a potential, with the requested rms and power-spectrum slope; NFW radii
distributed as the truncated enclosed-mass profile; haloes that replace
distinct particles within their r200; the batched boxes' layout and
growing-mode momenta.  CPU only."""
import math

import numpy as np
import pytest

from paper_1407_2600_gb300 import ics


@pytest.mark.parametrize("ng,n_index,rms", [(32, -2.0, 0.25), (48, -1.5, 0.6)])
def test_zeldovich_rms_and_gradient_field(ng, n_index, rms):
    psi = ics.zeldovich_displacement(ng, n_index, rms, 4)
    assert psi.shape == (ng ** 3, 3)
    assert abs(math.sqrt(np.mean(np.sum(psi * psi, axis=1))) - rms / ng) <= 1e-12 * rms / ng
    # curl-free: k x psi_k = 0 for every mode (psi is minus the gradient of a potential)
    f = [np.fft.fftn(psi[:, d].reshape(ng, ng, ng)) for d in range(3)]
    k = np.fft.fftfreq(ng, d=1.0 / ng)
    KX, KY, KZ = np.meshgrid(k, k, k, indexing="ij")
    curl = [KY * f[2] - KZ * f[1], KZ * f[0] - KX * f[2], KX * f[1] - KY * f[0]]
    scale = np.sqrt(KX ** 2 + KY ** 2 + KZ ** 2) * np.sqrt(sum(np.abs(c) ** 2 for c in f))
    assert max(np.abs(c).max() for c in curl) <= 1e-10 * scale.max()


@pytest.mark.parametrize("n_index", [-2.0, -1.5])
def test_zeldovich_power_spectrum_slope(n_index):
    """delta = -div psi has P(k) ~ k^n: the slope of the shell-averaged
    power over k in [4, 0.8 k_Ny] (in units of the fundamental mode)."""
    ng = 64
    psi = ics.zeldovich_displacement(ng, n_index, 0.25, 11)
    f = [np.fft.fftn(psi[:, d].reshape(ng, ng, ng)) for d in range(3)]
    k = np.fft.fftfreq(ng, d=1.0 / ng)
    KX, KY, KZ = np.meshgrid(k, k, k, indexing="ij")
    delta = -1j * 2 * math.pi * (KX * f[0] + KY * f[1] + KZ * f[2])
    kk = np.sqrt(KX ** 2 + KY ** 2 + KZ ** 2).ravel()
    pk = (np.abs(delta) ** 2).ravel()
    edges = np.geomspace(4.0, 0.8 * ng / 2, 12)
    lk, lp = [], []
    for lo, hi in zip(edges[:-1], edges[1:]):
        sel = (kk >= lo) & (kk < hi)
        lk.append(np.log(np.mean(kk[sel])))
        lp.append(np.log(np.mean(pk[sel])))
    slope = np.polyfit(lk, lp, 1)[0]
    assert abs(slope - n_index) <= 0.05, slope
    # nothing beyond the spherical Nyquist cut
    assert pk[kk > ng / 2 + 1e-9].max() <= 1e-20 * pk.max()


def test_nfw_radii_follow_the_enclosed_mass_profile():
    rng = np.random.Generator(np.random.PCG64(5))
    c, r200, n = 8.0, 0.02, 20000
    r = ics.nfw_radii(rng, n, c, r200)
    assert r.min() >= 0.0 and r.max() <= r200
    x = np.sort(r * c / r200)
    mu = lambda t: np.log1p(t) - t / (1.0 + t)
    cdf = mu(x) / mu(c)
    emp = np.arange(1, n + 1) / n
    ks = np.max(np.maximum(np.abs(emp - cdf), np.abs(emp - 1.0 / n - cdf)))
    assert ks <= 1.63 / math.sqrt(n)  # 1 % level of the Kolmogorov distribution


def test_haloes_replace_distinct_particles_within_r200():
    ng = 32
    q, psi = ics.zeldovich_particles(ng, -2.0, 0.6, 3)
    x = np.mod(q + psi, 1.0)
    xn, members, table = ics.add_nfw_haloes(x, 6, 50, 800, 5.0, 15.0, 77)
    assert xn.shape == x.shape
    assert len(np.unique(members)) == len(members) == int(table[:, 0].sum())
    untouched = np.setdiff1d(np.arange(len(x)), members)
    assert np.array_equal(xn[untouched], x[untouched])
    assert (xn >= 0).all() and (xn < 1).all()
    off = 0
    for cnt, conc, r200, cx, cy, cz in table:
        cnt = int(cnt)
        assert 50 <= cnt <= 800 and 5.0 <= conc <= 15.0
        # r200 encloses 200 times the mean density (n particles per unit volume)
        assert abs(cnt / (4.0 / 3.0 * math.pi * r200 ** 3) / len(x) - 200.0) <= 1e-9 * 200.0
        d = xn[members[off:off + cnt]] - np.array([cx, cy, cz])
        d -= np.round(d)
        assert np.linalg.norm(d, axis=1).max() <= r200 * (1 + 1e-12)
        off += cnt


def test_batched_boxes_layout_and_growing_mode():
    sizes = (8, 12, 16)
    a = 0.02
    x, p, off, eps = ics.config_batched(2, sizes=sizes, a=a)
    assert list(off) == [0, 512, 512 + 1728, 512 + 1728 + 4096]
    assert np.allclose(eps, [1.0 / (30 * s) for s in sizes], rtol=0, atol=0)
    h0 = math.sqrt(8.0 * math.pi / 3.0)
    for b, ng in enumerate(sizes):
        xb, pb = x[off[b]:off[b + 1]], p[off[b]:off[b + 1]]
        psi = xb - ics.lattice(ng)
        psi -= np.round(psi)  # displacements are far below half a box
        assert np.allclose(pb, h0 * math.sqrt(a) * psi, rtol=1e-12, atol=1e-15)
        assert abs(math.sqrt(np.mean(np.sum(psi * psi, axis=1))) - 0.25 / ng) <= 1e-9 / ng


def _crossed_waves(ng, A, B):
    q = ics.lattice(ng)
    k = 2 * math.pi
    psi1 = np.stack([A * np.sin(k * q[:, 0]), B * np.sin(k * q[:, 1]), 0 * q[:, 2]], axis=1)
    return q, psi1


def test_lpt2_crossed_waves_closed_form():
    """psi1 = (A sin kx, B sin ky, 0): phi1 = (A cos kx + B cos ky)/k, the
    source phi1_xx phi1_yy = A B k^2 cos kx cos ky, phi2 = -(A B / 2) cos kx
    cos ky and psi2 = (A B k / 2)(sin kx cos ky, cos kx sin ky, 0)."""
    ng, A, B = 16, 0.02, 0.013
    q, psi1 = _crossed_waves(ng, A, B)
    psi2 = ics.lpt2_displacement(psi1, ng)
    k = 2 * math.pi
    ref = np.stack([A * B * k / 2 * np.sin(k * q[:, 0]) * np.cos(k * q[:, 1]),
                    A * B * k / 2 * np.cos(k * q[:, 0]) * np.sin(k * q[:, 1]), 0 * q[:, 2]], axis=1)
    assert np.abs(psi2 - ref).max() <= 1e-12 * np.abs(ref).max()
    # one plane wave has no second-order displacement
    assert np.abs(ics.lpt2_displacement(_crossed_waves(ng, A, 0.0)[1], ng)).max() <= 1e-18


def test_lpt2_of_a_random_field_is_curl_free():
    ng = 24
    psi1 = ics.zeldovich_displacement(ng, -2.0, 0.25, 9)
    psi2 = ics.lpt2_displacement(psi1, ng)
    assert np.abs(psi2).max() > 0
    f = [np.fft.fftn(psi2[:, d].reshape(ng, ng, ng)) for d in range(3)]
    k = np.fft.fftfreq(ng, d=1.0 / ng)
    KX, KY, KZ = np.meshgrid(k, k, k, indexing="ij")
    curl = [KY * f[2] - KZ * f[1], KZ * f[0] - KX * f[2], KX * f[1] - KY * f[0]]
    scale = np.sqrt(KX ** 2 + KY ** 2 + KZ ** 2) * np.sqrt(sum(np.abs(c) ** 2 for c in f))
    assert max(np.abs(c).max() for c in curl) <= 1e-10 * scale.max()


def test_lpt2_follows_the_dynamics():
    """Sign and the 3/7 of the second-order term, by the oracle's own
    dynamics: crossed waves started from second-order positions and momenta
    at a = 0.5 and stepped to a = 1 (oracle tree forces, KDK) stay on the
    second-order prediction far more closely than on the first-order one
    (the remaining difference is third order, lattice discreteness and the
    integrator's error)."""
    import oracle as O
    ng, A, B = 16, 0.02, 0.013
    q, psi1 = _crossed_waves(ng, A, B)
    psi2 = ics.lpt2_displacement(psi1, ng)
    ai, af, S = 0.5, 1.0, 6
    x, p = ics.lpt2_state(q, psi1, psi2, ai, ai)  # D = a
    op = O.tree_params(1e-4, 0.5, 4, ewald=4, ew_grid=4)
    force = lambda xx: O.tree_forces(xx, None, op)
    g = force(x)
    a_list = [ai * (af / ai) ** (j / S) for j in range(S + 1)]
    for j in range(S):
        x, p, g = O.kdk_step(x, p, g, a_list[j], a_list[j + 1], force)

    def rms_off(pred):
        d = x - np.mod(pred, 1.0)
        d -= np.round(d)
        return math.sqrt(np.mean(np.sum(d * d, axis=1)))

    e1 = rms_off(q + af * psi1)
    e2 = rms_off(q + af * psi1 - 3.0 / 7.0 * af ** 2 * psi2)
    assert e2 <= 0.1 * e1, (e1, e2)
    # the wrong sign of the second-order term does worse than first order
    assert rms_off(q + af * psi1 + 3.0 / 7.0 * af ** 2 * psi2) > e1
