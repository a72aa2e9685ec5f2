"""Pins of the orbital-dipole oracle (Sect. 3.3: Eqs. dipole, dipole_fast and the
subsampled rotation with a spline in between) against things other than itself:
quadrature with scipy's spherical harmonics, the Sect. 2.1 convolution oracle on
the dipole sky, scipy's natural cubic spline, and closed-form special cases."""
import math

import numpy as np
import pytest

import oracle
from oracle import orbital as orb

sp = pytest.importorskip("scipy.special")


def _ylm(l, m, theta, phi):
    return sp.sph_harm_y(l, m, theta, phi)   # Condon-Shortley phase, theta polar


def _random_beam(L, K, seed):
    rng = np.random.default_rng(seed)
    b = (rng.standard_normal((K + 1, L + 1)) + 1j * rng.standard_normal((K + 1, L + 1)))
    for k in range(K + 1):
        b[k, :k] = 0.0
    b[0].imag = 0.0
    return b


def _quad_grid(nth=16, nph=32):
    x, w = np.polynomial.legendre.leggauss(nth)
    th = np.arccos(x)
    ph = 2 * np.pi * np.arange(nph) / nph
    TH, PH = np.meshgrid(th, ph, indexing="ij")
    W = np.outer(w, np.full(nph, 2 * np.pi / nph))
    return TH, PH, W


def _beam_on_grid(b, TH, PH):
    K1, L1 = b.shape
    B = np.zeros(TH.shape, dtype=np.complex128)
    for l in range(L1):
        for k in range(min(l, K1 - 1) + 1):
            B += b[k, l] * _ylm(l, k, TH, PH)
            if k > 0:
                B += (-1) ** k * np.conj(b[k, l]) * _ylm(l, -k, TH, PH)
    assert np.max(np.abs(B.imag)) < 1e-12
    return B.real


def test_moments_equal_quadrature_of_beam():
    """S_v = int v B dOmega by exact quadrature (degree <= 6 integrand)."""
    b = _random_beam(4, 4, seed=11)
    TH, PH, W = _quad_grid()
    B = _beam_on_grid(b, TH, PH)
    x, y, z = np.sin(TH) * np.cos(PH), np.sin(TH) * np.sin(PH), np.cos(TH)
    want = [np.sum(W * v * B) for v in (x, y, z, x * x, y * y, z * z, x * y, x * z, y * z)]
    got = orb.moments(b)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12 * np.max(np.abs(want)))


def test_moments_ignore_beam_above_l2_and_handle_small_kmax():
    b = _random_beam(6, 5, seed=3)
    S_full = orb.moments(b)
    S_trunc = orb.moments(b[:3, :3])
    np.testing.assert_array_equal(S_full, S_trunc)
    # kmax = 0: only the axisymmetric part
    S0 = orb.moments(b[:1])
    assert S0[0] == S0[1] == S0[6] == S0[7] == S0[8] == 0.0
    assert S0[3] == S0[4]


def _dipole_sky_alm(L, T0, q, beta):
    """a_lm (m >= 0, m-major packing) of D(n) = T0 [beta.n + q (beta.n)^2] by quadrature."""
    TH, PH, W = _quad_grid()
    n = np.stack([np.sin(TH) * np.cos(PH), np.sin(TH) * np.sin(PH), np.cos(TH)], -1)
    bn = n @ np.asarray(beta)
    D = T0 * (bn + q * bn * bn)
    alm = np.zeros((L + 1) * (L + 2) // 2, dtype=np.complex128)
    for m in range(L + 1):
        for l in range(m, L + 1):
            alm[m * (2 * L + 1 - m) // 2 + l] = np.sum(W * D * np.conj(_ylm(l, m, TH, PH)))
    return alm


def test_dipole_equals_convolution_of_dipole_sky():
    """Eq. dipole is Eq. convolution with the sky D(n): the rotation convention and the
    moments must agree with the (quadrature-pinned) total-convolution oracle."""
    L = K = 4
    T0, q = 2.7255, 1.25
    beta = np.array([0.3, -0.5, 0.8])
    b = _random_beam(L, K, seed=5)
    sky = _dipole_sky_alm(L, T0, q, beta)
    rng = np.random.default_rng(2)
    n = 64
    th = np.arccos(rng.uniform(-1, 1, n))
    ph = rng.uniform(0, 2 * np.pi, n)
    ps = rng.uniform(0, 2 * np.pi, n)
    want = oracle.conv_exact(sky[None], b[None], th, ph, ps)
    got = orb.dipole_exact(orb.moments(b), T0, q, th, ph, ps, np.broadcast_to(beta, (n, 3)))
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-11 * np.max(np.abs(want)))


def test_isotropic_and_boresight_dipole_beams():
    """b_00 only: the response is T0 q |beta|^2 b_00 sqrt(4 pi)/3 at every pointing;
    b_10 only: T0 sqrt(4 pi/3) b_10 (beta . boresight)."""
    rng = np.random.default_rng(7)
    n = 50
    th = np.arccos(rng.uniform(-1, 1, n))
    ph = rng.uniform(0, 2 * np.pi, n)
    ps = rng.uniform(0, 2 * np.pi, n)
    beta = rng.standard_normal((n, 3)) * 1e-4
    T0, q = 2.7255, 1.7
    b = np.zeros((3, 3), dtype=np.complex128)
    b[0, 0] = 0.9
    got = orb.dipole_exact(orb.moments(b), T0, q, th, ph, ps, beta)
    want = T0 * q * np.sum(beta ** 2, 1) * 0.9 * math.sqrt(4 * math.pi) / 3
    np.testing.assert_allclose(got, want, rtol=1e-13)
    b[:] = 0
    b[0, 1] = 0.6
    got = orb.dipole_exact(orb.moments(b), T0, q, th, ph, ps, beta)
    n0 = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], -1)
    want = T0 * math.sqrt(4 * math.pi / 3) * 0.6 * np.sum(beta * n0, 1)
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-18)


def test_quad_factor_limits():
    T0 = 2.7255
    # a -> 0: q -> 1 + a^2/12
    nu = 1e6
    a = orb.H_PLANCK * nu / (orb.K_BOLTZMANN * T0)
    assert abs(orb.quad_factor(nu, T0) - (1 + a * a / 12)) < 1e-12
    # large a: q -> a/2
    nu = 5e12
    a = orb.H_PLANCK * nu / (orb.K_BOLTZMANN * T0)
    assert abs(orb.quad_factor(nu, T0) / (a / 2) - 1) < 1e-12


def test_natural_spline_matches_scipy():
    interp = pytest.importorskip("scipy.interpolate")
    rng = np.random.default_rng(4)
    for n in (2, 3, 4, 17, 200):
        y = rng.standard_normal(n)
        h = 20.0
        M = orb.natural_spline_second_derivs(y, h)
        t = np.sort(rng.uniform(0, h * (n - 1), 300))
        t = np.concatenate([t, h * np.arange(n)])
        want = interp.CubicSpline(h * np.arange(n), y, bc_type="natural")(t)
        np.testing.assert_allclose(orb.spline_eval(y, M, h, t), want, rtol=0, atol=1e-13 * np.max(np.abs(y)))


def _periods(n, lens):
    starts = np.concatenate([[0], np.cumsum(lens)])
    assert starts[-1] == n
    return starts


def test_subsampled_nodes_remainder_and_accuracy():
    """Exact at the nodes and in each period's remainder; s = 1 is the exact TOD; on a
    smooth scan the spline is close to the exact values."""
    import workloads as W
    lens = [1, 5, 20, 21, 40, 41, 1000, 1957, 4000]
    n = int(sum(lens))
    th, ph, ps = W.pointings_scan(n)
    starts = _periods(n, lens)
    rng = np.random.default_rng(9)
    beta = rng.standard_normal((len(lens), 3)) * 1e-4
    b = _random_beam(4, 4, seed=1)
    S = orb.moments(b)
    T0, q = 2.7255, orb.quad_factor(70e9, 2.7255)
    per_sample = np.repeat(beta, lens, axis=0)
    exact = orb.dipole_exact(S, T0, q, th, ph, ps, per_sample)
    np.testing.assert_array_equal(orb.dipole_subsampled(S, T0, q, th, ph, ps, starts, beta, 1), exact)
    s = 20
    sub = orb.dipole_subsampled(S, T0, q, th, ph, ps, starts, beta, s)
    for p, L_p in enumerate(lens):
        a = starts[p]
        M = orb.nodes_of_period(L_p, s)
        last = s * (M - 1)
        nodes = a + s * np.arange(M)
        np.testing.assert_array_equal(sub[nodes], exact[nodes])
        np.testing.assert_array_equal(sub[a + last + 1:a + L_p], exact[a + last + 1:a + L_p])
    # long periods: away from the period ends the spline through ~100 nodes per spin
    # period is close (~3e-8); the natural end condition costs ~1e-4 over the first and
    # last few nodes (periods with 2-3 nodes are nearly linear, exact at nodes only)
    for p in (6, 7, 8):
        r = slice(starts[p], starts[p + 1])
        err, ref = sub[r] - exact[r], np.max(np.abs(exact[r]))
        assert np.max(np.abs(err[200:-200])) < 1e-6 * ref
        assert np.max(np.abs(err)) < 1e-3 * ref
