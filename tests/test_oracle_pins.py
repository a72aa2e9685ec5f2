"""Pins of the CPU oracle against things other than itself.

Each test names the passage of Galloway et al. (BeyondPlanck VIII, Sect. 2.1)
it pins and what fixes the expected value: Wigner's explicit formula, the
textbook d^1 / d^2 tables, scipy's spherical harmonics (a library routine),
mpmath's Jacobi polynomials at 50 digits, brute-force quadrature of the
convolution integral (Eq. convolution), closed forms, invariants and the
adjoint identity.
"""
import math

import numpy as np
import pytest

from tests.conftest import rel_l2
import workloads as W

sph_harm_y = pytest.importorskip("scipy.special").sph_harm_y


# --------------------------------------------------------------------------- helpers
def _rand_sky(rng, L, ncomp=1):
    n = W.nalm(L)
    z = rng.standard_normal((ncomp, n)) + 1j * rng.standard_normal((ncomp, n))
    z[:, :L + 1] = z[:, :L + 1].real          # m = 0 block is real
    return z


def _rand_beam(rng, L, K, ncomp=1):
    b = rng.standard_normal((ncomp, K + 1, L + 1)) + 1j * rng.standard_normal((ncomp, K + 1, L + 1))
    b[:, 0] = b[:, 0].real
    for k in range(K + 1):
        b[:, k, :k] = 0
    return b


def _ext(arr, L, l, m, packed_sky=True, K=None):
    """Real-field extension for negative m (sky) or k (beam)."""
    am = abs(m)
    if packed_sky:
        v = arr[am * (2 * L + 1 - am) // 2 + l]
    else:
        if am > K:
            return 0.0
        v = arr[am, l]
    if am == 0:
        return v.real
    return v if m > 0 else (-1) ** am * np.conj(v)


def _field(coef, L, th, ph):
    v = np.zeros(np.shape(th), complex)
    for l in range(L + 1):
        for m in range(-l, l + 1):
            c = coef(l, m)
            if c != 0:
                v = v + c * sph_harm_y(l, m, th, ph)
    return v


def _Rz(a):
    return np.array([[math.cos(a), -math.sin(a), 0], [math.sin(a), math.cos(a), 0], [0, 0, 1.0]])


def _Ry(b):
    return np.array([[math.cos(b), 0, math.sin(b)], [0, 1.0, 0], [-math.sin(b), 0, math.cos(b)]])


def _quadrature_grid(L):
    x, w = np.polynomial.legendre.leggauss(L + 2)
    nph = 2 * L + 2
    tq = np.arccos(x)
    pq = 2 * np.pi * np.arange(nph) / nph
    T, P = np.meshgrid(tq, pq, indexing="ij")
    Wt = np.repeat(w[:, None], nph, 1) * 2 * np.pi / nph
    n = np.stack([np.sin(T) * np.cos(P), np.sin(T) * np.sin(P), np.cos(T)], -1)
    return T, P, Wt, n


def _conv_quadrature(sky, beam, L, K, th, ph, ps):
    """Eq. convolution by exact quadrature: c = int s(n) b(R^-1 n) dOmega with
    R = Rz(phi) Ry(theta) Rz(psi).  No Wigner function is involved."""
    T, P, Wt, n = _quadrature_grid(L)
    out = 0.0
    for X in range(sky.shape[0]):
        s = _field(lambda l, m: _ext(sky[X], L, l, m), L, T, P)
        R = _Rz(ph) @ _Ry(th) @ _Rz(ps)
        n2 = n @ R                               # R^T n for every node
        t2 = np.arccos(np.clip(n2[..., 2], -1, 1))
        p2 = np.arctan2(n2[..., 1], n2[..., 0])
        b = _field(lambda l, k: _ext(beam[X], L, l, k, packed_sky=False, K=K), L, t2, p2)
        out += np.sum(Wt * s * b)
    return out


# --------------------------------------------------------------------------- Wigner d
def test_recurrence_matches_wigner_explicit_sum(oracle_lib):
    """Seeds + three-term recurrence vs Wigner's explicit sum, l <= 16."""
    worst = 0.0
    for l in range(0, 17):
        for m in range(-l, l + 1):
            for k in range(-l, l + 1):
                for b in (0.0, 0.31, 1.7, math.pi - 1e-3, math.pi):
                    e = oracle_lib.wigner_d_explicit(l, m, k, b)
                    s = oracle_lib.wigner_d_seq(l, m, k, b)[l]
                    worst = max(worst, abs(e - s))
    assert worst < 1e-13


def test_spin0_column_matches_scipy_harmonics(oracle_lib):
    """Sect. 2.1 (k = 0 is a spin-0 transform): d^l_{m0}(t) = sqrt(4 pi/(2l+1)) Y_lm(t, 0)
    with scipy's Condon-Shortley Y_lm."""
    for m in (0, 1, 5, 40, 199):
        for t in (0.05, 0.9, 1.9, 3.0):
            d = oracle_lib.wigner_d_seq(200, m, 0, t)
            ls = np.arange(max(m, 0), 201)
            y = np.sqrt(4 * np.pi / (2 * ls + 1)) * sph_harm_y(ls, m, t, 0.0).real
            np.testing.assert_allclose(d[ls], y, rtol=1e-11, atol=1e-13)


def test_textbook_d1_d2_tables(oracle_lib):
    """Closed forms of d^1 and d^2 (standard tables)."""
    for b in (0.2, 1.0, 2.4):
        c, s = math.cos(b), math.sin(b)
        table = {
            (1, 1, 1): (1 + c) / 2, (1, 1, 0): -s / math.sqrt(2), (1, 1, -1): (1 - c) / 2,
            (1, 0, 0): c, (1, 0, 1): s / math.sqrt(2), (1, 0, -1): -s / math.sqrt(2),
            (2, 2, 2): ((1 + c) / 2) ** 2, (2, 2, 1): -(1 + c) * s / 2,
            (2, 2, 0): math.sqrt(3.0 / 8.0) * s * s, (2, 2, -1): -(1 - c) * s / 2,
            (2, 2, -2): ((1 - c) / 2) ** 2, (2, 1, 1): (1 + c) * (2 * c - 1) / 2,
            (2, 1, 0): -math.sqrt(1.5) * s * c, (2, 1, -1): (1 - c) * (2 * c + 1) / 2,
            (2, 0, 0): (3 * c * c - 1) / 2,
        }
        for (l, m, k), v in table.items():
            assert abs(oracle_lib.wigner_d_seq(l, m, k, b)[l] - v) < 1e-14, (l, m, k, b)


def _d_mpmath(l, m, k, beta):
    """d^l_{mk} at 50 digits through the Jacobi-polynomial form (m >= |k|):
    (-1)^{m-k} sqrt((l+m)!(l-m)!/((l+k)!(l-k)!)) sin(b/2)^{m-k} cos(b/2)^{m+k}
    P^{(m-k,m+k)}_{l-m}(cos b)."""
    import mpmath as mp
    mp.mp.dps = 50
    b = mp.mpf(beta)
    pref = mp.sqrt(mp.factorial(l + m) * mp.factorial(l - m) /
                   (mp.factorial(l + k) * mp.factorial(l - k)))
    sgn = -1 if (m - k) % 2 else 1
    return sgn * pref * mp.sin(b / 2) ** (m - k) * mp.cos(b / 2) ** (m + k) * \
        mp.jacobi(l - m, m - k, m + k, mp.cos(b))


@pytest.mark.parametrize("m,k", [(0, 0), (3, 2), (16, -16), (200, 16), (700, -5)])
def test_high_l_recurrence_vs_mpmath(oracle_lib, m, k):
    """Scaled recurrence at l ~ 1000, including polar rings where the seed is far
    below double range, against 50-digit Jacobi polynomials.  Tolerance: rounding
    x = cos(beta) to double moves beta by ~eps/sin(beta), which moves d^l by about
    l times that; near the pole this input conditioning dominates."""
    lmax = 1024
    for beta in (math.pi / 2048, 0.37, 1.5707, 2.9):
        d = oracle_lib.wigner_d_seq(lmax, m, k, beta)
        for l in (m + 1, 512, 900, 1024):
            if l < max(abs(m), abs(k)):
                continue
            ref = float(_d_mpmath(l, m, k, beta))
            tol = 2e-15 + l * 2.0 ** -53 / math.sin(beta)
            assert abs(d[l] - ref) <= tol, (l, m, k, beta, d[l], ref)


def test_unitarity_rows(oracle_lib):
    """sum_k (d^l_{mk})^2 = 1 (d^l is orthogonal), at l = 300 near a pole and at the equator."""
    l = 300
    for beta in (math.pi / 1024, 1.2):
        for m in (0, 17, 250):
            tot = sum(oracle_lib.wigner_d_seq(l, m, k, beta)[l] ** 2 for k in range(-l, l + 1))
            assert abs(tot - 1.0) < 1e-11


# --------------------------------------------------------------------------- convolution
@pytest.mark.parametrize("ncomp", [1, 3])
def test_exact_sum_equals_quadrature_of_convolution_integral(oracle_lib, ncomp):
    """Eq. totalconvolver (Wigner-D sum) == Eq. convolution (direct integral with the
    beam rotated by R = Rz(phi) Ry(theta) Rz(psi)); fixes every sign and the meaning
    of psi."""
    rng = np.random.default_rng(11)
    L, K = 5, 3
    sky = _rand_sky(rng, L, ncomp)
    beam = _rand_beam(rng, L, K, ncomp)
    pts = [(0.7, 1.3, 2.1), (2.5, 5.0, 0.4), (0.0, 1.0, 0.5), (math.pi, 0.3, 4.0), (1.9, 6.1, 3.3)]
    th, ph, ps = (np.array(v) for v in zip(*pts))
    re, im = oracle_lib.conv_exact(sky, beam, th, ph, ps, return_imag=True)
    for i, p in enumerate(pts):
        q = _conv_quadrature(sky, beam, L, K, *p)
        assert abs(re[i] - q.real) < 1e-11 * max(1, abs(q))
        assert abs(q.imag) < 1e-11
    assert np.max(np.abs(im)) < 1e-12          # F_{-k} = conj(F_k): the sum is real


def test_axisymmetric_beam_is_spin0_synthesis(oracle_lib):
    """Sect. 2.1: with b_lk = 0 for k > 0 the convolution is psi-independent and is
    the spin-0 synthesis of sqrt(4 pi/(2l+1)) s_lm b_l0 (scipy Y_lm)."""
    rng = np.random.default_rng(3)
    L, K = 12, 3
    sky = _rand_sky(rng, L)
    beam = _rand_beam(rng, L, K)
    beam[:, 1:] = 0
    th = rng.uniform(0, np.pi, 6)
    ph = rng.uniform(0, 2 * np.pi, 6)
    c1 = oracle_lib.conv_exact(sky, beam, th, ph, np.zeros(6))
    c2 = oracle_lib.conv_exact(sky, beam, th, ph, rng.uniform(0, 2 * np.pi, 6))
    ref = _field(lambda l, m: math.sqrt(4 * math.pi / (2 * l + 1)) * _ext(sky[0], L, l, m) *
                 beam[0, 0, l].real, L, th, ph).real
    np.testing.assert_allclose(c1, ref, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(c2, ref, rtol=1e-12, atol=1e-12)


def test_single_alm_closed_forms(oracle_lib):
    """Dipole sky s_10 = 1: c = b_10 cos(t) + sqrt(2) sin(t) Re(conj(b_11) e^{i psi});
    quadrupole s_21 (+ its partner s_{2,-1}) from the d^2 table."""
    rng = np.random.default_rng(4)
    L, K = 2, 2
    beam = _rand_beam(rng, L, K)
    th, ph, ps = rng.uniform(0, np.pi, 5), rng.uniform(0, 2 * np.pi, 5), rng.uniform(0, 2 * np.pi, 5)
    sky = np.zeros((1, W.nalm(L)), complex)
    sky[0, W.alm_index(L, 1, 0)] = 1.0
    c = oracle_lib.conv_exact(sky, beam, th, ph, ps)
    b10, b11 = beam[0, 0, 1].real, beam[0, 1, 1]
    ref = b10 * np.cos(th) + math.sqrt(2) * np.sin(th) * (np.conj(b11) * np.exp(1j * ps)).real
    np.testing.assert_allclose(c, ref, rtol=1e-13, atol=1e-14)

    s21 = 0.3 - 0.8j
    sky = np.zeros((1, W.nalm(L)), complex)
    sky[0, W.alm_index(L, 2, 1)] = s21
    c = oracle_lib.conv_exact(sky, beam, th, ph, ps)

    def d2(m, k, b):
        """d^2_{1,k} from the standard table (only m = 1 is needed)."""
        assert m == 1
        cb, sb = np.cos(b), np.sin(b)
        t = {2: (1 + cb) * sb / 2, 1: (1 + cb) * (2 * cb - 1) / 2, 0: -np.sqrt(1.5) * sb * cb,
             -1: (1 - cb) * (2 * cb + 1) / 2, -2: -(1 - cb) * sb / 2}
        return t[k]

    ref = np.zeros(5, complex)
    for k in range(-2, 3):
        bk = _ext(beam[0], L, 2, k, packed_sky=False, K=K)
        # d^2_{-1,k} = d^2_{-k,1} = (-1)^{1+k} d^2_{1,-k}
        dm1 = (-1) ** (1 + k) * d2(1, -k, th)
        ref += np.conj(bk) * (s21 * d2(1, k, th) * np.exp(1j * ph) +
                              (-np.conj(s21)) * dm1 * np.exp(-1j * ph)) * np.exp(1j * k * ps)
    np.testing.assert_allclose(c, ref.real, rtol=1e-12, atol=1e-13)
    assert np.max(np.abs(ref.imag)) < 1e-12


def test_rotation_invariance(oracle_lib):
    """Rotating the sky by Q and the pointing by Q leaves c unchanged.
    (a) Q = Rz(alpha): s'_lm = e^{-im alpha} s_lm, phi -> phi + alpha (exact);
    (b) a general Q: s' obtained by quadrature projection of s(Q^-1 n) on scipy Y_lm;
        c'(R) must equal c(Q^-1 R)."""
    rng = np.random.default_rng(5)
    L, K = 6, 2
    sky = _rand_sky(rng, L)
    beam = _rand_beam(rng, L, K)
    th, ph, ps = rng.uniform(0.1, 3.0, 4), rng.uniform(0, 6.2, 4), rng.uniform(0, 6.2, 4)
    a = 0.77
    l_of, m_of = np.zeros(W.nalm(L), int), np.zeros(W.nalm(L), int)
    for m in range(L + 1):
        for l in range(m, L + 1):
            l_of[W.alm_index(L, l, m)], m_of[W.alm_index(L, l, m)] = l, m
    sky_r = sky * np.exp(-1j * m_of * a)[None]
    np.testing.assert_allclose(oracle_lib.conv_exact(sky_r, beam, th, ph + a, ps),
                               oracle_lib.conv_exact(sky, beam, th, ph, ps), rtol=1e-12, atol=1e-12)

    Q = _Rz(0.4) @ _Ry(1.1) @ _Rz(-0.9)
    T, P, Wt, n = _quadrature_grid(L)
    n_src = n @ Q                                   # Q^-1 n
    s_rot = _field(lambda l, m: _ext(sky[0], L, l, m), L,
                   np.arccos(np.clip(n_src[..., 2], -1, 1)), np.arctan2(n_src[..., 1], n_src[..., 0]))
    sky_q = np.zeros_like(sky)
    for m in range(L + 1):
        for l in range(m, L + 1):
            sky_q[0, W.alm_index(L, l, m)] = np.sum(Wt * s_rot * np.conj(sph_harm_y(l, m, T, P)))
    for i in range(4):
        Rm = _Rz(ph[i]) @ _Ry(th[i]) @ _Rz(ps[i])
        M = Q.T @ Rm
        t2 = math.acos(max(-1.0, min(1.0, M[2, 2])))
        p2 = math.atan2(M[1, 2], M[0, 2])
        s2 = math.atan2(M[2, 1], -M[2, 0])
        a1 = oracle_lib.conv_exact(sky_q, beam, [th[i]], [ph[i]], [ps[i]])[0]
        a2 = oracle_lib.conv_exact(sky, beam, [t2], [p2], [s2])[0]
        assert abs(a1 - a2) < 1e-10 * max(1, abs(a2))


def test_pole_depends_only_on_phi_plus_psi(oracle_lib):
    """At theta = 0 the rotation is Rz(phi + psi): c(0, phi, psi) = c(0, phi + a, psi - a)."""
    rng = np.random.default_rng(6)
    L, K = 8, 3
    sky, beam = _rand_sky(rng, L), _rand_beam(rng, L, K)
    ph, ps = rng.uniform(0, 6, 5), rng.uniform(0, 6, 5)
    c1 = oracle_lib.conv_exact(sky, beam, np.zeros(5), ph, ps)
    c2 = oracle_lib.conv_exact(sky, beam, np.zeros(5), ph + 1.3, ps - 1.3)
    np.testing.assert_allclose(c1, c2, rtol=1e-12, atol=1e-12)


def test_polarised_is_sum_of_scalar_convolutions_parity_unpinned(oracle_lib):
    """Polarised reading: T/E/B total = sum of three scalar convolutions (linear identity).

    PARITY UNPINNED: the paper shows T/Q/U sidelobe maps but states no polarised
    formula, so nothing outside this code fixes the T/E/B sum; this test checks
    only that the oracle's component sum is the sum of its (pinned) scalar
    convolutions."""
    rng = np.random.default_rng(7)
    L, K = 8, 3
    sky, beam = _rand_sky(rng, L, 3), _rand_beam(rng, L, K, 3)
    th, ph, ps = rng.uniform(0, 3, 7), rng.uniform(0, 6, 7), rng.uniform(0, 6, 7)
    tot = oracle_lib.conv_exact(sky, beam, th, ph, ps)
    parts = sum(oracle_lib.conv_exact(sky[X:X + 1], beam[X:X + 1], th, ph, ps) for X in range(3))
    np.testing.assert_allclose(tot, parts, rtol=1e-13, atol=1e-13)


# --------------------------------------------------------------------------- cube
@pytest.mark.parametrize("nphi", [24, 16, 8])
def test_cube_nodes_are_psi_fourier_coefficients(oracle_lib, nphi):
    """Step 1 of the two-step algorithm: the cube at a node equals the k-th Fourier
    coefficient in psi of the exact convolution there (nphi = 16 < 2L+1 also checks
    that folding m mod nphi is exact at the nodes; nphi = 8 <= L, that several
    aliases of one bin add up)."""
    rng = np.random.default_rng(8)
    L, K, R = 10, 3, 8
    sky, beam = _rand_sky(rng, L, 2), _rand_beam(rng, L, K, 2)
    rt = W.equiangular_ring_theta(R)
    cube = oracle_lib.cube(sky, beam, rt, nphi)
    npsi = 2 * K + 2
    psis = 2 * np.pi * np.arange(npsi) / npsi
    T = np.repeat(rt, nphi * npsi)
    P = np.tile(np.repeat(2 * np.pi * np.arange(nphi) / nphi, npsi), R)
    S = np.tile(psis, R * nphi)
    c = oracle_lib.conv_exact(sky, beam, T, P, S).reshape(R, nphi, npsi)
    for k in range(K + 1):
        Fk = np.mean(c * np.exp(-1j * k * psis)[None, None, :], axis=2)
        np.testing.assert_allclose(cube[:, :, k], Fk, rtol=0, atol=1e-11 * np.abs(c).max())


def test_cube_conjugate_pairs(oracle_lib):
    """Conjugate pairs (Sect. 2.1): with k = 0 the cube is real (spin-0 real map)."""
    rng = np.random.default_rng(9)
    L, K = 9, 2
    sky, beam = _rand_sky(rng, L), _rand_beam(rng, L, K)
    cube = oracle_lib.cube(sky, beam, W.healpix_ring_theta(4), 16)
    assert np.max(np.abs(cube[:, :, 0].imag)) < 1e-12 * np.max(np.abs(cube))


# --------------------------------------------------------------------------- interpolation
def _ring_list(rng, R):
    """A non-uniform, north/south-symmetric ring list in (0, pi)."""
    rt = np.sort(rng.uniform(0.05, np.pi / 2 - 0.02, R // 2))
    return np.concatenate([rt, (np.pi - rt)[::-1]])


@pytest.mark.parametrize("p", [2, 4, 6])
def test_lagrange_exact_on_polynomials_away_from_poles(oracle_lib, p):
    """Interpolation reading: p-point Lagrange reproduces data that are polynomials
    of degree p - 1 in theta and in the phi index, on a non-uniform ring list, for
    stencils without ghost rows."""
    rng = np.random.default_rng(10 + p)
    R, nphi, K = 40, 64, 3
    rt = _ring_list(rng, R)
    ca = rng.standard_normal((K + 1, p)) + 1j * rng.standard_normal((K + 1, p))
    cb = rng.standard_normal((K + 1, p)) + 1j * rng.standard_normal((K + 1, p))
    u = np.arange(nphi, dtype=float)
    cube = np.zeros((R, nphi, K + 1), complex)
    for k in range(K + 1):
        Pt = np.polyval(ca[k], rt)
        Qu = np.polyval(cb[k], (u - 30.0) / 10.0)
        cube[:, :, k] = Pt[:, None] * Qu[None, :]
    n = 300
    h = p // 2
    th = rng.uniform(rt[h], rt[-h - 1], n)
    uu = rng.uniform(h, nphi - h - 1, n)
    ph = uu * 2 * np.pi / nphi
    ps = rng.uniform(0, 2 * np.pi, n)
    got = oracle_lib.interp(cube, rt, th, ph, ps, p=p)
    ref = np.zeros(n)
    for k in range(K + 1):
        v = np.polyval(ca[k], th) * np.polyval(cb[k], (uu - 30.0) / 10.0)
        ref += (1 if k == 0 else 2) * (v * np.exp(1j * k * ps)).real
    np.testing.assert_allclose(got, ref, rtol=1e-10, atol=1e-10)


@pytest.mark.parametrize("p", [2, 4, 6])
def test_stencil_is_the_p_nearest_nodes_with_ghost_rows(oracle_lib, p):
    """Interpolation reading, pinned node by node: a sample reads exactly the p rows
    and p columns nearest to it (rows i - p/2 + 1 ... i + p/2 around the last ring
    at or above it, p/2 ghost rows deep past either pole) and is exact on data that
    are polynomials of degree p - 1 there.  For each sample a cube is built that
    holds the polynomial only on those p x p nodes and large random values on every
    other node, so reading any other node, a ghost row without the shift of phi by
    pi, without the (-1)^k sign, or at the wrong colatitude (-theta_i north,
    2 pi - theta_i south) breaks the equality."""
    rng = np.random.default_rng(20 + p)
    R, nphi, K = 24, 32, 3
    rt = _ring_list(rng, R)
    h = p // 2
    # extended colatitudes of rows -h .. R-1+h (the ghost rule's colatitudes)
    rows = np.arange(-h, R + h)
    ext = np.where(rows < 0, -rt[np.clip(-1 - rows, 0, R - 1)],
                   np.where(rows >= R, 2 * np.pi - rt[np.clip(2 * R - 1 - rows, 0, R - 1)],
                            rt[np.clip(rows, 0, R - 1)]))
    th = np.concatenate([rng.uniform(0, rt[h], 14), rng.uniform(rt[-h - 1], np.pi, 14),
                         rng.uniform(rt[h], rt[-h - 1], 12), [0.0, np.pi, rt[0], rt[-1]]])
    n = th.size
    uu = np.concatenate([rng.uniform(0, nphi, n - 4), [0.0, nphi - 1e-9, 0.5, nphi - 0.5]])
    ph = uu * 2 * np.pi / nphi
    ps = rng.uniform(0, 2 * np.pi, n)
    for s in range(n):
        i = R - 1 if th[s] >= rt[-1] else (-1 if th[s] < rt[0] else int(np.searchsorted(rt, th[s], "right") - 1))
        j = int(np.floor(uu[s]))
        ca = rng.standard_normal((K + 1, p)) + 1j * rng.standard_normal((K + 1, p))
        cb = rng.standard_normal((K + 1, p)) + 1j * rng.standard_normal((K + 1, p))
        cube = 1e3 * (rng.standard_normal((R, nphi, K + 1)) + 1j * rng.standard_normal((R, nphi, K + 1)))
        for a in range(p):
            row = i - h + 1 + a
            tha = ext[row + h]
            for b in range(p):
                col = j - h + 1 + b                     # unwrapped phi index
                for k in range(K + 1):
                    f = np.polyval(ca[k], tha) * np.polyval(cb[k], (col - uu[s]) / 3.0)
                    if 0 <= row < R:
                        cube[row, col % nphi, k] = f
                    else:                               # ghost: (-1)^k F_k(ring, phi + pi)
                        ring = -1 - row if row < 0 else 2 * R - 1 - row
                        cube[ring, (col + nphi // 2) % nphi, k] = (-1) ** k * f
        got = oracle_lib.interp(cube, rt, th[s:s + 1], ph[s:s + 1], ps[s:s + 1], p=p)[0]
        ref = sum((1 if k == 0 else 2) * (np.polyval(ca[k], th[s]) * np.polyval(cb[k], 0.0)
                                          * np.exp(1j * k * ps[s])).real for k in range(K + 1))
        assert abs(got - ref) < 1e-9 * max(1.0, abs(ref)), (p, s, th[s], uu[s], got, ref)


@pytest.mark.parametrize("p", [2, 4, 6])
def test_interpolation_converges_at_order_p_including_poles(oracle_lib, p):
    """Ghost-row reading at the poles: the interpolated TOD converges to the exact
    sum as h^p, also for samples within three ring spacings of each pole (a wrong
    ghost rule leaves an O(1) polar error that does not shrink)."""
    rng = np.random.default_rng(12)
    L, K = 6, 2
    sky, beam = _rand_sky(rng, L), _rand_beam(rng, L, K)
    errs = []
    for R in (32, 64, 128):
        rt = W.equiangular_ring_theta(R)
        h = np.pi / R
        th = np.concatenate([rng.uniform(0, 3 * h, 30), rng.uniform(np.pi - 3 * h, np.pi, 30),
                             np.arccos(rng.uniform(-1, 1, 60))])
        ph, ps = rng.uniform(0, 2 * np.pi, 120), rng.uniform(0, 2 * np.pi, 120)
        cube = oracle_lib.cube(sky, beam, rt, 2 * R)
        got = oracle_lib.interp(cube, rt, th, ph, ps, p=p)
        ex = oracle_lib.conv_exact(sky, beam, th, ph, ps)
        errs.append(np.max(np.abs(got - ex)) / np.max(np.abs(ex)))
    assert errs[0] < {2: 3e-2, 4: 1e-3, 6: 1e-4}[p], errs
    # halving h divides the error by about 2^p (at least 0.6 of it)
    assert errs[0] / errs[1] > 0.6 * 2 ** p and errs[1] / errs[2] > 0.6 * 2 ** p, errs


# --------------------------------------------------------------------------- adjoint
def _dot_c(a, b):
    return float(np.real(np.vdot(b.ravel(), a.ravel())))   # Re sum a conj(b)


def test_adjoint_dot_products(oracle_lib):
    """<Ax, y> = <x, A^T y> for each transposed step and for the whole chain."""
    rng = np.random.default_rng(13)
    L, K, R, nphi, n = 7, 3, 10, 14, 400
    rt = W.equiangular_ring_theta(R)
    th, ph, ps = np.arccos(rng.uniform(-1, 1, n)), rng.uniform(0, 6.3, n), rng.uniform(0, 6.3, n)
    # interpolation
    F = rng.standard_normal((R, nphi, K + 1)) + 1j * rng.standard_normal((R, nphi, K + 1))
    y = rng.standard_normal(n)
    for p in (2, 4, 6):
        lhs = np.dot(oracle_lib.interp(F, rt, th, ph, ps, p=p), y)
        rhs = _dot_c(F, oracle_lib.interp_adjoint(y, rt, nphi, K, th, ph, ps, p=p))
        assert abs(lhs - rhs) < 1e-12 * abs(lhs), p
    # synthesis along phi
    G = rng.standard_normal((K + 1, R, 2 * L + 1)) + 1j * rng.standard_normal((K + 1, R, 2 * L + 1))
    lhs = _dot_c(oracle_lib.cube_from_G(G, nphi), F)
    rhs = _dot_c(G, oracle_lib.cube_from_G_adjoint(F, L))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    # contraction over l, as a linear map of A (A built from sky x beam)
    sky, beam = _rand_sky(rng, L, 1), _rand_beam(rng, L, K, 1)
    Gf = oracle_lib.cube_G(sky, beam, rt)
    Ab = oracle_lib.cube_G_adjoint(G, rt)
    A = np.zeros((K + 1, 2 * L + 1, L + 1), complex)
    for k in range(K + 1):
        for m in range(-L, L + 1):
            for l in range(max(abs(m), k), L + 1):
                A[k, m + L, l] = _ext(sky[0], L, l, m) * np.conj(_ext(beam[0], L, l, k, False, K))
    lhs = _dot_c(Gf, G)
    rhs = _dot_c(A, Ab)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


@pytest.mark.parametrize("ncomp", [1, 3])
def test_gradients_by_central_differences(oracle_lib, ncomp):
    """Gradients of 0.5 |tod(s, b) - d|^2: the loss is quadratic in each real parameter,
    so central differences are exact up to roundoff; 16 sky and 16 beam entries."""
    rng = np.random.default_rng(14 + ncomp)
    L, K, nphi, n = 6, 2, 14, 300
    rt = W.equiangular_ring_theta(12)
    sky, beam = _rand_sky(rng, L, ncomp), _rand_beam(rng, L, K, ncomp)
    th, ph, ps = np.arccos(rng.uniform(-1, 1, n)), rng.uniform(0, 6.3, n), rng.uniform(0, 6.3, n)
    data = rng.standard_normal(n)

    def loss(s, b):
        t = oracle_lib.tod(s, b, rt, nphi, th, ph, ps)
        return 0.5 * np.sum((t - data) ** 2)

    res = oracle_lib.tod(sky, beam, rt, nphi, th, ph, ps) - data
    gs, gb = oracle_lib.adjoint_tod(res, sky, beam, rt, nphi, th, ph, ps)
    h = 1e-3
    for _ in range(16):
        X = rng.integers(ncomp)
        i = rng.integers(W.nalm(L))
        part = 1j if (i > L and rng.random() < 0.5) else 1.0
        sp, sm = sky.copy(), sky.copy()
        sp[X, i] += h * part
        sm[X, i] -= h * part
        fd = (loss(sp, beam) - loss(sm, beam)) / (2 * h)
        an = gs[X, i].imag if part == 1j else gs[X, i].real
        assert abs(fd - an) < 1e-7 * max(1, abs(an)), (X, i, part, fd, an)
    for _ in range(16):
        X = rng.integers(ncomp)
        k = rng.integers(K + 1)
        l = rng.integers(k, L + 1)
        part = 1j if (k > 0 and rng.random() < 0.5) else 1.0
        bp, bm = beam.copy(), beam.copy()
        bp[X, k, l] += h * part
        bm[X, k, l] -= h * part
        fd = (loss(sky, bp) - loss(sky, bm)) / (2 * h)
        an = gb[X, k, l].imag if part == 1j else gb[X, k, l].real
        assert abs(fd - an) < 1e-7 * max(1, abs(an)), (X, k, l, part, fd, an)


def test_golden_regression_fixture(oracle_lib):
    """Regression fixture written by tests/golden/make_golden.py (oracle only)."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "tiny_tod.txt")
    data = np.loadtxt(path)
    g = __import__("tests.golden.make_golden", fromlist=["case"]).case()
    tod = oracle_lib.tod(g["sky"], g["beam"], g["ring_theta"], g["nphi"], g["theta"], g["phi"], g["psi"])
    np.testing.assert_allclose(tod, data, rtol=1e-12, atol=1e-13)
