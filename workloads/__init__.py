"""Seeded synthetic inputs for the sidelobe convolution: skies, beams, ring
grids and pointings.

This module is shared by the CPU oracle's tests, the GPU parity tests and the
benchmark.  It holds no step of the convolution itself: it only draws random
numbers (numpy PCG64, fixed seeds) and lays them out in the packed formats the
library expects.

Packing (same for every consumer):

* sky ``a_lm``: complex array ``[ncomp, nalm]`` with ``nalm = (L+1)(L+2)/2`` and
  m-major index ``idx(l, m) = m(2L+1-m)/2 + l`` for ``0 <= m <= l <= L``.
  ``Im a_l0`` is zero.  Negative m follow the real-field relation
  ``a_{l,-m} = (-1)^m conj(a_lm)``.
* beam ``b_lk``: complex array ``[ncomp, K+1, L+1]`` (``k = 0..K``), zero for
  ``l < k``; ``Im b_l0`` is zero (real beam, Sect. 2.1 Eq. breal).
* pointings: three float64 arrays ``theta`` (colatitude), ``phi`` (longitude),
  ``psi`` (beam orientation), in radians.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "nalm", "alm_index", "healpix_ring_theta", "equiangular_ring_theta",
    "sky_gaussian", "sky_polarised", "beam_gaussian_taper", "beam_far_sidelobe",
    "pointings_uniform", "pointings_scan", "config_small", "config_lfi", "config_highres",
    "truncate_alm", "rotation_about", "config_detectors",
]


def nalm(lmax: int) -> int:
    return (lmax + 1) * (lmax + 2) // 2


def alm_index(lmax: int, l, m):
    """m-major packed index of (l, m), m >= 0."""
    return m * (2 * lmax + 1 - m) // 2 + l


def _mirror(north: np.ndarray, nrings: int) -> np.ndarray:
    """Complete a north half (plus the equator ring when nrings is odd) with its
    exact mirror ``theta -> pi - theta`` so that the list is N/S symmetric."""
    th = np.empty(nrings, dtype=np.float64)
    h = nrings // 2
    th[:h] = north[:h]
    if nrings % 2:
        th[h] = 0.5 * math.pi
    th[nrings - h:] = (math.pi - north[:h])[::-1]
    return th


def healpix_ring_theta(nside: int) -> np.ndarray:
    """Colatitudes of the 4*nside-1 HEALPix rings (Gorski et al. 2005 ring z
    formula), made exactly N/S symmetric."""
    nr = 4 * nside - 1
    i = np.arange(1, 2 * nside, dtype=np.float64)   # north rings incl. the equator
    z = np.where(i < nside, 1.0 - i * i / (3.0 * nside * nside),
                 4.0 / 3.0 - 2.0 * i / (3.0 * nside))
    return _mirror(np.arccos(z), nr)


def equiangular_ring_theta(nrings: int) -> np.ndarray:
    """theta_r = pi (r + 1/2) / nrings, made exactly N/S symmetric."""
    r = np.arange(nrings, dtype=np.float64)
    return _mirror(math.pi * (r + 0.5) / nrings, nrings)


def _complex_normal(rng: np.random.Generator, shape) -> np.ndarray:
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _packed_lm(lmax: int):
    m = np.concatenate([np.full(lmax + 1 - mm, mm) for mm in range(lmax + 1)])
    l = np.concatenate([np.arange(mm, lmax + 1) for mm in range(lmax + 1)])
    return l, m


def sky_gaussian(lmax: int, cl, seed: int = 0, ncomp_cls=None) -> np.ndarray:
    """Gaussian real-field sky: a_l0 = sqrt(C_l) N(0,1), a_lm = sqrt(C_l/2)(N+iN).

    ``cl`` is a list of per-component spectra (arrays of length lmax+1)."""
    rng = np.random.default_rng(seed)
    l, m = _packed_lm(lmax)
    out = np.zeros((len(cl), nalm(lmax)), dtype=np.complex128)
    for c, spec in enumerate(cl):
        spec = np.asarray(spec, dtype=np.float64)
        z = _complex_normal(rng, nalm(lmax))
        amp = np.sqrt(spec[l] * np.where(m == 0, 1.0, 0.5))
        vals = np.where(m == 0, z.real + 0j, z) * amp
        out[c] = vals
    return out


def sky_polarised(lmax: int, seed: int = 0) -> np.ndarray:
    """T/E/B sky with C^TT_l = (l+1)^-2, EE = 0.05 TT, BB = 0.01 TT (no TE);
    E and B vanish for l < 2."""
    ell = np.arange(lmax + 1, dtype=np.float64)
    tt = (ell + 1.0) ** -2
    pol = np.where(ell >= 2, 1.0, 0.0)
    return sky_gaussian(lmax, [tt, 0.05 * tt * pol, 0.01 * tt * pol], seed)


def _beam_from(lmax: int, kmax: int, ncomp: int, amp_lk, rng) -> np.ndarray:
    out = np.zeros((ncomp, kmax + 1, lmax + 1), dtype=np.complex128)
    ell = np.arange(lmax + 1)
    for c in range(ncomp):
        xi = _complex_normal(rng, (kmax + 1, lmax + 1))
        xi[0] = xi[0].real
        for k in range(kmax + 1):
            row = amp_lk(c, k) * xi[k]
            row[ell < k] = 0.0
            out[c, k] = row
    return out


def beam_gaussian_taper(lmax: int, kmax: int, sigma_l: float = 20.0, seed: int = 1,
                        ncomp: int = 1) -> np.ndarray:
    """b_lk = exp(-l^2 / (2 sigma_l^2)) 0.5^k xi_lk with xi complex normal
    (xi_l0 real normal), zero for l < k."""
    rng = np.random.default_rng(seed)
    ell = np.arange(lmax + 1, dtype=np.float64)
    taper = np.exp(-ell * ell / (2.0 * sigma_l * sigma_l))
    return _beam_from(lmax, kmax, ncomp, lambda c, k: taper * 0.5 ** k, rng)


def beam_far_sidelobe(lmax: int, kmax: int, seed: int = 1,
                      comp_amp=(1.0, 0.1, 0.1)) -> np.ndarray:
    """Polarised far-sidelobe-like beam: b^X_lk = a_X (l+1)^-1.5 xi^X_lk,
    zero for l < k (and for l < 2 in E and B)."""
    rng = np.random.default_rng(seed)
    ell = np.arange(lmax + 1, dtype=np.float64)
    base = (ell + 1.0) ** -1.5
    pol = np.where(ell >= 2, 1.0, 0.0)

    def amp(c, k):
        return comp_amp[c] * base * (pol if c > 0 else 1.0)
    return _beam_from(lmax, kmax, len(comp_amp), amp, rng)


def pointings_uniform(n: int, seed: int = 2):
    """cos(theta) ~ U(-1, 1); phi, psi ~ U[0, 2 pi)."""
    rng = np.random.default_rng(seed)
    ct = rng.uniform(-1.0, 1.0, n)
    phi = rng.uniform(0.0, 2.0 * math.pi, n)
    psi = rng.uniform(0.0, 2.0 * math.pi, n)
    return np.arccos(ct), phi, psi


def pointings_scan(n: int, fsamp: float = 32.5, spin_rpm: float = 1.0,
                   opening_deg: float = 85.0, psi_offset: float = 0.0,
                   t0: float = 0.0, chunk: int = 1 << 22, offset=None):
    """Synthetic satellite scan: spin axis in the ecliptic plane at longitude
    2 pi t / (365.25 d), boresight at ``opening_deg`` from the spin axis,
    spinning at ``spin_rpm``; the beam x-axis points along the scan direction.
    (theta, phi, psi) are the zyz Euler angles of the beam-to-sky rotation
    R = [x_beam, y_beam, boresight].  ``offset`` (a 3x3 rotation) moves the
    detector within the focal plane: R -> R @ offset."""
    th = np.empty(n)
    ph = np.empty(n)
    ps = np.empty(n)
    year = 365.25 * 86400.0
    w = 2.0 * math.pi * spin_rpm / 60.0
    ca, sa = math.cos(math.radians(opening_deg)), math.sin(math.radians(opening_deg))
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        t = t0 + np.arange(s, e, dtype=np.float64) / fsamp
        lam = 2.0 * math.pi * t / year
        cl, sl = np.cos(lam), np.sin(lam)
        cw, sw = np.cos(w * t), np.sin(w * t)
        # spin axis a = (cl, sl, 0); e1 = z; e2 = z x a = (-sl, cl, 0)
        nx = ca * cl + sa * sw * (-sl)
        ny = ca * sl + sa * sw * cl
        nz = sa * cw
        # scan direction x = -sin(wt) e1 + cos(wt) e2
        xx = cw * (-sl)
        xy = cw * cl
        xz = -sw
        # y = n cross x
        yz = nx * xy - ny * xx
        if offset is not None:
            Q = np.asarray(offset, dtype=np.float64)
            yx = ny * xz - nz * xy
            yy = nz * xx - nx * xz
            cols = []
            for j in range(3):     # column j of R @ Q = sum_i R[:, i] Q[i, j]
                cols.append(tuple(Q[0, j] * a + Q[1, j] * b + Q[2, j] * c
                                  for a, b, c in ((xx, yx, nx), (xy, yy, ny), (xz, yz, nz))))
            (xx, xy, xz), (_, _, yz), (nx, ny, nz) = cols
        th[s:e] = np.arccos(np.clip(nz, -1.0, 1.0))
        ph[s:e] = np.mod(np.arctan2(ny, nx), 2.0 * math.pi)
        ps[s:e] = np.mod(np.arctan2(yz, -xz) + psi_offset, 2.0 * math.pi)
    return th, ph, ps


def config_small(n: int = 100_000):
    """Unpolarised small case: lmax=64, kmax=4, Nside=32 HEALPix-like rings with
    128 phi per ring, uniform pointings."""
    lmax, kmax = 64, 4
    ell = np.arange(lmax + 1, dtype=np.float64)
    sky = sky_gaussian(lmax, [(ell + 1.0) ** -2], seed=0)
    beam = beam_gaussian_taper(lmax, kmax, 20.0, seed=1)
    rings = healpix_ring_theta(32)
    th, ph, ps = pointings_uniform(n, seed=2)
    return dict(lmax=lmax, kmax=kmax, sky=sky, beam=beam, ring_theta=rings, nphi=128,
                theta=th, phi=ph, psi=ps)


def config_lfi(n: int = 100_000_000, with_pointings: bool = True):
    """LFI-like scale: polarised T/E/B sky and beam at lmax=1024, kmax=16;
    1024 equiangular rings x 2048 phi; synthetic scan pointings at 32.5 Hz."""
    lmax, kmax = 1024, 16
    d = dict(lmax=lmax, kmax=kmax, sky=sky_polarised(lmax, seed=0),
             beam=beam_far_sidelobe(lmax, kmax, seed=1),
             ring_theta=equiangular_ring_theta(1024), nphi=2048)
    if with_pointings:
        d["theta"], d["phi"], d["psi"] = pointings_scan(n)
    return d


def config_highres(n: int = 200_000_000, with_pointings: bool = True):
    """Precision-variant scale: the small case's generators (unpolarised sky with
    C_l = (l+1)^-2, Gaussian-taper beam with sigma_l = 20 and 0.5^k) at
    lmax=2048, kmax=32; 2048 equiangular rings x 4096 phi; uniform pointings."""
    lmax, kmax = 2048, 32
    ell = np.arange(lmax + 1, dtype=np.float64)
    d = dict(lmax=lmax, kmax=kmax, sky=sky_gaussian(lmax, [(ell + 1.0) ** -2], seed=0),
             beam=beam_gaussian_taper(lmax, kmax, 20.0, seed=1),
             ring_theta=equiangular_ring_theta(2048), nphi=4096)
    if with_pointings:
        d["theta"], d["phi"], d["psi"] = pointings_uniform(n, seed=2)
    return d


def truncate_alm(alm: np.ndarray, lmax: int, lnew: int) -> np.ndarray:
    """The packed coefficients [..., nalm(lmax)] restricted to l <= lnew."""
    idx = np.concatenate([alm_index(lmax, np.arange(m, lnew + 1), m) for m in range(lnew + 1)])
    return np.ascontiguousarray(alm[..., idx])


def rotation_about(axis, angle: float) -> np.ndarray:
    """Rotation matrix by ``angle`` about the unit vector ``axis`` (Rodrigues)."""
    a = np.asarray(axis, dtype=np.float64)
    a = a / np.linalg.norm(a)
    K = np.array([[0.0, -a[2], a[1]], [a[2], 0.0, -a[0]], [-a[1], a[0], 0.0]])
    return np.eye(3) + math.sin(angle) * K + (1.0 - math.cos(angle)) * (K @ K)


def config_detectors(ndet: int = 22, sky_lmax: int = 1500, seed: int = 3, with_pointings: bool = True):
    """Many detectors with uneven band limits sharing one polarised sky:
    detector d has lmax = (256, 512, 768, 1024, 1500)[d mod 5] and
    kmax = (4, 8, 12, 16, 24)[3d mod 5], its own far-sidelobe beam (seed 100+d),
    lmax_d equiangular rings x 2 lmax_d phi, a scan of n_d samples (log-uniform
    in [1e6, 5e7]) seen through a random 0-5 degree focal-plane offset and a
    psi offset uniform in [0, 2 pi).  The sky is the T/E/B sky at sky_lmax
    truncated to each lmax_d."""
    rng = np.random.default_rng(seed)
    sky = sky_polarised(sky_lmax, seed=0)
    dets = []
    for d in range(ndet):
        L = (256, 512, 768, 1024, 1500)[d % 5]
        K = (4, 8, 12, 16, 24)[(3 * d) % 5]
        n = int(round(math.exp(rng.uniform(math.log(1e6), math.log(5e7)))))
        axis = rng.standard_normal(3)
        offset = rotation_about(axis, math.radians(rng.uniform(0.0, 5.0)))
        psi_off = rng.uniform(0.0, 2.0 * math.pi)
        det = dict(lmax=L, kmax=K, sky=truncate_alm(sky, sky_lmax, L),
                   beam=beam_far_sidelobe(L, K, seed=100 + d), ring_theta=equiangular_ring_theta(L),
                   nphi=2 * L, n=n, offset=offset, psi_offset=psi_off)
        if with_pointings:
            det["theta"], det["phi"], det["psi"] = pointings_scan(n, psi_offset=psi_off, offset=offset)
        dets.append(det)
    return dets


def pointing_periods(n: int, fsamp: float = 32.5, minutes=(40.0, 70.0), seed: int = 4) -> np.ndarray:
    """Offsets (nper + 1 int64, 0 ... n) of consecutive pointing periods whose
    lengths are uniform in ``minutes`` at ``fsamp`` Hz (the last one truncated)."""
    rng = np.random.default_rng(seed)
    lo, hi = (int(round(m * 60.0 * fsamp)) for m in minutes)
    starts = [0]
    while starts[-1] < n:
        starts.append(min(n, starts[-1] + int(rng.integers(lo, hi + 1))))
    return np.asarray(starts, dtype=np.int64)


def orbital_velocity(starts: np.ndarray, fsamp: float = 32.5, seed: int = 5) -> np.ndarray:
    """beta = v / c per pointing period [nper, 3] (ecliptic frame of the scan):
    the Earth's orbital velocity (29.78 km/s along the orbit, longitude 2 pi t /
    (365.25 d) at mid-period) plus a 0.3 km/s Gaussian jitter per component."""
    rng = np.random.default_rng(seed)
    c = 299792458.0
    tmid = 0.5 * (starts[:-1] + starts[1:]) / fsamp
    lam = 2.0 * math.pi * tmid / (365.25 * 86400.0)
    v = 29.78e3 * np.stack([-np.sin(lam), np.cos(lam), np.zeros_like(lam)], -1)
    v += rng.standard_normal(v.shape) * 0.3e3
    return v / c


def config_orbital(n: int = 100_000_000, with_pointings: bool = True):
    """Orbital dipole through the 4pi beam: the LFI-like beam (lmax=1024, kmax=16,
    T/E/B; the temperature beam's l <= 2 coefficients enter), the 32.5 Hz scan,
    40-70 minute pointing periods, Earth-orbit velocities, T0 = 2.7255 K and a
    70 GHz channel."""
    d = dict(lmax=1024, kmax=16, beam=beam_far_sidelobe(1024, 16, seed=1),
             ring_theta=equiangular_ring_theta(1024), nphi=2048, T0=2.7255, nu=70e9)
    d["period_start"] = pointing_periods(n)
    d["beta"] = orbital_velocity(d["period_start"])
    if with_pointings:
        d["theta"], d["phi"], d["psi"] = pointings_scan(n)
    return d


def beam_elliptical(lmax: int, kmax: int, sigma_l: float = 0.0, ellipticity: float = 0.3) -> np.ndarray:
    """Elliptical-Gaussian-like beam [1][kmax+1][lmax+1] (boresight on +z): the
    Gaussian envelope sqrt((2l+1)/4pi) exp(-l(l+1) s^2/2) times, for even k, the
    ratio of modified Bessel functions I_{k/2}(x)/I_0(x) with x = l(l+1) s^2 e/4
    (odd k vanish for a beam symmetric under a half turn); s = 1.5/lmax unless
    sigma_l is given.  A timing stand-in with the shape and k structure of an
    elliptical beam."""
    from scipy.special import ive
    s = sigma_l if sigma_l > 0 else 1.5 / lmax
    ell = np.arange(lmax + 1, dtype=np.float64)
    ll = ell * (ell + 1.0)
    env = np.sqrt((2 * ell + 1) / (4 * math.pi)) * np.exp(-0.5 * ll * s * s)
    x = ll * s * s * ellipticity / 4.0
    b = np.zeros((1, kmax + 1, lmax + 1), dtype=np.complex128)
    i0 = ive(0, x)
    for k in range(0, kmax + 1, 2):
        b[0, k] = env * ive(k // 2, x) / i0
        b[0, k, :k] = 0.0
    return b
