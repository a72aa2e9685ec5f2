"""Plain FP64 CPU oracle for the orbital dipole and quadrupole seen through the
full 4pi beam (Galloway et al., BeyondPlanck VIII, Sect. 3.3: Eqs. dipole_simple,
dipole and dipole_fast, and the subsampled-rotation scheme described after them).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The CUDA library never
imports anything here, and nothing here imports the library.

What the method computes:

* ``moments``      -- the nine geometric factors S_x ... S_yz = int v(n) B(n) dOmega of
                      Eq. dipole_fast, in the beam frame (boresight on +z), for the
                      temperature beam B(n) = sum_lm b_lm Y_lm(n).  Only l <= 2 of the
                      beam contributes; the closed forms below follow from writing each
                      v in {x, y, z, x^2, y^2, z^2, xy, xz, yz} in spherical harmonics
                      (Condon-Shortley phase) and using b_{l,-m} = (-1)^m conj(b_lm).
* ``quad_factor``  -- q = (a/2)(e^a + 1)/(e^a - 1), a = h nu / (k_B T0).
* ``to_beam``      -- the velocity rotated into the beam frame: beta' = R^T beta with
                      R = Rz(phi) Ry(theta) Rz(psi), the beam-to-sky rotation of the
                      convolution (Sect. 2.1).
* ``dipole_exact`` -- Eq. dipole_fast at every sample.
* ``dipole_subsampled`` -- the paper's acceleration: within each pointing period the
                      rotation is evaluated at every s-th sample only (local indices
                      0, s, 2s, ...), a cubic spline through those node values gives
                      the samples in between, and the samples after the last node
                      (the remainder that does not divide evenly by s) are evaluated
                      exactly.  Reading of the unnamed spline: natural cubic spline on
                      the uniform node grid (second derivative zero at both ends),
                      solved by the tridiagonal (Thomas) elimination.

Pins live in ``tests/test_orbital_pins.py``: quadrature of the moments with
scipy's spherical harmonics, the convolution of the dipole sky through the
Sect. 2.1 oracle, scipy's natural cubic spline, and closed-form special cases.
"""
from __future__ import annotations

import math

import numpy as np

# physical constants (CODATA 2018 exact values for h and k_B)
H_PLANCK = 6.62607015e-34
K_BOLTZMANN = 1.380649e-23


def quad_factor(nu_hz: float, T0: float) -> float:
    """q of Eq. dipole_simple: (a/2) (e^a + 1) / (e^a - 1), a = h nu / (k_B T0)."""
    a = H_PLANCK * nu_hz / (K_BOLTZMANN * T0)
    return 0.5 * a * (math.exp(a) + 1.0) / math.expm1(a)


def moments(beam_t: np.ndarray) -> np.ndarray:
    """S = [S_x, S_y, S_z, S_xx, S_yy, S_zz, S_xy, S_xz, S_yz] of the temperature beam.

    ``beam_t`` is [K+1][L+1] complex, b_lk for k >= 0 (the beam layout of the
    convolution).  Coefficients with l > 2 or absent (L < 2, K < 2) do not enter.
    """
    b = np.asarray(beam_t, dtype=np.complex128)
    K1, L1 = b.shape

    def c(l, k):
        return complex(b[k, l]) if (k < K1 and l < L1 and l >= k) else 0j

    b00, b10, b11 = c(0, 0).real, c(1, 0).real, c(1, 1)
    b20, b21, b22 = c(2, 0).real, c(2, 1), c(2, 2)
    pi = math.pi
    # z = sqrt(4pi/3) Y10;  x + iy = -sqrt(8pi/3) Y11
    Sz = math.sqrt(4 * pi / 3) * b10
    Sx = -2.0 * math.sqrt(2 * pi / 3) * b11.real
    Sy = 2.0 * math.sqrt(2 * pi / 3) * b11.imag
    # 1 = sqrt(4pi) Y00;  z^2 = sqrt(4pi)/3 Y00 + (4/3) sqrt(pi/5) Y20
    # (x + iy)^2 = sqrt(32pi/15) Y22;  (x + iy) z = -sqrt(8pi/15) Y21
    mono = math.sqrt(4 * pi) / 3 * b00
    c22 = math.sqrt(32 * pi / 15)
    Szz = mono + 4.0 / 3.0 * math.sqrt(pi / 5) * b20
    Sxx = mono - 2.0 / 3.0 * math.sqrt(pi / 5) * b20 + 0.5 * c22 * b22.real
    Syy = mono - 2.0 / 3.0 * math.sqrt(pi / 5) * b20 - 0.5 * c22 * b22.real
    Sxy = -0.5 * c22 * b22.imag
    Sxz = -math.sqrt(8 * pi / 15) * b21.real
    Syz = math.sqrt(8 * pi / 15) * b21.imag
    return np.array([Sx, Sy, Sz, Sxx, Syy, Szz, Sxy, Sxz, Syz])


def to_beam(theta, phi, psi, beta) -> np.ndarray:
    """beta' = Rz(-psi) Ry(-theta) Rz(-phi) beta, per sample; beta is [n, 3]."""
    th, ph, ps = (np.asarray(a, dtype=np.float64) for a in (theta, phi, psi))
    b = np.asarray(beta, dtype=np.float64)
    ct, st = np.cos(th), np.sin(th)
    cp, sp = np.cos(ph), np.sin(ph)
    cs, ss = np.cos(ps), np.sin(ps)
    # R = Rz(phi) Ry(theta) Rz(psi) written out; beta' = R^T beta
    R = np.empty(th.shape + (3, 3))
    R[..., 0, 0] = cp * ct * cs - sp * ss
    R[..., 0, 1] = -cp * ct * ss - sp * cs
    R[..., 0, 2] = cp * st
    R[..., 1, 0] = sp * ct * cs + cp * ss
    R[..., 1, 1] = -sp * ct * ss + cp * cs
    R[..., 1, 2] = sp * st
    R[..., 2, 0] = -st * cs
    R[..., 2, 1] = st * ss
    R[..., 2, 2] = ct
    return np.einsum("...ji,...j->...i", R, b)


def dipole_exact(S, T0: float, q: float, theta, phi, psi, beta_per_sample) -> np.ndarray:
    """Eq. dipole_fast at each sample; beta_per_sample is [n, 3] (sky frame)."""
    S = np.asarray(S, dtype=np.float64)
    bp = to_beam(theta, phi, psi, beta_per_sample)
    x, y, z = bp[:, 0], bp[:, 1], bp[:, 2]
    lin = S[0] * x + S[1] * y + S[2] * z
    quad = (S[3] * x * x + S[4] * y * y + S[5] * z * z
            + 2.0 * S[6] * x * y + 2.0 * S[7] * x * z + 2.0 * S[8] * y * z)
    return T0 * (lin + q * quad)


def nodes_of_period(n_p: int, s: int) -> int:
    """Number of spline nodes (local indices 0, s, ..., s (M - 1) < n_p)."""
    return 0 if n_p <= 0 else (n_p - 1) // s + 1


def natural_spline_second_derivs(y: np.ndarray, h: float) -> np.ndarray:
    """Second derivatives of the natural cubic spline through y on a uniform grid of
    spacing h: M_0 = M_{n-1} = 0 and M_{j-1} + 4 M_j + M_{j+1} = 6 (y_{j+1} - 2 y_j
    + y_{j-1}) / h^2 inside, by forward elimination and back substitution."""
    n = y.size
    M = np.zeros(n)
    if n < 3:
        return M
    cp = np.zeros(n)
    dp = np.zeros(n)
    for j in range(1, n - 1):
        r = 6.0 * (y[j + 1] - 2.0 * y[j] + y[j - 1]) / (h * h)
        den = 4.0 - cp[j - 1]
        cp[j] = 1.0 / den
        dp[j] = (r - dp[j - 1]) / den
    M[n - 2] = dp[n - 2]
    for j in range(n - 3, 0, -1):
        M[j] = dp[j] - cp[j] * M[j + 1]
    return M


def spline_eval(y: np.ndarray, M: np.ndarray, h: float, t: np.ndarray) -> np.ndarray:
    """The spline (nodes at 0, h, 2h, ...) at positions t in [0, h (n - 1)]."""
    n = y.size
    if n == 1:
        return np.full(t.shape, y[0])
    j = np.minimum((t // h).astype(np.int64), n - 2)
    B = (t - j * h) / h
    A = 1.0 - B
    return A * y[j] + B * y[j + 1] + ((A ** 3 - A) * M[j] + (B ** 3 - B) * M[j + 1]) * (h * h) / 6.0


def dipole_subsampled(S, T0: float, q: float, theta, phi, psi, period_start, beta, s: int) -> np.ndarray:
    """The orbital TOD with the rotation at every s-th sample of each pointing period,
    a natural cubic spline in between and exact values after the last node.

    ``period_start`` has nper + 1 entries (0 ... n); ``beta`` is [nper, 3]."""
    th, ph, ps = (np.asarray(a, dtype=np.float64) for a in (theta, phi, psi))
    starts = np.asarray(period_start, dtype=np.int64)
    beta = np.asarray(beta, dtype=np.float64).reshape(-1, 3)
    out = np.zeros(th.size)
    for p in range(starts.size - 1):
        a, e = int(starts[p]), int(starts[p + 1])
        n_p = e - a
        if n_p <= 0:
            continue
        bp = np.broadcast_to(beta[p], (n_p, 3))
        if s <= 1:
            out[a:e] = dipole_exact(S, T0, q, th[a:e], ph[a:e], ps[a:e], bp)
            continue
        M_nodes = nodes_of_period(n_p, s)
        idx = a + s * np.arange(M_nodes)
        y = dipole_exact(S, T0, q, th[idx], ph[idx], ps[idx], bp[:M_nodes])
        last = s * (M_nodes - 1)            # local index of the last node
        M2 = natural_spline_second_derivs(y, float(s))
        t = np.arange(last + 1, dtype=np.float64)
        out[a:a + last + 1] = spline_eval(y, M2, float(s), t)
        if last + 1 < n_p:                  # the remainder: exact
            r = slice(a + last + 1, e)
            out[r] = dipole_exact(S, T0, q, th[r], ph[r], ps[r], bp[last + 1:])
    return out
