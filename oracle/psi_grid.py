"""Plain FP64 CPU oracle for the psi-grid variant of step 2 of the two-step
algorithm (Galloway et al., BeyondPlanck VIII, Sect. 2.1: the Fourier transform
over the beam order m_b = k that turns the cube c(theta, phi, k) into
c(theta, phi, psi), Eq. c_m, followed by interpolation in all three angles).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The CUDA library never
imports anything here, and nothing here imports the library.

* ``psi_cube``   -- c(theta_r, phi_j, psi_n) = Re F_0 + 2 sum_{k=1}^{K} Re(e^{ik psi_n} F_k),
                    psi_n = 2 pi n / npsi (the conjugate-pair sum of Eq. c_m at the
                    grid angles), as one matrix product with the explicit phases.
* ``interp_psi`` -- the TOD from that cube.  Reading (the paper leaves the scheme
                    open): the same separable p-point Lagrange interpolation as the
                    exact-phase path in theta (actual ring colatitudes, ghost rows
                    past the poles) and phi (uniform, periodic), times p-point
                    Lagrange on the uniform periodic psi grid.  A ghost row holds
                    (-1)^k F_k(ring, phi + pi), i.e. c(ring, phi + pi, psi + pi): it
                    is read at column + nphi/2 and psi index + npsi/2 (npsi even).

Pins in ``tests/test_psi_grid_pins.py``: at grid angles the result equals the
exact phase-sum TOD of the Sect. 2.1 oracle; single-k cubes give 2 cos(k psi_n);
the psi weights reproduce polynomials of degree < p; the error vanishes as npsi
grows.
"""
from __future__ import annotations


import numpy as np


def psi_nodes(npsi: int) -> np.ndarray:
    return 2.0 * np.pi * np.arange(npsi) / npsi


def psi_cube(cube: np.ndarray, npsi: int) -> np.ndarray:
    """[R, nphi, K+1] complex -> [R, nphi, npsi] real."""
    cube = np.asarray(cube, dtype=np.complex128)
    K1 = cube.shape[-1]
    k = np.arange(K1)
    n = np.arange(npsi)
    # exact integer phase k n mod npsi
    ph = np.exp(2j * np.pi * ((np.outer(n, k)) % npsi) / npsi)      # [npsi, K+1]
    ph[:, 1:] *= 2.0
    return np.real(cube @ ph.T)


def _uniform_weights(f: np.ndarray, p: int) -> np.ndarray:
    """Lagrange weights of nodes x_b = b - p/2 + 1 (b = 0..p-1) at f in [0, 1)."""
    x = np.arange(p) - p // 2 + 1
    w = np.ones(f.shape + (p,))
    for b in range(p):
        for c in range(p):
            if c != b:
                w[..., b] *= (f - x[c]) / (x[b] - x[c])
    return w


def interp_psi(cube_psi: np.ndarray, ring_theta: np.ndarray, theta, phi, psi, p: int = 4) -> np.ndarray:
    """TOD from the psi-grid cube [R, nphi, npsi] (see the module docstring)."""
    cp = np.asarray(cube_psi, dtype=np.float64)
    R, nphi, npsi = cp.shape
    rt = np.asarray(ring_theta, dtype=np.float64)
    th, ph, ps = (np.asarray(a, dtype=np.float64) for a in (theta, phi, psi))
    half = p // 2
    # extended rows -half .. R+half-1
    rows = np.arange(-half, R + half)
    ring = np.where(rows < 0, -1 - rows, np.where(rows >= R, 2 * R - 1 - rows, rows))
    text = np.where(rows < 0, -rt[ring], np.where(rows >= R, 2 * np.pi - rt[ring], rt[ring]))
    ghost = (rows < 0) | (rows >= R)
    base = np.searchsorted(text, th, side="right") - 1          # index into the extended rows
    base = np.clip(base, half - 1, R + half - 1)
    first = base - half + 1                                      # first stencil row (extended index)
    # theta weights: Lagrange through the p stencil colatitudes
    T = text[first[:, None] + np.arange(p)]                       # [n, p]
    wt = np.ones((th.size, p))
    for a in range(p):
        for b in range(p):
            if b != a:
                wt[:, a] *= (th - T[:, b]) / (T[:, a] - T[:, b])
    # phi and psi: uniform periodic grids
    u = np.mod(ph * (nphi / (2 * np.pi)), nphi)
    j0 = np.minimum(np.floor(u).astype(np.int64), nphi - 1)
    wp = _uniform_weights(u - j0, p)
    v = np.mod(ps * (npsi / (2 * np.pi)), npsi)
    n0 = np.minimum(np.floor(v).astype(np.int64), npsi - 1)
    wq = _uniform_weights(v - n0, p)
    out = np.zeros(th.size)
    for a in range(p):
        e = first + a
        rg, gh = ring[e], ghost[e]
        for b in range(p):
            col = np.mod(j0 + b - half + 1 + np.where(gh, nphi // 2, 0), nphi)
            for c in range(p):
                q = np.mod(n0 + c - half + 1 + np.where(gh, npsi // 2, 0), npsi)
                out += wt[:, a] * wp[:, b] * wq[:, c] * cp[rg, col, q]
    return out
