"""Plain FP64 CPU oracle for the spin-harmonic sidelobe convolution
(Galloway et al., BeyondPlanck VIII, Sect. 2.1).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The CUDA library never
imports or links anything here, and nothing here imports the library.

Heavy loops (Wigner recurrences, contraction over l, interpolation) live in
``oracle.c`` (plain C, double precision); the steps that are a single library
primitive (the DFT along phi as an explicit matrix product) and the final
l-local products are written here in numpy.

Every function follows one passage of the paper:

* ``conv_exact``      -- Eq. totalconvolver, evaluated term by term per sample.
* ``cube_G``          -- Eqs. c_m / S: the spin "Legendre" step for each k.
* ``cube_from_G``     -- step 1 of the two-step algorithm: synthesis along phi.
* ``interp``          -- the cube evaluated at pointings (interpolation reading:
                         p-point Lagrange with ghost rows past the poles), summed
                         over k with e^{ik psi} phases (conjugate pairs, Eq. between
                         c_m and S).
* ``*_adjoint`` / ``grad`` -- literal transposes of the above.

Parity pins for all of these are in ``tests/test_oracle_pins.py``.  The polarised
(T/E/B) sum is a reading (sum of three scalar convolutions): parity unpinned
beyond that linear identity.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, -O2, OpenMP, IEEE double)."""
    if force or not os.path.exists(_LIB_PATH) or \
            os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fopenmp", "-fPIC", "-shared",
                               "-fno-fast-math", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _L():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        i32, i64, f64 = ctypes.c_int, ctypes.c_int64, ctypes.c_double
        lib.or_wigner_d_explicit.restype = ctypes.c_longdouble
        lib.or_wigner_d_explicit.argtypes = [i32, i32, i32, ctypes.c_longdouble]
        lib.or_wigner_d_seq.restype = None
        lib.or_wigner_d_seq.argtypes = [i32, i32, i32, f64, P]
        lib.or_conv_exact.restype = None
        lib.or_conv_exact.argtypes = [i32, i32, i32, P, P, i64, P, P, P, P, P]
        lib.or_cube_G.restype = None
        lib.or_cube_G.argtypes = [i32, i32, i32, P, P, i32, P, P]
        lib.or_cube_G_adjoint.restype = None
        lib.or_cube_G_adjoint.argtypes = [i32, i32, i32, P, P, P]
        lib.or_interp.restype = None
        lib.or_interp.argtypes = [i32, i32, P, i32, i32, P, i64, P, P, P, P]
        lib.or_interp_adjoint.restype = None
        lib.or_interp_adjoint.argtypes = [i32, i32, P, i32, i32, i64, P, P, P, P, P]
        _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _c128(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _dims(sky, beam):
    sky = _c128(sky)
    beam = _c128(beam)
    if sky.ndim == 1:
        sky = sky[None]
    if beam.ndim == 2:
        beam = beam[None]
    ncomp, K1, L1 = beam.shape
    if sky.shape != (ncomp, L1 * (L1 + 1) // 2):
        raise ValueError("sky/beam shapes disagree")
    return sky, beam, L1 - 1, K1 - 1, ncomp


# ----------------------------------------------------------------------------- Wigner d
def wigner_d_explicit(l: int, m: int, k: int, beta: float) -> float:
    """Wigner's explicit sum (long double), small l only."""
    return float(_L().or_wigner_d_explicit(l, m, k, beta))


def wigner_d_seq(lmax: int, m: int, k: int, beta: float) -> np.ndarray:
    """d^l_{mk}(beta) for l = 0..lmax by the scaled three-term recurrence."""
    out = np.zeros(lmax + 1)
    _L().or_wigner_d_seq(lmax, m, k, float(beta), _p(out))
    return out


# ----------------------------------------------------------------------------- forward
def conv_exact(sky, beam, theta, phi, psi, return_imag=False):
    """Eq. totalconvolver summed term by term at each pointing (no grid)."""
    sky, beam, L, K, nc = _dims(sky, beam)
    th, ph, ps = _f64(theta), _f64(phi), _f64(psi)
    re = np.zeros(th.size)
    im = np.zeros(th.size)
    _L().or_conv_exact(L, K, nc, _p(sky), _p(beam), th.size, _p(th), _p(ph), _p(ps),
                       _p(re), _p(im))
    return (re, im) if return_imag else re


def cube_G(sky, beam, ring_theta):
    """G_k(r, m) = sum_l A_{k,lm} d^l_{mk}(theta_r); shape [K+1, R, 2L+1], m-slot m+L."""
    sky, beam, L, K, nc = _dims(sky, beam)
    rt = _f64(ring_theta)
    G = np.zeros((K + 1, rt.size, 2 * L + 1), dtype=np.complex128)
    _L().or_cube_G(L, K, nc, _p(sky), _p(beam), rt.size, _p(rt), _p(G))
    return G


def _dft_matrix(nphi: int, L: int) -> np.ndarray:
    """E[j, m+L] = exp(i m phi_j), phi_j = 2 pi j / nphi (exact integer phase)."""
    j = np.arange(nphi)[:, None]
    m = np.arange(-L, L + 1)[None, :]
    q = np.mod(j * m, nphi)                       # exact integer phase index
    return np.exp(2j * np.pi * q / nphi)


def cube_from_G(G, nphi: int) -> np.ndarray:
    """F_k(r, phi_j) = sum_m G_k(r, m) e^{i m phi_j}; returns [R, nphi, K+1]."""
    K1, R, nm = G.shape
    L = (nm - 1) // 2
    E = _dft_matrix(nphi, L)
    F = np.einsum("jm,krm->rjk", E, G, optimize=True)
    return np.ascontiguousarray(F)


def cube(sky, beam, ring_theta, nphi: int) -> np.ndarray:
    """The convolution cube c(theta_r, phi_j, k) of step 1, layout [R, nphi, K+1]."""
    return cube_from_G(cube_G(sky, beam, ring_theta), nphi)


def interp(cube_, ring_theta, theta, phi, psi, p: int = 4) -> np.ndarray:
    """TOD from the cube: p-point Lagrange per axis, ghost rows past the poles,
    c = Re S_0 + 2 sum_k Re(e^{ik psi} S_k)."""
    cb = _c128(cube_)
    R, nphi, K1 = cb.shape
    rt = _f64(ring_theta)
    th, ph, ps = _f64(theta), _f64(phi), _f64(psi)
    tod = np.zeros(th.size)
    _L().or_interp(K1 - 1, R, _p(rt), nphi, p, _p(cb), th.size, _p(th), _p(ph), _p(ps),
                   _p(tod))
    return tod


def tod(sky, beam, ring_theta, nphi, theta, phi, psi, p: int = 4) -> np.ndarray:
    return interp(cube(sky, beam, ring_theta, nphi), ring_theta, theta, phi, psi, p)


# ----------------------------------------------------------------------------- adjoint
def interp_adjoint(y, ring_theta, nphi: int, kmax: int, theta, phi, psi, p: int = 4):
    """Transpose of ``interp``: returns cube_bar [R, nphi, K+1]."""
    rt = _f64(ring_theta)
    th, ph, ps, yy = _f64(theta), _f64(phi), _f64(psi), _f64(y)
    cb = np.zeros((rt.size, nphi, kmax + 1), dtype=np.complex128)
    _L().or_interp_adjoint(kmax, rt.size, _p(rt), nphi, p, th.size, _p(th), _p(ph), _p(ps),
                           _p(yy), _p(cb))
    return cb


def cube_from_G_adjoint(cube_bar, lmax: int) -> np.ndarray:
    """Transpose of ``cube_from_G``: Ghat_k(r, m) = sum_j cube_bar[r, j, k] e^{-i m phi_j}."""
    R, nphi, K1 = cube_bar.shape
    E = _dft_matrix(nphi, lmax)
    return np.ascontiguousarray(np.einsum("jm,rjk->krm", E.conj(), cube_bar, optimize=True))


def cube_G_adjoint(Ghat, ring_theta) -> np.ndarray:
    """Transpose of ``cube_G`` w.r.t. A: Abar [K+1, 2L+1, L+1] (m-slot m+L)."""
    Gh = _c128(Ghat)
    K1, R, nm = Gh.shape
    L = (nm - 1) // 2
    rt = _f64(ring_theta)
    Ab = np.zeros((K1, nm, L + 1), dtype=np.complex128)
    _L().or_cube_G_adjoint(L, K1 - 1, R, _p(rt), _p(Gh), _p(Ab))
    return Ab


def grad_products(Abar, sky, beam):
    """Gradients of <c, y> with respect to the packed real parameters.

    With A_{k,lm} = sum_X s^X_lm conj(b^X_lk) (m in [-l, l], s_{l,-m} =
    (-1)^m conj(s_lm)), <c,y> = Re sum A conj(Abar).  Returned as complex
    arrays g = d/dRe + i d/dIm shaped like sky and beam; Im parts of the m=0
    and k=0 entries are not parameters and are returned as 0.
      sky,  m > 0: sum_k [b_lk Abar_{k,l,m} + (-1)^m conj(b_lk) conj(Abar_{k,l,-m})]
      sky,  m = 0: sum_k Re(b_lk Abar_{k,l,0})
      beam:        sum_{m=-l..l} s_lm conj(Abar_{k,lm})   (real part only for k = 0)
    """
    sky, beam, L, K, nc = _dims(sky, beam)
    Ab = _c128(Abar)
    gs = np.zeros_like(sky)
    gb = np.zeros_like(beam)
    for m in range(L + 1):
        ls = np.arange(m, L + 1)
        idx = m * (2 * L + 1 - m) // 2 + ls
        Ap = Ab[:, L + m, m:]                 # [K+1, nl]
        An = Ab[:, L - m, m:]
        sgn = -1.0 if m % 2 else 1.0
        for X in range(nc):
            b = beam[X][:, m:].copy()         # [K+1, nl]
            b[0] = b[0].real
            s = sky[X, idx].copy()
            if m == 0:
                s = s.real.astype(np.complex128)
                gs[X, idx] = np.sum((b * Ap).real, axis=0)
                gb[X][:, m:] += s[None, :] * np.conj(Ap)
            else:
                gs[X, idx] = np.sum(b * Ap + sgn * np.conj(b) * np.conj(An), axis=0)
                gb[X][:, m:] += s[None, :] * np.conj(Ap) + sgn * np.conj(s)[None, :] * np.conj(An)
    gb[:, 0, :] = gb[:, 0, :].real
    for k in range(K + 1):                    # b_lk for l < k is not a parameter
        gb[:, k, :k] = 0
    return gs, gb


def adjoint_tod(y, sky, beam, ring_theta, nphi, theta, phi, psi, p: int = 4):
    """Gradients of <tod(sky, beam), y> w.r.t. sky and beam (see grad_products)."""
    sky, beam, L, K, nc = _dims(sky, beam)
    cb = interp_adjoint(y, ring_theta, nphi, K, theta, phi, psi, p)
    Gh = cube_from_G_adjoint(cb, L)
    Ab = cube_G_adjoint(Gh, ring_theta)
    return grad_products(Ab, sky, beam)
