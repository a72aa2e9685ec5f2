"""Pins of the psi-grid oracle (Sect. 2.1, step 2 as a Fourier transform over
the beam order, then interpolation in theta, phi and psi) against the exact
phase-sum oracle, closed forms and polynomial exactness."""
import numpy as np
import pytest

import oracle
import workloads as W
from oracle import psi_grid as pg


@pytest.fixture(scope="module")
def small(oracle_lib):
    cfg = W.config_small(n=4000)
    cube = oracle_lib.cube(cfg["sky"], cfg["beam"], cfg["ring_theta"], cfg["nphi"])
    return cfg, cube


def test_single_k_cube_is_twice_cosine():
    R, nphi, K, npsi = 3, 8, 5, 12
    for k in range(K + 1):
        cube = np.zeros((R, nphi, K + 1), dtype=np.complex128)
        cube[..., k] = 1.0 + 0.5j
        got = pg.psi_cube(cube, npsi)
        psi = pg.psi_nodes(npsi)
        want = (1.0 if k == 0 else 2.0) * (np.cos(k * psi) - (0.5 * np.sin(k * psi) if k else 0.0))
        np.testing.assert_allclose(got, np.broadcast_to(want, got.shape), atol=1e-14)


def test_at_grid_angles_equals_exact_phase_sum(small):
    cfg, cube = small
    K = cfg["kmax"]
    npsi = 2 * K + 2
    cp = pg.psi_cube(cube, npsi)
    rng = np.random.default_rng(3)
    n = 2000
    th, ph = cfg["theta"][:n], cfg["phi"][:n]
    ps = pg.psi_nodes(npsi)[rng.integers(0, npsi, n)]
    want = oracle.interp(cube, cfg["ring_theta"], th, ph, ps)
    got = pg.interp_psi(cp, cfg["ring_theta"], th, ph, ps)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12 * np.max(np.abs(want)))


def test_psi_weights_reproduce_polynomials():
    """A cube whose values are a cubic in the psi index is interpolated exactly
    wherever the 4-point psi stencil does not wrap (theta, phi at nodes)."""
    R, nphi, npsi, p = 6, 8, 40, 4
    rt = (np.arange(R) + 0.5) * np.pi / R
    n = np.arange(npsi, dtype=np.float64)
    q = 0.3 - 0.2 * n + 0.05 * n ** 2 - 0.001 * n ** 3
    cp = np.broadcast_to(q, (R, nphi, npsi)).copy()
    rng = np.random.default_rng(1)
    v = rng.uniform(2.0, npsi - 3.0, 50)
    ps = v * 2 * np.pi / npsi
    th = rt[rng.integers(1, R - 1, 50)]
    ph = rng.integers(0, nphi, 50) * 2 * np.pi / nphi
    got = pg.interp_psi(cp, rt, th, ph, ps, p)
    want = 0.3 - 0.2 * v + 0.05 * v ** 2 - 0.001 * v ** 3
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12)


def test_error_vanishes_as_the_psi_grid_refines(small):
    cfg, cube = small
    K = cfg["kmax"]
    n = 1500
    th, ph, ps = cfg["theta"][:n], cfg["phi"][:n], cfg["psi"][:n]
    exact = oracle.interp(cube, cfg["ring_theta"], th, ph, ps)
    errs = []
    for npsi in (2 * K + 2, 4 * K, 16 * K, 64 * K):
        got = pg.interp_psi(pg.psi_cube(cube, npsi), cfg["ring_theta"], th, ph, ps)
        errs.append(np.linalg.norm(got - exact) / np.linalg.norm(exact))
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < 1e-6, errs
