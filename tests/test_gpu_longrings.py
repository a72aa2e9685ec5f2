"""Rings longer than one CTA's shared memory (the ring FFT and its adjoint on a
cluster of 2 or 4 CTAs: nphi = 7680, 8192, 16384) and beam band limits above
64 (kmax = 100, the production-like case lmax 512 / kmax 100 scaled down)
against the oracle: cube, TOD and gradients."""
import numpy as np
import pytest
import torch

import workloads as W
from tests.conftest import MAX32, MAX64, check_close

pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _case(L, K, R, seed=0):
    ell = np.arange(L + 1, dtype=np.float64)
    sky = W.sky_gaussian(L, [(ell + 1.0) ** -2], seed=seed)
    beam = W.beam_gaussian_taper(L, K, 20.0, seed=seed + 1)
    th, ph, ps = W.pointings_uniform(3000, seed=seed + 2)
    return sky, beam, W.equiangular_ring_theta(R), th, ph, ps


@pytest.mark.parametrize("prec,nphi,tol", [("fp64", 8192, 1e-10), ("fp64", 7680, 1e-10), ("fp64", 16384, 1e-10),
                                           ("fp32", 16384, 1e-5), ("df64", 8192, 1e-10)])
def test_long_rings_cube_and_tod(oracle_lib, prec, nphi, tol):
    import paper_2201_03478_gb300 as sl
    L, K, R = 96, 6, 12
    sky, beam, rt, th, ph, ps = _case(L, K, R)
    plan = sl.sidelobe_plan_create(L, K, rt, nphi, ncomp=1, precision=prec)
    try:
        maps = sl.synth_spin_maps(plan, _dev(sky), _dev(beam))
        tod = sl.interp_tod(plan, maps, _dev(th), _dev(ph), _dev(ps))
        plan.sync()
        got_cube, got_tod = maps.cpu().numpy().astype(np.complex128), tod.cpu().numpy()
    finally:
        sl.plan_destroy(plan)
    ref_cube = oracle_lib.cube(sky, beam, rt, nphi)
    ref_tod = oracle_lib.interp(ref_cube, rt, th, ph, ps)
    mx = MAX64 if tol <= 1e-10 else MAX32
    check_close(got_cube, ref_cube, tol, mx, "long rings %s nphi=%d cube" % (prec, nphi))
    check_close(got_tod, ref_tod, tol, mx, "long rings %s nphi=%d tod" % (prec, nphi))


def test_long_rings_adjoint(oracle_lib):
    import paper_2201_03478_gb300 as sl
    L, K, R, nphi = 64, 4, 8, 16384
    sky, beam, rt, th, ph, ps = _case(L, K, R, seed=4)
    y = np.random.default_rng(1).standard_normal(th.size)
    plan = sl.sidelobe_plan_create(L, K, rt, nphi, ncomp=1, precision="fp64")
    try:
        gs, gb = sl.adjoint_tod(plan, _dev(th), _dev(ph), _dev(ps), _dev(y), _dev(sky), _dev(beam))
        plan.sync()
        gs, gb = gs.cpu().numpy(), gb.cpu().numpy()
    finally:
        sl.plan_destroy(plan)
    rs, rb = oracle_lib.adjoint_tod(y, sky, beam, rt, nphi, th, ph, ps)
    check_close(gs, rs, 1e-10, MAX64, "long rings adjoint sky")
    check_close(gb, rb, 1e-10, MAX64, "long rings adjoint beam")


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 1e-5), ("df64", 1e-10)])
def test_kmax_100(oracle_lib, prec, tol):
    import paper_2201_03478_gb300 as sl
    L, K, R, nphi = 128, 100, 16, 256
    sky, beam, rt, th, ph, ps = _case(L, K, R, seed=7)
    plan = sl.sidelobe_plan_create(L, K, rt, nphi, ncomp=1, precision=prec)
    try:
        maps = sl.synth_spin_maps(plan, _dev(sky), _dev(beam))
        tod = sl.interp_tod(plan, maps, _dev(th), _dev(ph), _dev(ps))
        plan.sync()
        got = tod.cpu().numpy()
    finally:
        sl.plan_destroy(plan)
    ref = oracle_lib.tod(sky, beam, rt, nphi, th, ph, ps)
    check_close(got, ref, tol, MAX64 if tol <= 1e-10 else MAX32, "kmax 100 %s tod" % prec)
