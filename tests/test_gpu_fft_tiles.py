"""The ring FFT of the cube build (Sect. 2.1, step 1: F_k(r, phi_j) = sum_m
G_k(r, m) e^{i m phi_j}, aliases folded) in every CTA tiling of the in-place
form -- 1, 2 or 4 rings x 1 or 2 orders k per CTA -- on ragged ring and k
counts, mixed radices (nphi = 120 = 4 2 3 5, 60) and bands wider than the ring
(L >= nphi / 2, and L >= nphi: several aliases per bin): every tiling gives the same bits, and the cube matches the
oracle.  Also the setter's argument checks and the cluster form's refusal."""
import numpy as np
import pytest
import torch

import workloads as W
from tests.conftest import MAX32, MAX64, check_close

pytestmark = pytest.mark.gpu

TILES = [(4, 2), (2, 2), (4, 1), (2, 1), (1, 2), (1, 1)]
CASES = [  # name, lmax, kmax, rings, nphi
    ("mixed_radix_ragged", 40, 5, 13, 120),
    ("alias_wide_band", 70, 4, 11, 128),
    ("k0_only", 33, 0, 9, 60),
    ("odd_k_count", 24, 6, 6, 64),
    ("band_over_twice_ring", 40, 3, 7, 24),
]


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("name,L,K,R,nphi", CASES)
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 1e-5)])
def test_every_tiling_same_bits_and_oracle(oracle_lib, name, L, K, R, nphi, prec, tol):
    import paper_2201_03478_gb300 as sl
    ell = np.arange(L + 1, dtype=np.float64)
    sky = W.sky_gaussian(L, [(ell + 1.0) ** -2], seed=3)
    beam = W.beam_gaussian_taper(L, K, 20.0, seed=4)
    rt = W.equiangular_ring_theta(R)
    plan = sl.sidelobe_plan_create(L, K, rt, nphi, ncomp=1, precision=prec)
    try:
        ds, db = _dev(sky), _dev(beam)
        base = sl.synth_spin_maps(plan, ds, db).clone()
        default = (plan.sizes()["fft_rings"], plan.sizes()["fft_korders"])
        assert default in TILES
        for rg, kg in TILES:
            plan.set_fft_tile(rg, kg)
            assert (plan.sizes()["fft_rings"], plan.sizes()["fft_korders"]) == (rg, kg)
            got = sl.synth_spin_maps(plan, ds, db)
            assert torch.equal(got, base), (rg, kg)
        plan.set_fft_tile(0, 0)
        assert (plan.sizes()["fft_rings"], plan.sizes()["fft_korders"]) == default
        cube = base.cpu().numpy().astype(np.complex128)
    finally:
        sl.plan_destroy(plan)
    ref = oracle_lib.cube(sky, beam, rt, nphi)
    check_close(cube, ref, tol, MAX64 if tol <= 1e-10 else MAX32, "%s %s cube (default tile %s)" % (name, prec, default))


def test_setter_checks():
    import paper_2201_03478_gb300 as sl
    L, K, R = 16, 2, 8
    rt = W.equiangular_ring_theta(R)
    plan = sl.sidelobe_plan_create(L, K, rt, 64, ncomp=1, precision="fp64")
    try:
        for bad in [(3, 1), (4, 3), (0, 1), (8, 1), (-1, 2)]:
            with pytest.raises(sl.SidelobeError):
                plan.set_fft_tile(*bad)
    finally:
        sl.plan_destroy(plan)
    # rings too long for one CTA run on clusters: no in-place tile to set
    plan = sl.sidelobe_plan_create(L, K, rt, 16384, ncomp=1, precision="fp64")
    try:
        assert (plan.sizes()["fft_rings"], plan.sizes()["fft_korders"]) == (0, 0)
        with pytest.raises(sl.SidelobeError):
            plan.set_fft_tile(1, 1)
    finally:
        sl.plan_destroy(plan)
