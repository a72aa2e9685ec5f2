"""Multi-sky cube build on the tensor cores (synth_spin_maps_multi, FP32 plans):
every sky's cube against the single-sky FP32 path (the same rescaled
recurrence, CUDA-core sums) and against the oracle, across sky-group
boundaries (more than 64 skies), polarised input, K = 0, odd ring counts and
deep polar evanescent zones (CTAs whose rings all start past lmax)."""
import numpy as np
import pytest
import torch

import workloads as W
from tests.conftest import MAXTC, TOL32, check_close, rel_l2, rms

pytestmark = pytest.mark.gpu

CASES = {
    # (L, K, rings, nphi, ncomp, nsky)
    "small_healpix_5": (64, 4, W.healpix_ring_theta(32), 128, 1, 5),
    "polarised_k0_70": (24, 0, W.equiangular_ring_theta(23), 48, 3, 70),
    "polar_scan_12": (200, 6, W.equiangular_ring_theta(200), 400, 1, 12),
    "kmax_eq_lmax_4": (12, 12, W.healpix_ring_theta(4), 50, 3, 4),
}


def _skies(L, ncomp, nsky, seed):
    ell = np.arange(L + 1, dtype=float)
    if ncomp == 1:
        return np.stack([W.sky_gaussian(L, [(ell + 1.0) ** -2], seed=seed + s) for s in range(nsky)])
    return np.stack([W.sky_polarised(L, seed=seed + s) for s in range(nsky)])


@pytest.mark.parametrize("name", sorted(CASES))
def test_multisky_matches_single_sky_and_oracle(name, oracle_lib):
    import paper_2201_03478_gb300 as sl
    L, K, rt, nphi, ncomp, nsky = CASES[name]
    skies = _skies(L, ncomp, nsky, 40)
    beam = W.beam_gaussian_taper(L, K, max(4.0, L / 3.0), seed=3, ncomp=ncomp) if ncomp == 1 else \
        W.beam_far_sidelobe(L, K, seed=3)
    plan = sl.sidelobe_plan_create(L, K, rt, nphi, ncomp=ncomp, precision="fp32")
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    multi = sl.synth_spin_maps_multi(plan, dev(skies), dev(beam))
    plan.sync()
    got = multi.cpu().numpy()
    worst_single, worst_single_max = 0.0, 0.0
    for s in range(nsky):
        single = sl.synth_spin_maps(plan, dev(skies[s]), dev(beam)).cpu().numpy()
        worst_single = max(worst_single, rel_l2(got[s], single))
        worst_single_max = max(worst_single_max, float(np.max(np.abs(got[s] - single)) / rms(single)))
        if s in (0, nsky - 1):
            ref = oracle_lib.cube(skies[s], beam, rt, nphi)
            check_close(got[s].astype(np.complex128), ref, TOL32, MAXTC, "%s sky %d vs oracle" % (name, s))
    print("%s: nsky %d, tensor-core cube vs FP32 single-sky: rel L2 %.2e, max|err|/rms %.2e"
          % (name, nsky, worst_single, worst_single_max))
    assert worst_single < 5e-6 and worst_single_max < MAXTC


def test_multisky_rejects_fp64_plans():
    import paper_2201_03478_gb300 as sl
    L, K, rt, nphi, ncomp, nsky = CASES["small_healpix_5"]
    plan = sl.sidelobe_plan_create(L, K, rt, nphi, ncomp=1, precision="fp64")
    sky = torch.zeros((2, 1, (L + 1) * (L + 2) // 2), dtype=torch.complex128, device="cuda")
    beam = torch.zeros((1, K + 1, L + 1), dtype=torch.complex128, device="cuda")
    with pytest.raises(ValueError):
        sl.synth_spin_maps_multi(plan, sky, beam)
    from paper_2201_03478_gb300 import _lib
    st = _lib.load().synth_spin_maps_multi(plan.ptr, 2, sky.data_ptr(), beam.data_ptr(), sky.data_ptr())
    assert st == -2
    sl.plan_destroy(plan)
    # more skies than the ring FFT's grid rows: refused before any buffer is touched
    plan = sl.sidelobe_plan_create(L, K, rt, nphi, ncomp=1, precision="fp32")
    st = _lib.load().synth_spin_maps_multi(plan.ptr, 65536, sky.data_ptr(), beam.data_ptr(), sky.data_ptr())
    assert st == -2
    st = _lib.load().synth_spin_maps_multi(plan.ptr, 0, sky.data_ptr(), beam.data_ptr(), sky.data_ptr())
    assert st == -1
    sl.plan_destroy(plan)


def test_bounded_wait_expires_and_is_reported():
    """A device-side wait that nothing satisfies gives up after its bound, raises
    the plan's flag and is reported as SL_ERR_TIMEOUT; the context stays usable."""
    import paper_2201_03478_gb300 as sl
    from paper_2201_03478_gb300 import _lib
    L, K, rt, nphi, ncomp, nsky = CASES["small_healpix_5"]
    plan = sl.sidelobe_plan_create(L, K, rt, nphi, ncomp=1, precision="fp32")
    lib = _lib.load()
    assert lib.sl_plan_selftest_timeout(plan.ptr) == 0
    assert lib.sl_plan_sync(plan.ptr) == -5
    assert b"bounded wait" in lib.sl_last_error()
    assert lib.sl_plan_sync(plan.ptr) == 0           # the flag was cleared
    skies = torch.from_numpy(_skies(L, 1, 2, 7)).cuda()
    beam = torch.from_numpy(W.beam_gaussian_taper(L, K, 20.0, seed=3)).cuda()
    maps = sl.synth_spin_maps_multi(plan, skies, beam)
    plan.sync()
    assert torch.isfinite(torch.view_as_real(maps)).all()
