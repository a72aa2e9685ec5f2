"""Orbital dipole through the 4pi beam on the GPU (k_orbital.cu through the C ABI)
against the oracle (Sect. 3.3, Eq. dipole_fast and the subsampled rotation with a
natural cubic spline): the moments, every sample of small scans with edge-case
pointing periods (empty, one sample, shorter than and equal to the node
spacing, with and without a remainder), s = 1 (exact), accumulate, and whole
periods of the full-size benchmark workload."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import orbital as orb

pytestmark = pytest.mark.gpu

TOL = 1e-12    # FP64: relative to the largest |value| of the reference


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module")
def small():
    import paper_2201_03478_gb300 as sl
    cfg = W.config_small(n=10)
    plan = sl.sidelobe_plan_create(cfg["lmax"], cfg["kmax"], cfg["ring_theta"], cfg["nphi"], ncomp=1,
                                   precision="fp64")
    yield sl, plan, cfg
    sl.plan_destroy(plan)


def _case(lens, seed=9):
    n = int(sum(lens))
    th, ph, ps = W.pointings_scan(n, t0=1234.5)
    starts = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    beta = np.random.default_rng(seed).standard_normal((len(lens), 3)) * 1e-4
    return th, ph, ps, starts, beta


def test_moments_match_oracle(small):
    sl, plan, cfg = small
    beam = _dev(cfg["beam"])
    got = sl.orbital_moments(plan, beam)
    want = orb.moments(cfg["beam"][0])
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-14 * np.max(np.abs(want)))


LENS = [0, 1, 5, 20, 21, 40, 41, 0, 1000, 1957, 4000, 60001, 123457]


@pytest.mark.parametrize("s", [1, 7, 20, 64])
def test_every_sample_matches_oracle(small, s):
    sl, plan, cfg = small
    th, ph, ps, starts, beta = _case(LENS)
    T0 = 2.7255
    q = sl.quad_factor(70e9, T0)
    got = sl.orbital_dipole_tod(plan, _dev(cfg["beam"]), T0, q, _dev(th), _dev(ph), _dev(ps), starts, beta,
                                subsample=s).cpu().numpy()
    want = orb.dipole_subsampled(orb.moments(cfg["beam"][0]), T0, orb.quad_factor(70e9, T0), th, ph, ps,
                                 starts, beta, s)
    err = np.max(np.abs(got - want)) / np.max(np.abs(want))
    print("orbital s=%d: max |gpu - oracle| / max |oracle| = %.2e" % (s, err))
    assert err < TOL


def test_accumulate_and_single_period(small):
    sl, plan, cfg = small
    lens = [77777]
    th, ph, ps, starts, beta = _case(lens, seed=3)
    T0, q = 2.7255, 1.5
    beam = _dev(cfg["beam"])
    base = torch.linspace(-1e-3, 1e-3, th.size, dtype=torch.float64, device="cuda")
    out = base.clone()
    sl.orbital_dipole_tod(plan, beam, T0, q, _dev(th), _dev(ph), _dev(ps), starts, beta, subsample=20,
                          tod=out, accumulate=True)
    want = orb.dipole_subsampled(orb.moments(cfg["beam"][0]), T0, q, th, ph, ps, starts, beta, 20)
    got = (out - base).cpu().numpy()
    assert np.max(np.abs(got - want)) / np.max(np.abs(want)) < 1e-10


def test_bad_periods_are_rejected(small):
    sl, plan, cfg = small
    th, ph, ps, starts, beta = _case([10, 10])
    beam = _dev(cfg["beam"])
    args = (_dev(th), _dev(ph), _dev(ps))
    with pytest.raises(sl.SidelobeError):
        sl.orbital_dipole_tod(plan, beam, 2.7, 1.0, *args, np.array([0, 12, 19]), beta)     # does not end at n
    with pytest.raises(sl.SidelobeError):
        sl.orbital_dipole_tod(plan, beam, 2.7, 1.0, *args, np.array([0, 15, 12, 20]), np.zeros((3, 3)))
    with pytest.raises(sl.SidelobeError):
        sl.orbital_dipole_tod(plan, beam, 2.7, 1.0, *args, starts, beta, subsample=0)


def test_fullsize_workload_whole_periods():
    """The benchmark's workload (1e8 scan samples, 40-70 minute periods, the
    LFI-like beam) in the launch configuration bench.py times; whole periods
    (first, middle, last) against the oracle."""
    import paper_2201_03478_gb300 as sl
    cfg = W.config_orbital(n=100_000_000)
    plan = sl.sidelobe_plan_create(cfg["lmax"], cfg["kmax"], cfg["ring_theta"], cfg["nphi"], ncomp=3,
                                   precision="fp64")
    try:
        q = sl.quad_factor(cfg["nu"], cfg["T0"])
        th, ph, ps = _dev(cfg["theta"]), _dev(cfg["phi"]), _dev(cfg["psi"])
        tod = sl.orbital_dipole_tod(plan, _dev(cfg["beam"]), cfg["T0"], q, th, ph, ps, cfg["period_start"],
                                    cfg["beta"], subsample=20)
        got = tod.cpu().numpy()
        del th, ph, ps, tod
    finally:
        sl.plan_destroy(plan)
        torch.cuda.empty_cache()
    starts, beta = cfg["period_start"], cfg["beta"]
    S = orb.moments(cfg["beam"][0])
    qo = orb.quad_factor(cfg["nu"], cfg["T0"])
    nper = starts.size - 1
    for p in (0, nper // 2, nper - 1):
        a, e = int(starts[p]), int(starts[p + 1])
        want = orb.dipole_subsampled(S, cfg["T0"], qo, cfg["theta"][a:e], cfg["phi"][a:e], cfg["psi"][a:e],
                                     np.array([0, e - a]), beta[p:p + 1], 20)
        err = np.max(np.abs(got[a:e] - want)) / np.max(np.abs(want))
        print("full-size orbital period %d (%d samples): %.2e" % (p, e - a, err))
        assert err < TOL
