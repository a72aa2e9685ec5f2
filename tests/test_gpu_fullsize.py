"""Parity at the benchmark's full size (LFI-like: T/E/B, lmax = 1024, kmax = 16,
1024 x 2048 equiangular rings, 1e8 scan pointings), in the launch
configuration bench.py times, on outputs the oracle can compute one by one:
whole cube rings (polar, mid-latitude, equatorial) and TOD samples whose
stencil rings the oracle synthesises."""
import numpy as np
import pytest
import torch

import workloads as W
from tests.conftest import MAX32, MAX64, check_close, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lfi(oracle_lib):
    import paper_2201_03478_gb300 as sl
    cfg = W.config_lfi(n=100_000_000)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    out = {"cfg": cfg}
    for prec in ("fp64", "fp32", "df64"):
        plan = sl.sidelobe_plan_create(cfg["lmax"], cfg["kmax"], cfg["ring_theta"], cfg["nphi"], ncomp=3,
                                       precision=prec)
        maps = sl.synth_spin_maps(plan, dev(cfg["sky"]), dev(cfg["beam"]))
        th, ph, ps = dev(cfg["theta"]), dev(cfg["phi"]), dev(cfg["psi"])
        tod = sl.interp_tod(plan, maps, th, ph, ps)
        plan.sync()
        out[prec] = (maps.cpu().numpy(), tod.cpu().numpy())
        del maps, th, ph, ps, tod
        sl.plan_destroy(plan)
        torch.cuda.empty_cache()
    return out


RINGS = [0, 1, 37, 300, 511, 512, 880, 1023]


def test_fullsize_cube_rings(lfi, oracle_lib):
    cfg = lfi["cfg"]
    rt = cfg["ring_theta"]
    G = oracle_lib.cube_G(cfg["sky"], cfg["beam"], rt[RINGS])
    ref = oracle_lib.cube_from_G(G, cfg["nphi"])            # [len(RINGS), nphi, K+1]
    for prec, tol, mx in (("fp64", 1e-10, MAX64), ("fp32", 1e-5, MAX32), ("df64", 1e-10, MAX64)):
        got = lfi[prec][0][RINGS].astype(np.complex128)
        check_close(got, ref, tol, mx, "full-size cube rings %s" % prec)


def _band_samples(theta, rt, bands, per_band, seed):
    """Indices of up to per_band samples per band whose 4 x 4 stencil rows
    (i - 1 .. i + 2 around the base row i) all lie inside the band."""
    i = np.searchsorted(rt, theta, side="right") - 1
    rng = np.random.default_rng(seed)
    out = []
    for a, b in bands:
        sel = np.nonzero((i >= a + 1) & (i <= b - 2))[0]
        out.append(np.sort(rng.choice(sel, min(per_band, sel.size), replace=False)))
    return out


def test_fullsize_tod_samples(lfi, oracle_lib):
    """Samples of the full 1e8-sample scan in four ring bands: around the scan's
    northern and southern turning points (its most polar samples), mid-latitude
    and equatorial; the oracle synthesises only each band's rings."""
    cfg = lfi["cfg"]
    rt, nphi = cfg["ring_theta"], cfg["nphi"]
    th_all = cfg["theta"]
    i_n = int(np.searchsorted(rt, th_all.min(), side="right")) - 1
    i_s = int(np.searchsorted(rt, th_all.max(), side="right")) - 1
    bands = [(i_n - 1, i_n + 10), (300, 311), (506, 517), (i_s - 9, i_s + 2)]
    subsets = _band_samples(th_all, rt, bands, 1500, seed=7)
    assert all(s.size >= 500 for s in subsets), [s.size for s in subsets]
    refs = []
    for (a, b), idx in zip(bands, subsets):
        band = rt[a:b + 1]
        cube = oracle_lib.cube_from_G(oracle_lib.cube_G(cfg["sky"], cfg["beam"], band), nphi)
        refs.append(oracle_lib.interp(cube, band, th_all[idx], cfg["phi"][idx], cfg["psi"][idx]))
    ref = np.concatenate(refs)
    idx = np.concatenate(subsets)
    for prec, tol, mx in (("fp64", 1e-10, MAX64), ("fp32", 1e-5, MAX32), ("df64", 1e-10, MAX64)):
        check_close(lfi[prec][1][idx], ref, tol, mx, "full-size TOD, %d band samples, %s" % (ref.size, prec))
    # every sample finite, and FP32 / DF64 close to FP64 over the whole 1e8-sample TOD
    t64 = lfi["fp64"][1]
    check_close(lfi["fp32"][1], t64, 1e-5, MAX32, "full-size TOD fp32 vs fp64, all samples")
    check_close(lfi["df64"][1], t64, 1e-10, MAX64, "full-size TOD df64 vs fp64, all samples")
