"""Precision variant at lmax = 2048, kmax = 32 (2048 x 4096 equiangular rings,
2e8 uniform pointings): the error of each precision mode (FP64, FP32, DF64 and
the 3xTF32 tensor-core contraction) against the oracle on a subset of about 1e6
samples, and FP32 against FP64 over the whole TOD.

The oracle synthesises only the rings of three bands (polar, mid-latitude,
equatorial); the subset is every pointing whose 4 x 4 stencil lies inside a
band, so its interpolation reads only rings the oracle has."""
import numpy as np
import pytest
import torch

import workloads as W
from tests.conftest import MAX32, MAX64, MAXTC, check_close, rel_l2

pytestmark = pytest.mark.gpu

BANDS = [(0, 11), (600, 611), (1018, 1029)]     # inclusive ring ranges
SUBSET = 1_000_000


@pytest.fixture(scope="module")
def highres():
    import paper_2201_03478_gb300 as sl
    cfg = W.config_highres(n=200_000_000)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    out = {"cfg": cfg}
    th, ph, ps = dev(cfg["theta"]), dev(cfg["phi"]), dev(cfg["psi"])
    for prec in ("fp64", "fp32", "df64", "tf32x3"):
        plan = sl.sidelobe_plan_create(cfg["lmax"], cfg["kmax"], cfg["ring_theta"], cfg["nphi"], ncomp=1,
                                       precision=prec)
        maps = sl.synth_spin_maps(plan, dev(cfg["sky"]), dev(cfg["beam"]))
        tod = sl.interp_tod(plan, maps, th, ph, ps)
        plan.sync()
        out[prec] = tod.cpu().numpy()
        del maps, tod
        sl.plan_destroy(plan)
        torch.cuda.empty_cache()
    del th, ph, ps
    torch.cuda.empty_cache()
    return out


def _band_subset(cfg):
    rt = cfg["ring_theta"]
    i = np.searchsorted(rt, cfg["theta"], side="right") - 1      # base row, -1 .. R-1
    sel = []
    for a, b in BANDS:
        lo = -1 if a == 0 else a + 1                              # rows i-1 .. i+2 inside [a, b]
        sel.append(np.nonzero((i >= lo) & (i <= b - 2))[0])
    rng = np.random.default_rng(11)
    out = []
    tot = sum(s.size for s in sel)
    for s in sel:
        take = min(s.size, int(round(SUBSET * s.size / tot)))
        out.append(np.sort(rng.choice(s, take, replace=False)))
    return out


def test_highres_precision_modes_vs_oracle(highres, oracle_lib):
    cfg = highres["cfg"]
    rt, nphi = cfg["ring_theta"], cfg["nphi"]
    subsets = _band_subset(cfg)
    assert sum(s.size for s in subsets) >= 900_000
    refs, got = [], {"fp64": [], "fp32": [], "df64": [], "tf32x3": []}
    for (a, b), idx in zip(BANDS, subsets):
        band = rt[a:b + 1]
        cube = oracle_lib.cube_from_G(oracle_lib.cube_G(cfg["sky"], cfg["beam"], band), nphi)
        refs.append(oracle_lib.interp(cube, band, cfg["theta"][idx], cfg["phi"][idx], cfg["psi"][idx]))
        for prec in got:
            got[prec].append(highres[prec][idx])
    ref = np.concatenate(refs)
    for prec, tol, mx in (("fp64", 1e-10, MAX64), ("fp32", 1e-5, MAX32), ("df64", 1e-10, MAX64),
                          ("tf32x3", 1e-5, MAXTC)):
        g = np.concatenate(got[prec])
        check_close(g, ref, tol, mx, "lmax=2048 kmax=32: %s TOD on %d-sample subset vs oracle" % (prec, ref.size))


def test_highres_fp32_vs_fp64_whole_tod(highres):
    t64, t32 = highres["fp64"], highres["fp32"]
    assert np.isfinite(t64).all() and np.isfinite(t32).all()
    err = rel_l2(t32, t64)
    print("lmax=2048 kmax=32: FP32 vs FP64 over 2e8 samples, rel L2 %.2e" % err)
    assert err < 1e-5
