"""Parity at the benchmark's full size (LFI-like: T/E/B, lmax = 1024, kmax = 16,
1024 x 2048 equiangular rings, 1e8 scan pointings), in the launch
configuration bench.py times, on outputs the oracle can compute one by one:
whole cube rings (polar, mid-latitude, equatorial) and TOD samples whose
stencil rings the oracle synthesises."""
import numpy as np
import pytest
import torch

import workloads as W
from tests.conftest import rel_l2

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
    for prec, tol in (("fp64", 1e-10), ("fp32", 1e-5), ("df64", 1e-10)):
        got = lfi[prec][0][RINGS].astype(np.complex128)
        err = rel_l2(got, ref)
        print("full-size cube rings %s rel L2 %.2e" % (prec, err))
        assert err < tol


def test_fullsize_tod_samples(lfi, oracle_lib):
    cfg = lfi["cfg"]
    rt, nphi = cfg["ring_theta"], cfg["nphi"]
    R = rt.size
    rng = np.random.default_rng(7)
    n = cfg["theta"].size
    idx = np.sort(np.concatenate([rng.choice(n, 6, replace=False),
                                  [int(np.argmin(cfg["theta"])), int(np.argmax(cfg["theta"]))]]))
    th, ph, ps = cfg["theta"][idx], cfg["phi"][idx], cfg["psi"][idx]
    rows = set()
    for t in th:
        i = int(np.searchsorted(rt, t, side="right")) - 1
        for r in range(i - 1, i + 3):
            rows.add(r if 0 <= r < R else (-1 - r if r < 0 else 2 * R - 1 - r))
    rows = sorted(rows)
    G = oracle_lib.cube_G(cfg["sky"], cfg["beam"], rt[rows])
    part = oracle_lib.cube_from_G(G, nphi)
    cube = np.zeros((R, nphi, cfg["kmax"] + 1), dtype=np.complex128)
    cube[rows] = part
    ref = oracle_lib.interp(cube, rt, th, ph, ps)
    for prec, tol in (("fp64", 1e-10), ("fp32", 1e-5), ("df64", 1e-10)):
        got = lfi[prec][1][idx]
        err = rel_l2(got, ref)
        print("full-size TOD samples %s rel L2 %.2e" % (prec, err))
        assert err < tol
    # every sample finite and FP32 close to FP64 over the whole 1e8-sample TOD
    t64, t32 = lfi["fp64"][1], lfi["fp32"][1]
    assert np.isfinite(t64).all() and np.isfinite(t32).all()
    err = rel_l2(t32, t64)
    print("full-size TOD fp32 vs fp64 rel L2 %.2e" % err)
    td = lfi["df64"][1]
    assert np.isfinite(td).all()
    err_d = rel_l2(td, t64)
    print("full-size TOD df64 vs fp64 rel L2 %.2e" % err_d)
    assert err_d < 1e-10
    assert err < 1e-5
