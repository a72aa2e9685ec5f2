"""psi-grid variant of step 2 on the GPU (k_psigrid.cu through the C ABI) against
the oracle (Sect. 2.1: the transform over the beam order to a psi grid, then
Lagrange interpolation in theta, phi and psi): the real cube element by
element, the TOD at random pointings (poles included), interpolation orders
2 and 6, FP32 plans, argument checks, and the full-size LFI-like cube."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import psi_grid as pg
from tests.conftest import MAX32, MAX64, check_close

pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module")
def small(oracle_lib):
    cfg = W.config_small(n=60_000)
    # pointings hugging both poles as well
    th = np.concatenate([cfg["theta"], np.linspace(1e-4, 0.08, 500), np.pi - np.linspace(1e-4, 0.08, 500)])
    rng = np.random.default_rng(8)
    ph = np.concatenate([cfg["phi"], rng.uniform(0, 2 * np.pi, 1000)])
    ps = np.concatenate([cfg["psi"], rng.uniform(-7, 7, 1000)])
    cube = oracle_lib.cube(cfg["sky"], cfg["beam"], cfg["ring_theta"], cfg["nphi"])
    return cfg, cube, th, ph, ps


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 1e-5), ("df64", 1e-10)])
@pytest.mark.parametrize("mult", [1, 3])
def test_psi_cube_and_tod_match_oracle(small, prec, tol, mult):
    import paper_2201_03478_gb300 as sl
    cfg, cube, th, ph, ps = small
    K = cfg["kmax"]
    npsi = mult * (2 * K + 2)
    plan = sl.sidelobe_plan_create(cfg["lmax"], K, cfg["ring_theta"], cfg["nphi"], ncomp=1, precision=prec)
    try:
        maps = sl.synth_spin_maps(plan, _dev(cfg["sky"]), _dev(cfg["beam"]))
        cp = sl.synth_psi_cube(plan, maps, npsi)
        tod = sl.interp_tod_psi(plan, cp, _dev(th), _dev(ph), _dev(ps))
        plan.sync()
        cp_h, tod_h = cp.cpu().numpy().astype(np.float64), tod.cpu().numpy()
    finally:
        sl.plan_destroy(plan)
    ref_cube = pg.psi_cube(cube, npsi)
    ref_tod = pg.interp_psi(ref_cube, cfg["ring_theta"], th, ph, ps)
    mx = MAX64 if tol <= 1e-10 else MAX32
    check_close(cp_h, ref_cube, tol, mx, "psi-grid %s npsi=%d cube" % (prec, npsi))
    check_close(tod_h, ref_tod, tol, mx, "psi-grid %s npsi=%d tod" % (prec, npsi))


@pytest.mark.parametrize("order", [2, 6])
def test_interpolation_orders(small, order):
    import paper_2201_03478_gb300 as sl
    cfg, cube, th, ph, ps = small
    K = cfg["kmax"]
    npsi = 2 * K + 2
    plan = sl.sidelobe_plan_create(cfg["lmax"], K, cfg["ring_theta"], cfg["nphi"], ncomp=1, precision="fp64",
                                   interp_order=order)
    try:
        maps = sl.synth_spin_maps(plan, _dev(cfg["sky"]), _dev(cfg["beam"]))
        tod = sl.interp_tod_psi(plan, sl.synth_psi_cube(plan, maps, npsi), _dev(th), _dev(ph), _dev(ps))
        tod_h = tod.cpu().numpy()
    finally:
        sl.plan_destroy(plan)
    ref = pg.interp_psi(pg.psi_cube(cube, npsi), cfg["ring_theta"], th, ph, ps, p=order)
    check_close(tod_h, ref, 1e-10, MAX64, "psi-grid order %d tod" % order)


def test_bad_npsi_is_rejected(small):
    import paper_2201_03478_gb300 as sl
    cfg = small[0]
    K = cfg["kmax"]
    plan = sl.sidelobe_plan_create(cfg["lmax"], K, cfg["ring_theta"], cfg["nphi"], ncomp=1, precision="fp64")
    try:
        maps = sl.synth_spin_maps(plan, _dev(cfg["sky"]), _dev(cfg["beam"]))
        for npsi in (2 * K, 2 * K + 3, 9000):
            with pytest.raises(sl.SidelobeError):
                sl.synth_psi_cube(plan, maps, npsi)
    finally:
        sl.plan_destroy(plan)


RINGS = [0, 1, 300, 511, 512, 1023]


def test_fullsize_psi_cube_rings_and_grid_angles(oracle_lib):
    """LFI-like full size (T/E/B, lmax 1024, kmax 16, 1024 x 2048), npsi = 34:
    whole psi-cube rings against the oracle, and at grid angles psi_n the
    psi-grid TOD equals the exact phase-sum TOD of interp_tod (1e7 scan samples)."""
    import paper_2201_03478_gb300 as sl
    cfg = W.config_lfi(with_pointings=False)
    K = cfg["kmax"]
    npsi = 2 * K + 2
    n = 10_000_000
    th, ph, _ = W.pointings_scan(n)
    ps = pg.psi_nodes(npsi)[np.random.default_rng(5).integers(0, npsi, n)]
    plan = sl.sidelobe_plan_create(cfg["lmax"], K, cfg["ring_theta"], cfg["nphi"], ncomp=3, precision="fp64")
    try:
        maps = sl.synth_spin_maps(plan, _dev(cfg["sky"]), _dev(cfg["beam"]))
        cp = sl.synth_psi_cube(plan, maps, npsi)
        dth, dph, dps = _dev(th), _dev(ph), _dev(ps)
        t_psi = sl.interp_tod_psi(plan, cp, dth, dph, dps)
        t_exact = sl.interp_tod(plan, maps, dth, dph, dps)
        plan.sync()
        rows = cp[RINGS].cpu().numpy()
        e_grid = float(torch.linalg.vector_norm(t_psi - t_exact) / torch.linalg.vector_norm(t_exact))
        del maps, cp, dth, dph, dps, t_psi, t_exact
    finally:
        sl.plan_destroy(plan)
        torch.cuda.empty_cache()
    G = oracle_lib.cube_G(cfg["sky"], cfg["beam"], cfg["ring_theta"][RINGS])
    ref = pg.psi_cube(oracle_lib.cube_from_G(G, cfg["nphi"]), npsi)
    print("full-size psi-grid vs exact TOD at grid angles %.2e" % e_grid)
    check_close(rows, ref, 1e-10, MAX64, "full-size psi cube rings")
    assert e_grid < 1e-12
