"""GPU parity: the CUDA path (through the C ABI) against the CPU FP64 oracle,
element by element on seeded inputs.

Tolerances (relative L2 over the whole output, the accuracy targets):
  FP64 plans: 1e-10 (oracle and kernels take different but equally exact
              routes: recurrence arrangement, FFT vs explicit DFT, sum order);
  DF64 plans (double-float contraction and interpolation): the FP64 target, 1e-10;
  FP32 plans: 1e-5, with the measured error printed.
Every comparison also bounds the largest element error, max|err| / rms(ref)
(MAX64, MAX32), so that an error on a few samples cannot hide in the norm.
Every case carries 240 extra pointings within two ring spacings of a pole or
exactly on the first and last rings, whose stencils read ghost rows.
"""
import math

import numpy as np
import pytest
import torch

import workloads as W
from tests.conftest import MAX32, MAX64, MAXTC, TOL32, TOL64, check_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sl():
    import paper_2201_03478_gb300 as sl
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return sl


def _dev(x, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(x))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def _case(L, K, rings, nphi, n, ncomp=1, seed=0, pointings="uniform"):
    rng = np.random.default_rng(seed)
    if ncomp == 1:
        ell = np.arange(L + 1, dtype=float)
        sky = W.sky_gaussian(L, [(ell + 1.0) ** -2], seed=seed)
        beam = W.beam_gaussian_taper(L, K, max(4.0, L / 3.0), seed=seed + 1)
    else:
        sky = W.sky_polarised(L, seed=seed)
        beam = W.beam_far_sidelobe(L, K, seed=seed + 1)
    if pointings == "uniform":
        th, ph, ps = W.pointings_uniform(n, seed=seed + 2)
    else:
        th, ph, ps = W.pointings_scan(n)
    th, ph, ps = _with_polar(rng, rings, th, ph, ps)
    return dict(L=L, K=K, sky=sky, beam=beam, rt=rings, nphi=nphi, th=th, ph=ph, ps=ps)


def _with_polar(rng, rt, th, ph, ps, m=100):
    """Append m pointings within two ring spacings of each pole (stencils with
    ghost rows), the poles themselves and the first and last ring colatitudes."""
    north = rng.uniform(0.0, rt[1], m)
    south = rng.uniform(rt[-2], np.pi, m)
    edge = np.array([0.0, np.pi, rt[0], rt[-1], rt[1], rt[-2]] * 6 + [1e-12, np.pi - 1e-12, 0.0, np.pi])
    t = np.concatenate([th, north, south, edge])
    k = t.size - th.size
    return (t, np.concatenate([ph, rng.uniform(-1.0, 2 * np.pi + 1.0, k)]),
            np.concatenate([ps, rng.uniform(-10.0, 10.0, k)]))


CASES = {
    # the small configuration: Nside=32 HEALPix-like rings (odd: equator ring), 128 phi
    "small_healpix": lambda: _case(64, 4, W.healpix_ring_theta(32), 128, 20000),
    # several CTAs of rings (600 rings -> 300 pairs: two ring blocks, ragged), nphi = 90 = 2*3^2*5 < 2L+1
    "ragged_mixed_radix": lambda: _case(40, 3, W.equiangular_ring_theta(600), 90, 5000, seed=3),
    # polarised, K = 0 edge, power-of-two phi with folding at m = +-L
    "polarised_k0": lambda: _case(24, 0, W.equiangular_ring_theta(24), 48, 3000, ncomp=3, seed=5),
    # polarised, nphi = 50 (radix 5), K = L
    "polarised_kmax_eq_lmax": lambda: _case(12, 12, W.healpix_ring_theta(4), 50, 3000, ncomp=3, seed=7),
    # larger band limit on equiangular rings: deep polar evanescent zones (recurrence
    # start states well past l0), nphi = 400 = 2^4 5^2 < 2L+1, scan pointings
    "medium_polar_scan": lambda: _case(200, 6, W.equiangular_ring_theta(200), 400, 20000, seed=9,
                                       pointings="scan"),
}


@pytest.fixture(scope="module", params=sorted(CASES))
def case(request, oracle_lib):
    c = CASES[request.param]()
    c["name"] = request.param
    c["cube"] = oracle_lib.cube(c["sky"], c["beam"], c["rt"], c["nphi"])
    c["tod"] = oracle_lib.interp(c["cube"], c["rt"], c["th"], c["ph"], c["ps"])
    return c


def _plan(sl, c, precision="fp64"):
    return sl.sidelobe_plan_create(c["L"], c["K"], c["rt"], c["nphi"], ncomp=c["sky"].shape[0],
                                   precision=precision)


def test_cube_fp64(sl, case):
    plan = _plan(sl, case)
    maps = sl.synth_spin_maps(plan, _dev(case["sky"]), _dev(case["beam"]))
    check_close(maps.cpu().numpy(), case["cube"], TOL64, MAX64, case["name"] + " cube fp64")


def test_interp_fp64_same_cube(sl, case):
    """Interpolation alone: the GPU reads the oracle's cube."""
    plan = _plan(sl, case)
    tod = sl.interp_tod(plan, _dev(case["cube"]), _dev(case["th"]), _dev(case["ph"]), _dev(case["ps"]))
    check_close(tod.cpu().numpy(), case["tod"], 1e-12, 1e-12, case["name"] + " interp fp64")


def test_tod_fp64(sl, case):
    plan = _plan(sl, case)
    maps = sl.synth_spin_maps(plan, _dev(case["sky"]), _dev(case["beam"]))
    tod = sl.interp_tod(plan, maps, _dev(case["th"]), _dev(case["ph"]), _dev(case["ps"]))
    check_close(tod.cpu().numpy(), case["tod"], TOL64, MAX64, case["name"] + " tod fp64")


def test_tod_fp32(sl, case):
    plan = _plan(sl, case, "fp32")
    maps = sl.synth_spin_maps(plan, _dev(case["sky"]), _dev(case["beam"]))
    assert maps.dtype == torch.complex64
    check_close(maps.cpu().numpy().astype(np.complex128), case["cube"], TOL32, MAX32, case["name"] + " cube fp32")
    tod = sl.interp_tod(plan, maps, _dev(case["th"]), _dev(case["ph"]), _dev(case["ps"]))
    check_close(tod.cpu().numpy(), case["tod"], TOL32, MAX32, case["name"] + " tod fp32")


def test_cube_and_tod_df64(sl, case):
    plan = _plan(sl, case, "df64")
    maps = sl.synth_spin_maps(plan, _dev(case["sky"]), _dev(case["beam"]))
    assert maps.dtype == torch.complex128
    check_close(maps.cpu().numpy(), case["cube"], TOL64, MAX64, case["name"] + " cube df64")
    tod = sl.interp_tod(plan, maps, _dev(case["th"]), _dev(case["ph"]), _dev(case["ps"]))
    check_close(tod.cpu().numpy(), case["tod"], TOL64, MAX64, case["name"] + " tod df64")


def test_cube_and_tod_tf32x3(sl, case):
    """FP32 plan with the contraction on the tensor cores (3xTF32, one sky)."""
    plan = _plan(sl, case, "tf32x3")
    maps = sl.synth_spin_maps(plan, _dev(case["sky"]), _dev(case["beam"]))
    plan.sync()
    assert maps.dtype == torch.complex64
    check_close(maps.cpu().numpy().astype(np.complex128), case["cube"], TOL32, MAXTC,
                case["name"] + " cube tf32x3")
    tod = sl.interp_tod(plan, maps, _dev(case["th"]), _dev(case["ph"]), _dev(case["ps"]))
    check_close(tod.cpu().numpy(), case["tod"], TOL32, MAXTC, case["name"] + " tod tf32x3")


def test_interp_df64_same_cube(sl, case):
    """Double-float interpolation alone, reading the oracle's cube."""
    plan = _plan(sl, case, "df64")
    tod = sl.interp_tod(plan, _dev(case["cube"]), _dev(case["th"]), _dev(case["ph"]), _dev(case["ps"]))
    check_close(tod.cpu().numpy(), case["tod"], 1e-12, MAX64, case["name"] + " interp df64")


@pytest.mark.parametrize("prec", ["fp64", "df64"])
def test_adjoint_interp(sl, case, oracle_lib, prec):
    plan = _plan(sl, case, prec)
    rng = np.random.default_rng(21)
    y = rng.standard_normal(case["th"].size)
    got = sl.adjoint_interp(plan, _dev(case["th"]), _dev(case["ph"]), _dev(case["ps"]), _dev(y)).cpu().numpy()
    ref = oracle_lib.interp_adjoint(y, case["rt"], case["nphi"], case["K"], case["th"], case["ph"], case["ps"])
    check_close(got, ref, 1e-12, MAX64, "%s %s adjoint interp" % (case["name"], prec))


@pytest.mark.parametrize("prec", ["fp64", "df64"])
def test_adjoint_synth(sl, case, oracle_lib, prec):
    """Transpose of the cube build + products, from the same adjoint cube."""
    plan = _plan(sl, case, prec)
    rng = np.random.default_rng(22)
    shp = (case["rt"].size, case["nphi"], case["K"] + 1)
    fbar = rng.standard_normal(shp) + 1j * rng.standard_normal(shp)
    gs, gb = sl.adjoint_synth(plan, _dev(fbar), _dev(case["sky"]), _dev(case["beam"]))
    Gh = oracle_lib.cube_from_G_adjoint(fbar, case["L"])
    Ab = oracle_lib.cube_G_adjoint(Gh, case["rt"])
    rs, rb = oracle_lib.grad_products(Ab, case["sky"], case["beam"])
    check_close(gs.cpu().numpy(), rs, TOL64, MAX64, "%s %s adjoint synth sky" % (case["name"], prec))
    check_close(gb.cpu().numpy(), rb, TOL64, MAX64, "%s %s adjoint synth beam" % (case["name"], prec))


@pytest.mark.parametrize("prec", ["fp64", "df64"])
def test_adjoint_tod_and_dot_product(sl, case, oracle_lib, prec):
    plan = _plan(sl, case, prec)
    rng = np.random.default_rng(23)
    y = rng.standard_normal(case["th"].size)
    sky, beam = _dev(case["sky"]), _dev(case["beam"])
    th, ph, ps = _dev(case["th"]), _dev(case["ph"]), _dev(case["ps"])
    gs, gb = sl.adjoint_tod(plan, th, ph, ps, _dev(y), sky, beam)
    rs, rb = oracle_lib.adjoint_tod(y, case["sky"], case["beam"], case["rt"], case["nphi"], case["th"],
                                    case["ph"], case["ps"])
    check_close(gs.cpu().numpy(), rs, TOL64, MAX64, "%s %s adjoint tod sky" % (case["name"], prec))
    check_close(gb.cpu().numpy(), rb, TOL64, MAX64, "%s %s adjoint tod beam" % (case["name"], prec))
    # <A(s), y> is linear in s: <A s, y> = <s, A^T y> with the real inner product on packed params
    tod = sl.interp_tod(plan, sl.synth_spin_maps(plan, sky, beam), th, ph, ps).cpu().numpy()
    lhs = float(np.dot(tod, y))
    s_np = case["sky"].copy()
    rhs = float(np.sum(s_np.real * gs.cpu().numpy().real + s_np.imag * gs.cpu().numpy().imag))
    # DF64: forward and adjoint each carry ~1e-14 of double-float rounding
    dot_tol = 1e-12 if prec == "fp64" else 1e-11
    assert abs(lhs - rhs) <= dot_tol * max(1.0, np.linalg.norm(tod) * np.linalg.norm(y))
    b_np = case["beam"]
    rhs_b = float(np.sum(b_np.real * gb.cpu().numpy().real + b_np.imag * gb.cpu().numpy().imag))
    assert abs(lhs - rhs_b) <= dot_tol * max(1.0, np.linalg.norm(tod) * np.linalg.norm(y))


def test_pointing_edge_cases(sl, oracle_lib):
    """Exact poles, exact ring colatitudes, phi outside [0, 2 pi), large psi, n = 0."""
    c = CASES["small_healpix"]()
    rt = c["rt"]
    th = np.array([0.0, math.pi, rt[0], rt[-1], rt[63], 1e-300, math.pi - 1e-15, 0.5 * rt[0], 1.0, 2.0])
    ph = np.array([0.0, 2 * math.pi, -0.3, 7.5, 1e-17, 100.0, -100.0, 3.0, 2 * math.pi - 1e-16, 0.25])
    ps = np.array([0.0, -1.0, 50.0, 1e3, 3.14, -7.0, 0.5, 2.0, 1.0, 6.2])
    cube = oracle_lib.cube(c["sky"], c["beam"], rt, 128)
    ref = oracle_lib.interp(cube, rt, th, ph, ps)
    plan = _plan(sl, c)
    got = sl.interp_tod(plan, _dev(cube), _dev(th), _dev(ph), _dev(ps)).cpu().numpy()
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
    e = torch.empty(0, dtype=torch.float64, device="cuda")
    out = sl.interp_tod(plan, _dev(cube), e, e, e)
    assert out.numel() == 0


def test_pointing_edge_cases_df64(sl, oracle_lib):
    """The double-float interpolation at the poles (ghost rows), on ring
    colatitudes, with phi outside [0, 2 pi) and large psi."""
    c = CASES["small_healpix"]()
    rt = c["rt"]
    th = np.array([0.0, math.pi, rt[0], rt[-1], rt[63], 1e-300, math.pi - 1e-15, 0.5 * rt[0], 1.0, 2.0])
    ph = np.array([0.0, 2 * math.pi, -0.3, 7.5, 1e-17, 100.0, -100.0, 3.0, 2 * math.pi - 1e-16, 0.25])
    ps = np.array([0.0, -1.0, 50.0, 1e3, 3.14, -7.0, 0.5, 2.0, 1.0, 6.2])
    cube = oracle_lib.cube(c["sky"], c["beam"], rt, 128)
    ref = oracle_lib.interp(cube, rt, th, ph, ps)
    plan = _plan(sl, c, "df64")
    got = sl.interp_tod(plan, _dev(cube), _dev(th), _dev(ph), _dev(ps)).cpu().numpy()
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


def test_df64_adjoint_matches_fp64_adjoint(sl):
    """The double-float adjoint (interpolation transpose and contraction
    transpose in double-float) against the FP64 adjoint on the same inputs."""
    c = CASES["small_healpix"]()
    y = _dev(np.random.default_rng(4).standard_normal(c["th"].size))
    outs = []
    for prec in ("fp64", "df64"):
        plan = _plan(sl, c, prec)
        gs, gb = sl.adjoint_tod(plan, _dev(c["th"]), _dev(c["ph"]), _dev(c["ps"]), y, _dev(c["sky"]),
                                _dev(c["beam"]))
        outs.append((gs.cpu().numpy(), gb.cpu().numpy()))
    check_close(outs[1][0], outs[0][0], 1e-11, MAX64, "df64 vs fp64 adjoint sky")
    check_close(outs[1][1], outs[0][1], 1e-11, MAX64, "df64 vs fp64 adjoint beam")


@pytest.fixture(scope="module")
def order_case(oracle_lib):
    """Small configuration plus pointings at and near the poles, on rings and
    with phi outside [0, 2 pi): ghost rows p/2 deep at both poles."""
    c = CASES["small_healpix"]()
    rt = c["rt"]
    # p = 6 stencils reach three rows past a pole: samples down to the third ring
    rng = np.random.default_rng(31)
    extra_th = np.concatenate([[0.0, math.pi, rt[0], rt[1], rt[2], rt[-1], 1e-9, math.pi - 1e-9, 0.5 * rt[0],
                                rt[63]], rng.uniform(0, rt[2], 100), rng.uniform(rt[-3], math.pi, 100)])
    extra_ph = np.concatenate([[0.1, 6.0, -0.3, 7.5, 2 * math.pi - 1e-16, 100.0, 0.0, 3.0, 1.0, 0.25],
                               rng.uniform(0, 2 * math.pi, 200)])
    extra_ps = np.linspace(-3.0, 40.0, extra_th.size)
    c["th"] = np.concatenate([c["th"], extra_th])
    c["ph"] = np.concatenate([c["ph"], extra_ph])
    c["ps"] = np.concatenate([c["ps"], extra_ps])
    c["cube"] = oracle_lib.cube(c["sky"], c["beam"], rt, c["nphi"])
    return c


@pytest.mark.parametrize("p", [2, 6])
@pytest.mark.parametrize("prec,tol,mx", [("fp64", TOL64, MAX64), ("df64", TOL64, MAX64), ("fp32", TOL32, MAX32)])
def test_interp_order_2_and_6(sl, oracle_lib, order_case, p, prec, tol, mx):
    c = order_case
    ref = oracle_lib.interp(c["cube"], c["rt"], c["th"], c["ph"], c["ps"], p=p)
    plan = sl.sidelobe_plan_create(c["L"], c["K"], c["rt"], c["nphi"], ncomp=1, precision=prec, interp_order=p)
    maps = sl.synth_spin_maps(plan, _dev(c["sky"]), _dev(c["beam"]))
    tod = sl.interp_tod(plan, maps, _dev(c["th"]), _dev(c["ph"]), _dev(c["ps"])).cpu().numpy()
    check_close(tod, ref, tol, mx, "p=%d %s tod" % (p, prec))
    if prec != "fp32":      # interpolation alone, on the oracle's cube
        got = sl.interp_tod(plan, _dev(c["cube"]), _dev(c["th"]), _dev(c["ph"]), _dev(c["ps"])).cpu().numpy()
        check_close(got, ref, 1e-12, MAX64, "p=%d %s interp" % (p, prec))


@pytest.mark.parametrize("p", [2, 6])
@pytest.mark.parametrize("prec", ["fp64", "df64"])
def test_adjoint_interp_order_2_and_6(sl, oracle_lib, order_case, p, prec):
    c = order_case
    y = np.random.default_rng(8).standard_normal(c["th"].size)
    ref = oracle_lib.interp_adjoint(y, c["rt"], c["nphi"], c["K"], c["th"], c["ph"], c["ps"], p=p)
    plan = sl.sidelobe_plan_create(c["L"], c["K"], c["rt"], c["nphi"], ncomp=1, interp_order=p, precision=prec)
    got = sl.adjoint_interp(plan, _dev(c["th"]), _dev(c["ph"]), _dev(c["ps"]), _dev(y)).cpu().numpy()
    check_close(got, ref, 1e-12, MAX64, "p=%d %s adjoint interp" % (p, prec))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_tod_from_host_pipeline(sl, prec):
    """The host-buffer end-to-end call (convolve_tod_host: upload in pieces beside
    the cube build, interpolation per piece, download) gives the device path's TOD
    bit for bit (every sample's arithmetic is the same whatever piece it falls in),
    for several piece counts including ragged ones and more pieces than samples,
    from pinned and from pageable host memory."""
    import ctypes
    from paper_2201_03478_gb300 import _lib
    c = CASES["small_healpix"]()
    plan = _plan(sl, c, prec)
    ref = sl.interp_tod(plan, sl.synth_spin_maps(plan, _dev(c["sky"]), _dev(c["beam"])), _dev(c["th"]),
                        _dev(c["ph"]), _dev(c["ps"])).cpu().numpy()
    host = [torch.from_numpy(np.ascontiguousarray(a)) for a in (c["sky"], c["beam"], c["th"], c["ph"], c["ps"])]
    pin = [t.pin_memory() for t in host]
    for chunks in (1, 3, 8, 64):
        got = sl.tod_from_host(plan, *pin, chunks=chunks).numpy()
        assert np.array_equal(got, ref), chunks
    assert np.array_equal(sl.tod_from_host(plan, *host, chunks=5).numpy(), ref)   # pageable
    few = [t[:5] for t in host[2:]]
    got = sl.tod_from_host(plan, host[0], host[1], *few, chunks=64).numpy()           # pieces > n
    assert np.array_equal(got, ref[:5])
    empty = [t[:0] for t in host[2:]]
    assert sl.tod_from_host(plan, host[0], host[1], *empty).numel() == 0
    lib = _lib.load()
    P = lambda t: ctypes.c_void_p(t.data_ptr())
    out = torch.empty(ref.size, dtype=torch.float64)
    for bad in (0, 65):
        st = lib.convolve_tod_host(plan.ptr, P(host[0]), P(host[1]), P(host[2]), P(host[3]), P(host[4]),
                                   ref.size, bad, P(out))
        assert st == _lib.SL_ERR_ARG
    sl.plan_destroy(plan)


def test_errors_are_reported(sl):
    c = CASES["small_healpix"]()
    with pytest.raises(sl.SidelobeError, match="SL_ERR_ARG"):
        sl.sidelobe_plan_create(64, 65, c["rt"], 128)
    with pytest.raises(sl.SidelobeError, match="SL_ERR_UNSUPPORTED"):
        sl.sidelobe_plan_create(64, 4, c["rt"], 14)       # 14 = 2 * 7
    with pytest.raises(sl.SidelobeError, match="SL_ERR_ARG"):
        sl.sidelobe_plan_create(64, 4, c["rt"][::-1].copy(), 128)
