"""convolve_tod: the whole forward operator in one call, the pointing sort on
a second stream beside the cube build.  It must give the cube and the TOD of
synth_spin_maps followed by interp_tod bit for bit, for every plan precision;
see pointings written on the plan's stream just before the call (the sort
stream forks after them); and agree with the oracle."""
import numpy as np
import pytest
import torch

import workloads as W
from tests.conftest import MAX32, MAX64, MAXTC, TOL32, TOL64, check_close

pytestmark = pytest.mark.gpu

L, K = 40, 6
RT = W.healpix_ring_theta(20)
NPHI = 80


def _setup(prec, n, seed=0):
    import paper_2201_03478_gb300 as sl
    ell = np.arange(L + 1, dtype=np.float64)
    sky = W.sky_gaussian(L, [(ell + 1.0) ** -2], seed=seed)
    beam = W.beam_gaussian_taper(L, K, 15.0, seed=seed + 1)
    th, ph, ps = W.pointings_uniform(n, seed=seed + 2)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    plan = sl.sidelobe_plan_create(L, K, RT, NPHI, precision=prec)
    return sl, plan, (sky, beam, th, ph, ps), [dev(a) for a in (sky, beam, th, ph, ps)]


@pytest.mark.parametrize("prec", ["fp64", "fp32", "df64", "tf32x3"])
def test_convolve_tod_equals_the_two_calls(prec, oracle_lib):
    sl, plan, host, (sky, beam, th, ph, ps) = _setup(prec, 60_000)
    maps_a = sl.synth_spin_maps(plan, sky, beam)
    tod_a = sl.interp_tod(plan, maps_a, th, ph, ps)
    maps_b, tod_b = sl.convolve_tod(plan, sky, beam, th, ph, ps)
    plan.sync()
    assert torch.equal(maps_a, maps_b)
    assert torch.equal(tod_a, tod_b)
    ref = oracle_lib.interp(oracle_lib.cube_from_G(oracle_lib.cube_G(host[0], host[1], RT), NPHI), RT,
                            host[2], host[3], host[4])
    tol, mx = {"fp32": (TOL32, MAX32), "tf32x3": (TOL32, MAXTC)}.get(prec, (TOL64, MAX64))
    check_close(tod_b.cpu().numpy(), ref, tol, mx, "convolve_tod %s" % prec)
    sl.plan_destroy(plan)


def test_convolve_tod_sees_pointings_written_just_before():
    """The pointings are rewritten on the plan's stream (torch's current stream)
    right before each call; the sort on the second stream must read the new
    values.  Alternating two pointing sets over several calls shows any stale read."""
    sl, plan, host, (sky, beam, th, ph, ps) = _setup("fp32", 200_000, seed=3)
    th2, ph2, ps2 = (torch.from_numpy(a).cuda() for a in W.pointings_uniform(200_000, seed=9))
    maps = sl.synth_spin_maps(plan, sky, beam)
    ref1 = sl.interp_tod(plan, maps, th, ph, ps).clone()
    ref2 = sl.interp_tod(plan, maps, th2, ph2, ps2).clone()
    cur = [t.clone() for t in (th, ph, ps)]
    tod = torch.empty_like(ref1)
    for it in range(6):
        src = (th2, ph2, ps2) if it % 2 else (th, ph, ps)
        for c, s_ in zip(cur, src):
            c.copy_(s_)                       # queued on the plan's stream just before the call
        sl.convolve_tod(plan, sky, beam, cur[0], cur[1], cur[2], maps=maps, tod=tod)
        plan.sync()
        assert torch.equal(tod, ref2 if it % 2 else ref1), it
    sl.plan_destroy(plan)


def test_convolve_tod_without_samples():
    sl, plan, host, (sky, beam, th, ph, ps) = _setup("fp64", 10)
    e = th[:0]
    maps_b, tod_b = sl.convolve_tod(plan, sky, beam, e, e, e)
    maps_a = sl.synth_spin_maps(plan, sky, beam)
    plan.sync()
    assert tod_b.numel() == 0 and torch.equal(maps_a, maps_b)
    sl.plan_destroy(plan)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "df64", "tf32x3"])
def test_convolve_tod_in_a_cuda_graph(prec):
    """convolve_tod captured into a CUDA graph on the plan's stream (thread-local
    capture, after a warm call on that stream has created the plan's second stream
    and sized its scratch).  Every replay gives the eager results bit for bit and
    reads the buffers' current contents: pointings rewritten between replays, then
    a doubled sky (every TOD value exactly doubled)."""
    n = 50_000
    sl, plan, host, (sky, beam, th, ph, ps) = _setup(prec, n, seed=5)
    th2, ph2, ps2 = (torch.from_numpy(a).cuda() for a in W.pointings_uniform(n, seed=11))
    cur = [t.clone() for t in (th, ph, ps)]
    maps = torch.empty(plan.maps_shape(), dtype=plan.maps_dtype, device="cuda")
    tod = torch.empty(n, dtype=torch.float64, device="cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        ref_maps, ref1 = (t.clone() for t in sl.convolve_tod(plan, sky, beam, th, ph, ps))
        ref2 = sl.interp_tod(plan, ref_maps, th2, ph2, ps2).clone()
        sl.convolve_tod(plan, sky, beam, cur[0], cur[1], cur[2], maps=maps, tod=tod)   # warm, on s
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s, capture_error_mode="thread_local"):
        sl.convolve_tod(plan, sky, beam, cur[0], cur[1], cur[2], maps=maps, tod=tod)
    torch.cuda.synchronize()
    for it in range(4):
        for c, x in zip(cur, (th2, ph2, ps2) if it % 2 else (th, ph, ps)):
            c.copy_(x)
        maps.zero_()
        tod.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(maps, ref_maps), it
        assert torch.equal(tod, ref2 if it % 2 else ref1), it
    for c, x in zip(cur, (th, ph, ps)):
        c.copy_(x)
    sky.mul_(2.0)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(tod, 2.0 * ref1)
    del g
    plan.sync()
    sl.plan_destroy(plan)
