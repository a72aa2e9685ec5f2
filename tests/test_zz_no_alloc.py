"""interp_tod_noalloc: the TOD evaluation for callers that cannot allocate
device memory during the call (for example while another component owns the
device-memory budget, or inside acquisition loops that cannot take the device
synchronisation of cudaMalloc/cudaFree).  Its sort scratch is a static device
array of fixed size, shared by all calls on a device.

Checked through the C ABI against interp_tod on two calls in a row (the second
with other pointings and another n, so stale scratch from the first call would
show), plus the size limit.  The file name sorts last so that a run stopping
at the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

import workloads as W
from tests.conftest import rel_l2

pytestmark = pytest.mark.gpu


def test_interp_tod_noalloc_matches_interp_tod():
    import paper_2201_03478_gb300 as sl
    from paper_2201_03478_gb300 import _lib
    lib = _lib.load()
    L, K, nphi = 48, 4, 96
    rt = W.healpix_ring_theta(24)
    ell = np.arange(L + 1, dtype=float)
    sky = torch.from_numpy(W.sky_gaussian(L, [(ell + 1.0) ** -2], seed=0)).cuda()
    beam = torch.from_numpy(W.beam_gaussian_taper(L, K, 16.0, seed=1)).cuda()
    plan = sl.sidelobe_plan_create(L, K, rt, nphi)
    maps = sl.synth_spin_maps(plan, sky, beam)
    P = lambda t: ctypes.c_void_p(t.data_ptr())

    for seed, n in ((2, 200_000), (5, 73_321)):
        th, ph, ps = (torch.from_numpy(a).cuda() for a in W.pointings_uniform(n, seed=seed))
        ref = torch.empty(n, dtype=torch.float64, device="cuda")
        got = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
        _lib.check(lib.interp_tod(plan.ptr, P(maps), P(th), P(ph), P(ps), n, P(ref)))
        _lib.check(lib.interp_tod_noalloc(plan.ptr, P(maps), P(th), P(ph), P(ps), n, P(got)))
        _lib.check(lib.sl_plan_sync(plan.ptr))
        err = rel_l2(got.cpu().numpy(), ref.cpu().numpy())
        assert err < 1e-12, (n, err)

    # sizes beyond the static scratch are rejected before any launch
    big = (1 << 18) + 1
    st = lib.interp_tod_noalloc(plan.ptr, P(maps), P(th), P(ph), P(ps), big, P(got))
    assert st == _lib.SL_ERR_ARG
    assert b"static scratch" in lib.sl_last_error()
    sl.plan_destroy(plan)
