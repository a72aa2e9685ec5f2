"""interp_tod_noalloc: the TOD evaluation for callers that cannot allocate
device memory during the call (for example while another component owns the
device-memory budget, or inside acquisition loops that cannot take the device
synchronisation of cudaMalloc/cudaFree).  Its sort scratch is a static device
array of fixed size, shared by all calls on a device.

Checked through the C ABI against interp_tod on two calls in a row (the second
with other pointings and another n, so stale scratch from the first call would
show), for every plan precision: FP64 plans gather per sample, FP32, TF32X3 and
DF64 plans run the tile-staged kernels over the per-tile work list that the
static scratch also holds.  The output is prefilled with NaN so that a sample the
call never writes fails.  Plus the size limit.  The file name sorts last so that
a run stopping at the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

import workloads as W
from tests.conftest import rel_l2

pytestmark = pytest.mark.gpu

# the tolerances of the parity tests: FP64-class plans, FP32-class plans
TOL = {"fp64": 1e-12, "df64": 1e-12, "fp32": 1e-6, "tf32x3": 1e-6}


@pytest.mark.parametrize("precision", ["fp64", "fp32", "tf32x3", "df64"])
def test_interp_tod_noalloc_matches_interp_tod(precision):
    import paper_2201_03478_gb300 as sl
    from paper_2201_03478_gb300 import _lib
    lib = _lib.load()
    L, K, nphi = 48, 4, 96
    rt = W.healpix_ring_theta(24)
    ell = np.arange(L + 1, dtype=float)
    sky = torch.from_numpy(W.sky_gaussian(L, [(ell + 1.0) ** -2], seed=0)).cuda()
    beam = torch.from_numpy(W.beam_gaussian_taper(L, K, 16.0, seed=1)).cuda()
    plan = sl.sidelobe_plan_create(L, K, rt, nphi, precision=precision)
    maps = sl.synth_spin_maps(plan, sky, beam)
    P = lambda t: ctypes.c_void_p(t.data_ptr())

    for seed, n in ((2, 200_000), (5, 73_321)):
        th, ph, ps = (torch.from_numpy(a).cuda() for a in W.pointings_uniform(n, seed=seed))
        ref = torch.empty(n, dtype=torch.float64, device="cuda")
        got = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
        _lib.check(lib.interp_tod(plan.ptr, P(maps), P(th), P(ph), P(ps), n, P(ref)))
        _lib.check(lib.interp_tod_noalloc(plan.ptr, P(maps), P(th), P(ph), P(ps), n, P(got)))
        _lib.check(lib.sl_plan_sync(plan.ptr))
        g, r = got.cpu().numpy(), ref.cpu().numpy()
        assert np.all(np.isfinite(g)), (precision, n, int(np.sum(~np.isfinite(g))))
        err = rel_l2(g, r)
        emax = float(np.max(np.abs(g - r)) / np.sqrt(np.mean(r * r)))
        assert err < TOL[precision] and emax < 10 * TOL[precision], (precision, n, err, emax)

    # sizes beyond the static scratch are rejected before any launch
    big = (1 << 18) + 1
    st = lib.interp_tod_noalloc(plan.ptr, P(maps), P(th), P(ph), P(ps), big, P(got))
    assert st == _lib.SL_ERR_ARG
    assert b"static scratch" in lib.sl_last_error()
    sl.plan_destroy(plan)
