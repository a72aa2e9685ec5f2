"""Batches of detectors (sl_batch_*): several plans with different lmax, kmax,
grids and precisions run as one CUDA graph.  Every detector's TOD must be
bit-identical to its own synth_spin_maps + interp_tod calls (the graph runs the
same kernels on the same inputs), with and without autotuning, and replays must
read the current contents of the input buffers."""
import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu

# (lmax, kmax, rings, nphi, precision, n)
DETECTORS = [
    (32, 2, W.equiangular_ring_theta(32), 64, "fp64", 20_000),
    (48, 5, W.healpix_ring_theta(16), 96, "fp32", 50_000),
    (64, 8, W.equiangular_ring_theta(64), 128, "fp64", 0),
    (24, 24, W.equiangular_ring_theta(30), 60, "fp32", 3_000),
    (100, 4, W.equiangular_ring_theta(100), 200, "fp64", 100_000),
    (40, 17, W.equiangular_ring_theta(40), 80, "fp32", 30_000),
]


def _make(sl, seed):
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    items = []
    for d, (L, K, rt, nphi, prec, n) in enumerate(DETECTORS):
        ell = np.arange(L + 1, dtype=np.float64)
        plan = sl.sidelobe_plan_create(L, K, rt, nphi, ncomp=1, precision=prec)
        th, ph, ps = W.pointings_uniform(n, seed=seed + d)
        items.append(dict(plan=plan, sky=dev(W.sky_gaussian(L, [(ell + 1.0) ** -2], seed=seed + d)),
                          beam=dev(W.beam_gaussian_taper(L, K, 20.0, seed=100 + d)),
                          maps=torch.empty(plan.maps_shape(), dtype=plan.maps_dtype, device="cuda"),
                          theta=dev(th), phi=dev(ph), psi=dev(ps),
                          tod=torch.zeros(n, dtype=torch.float64, device="cuda")))
    return items


def _individual(sl, items):
    out = []
    for it in items:
        maps = sl.synth_spin_maps(it["plan"], it["sky"], it["beam"])
        out.append(sl.interp_tod(it["plan"], maps, it["theta"], it["phi"], it["psi"]))
    torch.cuda.synchronize()
    return [t.cpu().numpy() for t in out]


@pytest.mark.parametrize("autotune", [False, True])
def test_batch_matches_individual_calls(autotune):
    import paper_2201_03478_gb300 as sl
    items = _make(sl, 5)
    ref = _individual(sl, items)
    batch = sl.sl_batch_create(items, autotune=autotune)
    info = batch.info()
    assert info["nitems"] == len(DETECTORS) and info["nstreams"] in (1, 2, 4, 8)
    assert info["kernel_nodes"] >= 2 * len(DETECTORS) and info["graph_nodes"] >= info["kernel_nodes"]
    if autotune:
        assert info["tuned_ms"] > 0 and info["serial_ms"] > 0
        for it in items:
            assert it["plan"].sizes()["tile_cols"] in (8, 16, 32)
    for it in items:
        it["tod"].zero_()
    batch.run()
    torch.cuda.synchronize()
    for it, r in zip(items, ref):
        assert np.array_equal(it["tod"].cpu().numpy(), r)
    # a replay reads the buffers' current contents: doubling every sky doubles every TOD exactly
    for it in items:
        it["sky"].mul_(2.0)
    batch.run()
    torch.cuda.synchronize()
    for it, r in zip(items, ref):
        assert np.array_equal(it["tod"].cpu().numpy(), 2.0 * r)
    sl.sl_batch_destroy(batch)


def test_batch_locks_plan_scratch():
    import paper_2201_03478_gb300 as sl
    items = _make(sl, 9)
    ref = _individual(sl, items[:1])[0]
    batch = sl.sl_batch_create(items)
    plan = items[0]["plan"]
    with pytest.raises(sl.SidelobeError):
        plan.reserve(10 * DETECTORS[0][5] + 1)           # would reallocate what the graph points into
    with pytest.raises(sl.SidelobeError):
        plan.set_tile_cols(8 if plan.sizes()["tile_cols"] != 8 else 16)
    plan.reserve(DETECTORS[0][5])                          # within capacity: fine
    sl.sl_batch_destroy(batch)
    plan.reserve(10 * DETECTORS[0][5] + 1)
    plan.set_tile_cols(8)
    assert plan.sizes()["tile_cols"] == 8
    # the plan still computes the same TOD after re-tiling
    maps = sl.synth_spin_maps(plan, items[0]["sky"], items[0]["beam"])
    tod = sl.interp_tod(plan, maps, items[0]["theta"], items[0]["phi"], items[0]["psi"])
    assert np.array_equal(tod.cpu().numpy(), ref)


def test_batch_rejects_shared_plans():
    import paper_2201_03478_gb300 as sl
    items = _make(sl, 3)[:2]
    items[1]["plan"] = items[0]["plan"]
    items[1]["maps"] = items[0]["maps"]
    items[1]["sky"], items[1]["beam"] = items[0]["sky"], items[0]["beam"]
    with pytest.raises(sl.SidelobeError):
        sl.sl_batch_create(items)


# FP32 detectors of uneven lmax, kmax, grids and sample counts (one of them empty)
PERSISTENT_DETECTORS = [
    (32, 2, W.equiangular_ring_theta(32), 64, 20_000),
    (48, 5, W.healpix_ring_theta(16), 96, 50_000),
    (64, 8, W.equiangular_ring_theta(64), 128, 0),
    (24, 24, W.equiangular_ring_theta(30), 60, 3_000),
    (100, 4, W.equiangular_ring_theta(100), 200, 100_000),
    (40, 17, W.equiangular_ring_theta(40), 80, 30_000),
    (300, 3, W.equiangular_ring_theta(300), 600, 200_000),
]


def _make_fp32(sl, seed):
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    items = []
    for d, (L, K, rt, nphi, n) in enumerate(PERSISTENT_DETECTORS):
        ell = np.arange(L + 1, dtype=np.float64)
        plan = sl.sidelobe_plan_create(L, K, rt, nphi, ncomp=1, precision="fp32")
        th, ph, ps = W.pointings_uniform(n, seed=seed + d)
        items.append(dict(plan=plan, sky=dev(W.sky_gaussian(L, [(ell + 1.0) ** -2], seed=seed + d)),
                          beam=dev(W.beam_gaussian_taper(L, K, 20.0, seed=100 + d)),
                          maps=torch.empty(plan.maps_shape(), dtype=plan.maps_dtype, device="cuda"),
                          theta=dev(th), phi=dev(ph), psi=dev(ps),
                          tod=torch.zeros(n, dtype=torch.float64, device="cuda")))
    return items


@pytest.mark.parametrize("autotune", [False, True])
def test_persistent_batch_matches_individual_calls(autotune):
    """The persistent form (one contraction launch and one interpolation launch
    for all detectors) gives every detector's TOD bit for bit: the same
    arithmetic per recurrence and per sample, whatever the tuning (ring pairs
    per thread, FFT tile, tile width) decides."""
    import paper_2201_03478_gb300 as sl
    items = _make_fp32(sl, 11)
    ref = _individual(sl, items)
    batch = sl.sl_batch_create(items, autotune=autotune, persistent=True)
    info = batch.info()
    assert info["persistent"] == 1 and info["nitems"] == len(PERSISTENT_DETECTORS)
    widths = {it["plan"].sizes()["tile_cols"] for it in items}
    assert len(widths) == 1 and widths <= {8, 16, 32}
    for it in items:
        assert it["plan"].sizes()["contraction_pairs"] in (2, 4, 8)
    for it in items:
        it["tod"].zero_()
    batch.run()
    batch.sync()
    for it, r in zip(items, ref):
        assert np.array_equal(it["tod"].cpu().numpy(), r)
    for it in items:                                   # replays read the current inputs
        it["sky"].mul_(2.0)
    batch.run()
    batch.sync()
    for it, r in zip(items, ref):
        assert np.array_equal(it["tod"].cpu().numpy(), 2.0 * r)
    sl.sl_batch_destroy(batch)


def test_persistent_batch_rejects_other_precisions():
    import paper_2201_03478_gb300 as sl
    items = _make(sl, 13)[:2]                          # an FP64 and an FP32 plan
    with pytest.raises(sl.SidelobeError, match="SL_ERR_UNSUPPORTED"):
        sl.sl_batch_create(items, persistent=True)
