"""Parity at a runtime-sweep point beyond the headline size: lmax = 4096,
kmax = 10 (the paper's m_max = 10 curve of Fig. speed), the sweep's
elliptical-Gaussian-like beam and C_l = (l+1)^-2 sky, 4096 equiangular rings x
8192 phi, in the launch configuration the sweep times.

The oracle synthesises only the rings of three bands (north polar,
equatorial, south polar): whole cube rings are compared there, and TOD samples
whose 4 x 4 stencils stay inside a band (at the poles the stencil's ghost rows
map back into the band).

Accuracy at this point.  Unlike the sidelobe beams of the other tests (whose
coefficients fall off with l), this beam keeps its power up to l ~ lmax, where
the l-recurrence has accumulated lmax steps of rounding: the error grows about
as lmax x the unit roundoff of each mode, and is largest in k = 0 at the polar
rings.  Measured (relative L2 / max|err|/rms of the cube): FP64 1.7e-12 /
1.4e-11, DF64 1.7e-10 / 1.5e-9, FP32 3.1e-3 / 2.3e-2 (at lmax 1024 with the same
beam: FP64 3.0e-13, DF64 2.8e-11, FP32 2.0e-4).  The bounds below sit a few
times above those values: FP64 meets the 1e-10 target; the FP32 mode's 1e-5
holds for sidelobe-like beams, not for this one."""
import numpy as np
import pytest
import torch

import workloads as W
from tests.conftest import check_close

pytestmark = pytest.mark.gpu

L, K, R, NPHI = 4096, 10, 4096, 8192
BANDS = [(0, 11), (2042, 2053), (4084, 4095)]      # inclusive ring ranges
RINGS = [0, 1, 2, 2047, 2048, 4093, 4095]            # compared whole (inside the bands)
PER_BAND = 40_000
# (relative L2, max|err|/rms) bounds per plan precision at this point (see above)
BOUNDS = {"fp64": (1e-10, 1e-10), "df64": (1e-9, 1e-8), "fp32": (1e-2, 1e-1)}


@pytest.fixture(scope="module")
def sweep_case():
    ell = np.arange(L + 1, dtype=np.float64)
    sky = W.sky_gaussian(L, [(ell + 1.0) ** -2], seed=0)
    beam = W.beam_elliptical(L, K)
    rt = W.equiangular_ring_theta(R)
    rng = np.random.default_rng(17)
    th, ph, ps = [], [], []
    for a, b in BANDS:
        lo = rt[0] * 0.0 if a == 0 else rt[a + 1]      # base row >= -1 at the north pole, a + 1 inside
        hi = np.pi if b == R - 1 else rt[b - 2]         # base row <= R - 1 at the south pole, b - 2 inside
        t = rng.uniform(lo, hi, PER_BAND)
        th.append(t)
        ph.append(rng.uniform(0, 2 * np.pi, PER_BAND))
        ps.append(rng.uniform(0, 2 * np.pi, PER_BAND))
    return dict(sky=sky, beam=beam, rt=rt, th=np.concatenate(th), ph=np.concatenate(ph), ps=np.concatenate(ps))


@pytest.fixture(scope="module")
def gpu_results(sweep_case):
    import paper_2201_03478_gb300 as sl
    c = sweep_case
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    th, ph, ps = dev(c["th"]), dev(c["ph"]), dev(c["ps"])
    out = {}
    for prec in ("fp64", "fp32", "df64"):
        plan = sl.sidelobe_plan_create(L, K, c["rt"], NPHI, ncomp=1, precision=prec)
        try:
            maps = sl.synth_spin_maps(plan, dev(c["sky"]), dev(c["beam"]))
            tod = sl.interp_tod(plan, maps, th, ph, ps)
            plan.sync()
            out[prec] = (maps[RINGS].cpu().numpy().astype(np.complex128), tod.cpu().numpy())
            del maps, tod
        finally:
            sl.plan_destroy(plan)
            torch.cuda.empty_cache()
    return out


@pytest.fixture(scope="module")
def band_cubes(sweep_case, oracle_lib):
    c = sweep_case
    return [oracle_lib.cube_from_G(oracle_lib.cube_G(c["sky"], c["beam"], c["rt"][a:b + 1]), NPHI) for a, b in BANDS]


def test_sweep_point_cube_rings(band_cubes, gpu_results):
    rows = []
    for r in RINGS:
        q = next(q for q, (a, b) in enumerate(BANDS) if a <= r <= b)
        rows.append(band_cubes[q][r - BANDS[q][0]])
    ref = np.stack(rows)
    for prec, (tol, mx) in BOUNDS.items():
        check_close(gpu_results[prec][0], ref, tol, mx, "lmax=4096 kmax=10 cube rings %s" % prec)


def test_sweep_point_tod_bands(sweep_case, band_cubes, gpu_results, oracle_lib):
    c = sweep_case
    rt = c["rt"]
    refs = []
    for q, (a, b) in enumerate(BANDS):
        sl_ = slice(q * PER_BAND, (q + 1) * PER_BAND)
        band = rt[a:b + 1]
        i = np.searchsorted(band, c["th"][sl_], side="right") - 1
        lo, hi = (-1 if a == 0 else 1), (len(band) - 1 if b == R - 1 else len(band) - 3)
        assert i.min() >= lo and i.max() <= hi, (a, b, i.min(), i.max())
        refs.append(oracle_lib.interp(band_cubes[q], band, c["th"][sl_], c["ph"][sl_], c["ps"][sl_]))
    ref = np.concatenate(refs)
    for prec, (tol, mx) in BOUNDS.items():
        check_close(gpu_results[prec][1], ref, tol, mx, "lmax=4096 kmax=10 TOD, %d band samples, %s" % (ref.size, prec))
