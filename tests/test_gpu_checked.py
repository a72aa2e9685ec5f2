"""The bounds-checked library variant (compiled with -DSL_CHECKED: every data-
dependent gather and scatter index of the binning, scatter, interpolation in all
precisions and directions, psi-grid and orbital kernels is tested before the
access; the forward also runs through interp_tod_noalloc) on the parity workloads, including pointings at and near both poles and
at phi = 0 and 2 pi: no guard may fire, and the results must still match the
oracle.  This stands in for a memory checker, which is not available here; it
runs in a child process because a process loads one library variant."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r'''
import ctypes
import sys
import numpy as np
import torch
sys.path.insert(0, ROOT)
from paper_2201_03478_gb300 import _lib
_lib.use_checked_build()
import paper_2201_03478_gb300 as sl
import oracle
oracle.build()
import workloads as W
from oracle import psi_grid as pg, orbital as orb
lib = _lib.load()
assert lib._name.endswith("libsidelobe_checked.so"), lib._name
dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
rel = lambda a, b: float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))
cfg = W.config_small(n=40_000)
th = np.concatenate([cfg["theta"], [0.0, 1e-9, np.pi, np.pi - 1e-9], np.linspace(1e-4, 0.1, 300)])
ph = np.concatenate([cfg["phi"], [0.0, 2 * np.pi - 1e-12, 0.0, np.pi], np.linspace(0, 2 * np.pi, 300)])
ps = np.concatenate([cfg["psi"], [0.0, -3.0, 7.0, 100.0], np.linspace(-10, 10, 300)])
L, K, rt, nphi = cfg["lmax"], cfg["kmax"], cfg["ring_theta"], cfg["nphi"]
ref_cube = oracle.cube(cfg["sky"], cfg["beam"], rt, nphi)
ref_tod = oracle.interp(ref_cube, rt, th, ph, ps)
y = np.random.default_rng(1).standard_normal(th.size)
rs, rb = oracle.adjoint_tod(y, cfg["sky"], cfg["beam"], rt, nphi, th, ph, ps)
for prec, tol in (("fp64", 1e-10), ("fp32", 1e-5), ("df64", 1e-10)):
    plan = sl.sidelobe_plan_create(L, K, rt, nphi, ncomp=1, precision=prec)
    maps = sl.synth_spin_maps(plan, dev(cfg["sky"]), dev(cfg["beam"]))
    tod = sl.interp_tod(plan, maps, dev(th), dev(ph), dev(ps)).cpu().numpy()
    gs, gb = sl.adjoint_tod(plan, dev(th), dev(ph), dev(ps), dev(y), dev(cfg["sky"]), dev(cfg["beam"]))
    npsi = 2 * K + 2
    tp = sl.interp_tod_psi(plan, sl.synth_psi_cube(plan, maps, npsi), dev(th), dev(ph), dev(ps)).cpu().numpy()
    tna = torch.full((th.size,), float("nan"), dtype=torch.float64, device="cuda")
    P = lambda t: ctypes.c_void_p(t.data_ptr())
    dth, dph, dps = dev(th), dev(ph), dev(ps)
    _lib.check(lib.interp_tod_noalloc(plan.ptr, P(maps), P(dth), P(dph), P(dps), th.size, P(tna)))
    plan.sync()
    tna = tna.cpu().numpy()
    st = lib.sl_debug_check_status()
    assert st == 0, (prec, hex(st))
    assert rel(tod, ref_tod) < tol, (prec, rel(tod, ref_tod))
    assert rel(tna, ref_tod) < tol, (prec, "noalloc", rel(tna, ref_tod))
    assert rel(gs.cpu().numpy(), rs) < 1e-10 and rel(gb.cpu().numpy(), rb) < 1e-10, prec   # adjoint: FP64
    ref_tp = pg.interp_psi(pg.psi_cube(ref_cube, npsi), rt, th, ph, ps)
    assert rel(tp, ref_tp) < tol, (prec, rel(tp, ref_tp))
    print("checked build %s: tod %.1e, psi-grid %.1e, no guard fired" % (prec, rel(tod, ref_tod), rel(tp, ref_tp)))
    sl.plan_destroy(plan)
plan = sl.sidelobe_plan_create(L, K, rt, nphi, ncomp=1, precision="fp64")
lens = [0, 1, 20, 21, 5000, 12345]
n = sum(lens)
oth, oph, ops = W.pointings_scan(n)
starts = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
beta = np.random.default_rng(2).standard_normal((len(lens), 3)) * 1e-4
got = sl.orbital_dipole_tod(plan, dev(cfg["beam"]), 2.7255, 1.2, dev(oth), dev(oph), dev(ops), starts, beta,
                            subsample=20).cpu().numpy()
want = orb.dipole_subsampled(orb.moments(cfg["beam"][0]), 2.7255, 1.2, oth, oph, ops, starts, beta, 20)
assert lib.sl_debug_check_status() == 0
assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want))
sl.plan_destroy(plan)
print("checked build: orbital ok")
'''


def test_checked_build_fires_no_guard_and_matches_oracle():
    code = "ROOT = %r\n" % ROOT + SCRIPT
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=1200)
    print(r.stdout[-3000:])
    assert r.returncode == 0, r.stderr[-4000:]
