"""Differentiation: torch.autograd through the C ABI (forward = cube build +
interpolation, backward = adjoint kernels).

- small case: autograd gradients against the CPU oracle's adjoint;
- the differentiation workload: the small configuration's sky, beam and
  Nside=32 grid with 1e8 uniform pointings, an FP32-stored TOD residual (white
  noise, sigma = 1e-3 of the signal RMS), loss 0.5 |tod - d|^2: dot-product
  test and central differences on 16 sky + 16 beam entries.  The loss is
  quadratic in each real parameter, so central differences are exact up to
  roundoff.
"""
import numpy as np
import pytest
import torch

import workloads as W
from tests.conftest import MAX64, check_close

pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_autograd_matches_oracle_adjoint(oracle_lib):
    import paper_2201_03478_gb300 as sl
    c = W.config_small(n=20000)
    plan = sl.sidelobe_plan_create(c["lmax"], c["kmax"], c["ring_theta"], c["nphi"])
    sky = _dev(c["sky"]).requires_grad_(True)
    beam = _dev(c["beam"]).requires_grad_(True)
    th, ph, ps = _dev(c["theta"]), _dev(c["phi"]), _dev(c["psi"])
    data = _dev(np.random.default_rng(3).standard_normal(th.numel()))
    tod = sl.sidelobe_tod(plan, sky, beam, th, ph, ps)
    loss = 0.5 * ((tod - data) ** 2).sum()
    loss.backward()
    res = (tod - data).detach().cpu().numpy()
    rs, rb = oracle_lib.adjoint_tod(res, c["sky"], c["beam"], c["ring_theta"], c["nphi"], c["theta"], c["phi"],
                                    c["psi"])
    check_close(sky.grad.cpu().numpy(), rs, 1e-10, MAX64, "autograd sky grad")
    check_close(beam.grad.cpu().numpy(), rb, 1e-10, MAX64, "autograd beam grad")


def test_differentiation_workload_fd_and_dot_product():
    import paper_2201_03478_gb300 as sl
    c = W.config_small(n=100_000_000)
    plan = sl.sidelobe_plan_create(c["lmax"], c["kmax"], c["ring_theta"], c["nphi"])
    sky0, beam0 = _dev(c["sky"]), _dev(c["beam"])
    th, ph, ps = _dev(c["theta"]), _dev(c["phi"]), _dev(c["psi"])
    with torch.no_grad():
        sig = sl.sidelobe_tod(plan, sky0, beam0, th, ph, ps)
        rms = float(sig.square().mean().sqrt())
        gen = torch.Generator(device="cuda").manual_seed(11)
        noise = torch.randn(sig.shape, generator=gen, device="cuda", dtype=torch.float64) * (1e-3 * rms)
        # data = signal of a perturbed sky/beam + noise, stored in FP32
        data32 = (0.97 * sig + noise).to(torch.float32)
    data = data32.to(torch.float64)

    def loss_of(s, b):
        with torch.no_grad():
            t = sl.sidelobe_tod(plan, s, b, th, ph, ps)
            return float(0.5 * (t - data).square().sum())

    sky = sky0.clone().requires_grad_(True)
    beam = beam0.clone().requires_grad_(True)
    tod = sl.sidelobe_tod(plan, sky, beam, th, ph, ps)
    r = tod - data
    (0.5 * r.square().sum()).backward()
    gs, gb = sky.grad.clone(), beam.grad.clone()

    # dot-product test: <A(s), y> = <s, A^T y> (and the same for the beam)
    with torch.no_grad():
        y = r.detach()
        lhs = float(torch.dot(tod.detach(), y))
        rhs_s = float((sky0.real * gs.real + sky0.imag * gs.imag).sum())
        rhs_b = float((beam0.real * gb.real + beam0.imag * gb.imag).sum())
    scale = float(tod.detach().norm() * y.norm())
    print("dot products: <As,y> %.12e  <s,A^T y> %.12e  <b,B^T y> %.12e" % (lhs, rhs_s, rhs_b))
    assert abs(lhs - rhs_s) <= 1e-11 * scale
    assert abs(lhs - rhs_b) <= 1e-11 * scale

    rng = np.random.default_rng(5)
    L, K = c["lmax"], c["kmax"]
    worst = 0.0
    for which in ("sky", "beam"):
        for _ in range(16):
            if which == "sky":
                i = int(rng.integers(W.nalm(L)))
                part = 1j if (i > L and rng.random() < 0.5) else 1.0
                base = sky0
                an = gs[0, i]
                idx = (0, i)
            else:
                k = int(rng.integers(K + 1))
                l = int(rng.integers(k, L + 1))
                part = 1j if (k > 0 and rng.random() < 0.5) else 1.0
                base = beam0
                an = gb[0, k, l]
                idx = (0, k, l)
            an = float(an.imag if part == 1j else an.real)
            h = 0.05 * max(abs(complex(base[idx].item())), 1e-3)
            p, m = base.clone(), base.clone()
            p[idx] += h * part
            m[idx] -= h * part
            fd = ((loss_of(p, beam0) - loss_of(m, beam0)) if which == "sky"
                  else (loss_of(sky0, p) - loss_of(sky0, m))) / (2 * h)
            err = abs(fd - an) / max(abs(an), 1e-12 * scale)
            worst = max(worst, err)
            assert err < 1e-6, (which, idx, part, fd, an)
    print("central differences: worst relative error %.2e" % worst)
