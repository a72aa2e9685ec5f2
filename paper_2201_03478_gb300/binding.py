"""Python binding of the C ABI (include/sidelobe.h), argument marshalling only.

PyTorch supplies device memory and the stream; every step of the computation
runs in libsidelobe.so.  The functions keep the C names:

    plan = sidelobe_plan_create(lmax, kmax, ring_theta, nphi, ncomp=1, precision="fp64")
    synth_spin_maps(plan, sky, beam, maps=None)        -> maps  [R, nphi, K+1] complex
    interp_tod(plan, maps, theta, phi, psi, tod=None)  -> tod   [n] float64
    adjoint_tod(plan, theta, phi, psi, tod, sky, beam) -> (sky_grad, beam_grad)
    plan_destroy(plan)

``sky`` is a complex128 tensor [ncomp, nalm] (m-major packing), ``beam`` a
complex128 tensor [ncomp, K+1, L+1]; both on the plan's device.  Gradients
come back in the same layouts, as d/dRe + i d/dIm of sum_i tod_i c_i.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib
from ._lib import SL_DF64, SL_FP32, SL_FP64, SL_TF32X3, check

_PREC = {"fp64": SL_FP64, "fp32": SL_FP32, "df64": SL_DF64, "tf32x3": SL_TF32X3,
         SL_FP64: SL_FP64, SL_FP32: SL_FP32, SL_DF64: SL_DF64, SL_TF32X3: SL_TF32X3}


class Plan:
    """Owns one sl_plan*.  Not thread-safe; all work goes to one CUDA stream."""

    def __init__(self, ptr, lmax, kmax, ncomp, ring_theta, nphi, precision, device, stream):
        self.ptr = ptr
        self.lmax, self.kmax, self.ncomp = lmax, kmax, ncomp
        self.ring_theta = np.asarray(ring_theta, dtype=np.float64)
        self.nrings, self.nphi = self.ring_theta.size, nphi
        self.precision, self.device = precision, device
        self._stream = stream
        self.nalm = (lmax + 1) * (lmax + 2) // 2

    @property
    def maps_dtype(self):
        return torch.complex64 if self.precision in (SL_FP32, SL_TF32X3) else torch.complex128

    def maps_shape(self):
        return (self.nrings, self.nphi, self.kmax + 1)

    def _sync_stream(self):
        s = torch.cuda.current_stream(self.device).cuda_stream
        if s != self._stream:
            check(_lib.load().sl_plan_set_stream(self.ptr, ctypes.c_void_p(s)))
            self._stream = s

    def sizes(self):
        out = _lib.PlanSizes()
        check(_lib.load().sl_plan_get_sizes(self.ptr, ctypes.byref(out)))
        return {f: getattr(out, f) for f, _ in out._fields_}

    def enable_timing(self, on=True):
        check(_lib.load().sl_plan_enable_timing(self.ptr, int(bool(on))))

    def kernel_stats(self, reset=False):
        arr = (_lib.KernelStat * 64)()
        n = ctypes.c_int(0)
        check(_lib.load().sl_plan_kernel_stats(self.ptr, arr, 64, ctypes.byref(n), int(bool(reset))))
        return {arr[i].name.decode(): (arr[i].launches, arr[i].total_ms) for i in range(min(n.value, 64))}

    def sync(self):
        check(_lib.load().sl_plan_sync(self.ptr))

    def reserve(self, n):
        """Grow the pointing-sort scratch to n samples now (sl_plan_reserve)."""
        check(_lib.load().sl_plan_reserve(self.ptr, int(n)))

    def set_tile_cols(self, tile_cols):
        """Sort-tile width in phi columns: 8, 16 or 32 (sl_plan_set_tile_cols)."""
        check(_lib.load().sl_plan_set_tile_cols(self.ptr, int(tile_cols)))

    def set_fft_tile(self, rings, korders):
        """Rings (1, 2, 4) x beam orders (1, 2) per CTA of the ring FFT; 0, 0 for the
        default (sl_plan_set_fft_tile)."""
        check(_lib.load().sl_plan_set_fft_tile(self.ptr, int(rings), int(korders)))

    def set_contraction_pairs(self, pairs):
        """Ring pairs (2, 4, 8) per thread of the FP32 contraction; 0 for the automatic
        choice (sl_plan_set_contraction_pairs)."""
        check(_lib.load().sl_plan_set_contraction_pairs(self.ptr, int(pairs)))

    def __del__(self):
        try:
            plan_destroy(self)
        except Exception:
            pass


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _dev_tensor(x, dtype, device, name, shape=None):
    if not isinstance(x, torch.Tensor):
        raise TypeError("%s must be a torch tensor on cuda:%d" % (name, device))
    if x.device.type != "cuda" or x.device.index != device:
        raise ValueError("%s must live on cuda:%d (got %s)" % (name, device, x.device))
    if x.dtype != dtype:
        raise TypeError("%s must be %s (got %s)" % (name, dtype, x.dtype))
    if not x.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if shape is not None and tuple(x.shape) != tuple(shape):
        raise ValueError("%s has shape %s, expected %s" % (name, tuple(x.shape), tuple(shape)))
    return x


def sidelobe_plan_create(lmax, kmax, ring_theta, nphi, ncomp=1, precision="fp64", interp_order=4,
                         device=None):
    lib = _lib.load()
    if device is None:
        device = torch.cuda.current_device()
    rt = np.ascontiguousarray(ring_theta, dtype=np.float64)
    stream = torch.cuda.current_stream(device).cuda_stream
    d = _lib.PlanDesc(lmax=int(lmax), kmax=int(kmax), ncomp=int(ncomp), nrings=int(rt.size),
                      ring_theta=rt.ctypes.data_as(ctypes.c_void_p), nphi=int(nphi),
                      interp_order=int(interp_order), precision=_PREC[precision], device=int(device),
                      stream=ctypes.c_void_p(stream))
    out = ctypes.c_void_p()
    check(lib.sidelobe_plan_create(ctypes.byref(out), ctypes.byref(d)))
    return Plan(out, int(lmax), int(kmax), int(ncomp), rt, int(nphi), _PREC[precision], int(device), stream)


def plan_destroy(plan: Plan) -> None:
    if plan is not None and plan.ptr:
        _lib.load().plan_destroy(plan.ptr)
        plan.ptr = None


def _sky_beam(plan, sky, beam):
    sky = _dev_tensor(sky, torch.complex128, plan.device, "sky", (plan.ncomp, plan.nalm))
    beam = _dev_tensor(beam, torch.complex128, plan.device, "beam", (plan.ncomp, plan.kmax + 1, plan.lmax + 1))
    return sky, beam


def synth_spin_maps(plan: Plan, sky, beam, maps=None):
    """Cube F_k(theta_r, phi_j), k = 0..kmax (Sect. 2.1, step 1)."""
    sky, beam = _sky_beam(plan, sky, beam)
    if maps is None:
        maps = torch.empty(plan.maps_shape(), dtype=plan.maps_dtype, device=sky.device)
    _dev_tensor(maps, plan.maps_dtype, plan.device, "maps", plan.maps_shape())
    plan._sync_stream()
    check(_lib.load().synth_spin_maps(plan.ptr, _ptr(sky), _ptr(beam), _ptr(maps)))
    return maps


def synth_spin_maps_multi(plan: Plan, sky, beam, maps=None):
    """Cubes of several skies that share one beam (FP32 plans; the l-contraction
    runs on the tensor cores).  sky: complex128 [nsky, ncomp, nalm]; returns
    complex64 maps [nsky, R, nphi, K+1]."""
    if plan.precision not in (SL_FP32, SL_TF32X3):
        raise ValueError("synth_spin_maps_multi needs an FP32 plan")
    if not isinstance(sky, torch.Tensor) or sky.dim() != 3:
        raise ValueError("sky must be a [nsky, ncomp, nalm] tensor")
    nsky = sky.shape[0]
    _dev_tensor(sky, torch.complex128, plan.device, "sky", (nsky, plan.ncomp, plan.nalm))
    beam = _dev_tensor(beam, torch.complex128, plan.device, "beam", (plan.ncomp, plan.kmax + 1, plan.lmax + 1))
    shape = (nsky,) + plan.maps_shape()
    if maps is None:
        maps = torch.empty(shape, dtype=torch.complex64, device=sky.device)
    _dev_tensor(maps, torch.complex64, plan.device, "maps", shape)
    plan._sync_stream()
    check(_lib.load().synth_spin_maps_multi(plan.ptr, int(nsky), _ptr(sky), _ptr(beam), _ptr(maps)))
    return maps


def _ptg(plan, theta, phi, psi):
    n = theta.numel()
    for name, t in (("theta", theta), ("phi", phi), ("psi", psi)):
        _dev_tensor(t, torch.float64, plan.device, name, (n,))
    return n


def interp_tod(plan: Plan, maps, theta, phi, psi, tod=None):
    """TOD at the pointings (Sect. 2.1, step 2 with conjugate-pair phases)."""
    _dev_tensor(maps, plan.maps_dtype, plan.device, "maps", plan.maps_shape())
    n = _ptg(plan, theta, phi, psi)
    if tod is None:
        tod = torch.empty(n, dtype=torch.float64, device=theta.device)
    _dev_tensor(tod, torch.float64, plan.device, "tod", (n,))
    plan._sync_stream()
    check(_lib.load().interp_tod(plan.ptr, _ptr(maps), _ptr(theta), _ptr(phi), _ptr(psi), n, _ptr(tod)))
    return tod


def convolve_tod(plan: Plan, sky, beam, theta, phi, psi, maps=None, tod=None):
    """The whole forward operator in one call (Sect. 2.1, steps 1 and 2): the cube
    and the TOD, as synth_spin_maps followed by interp_tod, with the pointing sort
    running beside the cube build.  Returns (maps, tod)."""
    sky, beam = _sky_beam(plan, sky, beam)
    if maps is None:
        maps = torch.empty(plan.maps_shape(), dtype=plan.maps_dtype, device=sky.device)
    _dev_tensor(maps, plan.maps_dtype, plan.device, "maps", plan.maps_shape())
    n = _ptg(plan, theta, phi, psi)
    if tod is None:
        tod = torch.empty(n, dtype=torch.float64, device=theta.device)
    _dev_tensor(tod, torch.float64, plan.device, "tod", (n,))
    plan._sync_stream()
    check(_lib.load().convolve_tod(plan.ptr, _ptr(sky), _ptr(beam), _ptr(maps), _ptr(theta), _ptr(phi), _ptr(psi),
                                   n, _ptr(tod)))
    return maps, tod


def synth_psi_cube(plan: Plan, maps, npsi: int, cube_psi=None):
    """psi-grid cube c(theta_r, phi_j, psi_n), psi_n = 2 pi n / npsi, from the spin
    cube (Sect. 2.1, step 2): float64 [R, nphi, npsi] for FP64/DF64 plans, float32
    for FP32 plans."""
    _dev_tensor(maps, plan.maps_dtype, plan.device, "maps", plan.maps_shape())
    rdt = torch.float64 if plan.maps_dtype == torch.complex128 else torch.float32
    shape = (plan.nrings, plan.nphi, int(npsi))
    if cube_psi is None:
        cube_psi = torch.empty(shape, dtype=rdt, device=maps.device)
    _dev_tensor(cube_psi, rdt, plan.device, "cube_psi", shape)
    plan._sync_stream()
    check(_lib.load().synth_psi_cube(plan.ptr, _ptr(maps), int(npsi), _ptr(cube_psi)))
    return cube_psi


def interp_tod_psi(plan: Plan, cube_psi, theta, phi, psi, tod=None):
    """TOD from the psi-grid cube: Lagrange in theta, phi and psi (plan's order)."""
    if cube_psi.dim() != 3:
        raise ValueError("cube_psi must be [nrings, nphi, npsi]")
    npsi = cube_psi.shape[2]
    rdt = torch.float64 if plan.maps_dtype == torch.complex128 else torch.float32
    _dev_tensor(cube_psi, rdt, plan.device, "cube_psi", (plan.nrings, plan.nphi, npsi))
    n = _ptg(plan, theta, phi, psi)
    if tod is None:
        tod = torch.empty(n, dtype=torch.float64, device=theta.device)
    _dev_tensor(tod, torch.float64, plan.device, "tod", (n,))
    plan._sync_stream()
    check(_lib.load().interp_tod_psi(plan.ptr, _ptr(cube_psi), int(npsi), _ptr(theta), _ptr(phi), _ptr(psi), n,
                                     _ptr(tod)))
    return tod


def quad_factor(nu_hz: float, T0: float) -> float:
    """The quadrupole factor of the orbital dipole (sl_quad_factor)."""
    out = ctypes.c_double(0.0)
    check(_lib.load().sl_quad_factor(float(nu_hz), float(T0), ctypes.byref(out)))
    return float(out.value)


def orbital_moments(plan: Plan, beam):
    """The nine moments [S_x, S_y, S_z, S_xx, S_yy, S_zz, S_xy, S_xz, S_yz] of the
    temperature beam (component 0 of the plan's beam layout), as numpy float64."""
    beam = _dev_tensor(beam, torch.complex128, plan.device, "beam", (plan.ncomp, plan.kmax + 1, plan.lmax + 1))
    S = np.zeros(9, dtype=np.float64)
    plan._sync_stream()
    check(_lib.load().sl_orbital_moments(plan.ptr, _ptr(beam), S.ctypes.data_as(ctypes.c_void_p)))
    return S


def orbital_dipole_tod(plan: Plan, beam, T0, q, theta, phi, psi, period_start, beta, subsample=20, tod=None,
                       accumulate=False):
    """Orbital dipole and quadrupole through the 4pi beam (Sect. 3.3, Eq. dipole_fast).

    period_start: nper + 1 sample offsets (host, 0 ... n); beta: [nper, 3] velocity / c
    per pointing period (host); subsample: rotation at every s-th sample of a period,
    natural cubic spline in between, the remainder exact (s = 1: exact everywhere)."""
    beam = _dev_tensor(beam, torch.complex128, plan.device, "beam", (plan.ncomp, plan.kmax + 1, plan.lmax + 1))
    n = _ptg(plan, theta, phi, psi)
    starts = np.ascontiguousarray(np.asarray(period_start, dtype=np.int64))
    bet = np.ascontiguousarray(np.asarray(beta, dtype=np.float64).reshape(-1, 3))
    nper = starts.size - 1
    if nper < 1 or bet.shape[0] != nper:
        raise ValueError("period_start must have nper + 1 entries and beta nper rows")
    if tod is None:
        tod = torch.empty(n, dtype=torch.float64, device=theta.device)
    _dev_tensor(tod, torch.float64, plan.device, "tod", (n,))
    plan._sync_stream()
    check(_lib.load().orbital_dipole_tod(plan.ptr, _ptr(beam), float(T0), float(q), _ptr(theta), _ptr(phi),
                                         _ptr(psi), n, starts.ctypes.data_as(ctypes.c_void_p),
                                         bet.ctypes.data_as(ctypes.c_void_p), nper, int(subsample), _ptr(tod),
                                         1 if accumulate else 0))
    return tod


def adjoint_tod(plan: Plan, theta, phi, psi, tod, sky, beam, sky_grad=None, beam_grad=None,
                accumulate=False, want_sky=True, want_beam=True):
    """Gradients of sum_i tod_i c_i w.r.t. the packed sky and beam (d/dRe + i d/dIm)."""
    sky, beam = _sky_beam(plan, sky, beam)
    n = _ptg(plan, theta, phi, psi)
    _dev_tensor(tod, torch.float64, plan.device, "tod", (n,))
    if want_sky and sky_grad is None:
        sky_grad = torch.zeros_like(sky)
    if want_beam and beam_grad is None:
        beam_grad = torch.zeros_like(beam)
    if sky_grad is not None:
        _dev_tensor(sky_grad, torch.complex128, plan.device, "sky_grad", tuple(sky.shape))
    if beam_grad is not None:
        _dev_tensor(beam_grad, torch.complex128, plan.device, "beam_grad", tuple(beam.shape))
    plan._sync_stream()
    check(_lib.load().adjoint_tod(plan.ptr, _ptr(theta), _ptr(phi), _ptr(psi), _ptr(tod), n, _ptr(sky),
                                  _ptr(beam), _ptr(sky_grad) if sky_grad is not None else None,
                                  _ptr(beam_grad) if beam_grad is not None else None, int(bool(accumulate))))
    return sky_grad, beam_grad


def adjoint_tod_sharded(plan: Plan, theta, phi, psi, tod, sky, beam, sky_grad=None, beam_grad=None,
                        group=None):
    """Adjoint of a TOD whose samples are split over the ranks of a process group
    (every rank holds the whole cube and its own stretch of pointings; the TOD is
    linear in the cube, Sect. 2.1): the local adjoint_tod, then one sum all-reduce
    of each gradient, so that every rank holds the gradients of the whole TOD.
    Without an initialised process group, or with one rank, it is adjoint_tod."""
    import torch.distributed as dist
    gs, gb = adjoint_tod(plan, theta, phi, psi, tod, sky, beam, sky_grad, beam_grad)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        for g in (gs, gb):
            dist.all_reduce(torch.view_as_real(g), op=dist.ReduceOp.SUM, group=group)
    return gs, gb


def adjoint_interp(plan: Plan, theta, phi, psi, tod, maps_bar=None):
    """Transpose of interp_tod: the adjoint cube [R, nphi, K+1] complex128."""
    n = _ptg(plan, theta, phi, psi)
    _dev_tensor(tod, torch.float64, plan.device, "tod", (n,))
    if maps_bar is None:
        maps_bar = torch.empty(plan.maps_shape(), dtype=torch.complex128, device=theta.device)
    _dev_tensor(maps_bar, torch.complex128, plan.device, "maps_bar", plan.maps_shape())
    plan._sync_stream()
    check(_lib.load().adjoint_interp(plan.ptr, _ptr(theta), _ptr(phi), _ptr(psi), _ptr(tod), n, _ptr(maps_bar)))
    return maps_bar


def adjoint_synth(plan: Plan, maps_bar, sky, beam, sky_grad=None, beam_grad=None, accumulate=False):
    """Transpose of synth_spin_maps followed by the sky x beam products."""
    sky, beam = _sky_beam(plan, sky, beam)
    _dev_tensor(maps_bar, torch.complex128, plan.device, "maps_bar", plan.maps_shape())
    if sky_grad is None:
        sky_grad = torch.zeros_like(sky)
    if beam_grad is None:
        beam_grad = torch.zeros_like(beam)
    plan._sync_stream()
    check(_lib.load().adjoint_synth(plan.ptr, _ptr(maps_bar), _ptr(sky), _ptr(beam), _ptr(sky_grad),
                                    _ptr(beam_grad), int(bool(accumulate))))
    return sky_grad, beam_grad


def tod_from_host(plan: Plan, sky, beam, theta, phi, psi, chunks: int = 8, out=None):
    """End-to-end call from host arrays (convolve_tod_host): the library copies
    the inputs to the device, builds the cube, uploads the pointings in `chunks`
    pieces while the cube is built, interpolates each piece as soon as it has
    arrived and copies its TOD back into `out` (a host float64 tensor; a pinned
    one is allocated when None), and returns `out` when all of it is there.
    Pinned host tensors let the copies overlap the computation; reusing `out`
    across calls avoids a pinned allocation per call."""
    def host(x, dtype, name, shape):
        t = x if isinstance(x, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(x))
        if t.device.type != "cpu" or t.dtype != dtype or tuple(t.shape) != tuple(shape) or not t.is_contiguous():
            raise ValueError("%s must be a contiguous host %s array of shape %s" % (name, dtype, tuple(shape)))
        return t
    n = int(theta.numel() if isinstance(theta, torch.Tensor) else np.size(theta))
    sky = host(sky, torch.complex128, "sky", (plan.ncomp, plan.nalm))
    beam = host(beam, torch.complex128, "beam", (plan.ncomp, plan.kmax + 1, plan.lmax + 1))
    th, ph, ps = (host(x, torch.float64, nm, (n,)) for x, nm in ((theta, "theta"), (phi, "phi"), (psi, "psi")))
    if out is None:
        out = torch.empty(n, dtype=torch.float64, pin_memory=True)
    host(out, torch.float64, "out", (n,))
    plan._sync_stream()
    check(_lib.load().convolve_tod_host(plan.ptr, _ptr(sky), _ptr(beam), _ptr(th), _ptr(ph), _ptr(ps), n,
                                        int(max(1, min(int(chunks), 64))), _ptr(out)))
    return out


class Batch:
    """Owns one sl_batch*: the forward path of several detectors as one CUDA
    graph.  Holds references to every item's tensors and plan, whose buffers
    the graph reads and writes on each run."""

    def __init__(self, ptr, items, device):
        self.ptr = ptr
        self.items = items
        self.device = device

    def run(self):
        check(_lib.load().sl_batch_run(self.ptr))

    def sync(self):
        """Waits for the batch's stream; raises on a device fault or an expired
        bounded wait (sl_batch_sync)."""
        check(_lib.load().sl_batch_sync(self.ptr))

    def info(self):
        out = _lib.BatchInfo()
        check(_lib.load().sl_batch_get_info(self.ptr, ctypes.byref(out)))
        return {f: getattr(out, f) for f, _ in out._fields_}

    def __del__(self):
        try:
            sl_batch_destroy(self)
        except Exception:
            pass


def sl_batch_create(items, autotune: bool = False, persistent: bool = False) -> Batch:
    """items: sequence of dicts with keys plan, sky, beam, maps, theta, phi, psi, tod
    (device tensors in the layouts of synth_spin_maps and interp_tod, one plan per
    item).  Captured on the current torch stream of the first plan's device.
    persistent: the persistent form (SL_BATCH_PERSISTENT; SL_FP32 plans)."""
    lib = _lib.load()
    items = [dict(it) for it in items]
    if not items:
        raise ValueError("a batch needs at least one item")
    device = items[0]["plan"].device
    arr = (_lib.BatchItem * len(items))()
    for i, it in enumerate(items):
        plan = it["plan"]
        sky, beam = _sky_beam(plan, it["sky"], it["beam"])
        _dev_tensor(it["maps"], plan.maps_dtype, plan.device, "maps", plan.maps_shape())
        n = _ptg(plan, it["theta"], it["phi"], it["psi"])
        _dev_tensor(it["tod"], torch.float64, plan.device, "tod", (n,))
        arr[i] = _lib.BatchItem(plan=plan.ptr, sky=_ptr(sky), beam=_ptr(beam), maps=_ptr(it["maps"]),
                                theta=_ptr(it["theta"]), phi=_ptr(it["phi"]), psi=_ptr(it["psi"]), n=n,
                                tod=_ptr(it["tod"]))
    stream = torch.cuda.current_stream(device).cuda_stream
    out = ctypes.c_void_p()
    flags = (_lib.SL_BATCH_AUTOTUNE if autotune else 0) | (_lib.SL_BATCH_PERSISTENT if persistent else 0)
    check(lib.sl_batch_create(ctypes.byref(out), arr, len(items), ctypes.c_void_p(stream), flags))
    return Batch(out, items, device)


def sl_batch_run(batch: Batch) -> None:
    batch.run()


def sl_batch_destroy(batch: Batch) -> None:
    if batch is not None and batch.ptr:
        _lib.load().sl_batch_destroy(batch.ptr)
        batch.ptr = None


def measure_alu_peak(kind: str = "fp64", device: int = 0) -> float:
    """Measured arithmetic peak of ``device`` in flops/s (sl_measure_alu_peak):
    kind "fp64", "fp32" or "fp32x2" (packed two-lane FP32 multiply-add)."""
    code = {"fp64": 0, "fp32": 1, "fp32x2": 2}[kind]
    out = ctypes.c_double(0.0)
    check(_lib.load().sl_measure_alu_peak(int(device), code, ctypes.byref(out)))
    return float(out.value)
