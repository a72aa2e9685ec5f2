"""GB300-native spin-harmonic sidelobe convolution (Galloway et al., BeyondPlanck
VIII, arXiv:2201.03478, Sect. 2.1): cube build, TOD interpolation and adjoint,
implemented as sm_103a CUDA kernels behind the C ABI in include/sidelobe.h.
"""
from .binding import (Batch, Plan, adjoint_interp, adjoint_synth, adjoint_tod, adjoint_tod_sharded, convolve_tod, interp_tod,
                      orbital_dipole_tod,
                      orbital_moments, plan_destroy, quad_factor, sidelobe_plan_create, sl_batch_create, sl_batch_destroy,
                      sl_batch_run, synth_spin_maps, synth_spin_maps_multi, tod_from_host, synth_psi_cube,
                      interp_tod_psi, measure_alu_peak)
from ._lib import SL_DF64, SL_FP32, SL_FP64, SL_TF32X3, SidelobeError
from .autograd import SidelobeConvolution, sidelobe_tod

__all__ = ["Plan", "sidelobe_plan_create", "synth_spin_maps", "interp_tod", "convolve_tod", "adjoint_tod", "adjoint_tod_sharded",
           "adjoint_interp",
           "adjoint_synth", "plan_destroy", "tod_from_host", "SidelobeError", "SL_FP64", "SL_FP32", "SL_DF64", "SL_TF32X3",
           "SidelobeConvolution", "sidelobe_tod", "Batch", "sl_batch_create", "sl_batch_run", "sl_batch_destroy",
           "synth_spin_maps_multi", "orbital_moments", "orbital_dipole_tod", "quad_factor", "synth_psi_cube", "interp_tod_psi",
           "measure_alu_peak"]
