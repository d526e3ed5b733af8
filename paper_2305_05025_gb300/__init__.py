"""GB300 (sm_103a) coupled lattice-Boltzmann / molecular-dynamics step.

After Lauricella et al., "Multiscale Hybrid Modeling of Proteins in Solvent"
(arXiv 2305.05025), Sec. 2.2. The compute runs in ``liblbmd.so`` (CUDA kernels
behind the C ABI of ``include/lbmd.h``); ``lbmd`` is its ctypes binding with
the same call names, ``synth`` the seeded synthetic inputs.
"""
from .lbmd import (LBMDError, OBS_DRAG_X, OBS_RG2, lbmd_analysis_begin, lbmd_analysis_frame, lbmd_analysis_result,
                   lbmd_backward, lbmd_backward_state, lbmd_cell_list, lbmd_check, lbmd_create, lbmd_destroy, lbmd_get_fields,
                   lbmd_get_stats, lbmd_last_error, lbmd_load_state, lbmd_params, lbmd_save_state, lbmd_set_charges, lbmd_set_md_timing_events,
                   lbmd_set_physics, lbmd_set_reinterpolation, lbmd_set_state, lbmd_set_thermal, lbmd_set_timing_events, lbmd_step,
                   lbmd_version, params_from)

__all__ = ["LBMDError", "OBS_DRAG_X", "OBS_RG2", "lbmd_analysis_begin", "lbmd_analysis_frame",
           "lbmd_analysis_result", "lbmd_backward", "lbmd_backward_state", "lbmd_cell_list", "lbmd_check", "lbmd_create",
           "lbmd_destroy", "lbmd_get_fields", "lbmd_get_stats", "lbmd_last_error", "lbmd_load_state", "lbmd_params",
           "lbmd_save_state",
           "lbmd_set_charges", "lbmd_set_md_timing_events", "lbmd_set_physics", "lbmd_set_reinterpolation",
           "lbmd_set_state",
           "lbmd_set_thermal", "lbmd_set_timing_events", "lbmd_step", "lbmd_version", "params_from"]
