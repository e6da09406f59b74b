"""ffgpu: exact fgemm / ftrsm / LQUP over Z/pZ on GB300 (sm_103a).

The computation lives in the CUDA library ``libffgpu.so`` (C ABI declared in
``include/ffgpu.h``); ``ffgpu`` is its thin Python binding.  ``workloads``
draws the seeded synthetic inputs.
"""
from .ffgpu import (FFGPUError, fgemm, fgemm_noalloc_ptr, fgemm_plan, fgemm_ptr, fgemm_workspace_size, fgemm_ws, ftrsm,
                    ftrsm_cascade_params,
                    fgemm_batched, batched_descs, fgemm_batched_descs, BatchedPlan, fgemm_multimod, fgemm_multimod_batched, multimod_descs, fgemm_multimod_batched_descs, fgemm_ex, Server, selftest_wait_timeout,
                    autotune, autotune_lookup, autotune_save, autotune_load, autotune_clear, fgemm_auto, autotune_batched,
                    profile_enable, profile_read, lqup, rank, det, inverse, set_small_threshold, get_small_threshold,
                    winograd_unreduced_kmax, peak_probe,
                    last_device_error, lib, release_workspaces, status_string, version)

__all__ = ["FFGPUError", "ftrsm_cascade_params", "fgemm", "fgemm_noalloc_ptr", "fgemm_plan", "fgemm_ptr", "fgemm_workspace_size", "fgemm_ws", "ftrsm", "fgemm_batched", "batched_descs", "fgemm_batched_descs", "BatchedPlan", "fgemm_multimod", "fgemm_multimod_batched", "multimod_descs", "fgemm_multimod_batched_descs", "fgemm_ex", "Server", "selftest_wait_timeout", "autotune", "autotune_lookup", "autotune_save",
           "autotune_load", "autotune_clear", "fgemm_auto", "autotune_batched", "lqup", "rank", "det", "inverse", "set_small_threshold",
           "get_small_threshold", "winograd_unreduced_kmax", "peak_probe",
           "last_device_error", "lib", "release_workspaces", "status_string", "version"]
