"""LinMin fully constrained unmixing on GB300 (sm_103a).

The product is the C-ABI library ``liblinmin.so`` (include/linmin.h) built
from ``csrc/``; ``linmin`` is its ctypes binding.
"""
from .linmin import (EXPORTED, LinminError, Server, Unmixer, library_path, linmin_create,  # noqa: F401
                     linmin_default_options, linmin_destroy, linmin_last_error,
                     linmin_options, linmin_phase_times, linmin_phase_times_at, linmin_unmix,
                     linmin_unmix_cov, linmin_unmix_batch, linmin_unmix_noalloc, linmin_noalloc_scratch_bytes, linmin_fp32_peak, linmin_live_allocations,
                     linmin_autotune, linmin_get_lanes, linmin_last_launches, linmin_set_lanes,
                     linmin_version,
                     linmin_server_create, linmin_server_default_options,
                     linmin_server_destroy, linmin_server_get_stats, linmin_server_handle_bytes, linmin_server_last_error,
                     linmin_server_poll, linmin_server_submit, linmin_server_wait,
                     linmin_wait, load,
                     linmin_detect, linmin_extra_spectra, linmin_threshold_stats,
                     linmin_thresholds, linmin_detection, linmin_threshold_sums,
                     detection_summary, threshold_sums, linmin_autofit,
                     linmin_second_pass, linmin_unmix_masked)
