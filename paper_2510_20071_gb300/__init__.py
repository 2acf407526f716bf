"""GB300 (sm_103a) FIBAR: filter-based reconstruction of images from events.

Python binding of the C ABI in ``include/fibar.h`` (``lib/libfibar.so``).  The binding
only marshals arguments; every step of the reconstruction runs in the library's CUDA
kernels.  There is no CPU fallback: importing the binding without the built library or
without a CUDA device raises.
"""
from .binding import (  # noqa: F401
    FIBAR_OK, FIBAR_EINVAL, FIBAR_ENOMEM, FIBAR_EORDER, FIBAR_ECUDA, FIBAR_ETIMEOUT,
    FibarError, FibarParams, FibarStats, FibarStateView, Fibar, load_library, library_path,
    fibar_default_params, fibar_create, fibar_push_events, fibar_readout, fibar_flush,
    fibar_debug_state, fibar_stats, fibar_set_timing, fibar_stage_times, fibar_last_error,
    fibar_destroy, fibar_queue_counts_noalloc, fibar_readout_batch, fibar_memory_bytes,
    memory_bytes, readout_batch, relative_thresholds, fibar_relative_thresholds, fibar_set_pixel_gain,
    EXPORTED, STAGES, FibarStageTimes, FIBAR_FILL_NPARAMS, fill_forward, fibar_fill_set_weights,
    fibar_fill_features, fibar_fill_forward, fibar_fill_train_step, fibar_readout_host_async, fibar_wait,
    fibar_set_grid_share, fibar_push_batch, push_batch, Group, FibarGroupStats, fibar_group_create,
    fibar_group_readout, fibar_group_latency, fibar_group_stats, fibar_group_last_error, fibar_group_destroy,
    fibar_group_join,
)
