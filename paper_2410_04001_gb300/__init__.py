"""GB300 (sm_103a) FastLRNR / sparse physics-informed backpropagation library.

The compute path is ``liblrnr.so`` (hand-written CUDA, C ABI in
``include/lrnr.h``); ``binding`` exposes its entry points under the same names,
``autograd`` wraps the adjoint as a ``torch.autograd.Function``.
"""
from . import binding  # noqa: F401
from .binding import (DeviceBatch, LrnrError, Model, fastlrnr_select_rows, lrnr_build,  # noqa: F401
                      lrnr_destroy, lrnr_last_device_status, lrnr_model_info, lrnr_reserve,
                      lrnr_residual, lrnr_residual_grad, lrnr_snapshots, lrnr_status_string,
                      lrnr_residual_grad_noalloc, lrnr_set_tuning, lrnr_timing, lrnr_timing_read, spinprop_step,
                      lrnr_measure_peaks, lrnr_set_wait_limit, lrnr_pod, lrnr_deim_rows,
                      fastlrnr_select_rows_deim, lrnr_adam_update, lrnr_copy_pinned)
