"""GB300-native ACCORD-FBS (HP-ACCORD, arXiv 2412.11554).

The solver lives in the CUDA library libaccord.so (C ABI in include/accord.h);
this package holds its sources (csrc/), the build step and the ctypes binding.
"""
from .accord import (  # noqa: F401
    AccordError,
    FitStats,
    accord_default_opts,
    accord_device_check,
    accord_fit,
    accord_fit_rows,
    accord_fit_rows_workspace_bytes,
    accord_grad_x,
    accord_postprocess,
    accord_to_csr,
    accord_dloss_dloglam,
    accord_path,
    accord_path_workspace_bytes,
    PathResult,
    accord_refit,
    accord_grad,
    accord_last_error,
    accord_loss,
    accord_loss_f64_noalloc,
    accord_status_string,
    accord_test_wait_limit,
    accord_workspace_bytes,
    dist_exchange,
    load_library,
)
from .autograd import SmoothLoss, smooth_loss  # noqa: F401,E402
