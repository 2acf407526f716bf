"""FIBAR FP64 oracle - test infrastructure only.

Plain CPU restatement of the paper's per-event procedure (C source in
``fibar_oracle.c``) plus a ctypes wrapper.  Only the tests, the smoke check and the
benchmark's CPU-baseline leg may import this package; the CUDA library never does.
"""
from .oracle import (  # noqa: F401
    Oracle, build, coefficients, blur_image, default_params, lib_path, relative_thresholds,
)
