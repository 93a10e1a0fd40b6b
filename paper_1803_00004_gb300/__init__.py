"""GB300-native joint-acceleration bilateral filter (Dai, Yuan, Zhang).

The filter runs in libbf.so (hand-written CUDA for sm_103a behind the C ABI of
include/bf.h); this package is its thin Python binding plus the seeded input
generators in ``synth``.  Importing the package does not load the library; the
first call does, and raises if it has not been built.
"""
from ._binding import (BFError, Cache, Plan, Server, bf_coeffs, bf_exact, bf_exact_lut, bf_filter, bf_filter_batch,  # noqa: F401
                       bf_filter_host,
                       bf_autotune_batch,
                       bf_version,
                       bf_launch_info, bf_autotune, bf_autotune_group, bf_autotune_image, bf_launch_candidates, bf_set_launch,
                       bf_debug_fail_launches, bf_debug_range_checks, bf_fp32_peak, desc, lib, LIB_PATH, EXPORTS)
from ._binding import (KERNEL_GAUSSIAN, KERNEL_EXPONENTIAL, KERNEL_BOX, RANGE_TRUNCATED_MIN_PERIOD,  # noqa: F401
                       RANGE_UNTRUNCATED_FULL, RANGE_PAPER_3D, SERIES_COSINE, SERIES_HAAR, PREC_FP32, PREC_BF16,
                       PREC_FP16)
from ._binding import (OK, ERR_INVALID_ARG, ERR_UNSUPPORTED, ERR_OOM, ERR_CUDA, ERR_ADMISSION, ERR_TIMEOUT,  # noqa: F401
                       ERR_DEVICE_TIMEOUT, ERR_RANGE, ERR_NO_DEVICE, ERR_NOT_FOUND, ERR_CANCELLED, ERR_SCRATCH,
                       MEM_DEVICE, MEM_HOST)
