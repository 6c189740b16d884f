"""GB300-native higher-order DMAS photoacoustic beamformer.

The compute path is the CUDA library built from ``csrc/`` (C ABI in
``include/pa_hodmas.h``); this package only marshals arguments to it.
PyTorch, when used by callers, provides device memory and streams.
"""

from ._native import (  # noqa: F401
    PA_OUT_DAS,
    PA_OUT_DMAS,
    PA_OUT_HODMAS,
    PA_RF_BF16,
    PA_RF_F16,
    PA_RF_F32,
    PA_STAGE_ENV,
    PA_STAGE_LOG,
    PA_STAGE_RAW,
    PAError,
    Plan,
    PlanDesc,
    footprint,
    load,
    make_desc,
    make_grid,
    pipe_schedule,
    pipe_time,
)
from .torch_api import beamform, beamform_host, image_metrics  # noqa: F401
