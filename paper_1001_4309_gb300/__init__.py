"""GB300 (sm_103a) Shifted-Fresnel multi-view reconstruction.

The computation lives in the CUDA library built from ``csrc/`` (C ABI in
``include/shifted_fresnel.h``); ``binding`` marshals arguments to it.
"""

from .binding import (  # noqa: F401
    ShiftedFresnel,
    SFError,
    sf_view,
    load,
    make_view,
    shifted_fresnel_plan,
    shifted_fresnel_execute,
    shifted_fresnel_execute_static,
    shifted_fresnel_destroy,
    shifted_fresnel_adjoint,
    shifted_fresnel_execute_batch,
    shifted_fresnel_batch_status,
    shifted_fresnel_strerror,
    shifted_fresnel_plan_query,
    shifted_fresnel_plan_update,
    shifted_fresnel_intensity_loss,
    shifted_fresnel_kernel_launches,
    shifted_fresnel_set_profile_events,
    shifted_fresnel_fft_length,
    SF_OK, SF_ERR_INVALID_ARG, SF_ERR_UNSUPPORTED_SIZE, SF_ERR_CUDA, SF_ERR_OOM,
    SF_ERR_TIMEOUT, SF_ERR_DEVICE_MISMATCH,
    SF_OUT_INTENSITY, SF_OUT_PHASE, SF_NO_PREFACTOR, SF_IN_COMPLEX, SF_PREC_FP32, SF_PREC_FP16TC, SF_PREC_BF16TC,
    SF_MAX_CONV_LENGTH,
)
