"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle runs.

This package generates holograms, object fields and view parameter sets.  It
contains none of the Shifted-Fresnel arithmetic: the in-line holograms are
recorded with the band-limited angular-spectrum transfer function (a different
diffraction model), so neither the CUDA path nor the oracle can leak into the
inputs they are compared on.
"""

from .gabor import (  # noqa: F401
    WAVELENGTH,
    PITCH,
    asm_propagate,
    bars_disks_object,
    target_blobs_object,
    gabor_hologram,
    random_field,
    view,
    config_c1,
    config_c2,
    config_c3,
    config_c4,
    config_c5,
    config_c5_inline,
    retrieval_object,
    poisson_intensity,
)
