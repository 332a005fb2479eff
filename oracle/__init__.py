"""FP64 CPU oracle for Shifted-Fresnel diffraction.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers.  The product path under
``paper_1001_4309_gb300`` never imports this package, and this package
imports nothing from it.

Functions and the passages they follow (Section 2.1 of the paper):

* ``forward``    -- Eqs. 1-4: the Shifted-Fresnel sum, evaluated as the plain
                    discretised Fresnel sum u1 = C Ky u0 Kx^T (no FFT).
* ``intensity``  -- Eq. 5: I = |u1|^2.
* ``phase``      -- the phase image atan2(Im u1, Re u1) in (-pi, pi].
* ``adjoint``    -- the conjugate transpose of ``forward`` (not in the paper;
                    pinned by the dot-product identity and brute force).
* ``forward_dz`` -- d u1 / d z of ``forward`` (not in the paper; pinned by
                    finite differences of ``forward``).
"""

from .driver import (  # noqa: F401
    build,
    forward,
    adjoint,
    forward_dz,
    intensity,
    phase,
    max_threads,
    OracleLib,
)
