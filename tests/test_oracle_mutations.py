"""The oracle's pins catch plausible mistakes (CPU only).

Each case plants one mistake in a temporary copy of the oracle's C source (a
flipped sign, a dropped term, a wrong index origin, a swapped operand),
compiles it, and checks that at least one pin rejects the mutant.  The real
oracle is never modified.
"""

import os

import numpy as np
import pytest

from oracle.driver import OracleLib, compile_oracle, _SRC
from synth import view, random_field, WAVELENGTH, PITCH
import test_oracle_pins as pins

MUTATIONS = {
    "kernel_sign": ("cexp(I * (M_PI * d * d", "cexp(-I * (M_PI * d * d"),
    "kernel_sum_not_difference": ("double d = x1 - x0;", "double d = x1 + x0;"),
    "index_origin": ("(double)(m - n / 2) * p", "(double)(m - (n - 1) / 2) * p"),
    "offset_sign": ("return o + (double)", "return -o + (double)"),
    "dropped_prefactor_denominator": ("/ (I * v->wavelength * v->z)", ""),
    "x_pitch_for_y": ("coord(n0, ny0, v->py0, v->oy0)", "coord(n0, ny0, v->px0, v->oy0)"),
    "output_pitch_swapped": ("coord(m1_begin + c, v->nx1, v->px1, v->ox1)",
                             "coord(m1_begin + c, v->nx1, v->px0, v->ox1)"),
    "adjoint_missing_conj": ("conj(Kx[(size_t)m1 * nx0 + m0])", "Kx[(size_t)m1 * nx0 + m0]"),
    "adjoint_prefactor_not_conjugated": ("const double complex Cc = conj(prefactor(v));",
                                         "const double complex Cc = prefactor(v);"),
    "dz_missing_y_term": ("+ Dy[(size_t)n1 * ny0 + n0] * tA[(size_t)n0 * nx1 + m1]", ""),
}


def battery(orc):
    """Return the names of the pins this oracle build fails."""
    failed = []
    for i, case in enumerate(pins.TINY_CASES[1:3]):
        nx0, ny0, nx1, ny1, z, p0, p1, o0, o1 = case
        v = view(WAVELENGTH, z, p0, p1, o0, o1, (nx0, ny0), (nx1, ny1))
        u0 = random_field(ny0, nx0, seed=100 + i)
        if pins.rel_l2(orc.forward(u0, v), pins.brute_force(u0, v)) > 1e-10:
            failed.append(f"brute_force[{i}]")
        if pins.rel_l2(orc.forward(u0, v), pins.paper_equations_1_to_4(u0, v)) > 1e-10:
            failed.append(f"paper_eqs[{i}]")
        g = random_field(ny1, nx1, seed=200 + i)
        lhs, rhs = np.vdot(g, orc.forward(u0, v)), np.vdot(orc.adjoint(g, v), u0)
        if abs(lhs - rhs) > 1e-10 * abs(lhs):
            failed.append(f"adjoint_dot[{i}]")
        h = 1e-9 * z
        fd = (orc.forward(u0, dict(v, z=z + h)) - orc.forward(u0, dict(v, z=z - h))) / (2 * h)
        if pins.rel_l2(orc.forward_dz(u0, v), fd) > 1e-5:
            failed.append(f"dz_fd[{i}]")
    return failed


def test_unmutated_oracle_passes_battery(tmp_path):
    orc = OracleLib()
    assert battery(orc) == []


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_mutant_is_caught(name, tmp_path):
    old, new = MUTATIONS[name]
    with open(_SRC) as f:
        src = f.read()
    assert src.count(old) >= 1, f"mutation anchor for {name} not found"
    mutated = tmp_path / "mutant.c"
    mutated.write_text(src.replace(old, new))
    lib = compile_oracle(str(mutated), str(tmp_path / "libmutant.so"))
    orc = OracleLib(lib)
    assert battery(orc), f"mutation {name} was not caught by any pin"
