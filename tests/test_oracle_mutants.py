"""Plant plausible mistakes in a copy of the oracle and check the pins catch
each one (dropped term, wrong sign, conjugate on the wrong side, transposed
operand, wrong index, dropped gain).  The copies are built in a temporary
directory; the committed oracle is untouched."""
import os
import shutil
import subprocess

import pytest

import oracle
from tests import oracle_pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "xc_oracle.c")

# (name, text to find, replacement, occurrence index to replace)
MUTANTS = [
    ("drop_imag_product_in_re", "re += ar * br + ai * bi;", "re += ar * br;", 0),
    ("wrong_sign_im", "im += ai * br - ar * bi;", "im += ai * br + ar * bi;", 0),
    ("conj_on_row", "im += ai * br - ar * bi;", "im += ar * bi - ai * br;", 0),
    ("transposed_pol", "in_off(t, f, s2, p2, F, N, P);", "in_off(t, f, s2, p1, F, N, P);", 0),
    ("wrong_baseline_index", "return s1 * (s1 + 1) / 2 + s2;", "return s1 * (s1 - 1) / 2 + s2;", 0),
    ("off_by_one_time", "for (int64_t t = 0; t < T; ++t) {", "for (int64_t t = 1; t < T; ++t) {", 0),
    ("float_drop_gain_phase", "const double ar = gar * a[0] - gai * a[1]", "const double ar = gar * a[0]", 0),
    ("float_wrong_sign_im", "im += ai * br - ar * bi;", "im += ai * br + ar * bi;", 1),
    ("adjoint_no_hermitian_part", "H[(b * n + a) * 2 + 1] -= go[1];", "H[(b * n + a) * 2 + 1] += go[1];", 0),
    ("adjoint_grad_x_no_conj", "gx[1] = gr * gyi - gi * gyr;", "gx[1] = gr * gyi + gi * gyr;", 0),
    ("adjoint_grad_g_conj", "+= x[0] * gyi - x[1] * gyr;", "+= x[0] * gyi + x[1] * gyr;", 0),
    ("fengine_exponent_sign", "wi[j] = -sin(", "wi[j] = sin(", 0),
    ("fengine_block_offset", "in + (a * T * F + t * F) * 2", "in + (a * T * F + t) * 2", 0),
    ("fengine_dropped_scale", "out[(o * n + a) * 2] = scale * re;", "out[(o * n + a) * 2] = re;", 0),
    ("fengine_station_pol_swapped", "in + (a * T * F + t * F) * 2",
     "in + (((a % P) * N + a / P) * T * F + t * F) * 2", 0),
    ("fengine_phase_index", "const int64_t j = (f * m) % F;", "const int64_t j = (f + m) % F;", 0),
    ("pfb_time_direction", "(t + p) * F + m) * 2;", "(t + ntaps - 1 - p) * F + m) * 2;", 0),
    ("pfb_tap_index", "yr += h[(int64_t)p * F + m] * x[0];", "yr += h[(int64_t)m * ntaps + p] * x[0];", 0),
    ("pfb_dropped_imag_tap", "yi += h[(int64_t)p * F + m] * x[1];", "yi += x[1];", 0),
]


def _replace_nth(text, old, new, n):
    pos = -1
    for _ in range(n + 1):
        pos = text.find(old, pos + 1)
        assert pos >= 0, "mutation site not found: %r" % old
    return text[:pos] + new + text[pos + len(old):]


@pytest.mark.parametrize("name,old,new,nth", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_mutant(name, old, new, nth, tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    with open(SRC) as fh:
        text = fh.read()
    mutated = _replace_nth(text, old, new, nth)
    assert mutated != text
    src = tmp_path / ("oracle_%s.c" % name)
    src.write_text(mutated)
    so = tmp_path / ("liboracle_%s.so" % name)
    subprocess.run(["gcc", "-O1", "-fopenmp", "-shared", "-fPIC", "-std=c11", "-o", str(so),
                    str(src), "-lm"], check=True)
    lib = oracle.load(str(so))
    caught = []
    for pin in oracle_pins.ALL_PINS:
        try:
            pin(lib)
        except AssertionError:
            caught.append(pin.__name__)
    assert caught, "no pin caught mutant %s" % name
