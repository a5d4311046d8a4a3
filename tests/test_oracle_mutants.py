"""The oracle's pins must reject plausible mistakes.

Each case plants one mistake in a copy of the oracle's C source (a flipped sign, a
dropped term, a transposed operand, an off-by-one), compiles it on the CPU, and runs
the pin suite against it in a subprocess; the suite has to fail.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "of_oracle.c")

MUTANTS = {
    "gradient_sign": ("ofo_bilinear(I2, H, W, px + 1.0, py) - ofo_bilinear(I2, H, W, px - 1.0, py)",
                      "ofo_bilinear(I2, H, W, px - 1.0, py) - ofo_bilinear(I2, H, W, px + 1.0, py)"),
    "dropped_linearisation_term": (" + gx[k] * u[k]", ""),
    "residual_sign": ("double e = P1[k] - Iw[k]", "double e = Iw[k] - P1[k]"),
    "i1grad_residual_sign": ("double et = P1[k] - Iw[k]", "double et = Iw[k] - P1[k]"),
    "transposed_solve": ("*xu = (c * d0 - b * e0) / det;", "*xu = (a * d0 - b * e0) / det;"),
    "wrong_product": ("p[1][k] = gx[k] * gy[k];", "p[1][k] = gx[k] * gx[k];"),
    "window_off_by_one": ("for (int dx = -r; dx <= r; ++dx)", "for (int dx = -r; dx < r; ++dx)"),
    "pyramid_normalisation": ("s / 256.0", "s / 255.0"),
    "upsample_not_doubled": ("2.0 * ofo_bilinear(fc, Hc, Wc, 0.5 * x, 0.5 * y)",
                             "ofo_bilinear(fc, Hc, Wc, 0.5 * x, 0.5 * y)"),
    "bilinear_weights_swapped": ("(1.0 - ax) * img[(size_t)y0 * W + x0] + ax * img[(size_t)y0 * W + x1]",
                                 "ax * img[(size_t)y0 * W + x0] + (1.0 - ax) * img[(size_t)y0 * W + x1]"),
    "bilinear_row_not_interpolated": ("const int y1 = y0 + 1 < H ? y0 + 1 : H - 1;", "const int y1 = y0;"),
    "i1grad_dropped_linearisation_term": (" + g1x[k] * u[k]", ""),
    "i1grad_gradient_sign": ("g1x[k] = (P1[(size_t)y * W + xp] - P1[(size_t)y * W + xm]) / 2.0;",
                             "g1x[k] = (P1[(size_t)y * W + xm] - P1[(size_t)y * W + xp]) / 2.0;"),
    "i1grad_gradient_rows_swapped": ("g1y[k] = (P1[(size_t)yp * W + x] - P1[(size_t)ym * W + x]) / 2.0;",
                                     "g1y[k] = (P1[(size_t)y * W + xp] - P1[(size_t)y * W + xm]) / 2.0;"),
    "guard_inverted": ("if (det <= OFO_SINGULAR_EPS * tr * tr) return 0;",
                       "if (det > OFO_SINGULAR_EPS * tr * tr) return 0;"),
    "second_numerator_wrong_entry": ("*xv = (a * e0 - b * d0) / det;", "*xv = (c * e0 - b * d0) / det;"),
    "window_rows_off_by_one": ("for (int dy = -r; dy <= r; ++dy) {", "for (int dy = -r; dy < r; ++dy) {"),
    "vertical_gradient_sign": ("ofo_bilinear(I2, H, W, px, py + 1.0) - ofo_bilinear(I2, H, W, px, py - 1.0)",
                               "ofo_bilinear(I2, H, W, px, py - 1.0) - ofo_bilinear(I2, H, W, px, py + 1.0)"),
    "pyramid_keeps_odd_rows": ("const int y = clampi(2 * i + a - 2, 0, H - 1);",
                               "const int y = clampi(2 * i + a - 1, 0, H - 1);"),
    "pyramid_taps_flattened": ("{1.0, 4.0, 6.0, 4.0, 1.0}", "{2.0, 4.0, 4.0, 4.0, 2.0}"),
    "normalisation_mean_not_subtracted": ("(I[(size_t)y * W + x] - mean) / sqrt(var + eps)",
                                          "I[(size_t)y * W + x] / sqrt(var + eps)"),
    "normalisation_printed_radicand": ("const double var = s2 / n - mean * mean;",
                                       "const double var = mean * mean - s2 / n;"),
    "sbubble_strict_threshold": ("if (u[k] <= Tv) ++c;", "if (u[k] < Tv) ++c;"),
    "sbubble_threshold_not_halved": ("return 0.5 * ((double)lo + (double)hi);", "return ((double)lo + (double)hi);"),
}


@pytest.mark.slow
@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_reject_planted_mistake(tmp_path, name):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not found exactly once"
    mut = tmp_path / "mut.c"
    mut.write_text(src.replace(old, new))
    so = tmp_path / "libmut.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-shared", "-fPIC", str(mut),
                    "-o", str(so), "-lm"], check=True, capture_output=True)
    env = dict(os.environ, OF_ORACLE_LIB=str(so))
    res = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", "test_oracle_pins.py"),
                          "-x", "-q", "-p", "no:cacheprovider"], env=env, capture_output=True, text=True,
                         cwd=ROOT, timeout=300)
    assert res.returncode != 0, f"pins did not catch mutant {name}:\n{res.stdout[-2000:]}"
