"""Plant plausible mistakes in a copy of the oracle source (on the CPU) and check that
the pins catch each one: a flipped or transposed filter, a wrong boundary rule, a
dropped or sign-flipped Harris term, a missing clamp scatter in an adjoint, a dropped
factor in the Harris chain rule and a flipped separable column pass."""
import os

import pytest

import oracle
import oracle_pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "imagecl_oracle.c")

MUTATIONS = {
    "flipped_taps": ("s += w[j * kw + i] * read_f64(x, W, H, px + i - rx, py + j - ry, border, bv);",
                     "s += w[j * kw + i] * read_f64(x, W, H, px - i + rx, py - j + ry, border, bv);"),
    "transposed_taps": ("s += w[j * kw + i] * read_f64(x, W, H, px + i - rx, py + j - ry, border, bv);",
                        "s += w[i * kh + j] * read_f64(x, W, H, px + i - rx, py + j - ry, border, bv);"),
    "wrap_not_clamp": ("    return x[clampi(qy, 0, H - 1) * W + clampi(qx, 0, W - 1)];\n}",
                       "    return x[((qy % H + H) % H) * W + ((qx % W + W) % W)];\n}"),
    "harris_k_sign": ("R[o] = sxx * syy - sxy * sxy - k * tr * tr;",
                      "R[o] = sxx * syy - sxy * sxy + k * tr * tr;"),
    "harris_no_sxy": ("R[o] = sxx * syy - sxy * sxy - k * tr * tr;",
                      "R[o] = sxx * syy - k * tr * tr;"),
    "harris_sobel_swapped": ("gx += sx[j * 3 + i] * v;", "gx += sx[i * 3 + j] * v;"),
    "adjoint_no_clamp_scatter": ("if (dx) dx[qy * W + qx] += w[j * kw + i] * gp;",
                                 "if (dx && inside) dx[qy * W + qx] += w[j * kw + i] * gp;"),
    "harris_bwd_factor": ("gI[p] = 2.0 * Ix[p] * gP[p] + Iy[p] * gP[2 * n + p];",
                          "gI[p] = Ix[p] * gP[p] + Iy[p] * gP[2 * n + p];"),
    "sep_column_flipped": ("int64_t qy = py + j - rc;\n                double v;",
                           "int64_t qy = py - j + rc;\n                double v;"),
    "harris_even_anchor": ("    const int rw = wk / 2;   /* anchor: odd wk centred, even wk offsets -wk/2 .. wk/2-1 */",
                           "    const int rw = (wk - 1) / 2;"),
    "int_no_wrap": ("out[(py - y0) * W + px] = (int32_t)(uint32_t)(uint64_t)s;",
                    "out[(py - y0) * W + px] = s > 2147483647 ? 2147483647 : (int32_t)s;"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_mutation(name, tmp_path):
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation anchor for {name} not found"
    mutated = tmp_path / "mutant.c"
    mutated.write_text(src.replace(old, new, 1))
    bad = oracle.from_source(str(mutated), str(tmp_path / "libmutant.so"))
    caught = []
    for check in oracle_pins.ALL_CHECKS:
        try:
            check(bad)
        except (AssertionError, ValueError):
            caught.append(check.__name__)
    assert caught, f"no pin caught the mutation {name}"
