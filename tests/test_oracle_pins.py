"""The oracle against facts the DFT fixes (CPU only), and planted mistakes.

Each planted mistake is a textual edit of a copy of oracle.c, compiled on the
CPU; the pins must reject every such copy while accepting the real oracle.
"""
import os

import pytest

import oracle
from tests import oracle_pins as P


@pytest.fixture(scope="module")
def o():
    return oracle.default()


@pytest.mark.parametrize("pin", P.ALL_PINS, ids=lambda p: p.__name__)
def test_pin(o, pin):
    pin(o)


# (name, original text, planted mistake)
MUTANTS = [
    ("root_sign", "*im = (double)sign * sin(a);", "*im = -(double)sign * sin(a);"),
    ("root_period", "double a = 2.0 * M_PI * (double)m / (double)n;",
     "double a = 2.0 * M_PI * (double)m / (double)(n + 1);"),
    ("naive_dropped_term", "si += xr * wi + xi * wr;\n        }\n        y[2 * k] = sr;",
     "si += xr * wi;\n        }\n        y[2 * k] = sr;"),
    ("butterfly_sign", "o[0] = e[0] - tr;", "o[0] = e[0] + tr;"),
    ("butterfly_conj_twiddle", "wi = w[2 * (j * step) + 1];", "wi = -w[2 * (j * step) + 1];"),
    ("no_bit_reversal", "r |= (int64_t)1 << (lg - 1 - b);", "r |= (int64_t)1 << b;"),
    ("butterfly_halved", "e[0] = e[0] + tr;", "e[0] = 0.5 * (e[0] + tr);"),
    ("split_wrong_bin", "fr = &f[2 * (r * n2 + (k % n2))];", "fr = &f[2 * (r * n2 + ((k + 1) % n2))];"),
    ("split_transposed", "sub[2 * t] = x[2 * (t * m + r)];", "sub[2 * t] = x[2 * ((r * n2 + t) % n)];"),
    ("bins_off_by_one", "int64_t k = ks[t] % n;", "int64_t k = (ks[t] + 1) % n;"),
    ("2d_column_reversed", "img[2 * (r * w + c)] = fc[2 * (c * h + r)];",
     "img[2 * (r * w + c)] = fc[2 * (c * h + (h - 1 - r))];"),
    ("conv_index_sign", "int64_t q = ((m - j) % n + n) % n;", "int64_t q = ((m + j) % n + n) % n;"),
    ("corr_missing_conj", "hr = h[2 * j]; hi = -h[2 * j + 1];", "hr = h[2 * j]; hi = h[2 * j + 1];"),
    ("2d_rows_only", "rc = oracle_fft_batch(col, fc, h, w, sign, nthreads);",
     "memcpy(fc, col, sizeof(double) * 2 * (size_t)(h * w)); rc = 0;"),
    ("ycc_luma_weight", "0.299 * R + 0.587 * G + 0.114 * B", "0.299 * R + 0.578 * G + 0.114 * B"),
    ("ycc_cb_sign", "128.0 - 0.168736 * R - 0.331264 * G + 0.5 * B", "128.0 - 0.168736 * R + 0.331264 * G + 0.5 * B"),
    ("ycc_cr_offset", "0.25 * (128.0 + 0.5 * R", "0.25 * (0.0 + 0.5 * R"),
    ("ycc_cb_cr_swapped", "0.25 * (128.0 - 0.168736 * R - 0.331264 * G + 0.5 * B)",
     "0.25 * (128.0 + 0.5 * R - 0.418688 * G - 0.081312 * B)"),
    ("chroma_half_weight", "cbb[k] += 0.25 *", "cbb[k] += 0.5 *"),
    ("chroma_wrong_block", "const int64_t k = (r / 2) * (w / 2) + c / 2;",
     "const int64_t k = (r / 2) * (w / 2) + c % (w / 2);"),
    ("deriv_border_central", "if (i == 0) return v[stride] - v[0];", "if (i == 0) return 0.5 * (v[stride] - v[0]);"),
    ("deriv_axes_swapped", "ux * deriv_1d(yb + r * w, c, w, 1) + uy * deriv_1d(yb + c, r, h, w)",
     "uy * deriv_1d(yb + r * w, c, w, 1) + ux * deriv_1d(yb + c, r, h, w)"),
    ("deriv_sign", "return 0.5 * (v[(i + 1) * stride] - v[(i - 1) * stride]);",
     "return 0.5 * (v[(i - 1) * stride] - v[(i + 1) * stride]);"),
]


@pytest.mark.parametrize("name,orig,bad", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(tmp_path, name, orig, bad):
    src = open(oracle.SOURCE).read()
    assert src.count(orig) == 1, f"mutation anchor not unique/present: {name}"
    p = tmp_path / f"mut_{name}.c"
    p.write_text(src.replace(orig, bad))
    lib = oracle.compile_source(str(p), str(tmp_path / f"mut_{name}.so"))
    failed = P.failing_pins(oracle.OracleLib(lib))
    assert failed, f"planted mistake {name} passed every pin"
