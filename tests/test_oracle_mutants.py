"""The pin battery must catch plausible mistakes planted in the oracle.

Each case rewrites one line of a copy of ``oracle/fft_oracle.c`` (on the
CPU, in a temporary directory), builds it, and checks that at least one pin
fails.  The unmodified source must pass every pin.  Each battery runs in a
child process, so a mutant that reads out of bounds and crashes counts as
caught without taking the test session down.
"""
import json
import os
import subprocess
import sys

import pytest

from oracle import oracle

SRC = os.path.join(os.path.dirname(oracle.__file__), "fft_oracle.c")

MUTANTS = {
    # butterfly: lower/upper output swapped sign (eq. 2 vs eq. 3)
    "butterfly_sign": ("e[0] = er + tr;", "e[0] = er - tr;"),
    # dropped term of the complex product
    "dropped_cross_term": ("double ti = wr * o[1] + wi * o[0];", "double ti = wr * o[1];"),
    # wrong sign of the rotation factor (conjugated twiddle)
    "twiddle_sign": ("*wi = sign * sin(ang);", "*wi = -sign * sin(ang);"),
    # twiddle of the wrong stage (W_{2^(s-1)} instead of W_{2^s})
    "twiddle_stage": ("oracle_twiddle(j, span, sign, &wr, &wi);",
                      "oracle_twiddle(j, half, sign, &wr, &wi);"),
    # scramble index not reversed
    "no_bitreverse": ("r |= 1L << (L - 1 - b);", "r |= 1L << b;"),
    # off-by-one: first butterfly of each block skipped
    "skip_j0": ("for (long j = 0; j < half; j++) {", "for (long j = 1; j < half; j++) {"),
    # inverse scaled by one side only
    "inverse_scale": ("1.0 / ((double)rows * (double)cols)", "1.0 / (double)rows"),
    # transposed operand: columns walked with row strides
    "column_strides": ("rc = oracle_lines_threaded(z, rows, cols, cols, 1, sign, col_stages,",
                       "rc = oracle_lines_threaded(z, rows, cols, 1, cols, sign, col_stages,"),
    # threads split the lines wrongly (first chunk offset ignored)
    "thread_chunks": ("jobs[t].z = z + 2 * first * line_stride;", "jobs[t].z = z;"),
    # direct DFT with a wrong exponent
    "dft_index": ("oracle_twiddle((m * k) % n, n, sign, &wr, &wi);",
                  "oracle_twiddle((m * (k + 1)) % n, n, sign, &wr, &wi);"),
    # low-pass distance not folded (no mirror symmetry)
    "lowpass_fold": ("const double dk = (double)(k < rows - k ? k : rows - k);",
                     "const double dk = (double)k;"),
    # quarter-turn value wrong
    "quarter_turn": ("static const double sq[4] = {0.0, 1.0, 0.0, -1.0};",
                     "static const double sq[4] = {0.0, -1.0, 0.0, 1.0};"),
    # DCT: half-sample shift dropped from the cosine phase (2j instead of 2j+1)
    "dct_phase": ("double c = ctab[(k * (2 * j + 1)) % (4 * n)];",
                  "double c = ctab[(k * (2 * j)) % (4 * n)];"),
    # DCT inverse: the k = 0 term weighted like the others
    "dct_inverse_weight": ("double w = inverse ? (b == 0 ? 1.0 : 2.0) : 1.0;",
                           "double w = inverse ? 2.0 : 1.0;"),
    # DCT inverse: 1/n missing
    "dct_inverse_scale": ("X[a * out_stride] = inverse ? s / (double)n : s;",
                          "X[a * out_stride] = s;"),
    # DCT: cosine table wrong at the half turn
    "dct_half_turn": ("            c[m] = -1.0;", "            c[m] = 1.0;"),
    # DCT: columns walked with row strides
    "dct_column_strides": ("oracle_dct_line_tab(z + c, cols, tmp, 1, rows, inverse, ccol);",
                           "oracle_dct_line_tab(z + c * rows, 1, tmp, 1, rows, inverse, ccol);"),
    # DCT single output: phase of the row factor off by one
    "dct_at_phase": ("long pm = (k * (2 * m + 1)) % (4 * rows);",
                     "long pm = (k * (2 * m + 2)) % (4 * rows);"),
}


HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _battery(tmp_path, name, text):
    """Build ``text`` as an oracle and run the pin battery on it in a child
    process.  Returns the failed pin names, or ["crashed"]."""
    src = tmp_path / f"{name}.c"
    src.write_text(text)
    lib = oracle.build(str(src), str(tmp_path / f"lib{name}.so"), force=True)
    code = ("import json, sys; sys.path[:0] = [%r, %r]; import _pins; "
            "from oracle import oracle; "
            "print(json.dumps(_pins.run_battery(oracle.Oracle(%r))))" % (ROOT, HERE, lib))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True,
                       timeout=300)
    if r.returncode != 0:
        return ["crashed"]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_unmodified_oracle_passes_all_pins(tmp_path):
    assert _battery(tmp_path, "clean", open(SRC).read()) == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name):
    old, new = MUTANTS[name]
    text = open(SRC).read()
    assert text.count(old) == 1, f"mutation anchor for {name} not found exactly once"
    failed = _battery(tmp_path, name, text.replace(old, new))
    assert failed, f"planted mistake {name} passed every pin"
