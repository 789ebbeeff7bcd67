"""The FP64 oracle under AddressSanitizer and UndefinedBehaviorSanitizer.

oracle/sanitize_driver.c drives every oracle entry point over small and
degenerate shapes and compares each radix-2 result with the direct DFT;
built here with -fsanitize=address,undefined and no recovery, any
out-of-bounds access, leak, overflow or wrong value ends it with a
non-zero status.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_oracle_is_clean_under_asan_and_ubsan(tmp_path):
    if not shutil.which("gcc"):
        pytest.skip("gcc not available")
    exe = str(tmp_path / "oracle_sanitized")
    build = subprocess.run(
        ["gcc", "-std=c11", "-O1", "-g", "-fno-omit-frame-pointer", "-ffp-contract=off",
         "-fsanitize=address,undefined", "-fno-sanitize-recover=all", "-pthread",
         os.path.join(ROOT, "oracle", "fft_oracle.c"),
         os.path.join(ROOT, "oracle", "sanitize_driver.c"), "-lm", "-o", exe],
        capture_output=True, text=True)
    if build.returncode != 0 and "sanitize" in build.stderr:
        pytest.skip("sanitizer runtime not available: " + build.stderr.strip()[:200])
    assert build.returncode == 0, build.stderr
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1:abort_on_error=0",
               UBSAN_OPTIONS="print_stacktrace=1")
    run = subprocess.run([exe], capture_output=True, text=True, env=env, timeout=300)
    assert run.returncode == 0, run.stdout + run.stderr
    assert "all checks passed" in run.stdout
