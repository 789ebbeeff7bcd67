"""The C-ABI library without a GPU: it loads, exports every symbol that
include/fft2d.h declares, validates arguments before touching CUDA, and
builds the rotation-factor tables the plans upload."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="session")
def fft():
    from conftest import build_lib
    build_lib()
    import paper_1505_08019_gb300 as fft
    return fft


def declared_symbols():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            names |= set(re.findall(r"^FFT2D_API\s+[^;(]*?\b(fft2d_\w+)\s*\(", text, re.M))
    return names


def test_library_exports_every_declared_symbol(fft):
    names = declared_symbols()
    assert len(names) >= 12
    missing = [n for n in sorted(names) if not hasattr(fft.lib, n)]
    assert not missing, f"declared in include/ but not exported: {missing}"


def test_version_and_strerror(fft):
    assert fft.fft2d_version() >= 100
    for st in range(9):
        assert fft.fft2d_strerror(st)
    assert fft.fft2d_strerror(99) == "unknown status"


@pytest.mark.parametrize("rows,cols,dtype,dir_,want", [
    (3, 4, 0, -1, 2),            # not a power of two
    (4, 0, 0, -1, 2),
    (-8, 4, 0, -1, 2),
    (32768, 4, 0, -1, 3),        # above FFT2D_MAX_SIDE
    (4, 1 << 15, 0, 1, 3),
    (8, 8, 0, 0, 1),             # bad direction
    (8, 8, 7, -1, 1),            # bad dtype
    (1, 8, 2, -1, 8),            # DCT plan with a side of 1: not provided
    (8, 1, 2, 1, 8),
    (1, 8, 1, -1, 8),            # half2 plan with a side of 1: not provided
    (6, 8, 2, -1, 2),            # DCT plan, side not a power of two
])
def test_plan_argument_errors(fft, rows, cols, dtype, dir_, want):
    import ctypes
    h = ctypes.c_void_p(123)
    st = fft.lib.fft2d_plan(rows, cols, dtype, dir_, ctypes.byref(h))
    assert st == want
    assert h.value is None


def test_null_arguments(fft):
    assert fft.lib.fft2d_exec(None, None, None, None) == fft.FFT2D_ERR_ARG
    assert fft.lib.fft2d_exec_pass(None, 0, None, None, None) == fft.FFT2D_ERR_ARG
    assert fft.lib.fft2d_destroy(None) == fft.FFT2D_OK
    assert fft.lib.fft2d_exec_batched(-1, None, None, None, None) == fft.FFT2D_ERR_ARG
    assert fft.lib.fft2d_exec_host_many(-1, None, None, None, None) == fft.FFT2D_ERR_ARG
    assert fft.lib.fft2d_exec_host_many(2, None, None, None, None) == fft.FFT2D_ERR_ARG
    assert fft.lib.fft2d_exec_host_many(0, None, None, None, None) == fft.FFT2D_OK
    assert fft.lib.fft2d_stage_table(15, -1, None) == fft.FFT2D_ERR_ARG


@pytest.mark.parametrize("L", [1, 2, 3, 5, 8, 12, 14])
@pytest.mark.parametrize("dir_", [-1, 1])
def test_stage_table(fft, L, dir_):
    t = fft.fft2d_stage_table(L, dir_)
    assert t.shape == ((1 << L) - 1,)
    for s in range(1, L + 1):
        half = 1 << (s - 1)
        j = np.arange(half)
        want = np.exp(dir_ * 2j * np.pi * j / (1 << s))       # float64
        got = t[half - 1: 2 * half - 1]
        # rounding FP64 to FP32: within half an FP32 ulp of the exact value
        err = np.abs(got.astype(np.complex128) - want)
        assert err.max() <= 2.0 ** -24 + 1e-15, f"stage {s}"
        # exact values at j = 0 and at the quarter turn
        assert got[0] == np.complex64(1)
        if s >= 2:
            assert got[half // 2] == np.complex64(dir_ * 1j)
    # conjugate symmetry between directions
    assert np.array_equal(fft.fft2d_stage_table(L, 1), np.conj(fft.fft2d_stage_table(L, -1)))


def test_no_gpu_plan_fails_cleanly(fft):
    """Without a usable GPU, plan creation returns FFT2D_ERR_CUDA (never a CPU path)."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import ctypes
    h = ctypes.c_void_p()
    st = fft.lib.fft2d_plan(8, 8, 0, -1, ctypes.byref(h))
    assert st == fft.FFT2D_ERR_CUDA
    assert h.value is None


def test_stage_tables_have_exact_quarter_turn_symmetry(fft):
    """The stage engine reads only the first quarter of each stage's rotation
    factors and rotates them by W_4^1 (-i forward, +i inverse) for the second
    quarter; that equals the table bit for bit only if the plan's FP64 -> FP32
    tables hold W^{j + M/4} = W_4^1 W^j exactly, which this checks for every
    axis length and both directions."""
    for L in range(2, 15):
        for d in (fft.FFT2D_FORWARD, fft.FFT2D_INVERSE):
            t = fft.fft2d_stage_table(L, d).view(np.float32).reshape(-1, 2)
            p = np.float32(-t[2, 1])                       # -Im W_4^1
            assert p == (1.0 if d == fft.FFT2D_FORWARD else -1.0)
            for s in range(2, L + 1):
                M = 1 << s
                off, q = M // 2 - 1, M // 4
                w, w2 = t[off:off + q], t[off + q:off + 2 * q]
                turned = np.stack([p * w[:, 1] + np.float32(0), -p * w[:, 0] + np.float32(0)],
                                  axis=1).astype(np.float32)
                assert np.array_equal(turned.view(np.uint32), w2.view(np.uint32)), (L, d, s)
