"""The FP64 oracle against its pins (no GPU).  See ``_pins.py``."""
import numpy as np
import pytest

import _pins
from synth import blob_image, uniform_complex, uniform_real


@pytest.mark.parametrize("pin", _pins.ALL_PINS, ids=lambda p: p.__name__)
def test_pin(orc, pin):
    pin(orc)


@pytest.mark.parametrize("shape,gen", [
    ((256, 256), "uniform_real"),       # the 256x256 gray-image case
    ((1024, 1024), "blob"),             # the paper's size, forward + inverse
    ((256, 1024), "uniform_real"),      # non-square, both orientations
    ((2048, 128), "uniform_real"),
])
def test_oracle_vs_library_config_sizes(orc, shape, gen):
    R, C = shape
    x = (uniform_real(R, C, 0) if gen == "uniform_real" else blob_image(R, C, 0))
    x = x.astype(np.complex128)
    X = orc.fft2d(x, threads=4)
    assert _pins.rel(X, np.fft.fft2(x)) < 1e-12
    back = orc.fft2d(X, inverse=True, threads=4)
    assert _pins.rel(back, x) < 1e-13
    assert _pins.rel(orc.fft2d(X, inverse=True), np.fft.ifft2(X)) < 1e-12


@pytest.mark.slow
def test_oracle_vs_library_4096(orc):
    x = blob_image(4096, 4096, 0).astype(np.complex128)
    X = orc.fft2d(x, threads=8)
    assert _pins.rel(X, np.fft.fft2(x)) < 1e-12


def test_threads_do_not_change_results(orc):
    x = uniform_complex(64, 128, 3).astype(np.complex128)
    a = orc.fft2d(x, threads=1)
    b = orc.fft2d(x, threads=5)
    assert np.array_equal(a, b)


def test_rejects_bad_sizes(orc):
    with pytest.raises(ValueError):
        orc.fft2d(np.zeros((3, 4), np.complex128))
    with pytest.raises(ValueError):
        orc.fft1d(np.zeros(8), nstages=4)


def test_table1_fixture_and_oracle_round_trip(orc):
    """tests/golden/table1.txt holds Table 1 as printed: five gray-image
    sides 128..2048 with a maximum error of 0.007 (read here only as the
    image sizes the paper used).  At the three smallest sides the FP64
    oracle's forward + inverse recovers a [0, 1) gray image within the
    radix-2 rounding bound: relative L2 error of order u log2(n) per
    transform (u = 2^-53, n = rows * cols), two transforms, times a slack
    of 8."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "table1.txt")
    rows = []
    with open(path) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                side, _, _, err = line.split()
                rows.append((int(side), float(err)))
    assert [r[0] for r in rows] == [128, 256, 512, 1024, 2048]
    assert all(e == 0.007 for _, e in rows)
    for side, _ in rows[:3]:
        x = uniform_real(side, side, seed=side).astype(np.complex128)
        back = orc.fft2d(orc.fft2d(x), inverse=True)
        bound = 8 * 2 * 2.0 ** -53 * np.log2(side * side)
        assert _pins.rel(back, x) <= bound


def test_gray_real_is_uniform_real_real_part():
    """The DCT's gray images are the same draws as the FFT's gray images."""
    from synth import gray_real
    for shape, seed in (((4, 8), 0), ((64, 32), 7)):
        g = gray_real(*shape, seed=seed)
        assert g.dtype == np.float32 and g.flags.c_contiguous
        assert np.array_equal(g, uniform_real(*shape, seed=seed).real)
