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
