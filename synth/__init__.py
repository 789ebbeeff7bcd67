"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module holds no FFT arithmetic: it only draws images (and, for the
serving workload, request streams) from numpy's PCG64 generator, so the CUDA
path and the CPU oracle can be fed identical data.  Every image is returned as
a C-contiguous ``complex64`` array; the oracle widens it to ``complex128``
exactly.

The paper's workload is "gray images" of 128x128 .. 2048x2048 (Section 4,
Table 1).  No image dataset is used: the recipes below stand in for it.
"""
from __future__ import annotations

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(seed)


def uniform_real(rows: int, cols: int, seed: int = 0) -> np.ndarray:
    """Gray-image stand-in: real part ~ U[0, 1), imaginary part 0."""
    g = rng(seed)
    re = g.random((rows, cols), dtype=np.float32)
    out = np.zeros((rows, cols), dtype=np.complex64)
    out.real = re
    return out


def gray_real(rows: int, cols: int, seed: int = 0) -> np.ndarray:
    """Real gray image (one float32 per pixel) ~ U[0, 1): the input of the
    discrete cosine transform; the same draws as ``uniform_real``'s real part."""
    return rng(seed).random((rows, cols), dtype=np.float32)


def blob_image(rows: int, cols: int, seed: int = 0, nblobs: int = 8) -> np.ndarray:
    """Smooth background of Gaussian blobs plus U[0, 1) noise, imaginary 0.

    re[m, n] = sum_b a_b exp(-((m-mu_b)^2 + (n-nu_b)^2) / (2 s_b^2)) + U[0,1)
    with a_b ~ U[0.5, 2), mu_b ~ U[0, rows), nu_b ~ U[0, cols),
    s_b ~ U[side/32, side/4), side = min(rows, cols).
    """
    g = rng(seed)
    side = min(rows, cols)
    a = g.uniform(0.5, 2.0, nblobs)
    mu = g.uniform(0, rows, nblobs)
    nu = g.uniform(0, cols, nblobs)
    s = g.uniform(side / 32, side / 4, nblobs)
    m = np.arange(rows, dtype=np.float64)[:, None]
    n = np.arange(cols, dtype=np.float64)[None, :]
    re = np.zeros((rows, cols), dtype=np.float64)
    for b in range(nblobs):
        re += a[b] * np.exp(-((m - mu[b]) ** 2 + (n - nu[b]) ** 2) / (2 * s[b] ** 2))
    re += g.random((rows, cols))
    out = np.zeros((rows, cols), dtype=np.complex64)
    out.real = re.astype(np.float32)
    return out


def uniform_complex(rows: int, cols: int, seed: int = 0) -> np.ndarray:
    """re, im ~ U[-1, 1) independently (the large-image precision workload)."""
    g = rng(seed)
    out = np.empty((rows, cols), dtype=np.complex64)
    out.real = g.uniform(-1.0, 1.0, (rows, cols)).astype(np.float32)
    out.imag = g.uniform(-1.0, 1.0, (rows, cols)).astype(np.float32)
    return out


def integer_image(rows: int, cols: int, seed: int = 0, lo: int = -8, hi: int = 8) -> np.ndarray:
    """Small integers in [lo, hi) for both parts: sums of these stay exact in FP32."""
    g = rng(seed)
    out = np.empty((rows, cols), dtype=np.complex64)
    out.real = g.integers(lo, hi, (rows, cols)).astype(np.float32)
    out.imag = g.integers(lo, hi, (rows, cols)).astype(np.float32)
    return out


def batch_shapes(n: int = 64, seed: int = 0, lo: int = 7, hi: int = 11) -> list[tuple[int, int]]:
    """n (rows, cols) pairs; log2 of each side drawn independently from U{lo..hi}."""
    g = rng(seed)
    lr = g.integers(lo, hi + 1, n)
    lc = g.integers(lo, hi + 1, n)
    return [(1 << int(a), 1 << int(b)) for a, b in zip(lr, lc)]


def batch_images(shapes, seed: int = 0) -> list[np.ndarray]:
    """One uniform_real image per shape, image i drawn with seed (seed, i)."""
    return [uniform_real(r, c, seed=(seed * 1_000_003 + i)) for i, (r, c) in enumerate(shapes)]
