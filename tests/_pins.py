"""Pins for the FP64 oracle: checks against facts that do not come from the
oracle itself.

Each pin takes an ``oracle.Oracle`` handle and raises ``AssertionError`` when
the oracle disagrees with
  * brute force: eq. 1 evaluated here with a numpy matrix on tiny inputs;
  * closed forms: delta, shifted delta, constant, single complex exponential;
  * invariants: Parseval, linearity, inverse round trip, Hermitian symmetry;
  * an independent library FFT (numpy.fft, pocketfft), which fixes the sign
    of W_N and the 1/(R*C) inverse scale;
  * decimation identities for partial stage counts (what the DIT butterfly
    recurrence of eqs. 2-3 must hold after k stages).
The same battery is run against deliberately broken builds of the oracle
(``test_oracle_mutants.py``) to show that it catches plausible mistakes.
"""
from __future__ import annotations

import numpy as np

from synth import uniform_complex, uniform_real

TOL_FFT = 1e-12     # FP64 radix-2 vs pocketfft / brute force, relative L2


def rel(a, b):
    a = np.asarray(a, np.complex128)
    b = np.asarray(b, np.complex128)
    d = np.linalg.norm(b.ravel())
    return np.linalg.norm((a - b).ravel()) / (d if d > 0 else 1.0)


def brute_dft(x, inverse=False):
    """Eq. 1 as a dense matrix product (tiny inputs only)."""
    x = np.asarray(x, np.complex128)
    n = x.size
    k = np.arange(n)
    sgn = 1.0 if inverse else -1.0
    F = np.exp(sgn * 2j * np.pi * np.outer(k, k) / n)
    return F @ x


def bitrev_brute(i, L):
    if L == 0:
        return 0
    return int(format(i, f"0{L}b")[::-1], 2)


def decimated_blocks(x, k):
    """What a line holds after k DIT stages: block b (2^k positions) is the
    2^k-point DFT of the subsequence x[rev_{L-k}(b) + m 2^(L-k)], m < 2^k."""
    x = np.asarray(x, np.complex128)
    n = x.size
    L = n.bit_length() - 1
    out = np.empty(n, np.complex128)
    for b in range(n >> k):
        start = bitrev_brute(b, L - k)
        sub = x[start::1 << (L - k)]
        out[b << k:(b + 1) << k] = np.fft.fft(sub)
    return out


# --------------------------------------------------------------------------
def pin_bitrev(orc):
    for L in range(0, 13):
        t = orc.bitrev(L)
        want = [bitrev_brute(i, L) for i in range(1 << L)]
        assert list(t) == want, f"bit-reversal table wrong for L={L}"


def pin_fft1d_brute(orc):
    g = np.random.default_rng(11)
    for L in range(0, 7):
        n = 1 << L
        x = g.standard_normal(n) + 1j * g.standard_normal(n)
        for inv in (False, True):
            got = orc.fft1d(x, inverse=inv)
            assert rel(got, brute_dft(x, inv)) < TOL_FFT, f"fft1d vs eq.1 n={n} inv={inv}"


def pin_dft1d_brute(orc):
    g = np.random.default_rng(12)
    for n in (1, 2, 3, 5, 8, 12, 16, 31, 64):
        x = g.standard_normal(n) + 1j * g.standard_normal(n)
        for inv in (False, True):
            assert rel(orc.dft1d(x, inverse=inv), brute_dft(x, inv)) < TOL_FFT, f"dft1d n={n}"


def pin_fft1d_library(orc):
    g = np.random.default_rng(13)
    for L in (7, 10, 12):
        n = 1 << L
        x = g.standard_normal(n) + 1j * g.standard_normal(n)
        assert rel(orc.fft1d(x), np.fft.fft(x)) < TOL_FFT, f"fft1d vs numpy n={n}"
        assert rel(orc.fft1d(x, inverse=True), n * np.fft.ifft(x)) < TOL_FFT


def pin_fft2d_library(orc, shapes=((1, 1), (2, 2), (4, 8), (16, 2), (32, 64), (64, 16), (128, 128))):
    for i, (R, C) in enumerate(shapes):
        x = uniform_complex(R, C, seed=100 + i).astype(np.complex128)
        assert rel(orc.fft2d(x), np.fft.fft2(x)) < TOL_FFT, f"fft2d vs numpy {R}x{C}"
        assert rel(orc.fft2d(x, inverse=True), np.fft.ifft2(x)) < TOL_FFT, f"ifft2d {R}x{C}"
        # the threaded split of lines must not change the result
        assert rel(orc.fft2d(x, threads=3), np.fft.fft2(x)) < TOL_FFT, f"threaded {R}x{C}"


def pin_dft2d(orc):
    g = np.random.default_rng(14)
    for R, C in ((1, 4), (4, 4), (8, 2), (6, 5), (16, 16)):
        x = g.standard_normal((R, C)) + 1j * g.standard_normal((R, C))
        assert rel(orc.dft2d(x), np.fft.fft2(x)) < TOL_FFT, f"dft2d {R}x{C}"
        assert rel(orc.dft2d(x, inverse=True), R * C * np.fft.ifft2(x)) < TOL_FFT


def pin_crops_brute(orc):
    """16x16 crops (top-left, centre) of the 256x256 gray image: radix-2 2D FFT
    of the crop equals the direct double sum of eq. 1."""
    img = uniform_real(256, 256, seed=0).astype(np.complex128)
    for (r0, c0) in ((0, 0), (120, 120)):
        crop = img[r0:r0 + 16, c0:c0 + 16]
        assert rel(orc.fft2d(crop), orc.dft2d(crop)) < TOL_FFT
        # and the double sum itself against the matrix form of eq. 1
        F = np.exp(-2j * np.pi * np.outer(np.arange(16), np.arange(16)) / 16)
        assert rel(orc.dft2d(crop), F @ crop @ F.T) < TOL_FFT


def pin_closed_forms(orc):
    for R, C in ((8, 8), (16, 64), (128, 32)):
        # delta at the origin -> all ones, exactly
        d = np.zeros((R, C), np.complex128)
        d[0, 0] = 1
        X = orc.fft2d(d)
        assert np.array_equal(X, np.ones((R, C))), f"delta {R}x{C}"
        # shifted delta -> pure phase W_R^{k m0} W_C^{l n0}
        m0, n0 = R // 4 + 1, C // 2 - 1
        d = np.zeros((R, C), np.complex128)
        d[m0, n0] = 1
        k = np.arange(R)[:, None]
        l = np.arange(C)[None, :]
        want = np.exp(-2j * np.pi * (k * m0 / R + l * n0 / C))
        assert rel(orc.fft2d(d), want) < TOL_FFT, "shifted delta"
        # constant c -> c R C at [0, 0] and zero elsewhere
        c = 0.75 - 0.25j
        X = orc.fft2d(np.full((R, C), c))
        assert abs(X[0, 0] - c * R * C) < 1e-12 * R * C
        Z = X.copy()
        Z[0, 0] = 0
        assert np.abs(Z).max() < 1e-12 * R * C, "constant leaks out of DC"
        # single complex exponential -> R C in exactly one bin
        k0, l0 = R // 2 + 1, C // 4 + 3
        m = np.arange(R)[:, None]
        n = np.arange(C)[None, :]
        e = np.exp(2j * np.pi * (k0 * m / R + l0 * n / C))
        X = orc.fft2d(e)
        assert abs(X[k0, l0] - R * C) < 1e-10 * R * C
        X[k0, l0] = 0
        assert np.abs(X).max() < 1e-10 * R * C, "exponential leaks"


def pin_invariants(orc):
    g = np.random.default_rng(15)
    for R, C in ((32, 32), (64, 8), (16, 128)):
        x = g.standard_normal((R, C)) + 1j * g.standard_normal((R, C))
        y = g.standard_normal((R, C)) + 1j * g.standard_normal((R, C))
        X, Y = orc.fft2d(x), orc.fft2d(y)
        # Parseval: sum |x|^2 = sum |X|^2 / (R C)
        px, pX = np.sum(np.abs(x) ** 2), np.sum(np.abs(X) ** 2) / (R * C)
        assert abs(px - pX) < 1e-12 * px, "Parseval"
        # linearity
        a, b = 1.5 - 0.5j, -0.25 + 2j
        assert rel(orc.fft2d(a * x + b * y), a * X + b * Y) < TOL_FFT, "linearity"
        # round trip
        assert rel(orc.fft2d(X, inverse=True), x) < 1e-14, "round trip"
        # Hermitian symmetry for real input: X[k, l] = conj(X[-k, -l])
        r = g.standard_normal((R, C)).astype(np.complex128)
        Xr = orc.fft2d(r)
        flip = np.conj(Xr[(-np.arange(R)) % R][:, (-np.arange(C)) % C])
        assert rel(Xr, flip) < 1e-13, "Hermitian symmetry"


def pin_partial_stages(orc):
    g = np.random.default_rng(16)
    for L in (1, 3, 6, 9):
        n = 1 << L
        x = g.standard_normal(n) + 1j * g.standard_normal(n)
        # zero stages: the scramble alone, an exact permutation
        perm = np.array([bitrev_brute(p, L) for p in range(n)])
        assert np.array_equal(orc.fft1d(x, nstages=0), x[perm]), "scramble"
        for k in range(1, L + 1):
            assert rel(orc.fft1d(x, nstages=k), decimated_blocks(x, k)) < TOL_FFT, \
                f"partial stages n={n} k={k}"
    # 2D: each axis obeys the same identity, rows first then columns
    R, C = 16, 32
    x = g.standard_normal((R, C)) + 1j * g.standard_normal((R, C))
    for kr, kc in ((0, 0), (2, 1), (5, 4), (3, 0)):
        want = np.array([decimated_blocks(row, kr) for row in x])
        want = np.array([decimated_blocks(col, kc) for col in want.T]).T
        got = orc.fft2d(x, row_stages=kr, col_stages=kc)
        assert rel(got, want) < TOL_FFT, f"2D partial {kr},{kc}"


def pin_lowpass(orc):
    """The Gaussian low-pass of the filtering workload: DC passes unchanged,
    the factor at distance d = sigma is exp(-1/2), it decreases with the
    frequency distance, the filter is separable and mirror-symmetric, and a
    real image stays real through FFT -> low-pass -> inverse."""
    R, C = 64, 32
    one = np.ones((R, C), np.complex128)
    H = orc.lowpass(one, 8.0, 4.0)
    assert H[0, 0] == 1.0
    assert abs(H[8, 0] - np.exp(-0.5)) < 1e-15 and abs(H[0, 4] - np.exp(-0.5)) < 1e-15
    assert abs(H[R - 8, 0] - np.exp(-0.5)) < 1e-15
    assert abs(H[8, 4] - np.exp(-1.0)) < 1e-15
    # decreasing with frequency distance up to the Nyquist bin on each axis
    assert np.all(np.diff(H[: R // 2 + 1, 0].real) < 0)
    assert np.all(np.diff(H[0, : C // 2 + 1].real) < 0)
    assert np.allclose(H, np.outer(H[:, 0], H[0, :]), rtol=1e-14, atol=0)
    g = np.random.default_rng(17)
    x = g.standard_normal((R, C)).astype(np.complex128)
    y = orc.filter_image(x)
    assert np.abs(y.imag).max() < 1e-12 * np.abs(y.real).max()
    # the mean (DC) of the image is preserved exactly in exact arithmetic
    assert abs(y.mean() - x.mean()) < 1e-12


def pin_dct_library(orc, shapes=((1, 1), (1, 8), (2, 2), (4, 8), (8, 4), (16, 32), (32, 16),
                                  (64, 64), (5, 3), (6, 10))):
    """The 2D DCT-II against an independent library: scipy's unnormalised type-2
    transform is twice this definition on every axis."""
    import scipy.fft as sf
    g = np.random.default_rng(11)
    for R, C in shapes:
        x = g.uniform(-1, 1, (R, C))
        want = sf.dctn(x, type=2, norm=None) / 4.0
        assert rel(orc.dct2d(x), want) <= 1e-13, (R, C)
        line = g.uniform(-1, 1, C)
        assert rel(orc.dct1d(line), sf.dct(line, type=2, norm=None) / 2.0) <= 1e-13, C


def pin_dct_brute(orc):
    """Every output of small 2D DCTs equals the unseparated double sum."""
    g = np.random.default_rng(12)
    for R, C in ((1, 1), (2, 4), (4, 4), (8, 2), (3, 5)):
        x = g.uniform(-1, 1, (R, C))
        X = orc.dct2d(x)
        for k in range(R):
            for l in range(C):
                assert abs(X[k, l] - orc.dct2d_at(x, k, l)) <= 1e-12 * max(1.0, abs(X[k, l])), (R, C, k, l)


def pin_dct_closed_forms(orc):
    """A constant lands only at [0][0] (c R C); the cosine basis image of
    (k0, l0) lands only there, with weight (R / (2 - [k0 == 0])) (C / (2 - [l0 == 0]))."""
    R, C = 8, 16
    X = orc.dct2d(np.full((R, C), 0.75))
    assert abs(X[0, 0] - 0.75 * R * C) <= 1e-12
    X[0, 0] = 0.0
    assert np.abs(X).max() <= 1e-12
    m = np.arange(R)[:, None]
    n = np.arange(C)[None, :]
    for k0, l0 in ((0, 0), (0, 5), (3, 0), (1, 1), (7, 15), (4, 8)):
        x = np.cos(np.pi * k0 * (2 * m + 1) / (2 * R)) * np.cos(np.pi * l0 * (2 * n + 1) / (2 * C))
        X = orc.dct2d(x)
        want = (R if k0 == 0 else R / 2) * (C if l0 == 0 else C / 2)
        assert abs(X[k0, l0] - want) <= 1e-11, (k0, l0)
        X[k0, l0] = 0.0
        assert np.abs(X).max() <= 1e-11, (k0, l0)


def pin_dct_round_trip(orc):
    """The inverse undoes the forward, square and non-square."""
    g = np.random.default_rng(13)
    for R, C in ((1, 1), (4, 4), (16, 8), (2, 64), (32, 32)):
        x = g.uniform(-1, 1, (R, C))
        assert np.abs(orc.dct2d(orc.dct2d(x), inverse=True) - x).max() <= 1e-12, (R, C)


ALL_PINS = [pin_dct_library, pin_dct_brute, pin_dct_closed_forms, pin_dct_round_trip,
            pin_lowpass, pin_bitrev, pin_fft1d_brute, pin_dft1d_brute, pin_fft1d_library,
            pin_fft2d_library, pin_dft2d, pin_crops_brute, pin_closed_forms,
            pin_invariants, pin_partial_stages]


def run_battery(orc):
    """Names of the pins that fail (empty when the oracle is sound)."""
    failed = []
    for p in ALL_PINS:
        try:
            p(orc)
        except (AssertionError, ValueError, FloatingPointError):
            failed.append(p.__name__)
    return failed
