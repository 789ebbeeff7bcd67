"""Python front end of the FP64 CPU oracle (``fft_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``; never by the library.  It shares no
code with the CUDA path.  Every function works on numpy ``complex128`` data
(interleaved re/im doubles) and follows the paper's method:

* ``bitrev``  -- the scramble index table (Section 3.2);
* ``fft1d``   -- scramble then log2(N) radix-2 DIT butterfly stages
                 (Section 2 eqs. 2-3, Section 3.1 eq. 4);
* ``fft2d``   -- rows, then columns (Section 2, separability), inverse scaled
                 by 1/(rows*cols);
* ``dft1d`` / ``dft2d`` -- eq. 1 evaluated directly (brute force);
* ``dct1d`` / ``dct2d`` / ``dct2d_at`` -- the discrete cosine transform (one
                 of the "similar transforms" of Section 5) from its definition,
                 real data.

``fft2d(..., threads=k)`` splits the lines of each axis over k POSIX threads
inside the C code; the arithmetic per line is the same single-threaded code.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fft_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD_DIR, "liboracle.so")

# -ffp-contract=off: no fused multiply-add, so the oracle gives the same
# IEEE double results on x86_64 and aarch64 hosts.
CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
          "-pthread"]

_lock = threading.Lock()


def build(src: str = _SRC, out: str = _LIB, force: bool = False) -> str:
    """Compile ``src`` into the shared library ``out`` with gcc (if stale)."""
    with _lock:
        if (not force and os.path.exists(out)
                and os.path.getmtime(out) >= os.path.getmtime(src)):
            return out
        os.makedirs(os.path.dirname(out), exist_ok=True)
        tmp = out + f".tmp{os.getpid()}"
        subprocess.run(["gcc", *CFLAGS, "-o", tmp, src, "-lm"], check=True)
        os.replace(tmp, out)
        return out


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


class Oracle:
    """ctypes handle on one build of the oracle library."""

    def __init__(self, lib_path: str | None = None):
        path = lib_path or build()
        self.path = path
        lib = ctypes.CDLL(path)
        L, P, I = ctypes.c_long, ctypes.c_void_p, ctypes.c_int
        lib.oracle_bitrev_table.argtypes = [I, P]
        lib.oracle_bitrev_table.restype = None
        lib.oracle_fft_line.argtypes = [P, L, L, I, I]
        lib.oracle_fft_line.restype = I
        lib.oracle_fft_lines.argtypes = [P, L, L, L, L, I, I]
        lib.oracle_fft_lines.restype = I
        lib.oracle_scale.argtypes = [P, L, ctypes.c_double]
        lib.oracle_scale.restype = None
        lib.oracle_fft2d.argtypes = [P, L, L, I, I, I, I, I]
        lib.oracle_fft2d.restype = I
        lib.oracle_dft_line.argtypes = [P, L, P, L, L, I]
        lib.oracle_dft_line.restype = I
        lib.oracle_dft2d.argtypes = [P, P, L, L, I]
        lib.oracle_dft2d.restype = I
        lib.oracle_gaussian_lowpass.argtypes = [P, L, L, ctypes.c_double, ctypes.c_double]
        lib.oracle_gaussian_lowpass.restype = None
        lib.oracle_dct_line.argtypes = [P, L, P, L, L, I]
        lib.oracle_dct_line.restype = I
        lib.oracle_dct2d.argtypes = [P, L, L, I]
        lib.oracle_dct2d.restype = I
        lib.oracle_dct2d_at.argtypes = [P, L, L, L, L]
        lib.oracle_dct2d_at.restype = ctypes.c_double
        self.lib = lib

    # -- Section 3.2 ---------------------------------------------------------
    def bitrev(self, L: int) -> np.ndarray:
        out = np.empty(1 << L, dtype=np.int64)
        self.lib.oracle_bitrev_table(L, _ptr(out))
        return out

    # -- Section 2 eqs. 2-3, one axis ------------------------------------------
    def fft1d(self, x, inverse: bool = False, nstages: int | None = None) -> np.ndarray:
        """Unscaled radix-2 DIT of a 1D power-of-two array (inverse: +i sign)."""
        z = np.array(x, dtype=np.complex128, copy=True).reshape(-1)
        n = z.size
        L = n.bit_length() - 1
        ns = L if nstages is None else nstages
        rc = self.lib.oracle_fft_line(_ptr(z), n, 1, 1 if inverse else -1, ns)
        if rc:
            raise ValueError(f"oracle_fft_line rc={rc} (n={n}, nstages={ns})")
        return z

    # -- Section 2 eq. 1 -------------------------------------------------------
    def dft1d(self, x, inverse: bool = False) -> np.ndarray:
        a = np.ascontiguousarray(x, dtype=np.complex128).reshape(-1)
        out = np.empty_like(a)
        rc = self.lib.oracle_dft_line(_ptr(a), 1, _ptr(out), 1, a.size, 1 if inverse else -1)
        if rc:
            raise ValueError(f"oracle_dft_line rc={rc}")
        return out

    def dft2d(self, x, inverse: bool = False) -> np.ndarray:
        a = np.ascontiguousarray(x, dtype=np.complex128)
        out = np.empty_like(a)
        rc = self.lib.oracle_dft2d(_ptr(a), _ptr(out), a.shape[0], a.shape[1],
                                   1 if inverse else -1)
        if rc:
            raise ValueError(f"oracle_dft2d rc={rc}")
        return out

    # -- Section 2 separability: rows then columns -----------------------------
    def fft2d(self, x, inverse: bool = False, row_stages: int | None = None,
              col_stages: int | None = None, scale: bool = True,
              threads: int = 1) -> np.ndarray:
        """2D radix-2 DIT: every row, then every column; inverse x 1/(R*C).

        ``row_stages``/``col_stages`` stop each axis after that many butterfly
        stages (0 = scramble only); ``None`` runs them all.  ``threads`` host
        threads share the lines of each axis (same arithmetic per line).
        """
        z = np.array(x, dtype=np.complex128, copy=True, order="C")
        if z.ndim != 2:
            raise ValueError("fft2d expects a 2D array")
        R, C = z.shape
        rs = -1 if row_stages is None else row_stages
        cs = -1 if col_stages is None else col_stages
        rc = self.lib.oracle_fft2d(_ptr(z), R, C, 1 if inverse else -1, rs, cs,
                                   1 if scale else 0, max(1, int(threads)))
        if rc:
            raise ValueError(f"oracle_fft2d rc={rc} ({R}x{C}, stages {rs},{cs})")
        return z


    # -- the filtering workload ------------------------------------------------
    def lowpass(self, X, sigma_rows: float, sigma_cols: float) -> np.ndarray:
        """Gaussian low-pass of an unshifted spectrum (copy)."""
        z = np.array(X, dtype=np.complex128, copy=True, order="C")
        self.lib.oracle_gaussian_lowpass(_ptr(z), z.shape[0], z.shape[1], sigma_rows, sigma_cols)
        return z

    def filter_image(self, x, threads: int = 1) -> np.ndarray:
        """FFT -> Gaussian low-pass (sigma = side/8 per axis) -> inverse FFT."""
        R, C = np.shape(x)
        X = self.fft2d(x, threads=threads)
        X = self.lowpass(X, R / 8.0, C / 8.0)
        return self.fft2d(X, inverse=True, threads=threads)

    # -- discrete cosine transform (Section 5's "similar transforms"),
    #    real data, evaluated from its definition (no FFT)
    def dct1d(self, x, inverse: bool = False) -> np.ndarray:
        """DCT-II of a real line, or (inverse) the scaled DCT-III that undoes it."""
        x = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
        X = np.empty_like(x)
        rc = self.lib.oracle_dct_line(_ptr(x), 1, _ptr(X), 1, x.shape[0], int(inverse))
        if rc != 0:
            raise ValueError(f"oracle_dct_line failed ({rc})")
        return X

    def dct2d(self, x, inverse: bool = False) -> np.ndarray:
        """2D DCT-II (rows, then columns) of a real image, or its inverse (copy)."""
        z = np.array(x, dtype=np.float64, copy=True, order="C")
        rc = self.lib.oracle_dct2d(_ptr(z), z.shape[0], z.shape[1], int(inverse))
        if rc != 0:
            raise ValueError(f"oracle_dct2d failed ({rc})")
        return z

    def dct2d_at(self, x, k: int, l: int) -> float:
        """One forward 2D DCT output X[k][l] as the direct double sum."""
        x = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
        return float(self.lib.oracle_dct2d_at(_ptr(x), x.shape[0], x.shape[1], k, l))


_default: Oracle | None = None


def get() -> Oracle:
    """The oracle built from ``fft_oracle.c`` (compiled on first use)."""
    global _default
    if _default is None:
        _default = Oracle()
    return _default


def fft2d(x, inverse=False, **kw):
    return get().fft2d(x, inverse=inverse, **kw)


def rel_l2(a, b) -> float:
    """||a - b||_2 / ||b||_2 in float64 (b is the reference)."""
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    den = np.linalg.norm(b.ravel())
    num = np.linalg.norm((a - b).ravel())
    return float(num / den) if den > 0 else float(num)


def default_threads() -> int:
    return max(1, len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count() or 1)
