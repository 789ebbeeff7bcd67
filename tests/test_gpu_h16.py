"""Half2 storage (FFT2D_C32H): half2 pixels with one power-of-two exponent
per line, FP32 butterflies.  Accuracy target: relative L2 <= 5e-3 against
the FP64 oracle applied to the dequantised half2 input.

The checking side never goes through the library's own conversions: inputs
are quantised and outputs dequantised here in numpy, from the format's
definition (value = q * 2^e, e = k - 14 for a line whose largest component
magnitude is f 2^k, f in [0.5, 1)).  The library's fft2d_h16_pack and
fft2d_h16_unpack are checked against that definition separately."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

TOL_H16 = 5e-3


@pytest.fixture(scope="module")
def env(orc):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from conftest import build_lib
    build_lib()
    import paper_1505_08019_gb300 as fft
    return torch, fft, orc


def rel(a, b, chunk=1 << 24):
    """||a - b|| / ||b|| in float64, in chunks (images up to 16384^2)."""
    a = np.asarray(a).reshape(-1)
    b = np.asarray(b).reshape(-1)
    num = den = 0.0
    for i in range(0, b.size, chunk):
        bb = b[i:i + chunk].astype(np.complex128)
        d = a[i:i + chunk].astype(np.complex128) - bb
        num += float(np.vdot(d, d).real)
        den += float(np.vdot(bb, bb).real)
    return float(np.sqrt(num / den))


def line_exponents(x, axis):
    """The format's exponent of every line (axis 0: one per row, 1: one per
    column) of a complex array: e = k - 14 with max |component| = f 2^k,
    f in [0.5, 1); 0 for an all-zero line."""
    m = np.maximum(np.abs(x.real), np.abs(x.imag)).max(axis=1 - axis).astype(np.float64)
    _, k = np.frexp(m)
    return np.where(m > 0, k - 14, 0).astype(np.int32)


def quantise_rows(x):
    """complex64 image -> (half2 array [R, C, 2], per-row int32 exponents):
    x scaled by 2^-e (exact in FP32) and rounded to half precision."""
    e = line_exponents(x, 0)
    f = np.ldexp(np.float32(1.0), -e).astype(np.float32)[:, None]
    q = np.empty(x.shape + (2,), np.float16)
    q[..., 0] = (x.real * f).astype(np.float16)
    q[..., 1] = (x.imag * f).astype(np.float16)
    return q, e


def dequantise(q, e, axis):
    """half2 [R, C, 2] + exponents per row (axis 0) or column (axis 1) ->
    complex128 values q * 2^e."""
    s = np.ldexp(1.0, e.astype(np.int64))
    s = s[:, None] if axis == 0 else s[None, :]
    return (q[..., 0].astype(np.float64) * s) + 1j * (q[..., 1].astype(np.float64) * s)


def check_column_format(q, e):
    """The stored-format invariants of a column-pass output, from q and e
    alone: the largest |component| of every nonzero column lies in
    [2^13, 2^14] (its exponent was chosen from that column's maximum)."""
    qa = np.maximum(np.abs(q[..., 0].astype(np.float32)), np.abs(q[..., 1].astype(np.float32)))
    colmax = qa.max(axis=0)
    nz = colmax > 0
    assert np.all(colmax[nz] >= 2.0 ** 13) and np.all(colmax[nz] <= 2.0 ** 14)
    assert np.all(np.abs(e) < 200)


def h16_fft(env, q, e, axis, direction):
    """Device transform of host half2 data q with exponents e; returns the
    raw half2 output and its per-column exponents as numpy arrays."""
    torch, fft, _ = env
    R, C = q.shape[0], q.shape[1]
    plan = fft.fft2d_plan(R, C, fft.FFT2D_C32H, direction)
    try:
        dq = torch.from_numpy(q).cuda()
        de = torch.from_numpy(e).cuda()
        out = torch.empty_like(dq)
        oe = torch.empty(C, dtype=torch.int32, device="cuda")
        fft.fft2d_exec_h16(plan, dq, de, axis, out, oe)
        torch.cuda.synchronize()
        return out.cpu().numpy(), oe.cpu().numpy()
    finally:
        fft.fft2d_destroy(plan)


@pytest.mark.parametrize("shape", [(2, 2), (16, 4096), (256, 256), (1024, 1024), (2048, 512),
                                   (64, 8192), (4096, 4096), (8192, 8192), (16384, 16384)],
                         ids=lambda s: f"{s[0]}x{s[1]}")
def test_h16_forward_matches_oracle(env, shape):
    torch, fft, orc = env
    R, C = shape
    x = synth.uniform_complex(R, C, seed=R ^ C)
    q, e = quantise_rows(x)
    xin = dequantise(q, e, 0)                               # the input as stored
    assert rel(xin, x) < 1e-3                               # half precision, per-row scale
    del x
    out, oe = h16_fft(env, q, e, fft.FFT2D_PASS_ROWS, fft.FFT2D_FORWARD)
    check_column_format(out, oe)
    want = orc.fft2d(xin, threads=16)
    del xin
    err = rel(dequantise(out, oe, 1), want)
    print(f"[h16] {R}x{C} fwd rel_l2={err:.3e}")
    assert err <= TOL_H16


@pytest.mark.parametrize("shape,direction", [((8192, 256), -1), ((8192, 256), 1),
                                             ((16384, 64), -1), ((16384, 64), 1),
                                             ((4096, 1024), 1)],
                         ids=lambda p: str(p))
def test_h16_cluster_and_tma_column_kernels_both_directions(env, shape, direction):
    """The half2 column kernels of 4096, 8192 and 16384 rows (one CTA, a CTA
    pair, four CTAs) in both directions, on narrow images: the inverse
    carries the 1/(rows cols) scale into the exponent choice."""
    torch, fft, orc = env
    R, C = shape
    x = synth.uniform_complex(R, C, seed=R + C + direction)
    q, e = quantise_rows(x)
    xin = dequantise(q, e, 0)
    out, oe = h16_fft(env, q, e, fft.FFT2D_PASS_ROWS, direction)
    check_column_format(out, oe)
    want = orc.fft2d(xin, inverse=(direction == 1), threads=16)
    err = rel(dequantise(out, oe, 1), want)
    print(f"[h16] {R}x{C} dir={direction} rel_l2={err:.3e}")
    assert err <= TOL_H16


def test_h16_round_trip(env):
    torch, fft, orc = env
    R, C = 1024, 2048
    x = synth.blob_image(R, C, seed=5)
    q, e = quantise_rows(x)
    xin = dequantise(q, e, 0)
    fq, fe = h16_fft(env, q, e, fft.FFT2D_PASS_ROWS, fft.FFT2D_FORWARD)
    check_column_format(fq, fe)
    # inverse of a column-scaled spectrum, against the oracle's inverse of
    # the stored spectrum and against the stored input
    bq, be = h16_fft(env, fq, fe, fft.FFT2D_PASS_COLS, fft.FFT2D_INVERSE)
    check_column_format(bq, be)
    back = dequantise(bq, be, 1)
    e_inv = rel(back, orc.fft2d(dequantise(fq, fe, 1), inverse=True, threads=16))
    err = rel(back, xin)
    print(f"[h16] {R}x{C} inverse rel_l2={e_inv:.3e}, round trip rel_l2={err:.3e}")
    assert e_inv <= TOL_H16 and err <= TOL_H16


@pytest.mark.parametrize("shape", [(4, 8), (64, 256), (512, 128)], ids=lambda s: f"{s[0]}x{s[1]}")
def test_h16_pack_unpack_follow_the_format(env, shape):
    """The library's conversions against the format's definition: packing is
    bit-exact (same exponent rule, same scaling by a power of two, round to
    nearest even), unpacking exact (q * 2^e fits in FP32), along both axes."""
    torch, fft, _ = env
    R, C = shape
    x = synth.uniform_complex(R, C, seed=R + C)
    x[R // 2] = 0                                            # an all-zero row
    x[1] *= np.float32(2.0 ** -30)                           # a tiny one
    q, e = quantise_rows(x)
    dx = torch.from_numpy(x).cuda()
    dq = torch.empty((R, C, 2), dtype=torch.float16, device="cuda")
    de = torch.empty(R, dtype=torch.int32, device="cuda")
    fft.fft2d_h16_pack(R, C, dx, dq, de)
    torch.cuda.synchronize()
    assert np.array_equal(de.cpu().numpy(), e)
    assert np.array_equal(dq.cpu().numpy().view(np.uint16), q.view(np.uint16))
    for axis, ex in ((0, e), (1, np.arange(C, dtype=np.int32) % 7 - 3)):
        out = torch.empty((R, C), dtype=torch.complex64, device="cuda")
        fft.fft2d_h16_unpack(R, C, torch.from_numpy(q).cuda(), torch.from_numpy(ex).cuda(),
                             axis, out)
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy().astype(np.complex128), dequantise(q, ex, axis))


def test_h16_rejects_complex64_calls(env):
    torch, fft, _ = env
    plan = fft.fft2d_plan(64, 64, fft.FFT2D_C32H, fft.FFT2D_FORWARD)
    try:
        x = torch.zeros(64, 64, dtype=torch.complex64, device="cuda")
        with pytest.raises(fft.FFT2DError):
            fft.fft2d_exec(plan, x, x)
    finally:
        fft.fft2d_destroy(plan)
    with pytest.raises(fft.FFT2DError):
        fft.fft2d_plan(1, 64, fft.FFT2D_C32H, fft.FFT2D_FORWARD)
