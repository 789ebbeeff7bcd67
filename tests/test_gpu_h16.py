"""Half2 storage (FFT2D_C32H): half2 pixels with one power-of-two exponent
per line, FP32 butterflies.  Accuracy target: relative L2 <= 5e-3 against
the FP64 oracle applied to the (dequantised) half2 input."""
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


def rel(a, b):
    a = np.asarray(a, np.complex128)
    b = np.asarray(b, np.complex128)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def pack(env, x):
    torch, fft, _ = env
    R, C = x.shape
    dx = torch.from_numpy(x).cuda()
    q = torch.empty((R, C, 2), dtype=torch.float16, device="cuda")
    e = torch.empty(R, dtype=torch.int32, device="cuda")
    fft.fft2d_h16_pack(R, C, dx, q, e)
    return q, e


def unpack(env, q, e, axis):
    torch, fft, _ = env
    R, C = q.shape[0], q.shape[1]
    out = torch.empty((R, C), dtype=torch.complex64, device="cuda")
    fft.fft2d_h16_unpack(R, C, q, e, axis, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def h16_fft(env, q, e, axis, direction):
    torch, fft, _ = env
    R, C = q.shape[0], q.shape[1]
    plan = fft.fft2d_plan(R, C, fft.FFT2D_C32H, direction)
    try:
        out = torch.empty_like(q)
        oe = torch.empty(C, dtype=torch.int32, device="cuda")
        fft.fft2d_exec_h16(plan, q, e, axis, out, oe)
        torch.cuda.synchronize()
        return out, oe
    finally:
        fft.fft2d_destroy(plan)


@pytest.mark.parametrize("shape", [(2, 2), (16, 4096), (256, 256), (1024, 1024), (2048, 512),
                                   (64, 8192), (4096, 4096), (8192, 8192)],
                         ids=lambda s: f"{s[0]}x{s[1]}")
def test_h16_forward_matches_oracle(env, shape):
    torch, fft, orc = env
    R, C = shape
    x = synth.uniform_complex(R, C, seed=R ^ C)
    q, e = pack(env, x)
    xin = unpack(env, q, e, fft.FFT2D_PASS_ROWS)          # the input as stored
    assert rel(xin, x) < 1e-3                                # packing itself is half precision
    out, oe = h16_fft(env, q, e, fft.FFT2D_PASS_ROWS, fft.FFT2D_FORWARD)
    got = unpack(env, out, oe, fft.FFT2D_PASS_COLS)
    want = orc.fft2d(xin, threads=16)
    err = rel(got, want)
    print(f"[h16] {R}x{C} fwd rel_l2={err:.3e}")
    assert err <= TOL_H16
    # every stored half lies below 2^14 and the exponents are in range
    qa = out.float().abs().max().item()
    assert 0 < qa <= 16384      # |q| < 2^14 before rounding to half
    assert int(oe.abs().max().item()) < 200


def test_h16_round_trip(env):
    torch, fft, orc = env
    R, C = 1024, 2048
    x = synth.blob_image(R, C, seed=5)
    q, e = pack(env, x)
    xin = unpack(env, q, e, fft.FFT2D_PASS_ROWS)
    fq, fe = h16_fft(env, q, e, fft.FFT2D_PASS_ROWS, fft.FFT2D_FORWARD)
    # inverse of a column-scaled spectrum
    bq, be = h16_fft(env, fq, fe, fft.FFT2D_PASS_COLS, fft.FFT2D_INVERSE)
    back = unpack(env, bq, be, fft.FFT2D_PASS_COLS)
    err = rel(back, xin)
    print(f"[h16] {R}x{C} round trip rel_l2={err:.3e}")
    assert err <= TOL_H16


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
