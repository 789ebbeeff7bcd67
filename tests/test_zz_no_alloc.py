"""fft2d_exec_noalloc -- the plan-free entry point for callers that cannot
allocate device memory (a plug-in in a host application that owns the whole
device, a process whose caching allocator holds the free memory, paths where
cudaMalloc's implicit synchronisation is not allowed) -- must give the same
results as fft2d_exec, within the FP32 tolerance of the other GPU tests, call
after call on its shared static scratch.  Collected last on purpose."""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from conftest import build_lib
    build_lib()
    import paper_1505_08019_gb300 as fft
    return torch, fft


def rel(a, b):
    a = np.asarray(a, np.complex128)
    b = np.asarray(b, np.complex128)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def via_plan(torch, fft, x, direction):
    R, C = x.shape
    plan = fft.fft2d_plan(R, C, fft.FFT2D_C64, direction)
    try:
        dx = torch.from_numpy(x).cuda()
        out = torch.empty_like(dx)
        fft.fft2d_exec(plan, dx, out)
        torch.cuda.synchronize()
        return out.cpu().numpy()
    finally:
        fft.fft2d_destroy(plan)


def test_noalloc_matches_plan_exec_on_consecutive_calls(env):
    torch, fft = env
    cases = [((4096, 4096), fft.FFT2D_FORWARD, 0),    # the benchmarked size
             ((256, 1024), fft.FFT2D_INVERSE, 1),     # next call: new shape, new direction
             ((4096, 4096), fft.FFT2D_FORWARD, 2)]    # and back, tables rewritten again
    for (R, C), direction, seed in cases:
        x = synth.uniform_complex(R, C, seed=seed)
        want = via_plan(torch, fft, x, direction)
        dx = torch.from_numpy(x).cuda()
        out = torch.empty_like(dx)
        fft.fft2d_exec_noalloc(R, C, direction, dx, out)
        torch.cuda.synchronize()
        err = rel(out.cpu().numpy(), want)
        print(f"[noalloc] {R}x{C} dir={direction}: rel_l2 vs fft2d_exec = {err:.2e}")
        assert err <= TOL


def test_noalloc_in_place_and_limits(env):
    torch, fft = env
    x = synth.blob_image(512, 512, seed=3)
    want = via_plan(torch, fft, x, fft.FFT2D_FORWARD)
    buf = torch.from_numpy(x).cuda()
    fft.fft2d_exec_noalloc(512, 512, fft.FFT2D_FORWARD, buf, buf)
    torch.cuda.synchronize()
    assert rel(buf.cpu().numpy(), want) <= TOL
    # beyond the static array's limit: rejected up front, nothing launched
    big = torch.zeros(8, dtype=torch.complex64, device="cuda")
    st = fft.lib.fft2d_exec_noalloc(8192, 8, fft.FFT2D_FORWARD, ctypes.c_void_p(big.data_ptr()),
                                    ctypes.c_void_p(big.data_ptr()), None)
    assert st == fft.FFT2D_ERR_TOO_LARGE
    st = fft.lib.fft2d_exec_noalloc(12, 8, fft.FFT2D_FORWARD, ctypes.c_void_p(big.data_ptr()),
                                    ctypes.c_void_p(big.data_ptr()), None)
    assert st == fft.FFT2D_ERR_NOT_POW2


@pytest.mark.parametrize("shape", [(1, 1024), (1024, 1), (1, 1)], ids=lambda s: f"{s[0]}x{s[1]}")
def test_noalloc_single_line_shapes(env, shape):
    """The entry point's own branches: a single row (the inverse scale rides
    on the row pass), a single column (the row pass is a copy, or nothing in
    place), both directions, in place and out of place."""
    torch, fft = env
    R, C = shape
    for direction in (fft.FFT2D_FORWARD, fft.FFT2D_INVERSE):
        x = synth.uniform_complex(R, C, seed=R + 2 * C + direction)
        want = via_plan(torch, fft, x, direction)
        dx = torch.from_numpy(x).cuda()
        out = torch.empty_like(dx)
        fft.fft2d_exec_noalloc(R, C, direction, dx, out)
        fft.fft2d_exec_noalloc(R, C, direction, dx, dx)
        torch.cuda.synchronize()
        assert rel(out.cpu().numpy(), want) <= TOL
        assert rel(dx.cpu().numpy(), want) <= TOL


@pytest.mark.parametrize("shape,direction", [((4096, 4096), -1), ((256, 1024), 1), ((2048, 32), -1)],
                         ids=["4096x4096_fwd", "256x1024_inv", "2048x32_fwd"])
def test_noalloc_matches_oracle(env, orc, shape, direction):
    """The entry point's rotation factors are computed on the device, not
    taken from the plan's FP64 tables, so it is also compared with the FP64
    oracle of eqs. 2-3 directly (inverse scaled by 1/(rows*cols))."""
    torch, fft = env
    R, C = shape
    x = synth.uniform_complex(R, C, seed=R + C)
    dx = torch.from_numpy(x).cuda()
    out = torch.empty_like(dx)
    fft.fft2d_exec_noalloc(R, C, fft.FFT2D_FORWARD if direction < 0 else fft.FFT2D_INVERSE, dx, out)
    torch.cuda.synchronize()
    want = orc.fft2d(x, inverse=direction > 0, threads=8)
    err = rel(out.cpu().numpy(), want)
    print(f"[noalloc] {R}x{C} dir={direction}: rel_l2 vs oracle = {err:.2e}")
    assert err <= TOL
