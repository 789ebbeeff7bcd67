"""GPU 2D DCT-II (plans of dtype FFT2D_R32_DCT2) against the FP64 oracle.

The oracle's DCT is the definition evaluated directly (no FFT), so these
tests check the whole GPU route -- the even/odd reordering fused into the
scrambled read, two real lines packed into one complex line, the radix-2
stages and the post-rotation by exp(-i pi k / (2N)) -- against it.

Tolerance: relative L2 error <= 1e-5 over whole outputs (the FP32 target of
the complex path; the DCT adds one rotation per output).  Where the oracle's
O(R C (R + C)) cost is too high (sides of 4096 and more), sampled outputs are
checked one by one against the unseparated double sum:

* zero-mean images: each output within 1e-5 (4 rms(X) + |X|), rms(X) =
  ||x||_2 / 2 being the root mean square of an unnormalised 2D DCT-II output
  (Parseval, up to the k = 0 rows);
* gray images in [0, 1): their large mean makes the radix-2 tree form
  outputs such as X[R/2][0] as differences of two partial sums of about
  R C / 4 each, so an output's FP32 error is set by ||X||_2, not by |X|:
  each within u log2(R C) sqrt(R C) ||x||_2 (u = 2^-24; the radix-2 error
  bound of order u log2(n) ||X||_2, with ||X||_2 <= sqrt(R C) ||x||_2).

A cosine basis image must also land on its single index, with every other
output small.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5


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
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    d = np.linalg.norm(b.ravel())
    return float(np.linalg.norm((a - b).ravel()) / (d if d > 0 else 1.0))


def gpu_dct(env, x, inplace=False, passes=None, inverse=False):
    torch, fft, _ = env
    R, C = x.shape
    plan = fft.fft2d_plan(R, C, fft.FFT2D_R32_DCT2,
                          fft.FFT2D_INVERSE if inverse else fft.FFT2D_FORWARD)
    try:
        dx = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()
        out = dx if inplace else torch.empty_like(dx)
        if passes is None:
            fft.fft2d_exec(plan, dx, out)
        else:
            src = dx
            for p in passes:
                fft.fft2d_exec_pass(plan, p, src, out)
                src = out
        torch.cuda.synchronize()
        return out.cpu().numpy()
    finally:
        fft.fft2d_destroy(plan)


@pytest.mark.parametrize("rows", [2, 4, 8, 16, 32])
@pytest.mark.parametrize("cols", [2, 4, 8, 16, 32])
def test_dct_small_shapes(env, rows, cols):
    """Every shape with sides 2..32: the in-register lines (up to 16 points,
    one stage group) and the shared-memory exchange (32 points)."""
    _, _, orc = env
    x = synth.gray_real(rows, cols, seed=rows * 100 + cols)
    err = rel(gpu_dct(env, x), orc.dct2d(x))
    assert err <= TOL, err


@pytest.mark.parametrize("rows,cols", [(64, 256), (256, 64), (2, 1024), (1024, 2),
                                       (512, 512), (128, 2048), (1024, 1024),
                                       (2048, 64), (4096, 32), (2048, 8), (4096, 4),
                                       (8192, 16), (8192, 8), (8192, 4), (16384, 8),
                                       (16384, 32), (16384, 4)])
def test_dct_whole_outputs(env, rows, cols):
    """Non-square and wide/tall images spanning several CTAs and a partly
    filled last CTA (2 rows: one complex line), whole outputs compared.
    Columns of 2048 and 4096 rows run on the TMA-fed column kernel when the
    image is at least two tiles wide (64 and 32 columns here) and on the
    plain kernel otherwise (8 and 4 columns).  Forward columns of 8192 and
    16384 rows run on the cluster kernels with two real columns per complex
    line when the width is a multiple of 8 (one to four 8-column tiles
    here); otherwise on the plain kernel (8192 x 4) or the four-CTA kernel
    with one complex line per real column (16384 x 4)."""
    _, _, orc = env
    x = synth.gray_real(rows, cols, seed=7)
    err = rel(gpu_dct(env, x), orc.dct2d(x))
    print(f"[dct] {rows}x{cols}: rel_l2={err:.3e}")
    assert err <= TOL, err


def test_dct_blob_in_place(env):
    """Smooth image (Gaussian blobs + noise), output written over the input."""
    _, _, orc = env
    x = np.ascontiguousarray(synth.blob_image(256, 512, seed=3).real)
    err = rel(gpu_dct(env, x, inplace=True), orc.dct2d(x))
    assert err <= TOL, err


@pytest.mark.parametrize("rows,cols", [(64, 128), (16, 2048), (2048, 16), (8, 4096)])
def test_dct_single_passes(env, rows, cols):
    """fft2d_exec_pass: the row pass alone is the 1D DCT-II of every row, the
    column pass alone that of every column; rows then columns is the 2D
    transform."""
    _, fft, orc = env
    x = synth.gray_real(rows, cols, seed=11)
    rows_only = np.stack([orc.dct1d(r) for r in x.astype(np.float64)])
    cols_only = np.stack([orc.dct1d(c) for c in x.astype(np.float64).T]).T
    assert rel(gpu_dct(env, x, passes=[fft.FFT2D_PASS_ROWS]), rows_only) <= TOL
    assert rel(gpu_dct(env, x, passes=[fft.FFT2D_PASS_COLS]), cols_only) <= TOL
    both = gpu_dct(env, x, passes=[fft.FFT2D_PASS_ROWS, fft.FFT2D_PASS_COLS])
    assert rel(both, orc.dct2d(x)) <= TOL


def sample_indices(R, C, n, seed):
    g = np.random.default_rng(seed)
    fixed = [(0, 0), (0, C // 2), (R // 2, 0), (R // 2, C // 2), (R - 1, C - 1), (1, C - 1),
             (R - 1, 1), (R // 2 - 1, C // 2 + 1)]
    rnd = [(int(a), int(b)) for a, b in zip(g.integers(0, R, n), g.integers(0, C, n))]
    return fixed + rnd


@pytest.mark.parametrize("side,nsamp", [(4096, 16), (8192, 6), (16384, 2)])
def test_dct_large_sampled(env, side, nsamp):
    """The full-size images: sampled outputs against the direct double sum."""
    _, _, orc = env
    idx = sample_indices(side, side, nsamp, seed=side)
    gray = synth.gray_real(side, side, seed=5)
    got = gpu_dct(env, gray)
    bound = 2.0 ** -24 * np.log2(side * side) * side * float(np.linalg.norm(gray.astype(np.float64)))
    for k, l in idx:
        want = orc.dct2d_at(gray, k, l)
        assert abs(float(got[k, l]) - want) <= bound, ("gray", k, l, float(got[k, l]), want)
    zm = gray - np.float32(0.5)   # exact in FP32
    got = gpu_dct(env, zm)
    rms = float(np.linalg.norm(zm.astype(np.float64))) / 2.0
    for k, l in idx:
        want = orc.dct2d_at(zm, k, l)
        assert abs(float(got[k, l]) - want) <= TOL * (4.0 * rms + abs(want)), \
            ("zero-mean", k, l, float(got[k, l]), want)


@pytest.mark.parametrize("rows,cols,inplace", [(4096, 4096, False), (2048, 16384, False),
                                               (8192, 8192, False), (16384, 512, False),
                                               (4096, 64, False), (2048, 1024, True),
                                               (4096, 8192, True), (16384, 256, True)])
def test_dct_separable_full(env, rows, cols, inplace):
    """A separable image x[m][n] = f[m] g[n] (small integers: the products
    are exact in FP32) has X[k][l] = F[k] G[l] with F, G the 1D transforms
    of f and g, which the oracle computes cheaply: every output of a dense
    full-size image is checked, in every column tile of every CTA."""
    _, _, orc = env
    g = np.random.default_rng(rows + cols)
    f = g.integers(0, 16, rows).astype(np.float64)
    h = g.integers(-8, 8, cols).astype(np.float64)
    x = np.outer(f, h).astype(np.float32)
    got = gpu_dct(env, x, inplace=inplace)
    want = np.outer(orc.dct1d(f), orc.dct1d(h))
    err = rel(got, want)
    print(f"[dct] separable {rows}x{cols}: rel_l2={err:.3e}")
    assert err <= TOL, err


@pytest.mark.parametrize("rows,cols,k0,l0", [(4096, 4096, 37, 1900), (4096, 4096, 2048, 0),
                                            (8192, 2048, 8191, 1023), (2048, 16384, 5, 16383)])
def test_dct_basis_image(env, rows, cols, k0, l0):
    """A cosine basis image cos(pi k0 (2m+1)/(2R)) cos(pi l0 (2n+1)/(2C)) lands
    on (k0, l0) alone, with weight (R/2 or R)(C/2 or C): every output is
    checked, at full size, without the oracle."""
    m = np.arange(rows, dtype=np.float64)
    n = np.arange(cols, dtype=np.float64)
    x = np.outer(np.cos(np.pi * k0 * (2 * m + 1) / (2 * rows)),
                 np.cos(np.pi * l0 * (2 * n + 1) / (2 * cols))).astype(np.float32)
    got = gpu_dct(env, x)
    spike = (rows if k0 == 0 else rows / 2) * (cols if l0 == 0 else cols / 2)
    assert abs(float(got[k0, l0]) - spike) <= 1e-5 * spike
    got[k0, l0] = 0.0
    assert float(np.abs(got).max()) <= 1e-5 * spike


def test_dct_plan_rules(env):
    """DCT plans: sides of 1 are not provided; the complex-only entry points
    refuse the plan; describe names the DCT passes."""
    torch, fft, _ = env
    import ctypes
    h = ctypes.c_void_p()
    assert fft.lib.fft2d_plan(1, 8, fft.FFT2D_R32_DCT2, fft.FFT2D_FORWARD,
                              ctypes.byref(h)) == fft.FFT2D_ERR_UNSUPPORTED
    plan = fft.fft2d_plan(16, 32, fft.FFT2D_R32_DCT2, fft.FFT2D_FORWARD)
    try:
        assert "dct2" in fft.fft2d_plan_describe(plan)
        assert fft.fft2d_plan_info(plan)[2] == fft.FFT2D_R32_DCT2
        d = torch.zeros(16, 32, device="cuda")
        assert fft.lib.fft2d_exec_stages(plan, d.data_ptr(), d.data_ptr(), 1, 1,
                                         None) == fft.FFT2D_ERR_ARG
        assert fft.lib.fft2d_autotune(plan, None) == fft.FFT2D_ERR_ARG
        assert fft.lib.fft2d_plan_set_variant(plan, 0, 0) == fft.FFT2D_ERR_ARG
    finally:
        fft.fft2d_destroy(plan)


def test_dct_host_buffers(env):
    """fft2d_exec_host on a DCT plan: 4-byte pixels copied in and out."""
    _, fft, orc = env
    x = synth.gray_real(128, 256, seed=2)
    out = np.empty_like(x)
    plan = fft.fft2d_plan(128, 256, fft.FFT2D_R32_DCT2, fft.FFT2D_FORWARD)
    try:
        fft.fft2d_exec_host(plan, x, out)
    finally:
        fft.fft2d_destroy(plan)
    assert rel(out, orc.dct2d(x)) <= TOL


# ------------------------------------------------------------------ inverse
@pytest.mark.parametrize("rows", [2, 4, 8, 16, 32])
@pytest.mark.parametrize("cols", [2, 8, 32])
def test_idct_small_shapes(env, rows, cols):
    """DCT-III (the oracle's scaled inverse) of small spectra."""
    _, _, orc = env
    X = synth.gray_real(rows, cols, seed=rows * 31 + cols) - np.float32(0.5)
    err = rel(gpu_dct(env, X, inverse=True), orc.dct2d(X, inverse=True))
    assert err <= TOL, err


@pytest.mark.parametrize("rows,cols", [(64, 256), (256, 64), (2, 1024), (1024, 2),
                                       (512, 512), (2048, 64), (4096, 32), (128, 2048),
                                       (8192, 16), (8192, 4), (16384, 4)])
def test_idct_whole_outputs(env, rows, cols):
    _, _, orc = env
    X = synth.gray_real(rows, cols, seed=9) - np.float32(0.5)
    err = rel(gpu_dct(env, X, inverse=True), orc.dct2d(X, inverse=True))
    print(f"[idct] {rows}x{cols}: rel_l2={err:.3e}")
    assert err <= TOL, err


def test_idct_plan_describe(env):
    _, fft, _ = env
    plan = fft.fft2d_plan(32, 64, fft.FFT2D_R32_DCT2, fft.FFT2D_INVERSE)
    try:
        assert fft.fft2d_plan_describe(plan) == \
            "rows:dct3(lines=16,points=64) cols:dct3(lines=32,points=32)"
    finally:
        fft.fft2d_destroy(plan)


def test_idct_in_place_and_passes(env):
    """In place; the row pass alone is the unscaled DCT-III of every row
    (cols times the oracle's inverse), the column pass alone carries the
    whole 1/(rows cols)."""
    _, fft, orc = env
    R, C = 64, 128
    X = synth.gray_real(R, C, seed=4) - np.float32(0.5)
    assert rel(gpu_dct(env, X, inplace=True, inverse=True), orc.dct2d(X, inverse=True)) <= TOL
    X64 = X.astype(np.float64)
    rows_only = np.stack([orc.dct1d(r, inverse=True) for r in X64]) * C
    cols_only = np.stack([orc.dct1d(c, inverse=True) for c in X64.T]).T / C
    assert rel(gpu_dct(env, X, passes=[fft.FFT2D_PASS_ROWS], inverse=True), rows_only) <= TOL
    assert rel(gpu_dct(env, X, passes=[fft.FFT2D_PASS_COLS], inverse=True), cols_only) <= TOL


@pytest.mark.parametrize("rows,cols,inplace", [(4096, 4096, False), (2048, 16384, False),
                                               (8192, 8192, False), (16384, 512, False),
                                               (2048, 1024, True), (4096, 8192, True),
                                               (16384, 256, True)])
def test_idct_separable_full(env, rows, cols, inplace):
    """Separable spectrum F[k] G[l] (small integers): the inverse is the outer
    product of the 1D inverses, every output checked."""
    _, _, orc = env
    g = np.random.default_rng(rows * 3 + cols)
    f = g.integers(-8, 8, rows).astype(np.float64)
    h = g.integers(-8, 8, cols).astype(np.float64)
    X = np.outer(f, h).astype(np.float32)
    got = gpu_dct(env, X, inverse=True, inplace=inplace)
    want = np.outer(orc.dct1d(f, inverse=True), orc.dct1d(h, inverse=True))
    err = rel(got, want)
    print(f"[idct] separable {rows}x{cols}: rel_l2={err:.3e}")
    assert err <= TOL, err


@pytest.mark.parametrize("rows,cols", [(4096, 4096), (8192, 1024), (256, 16384), (16384, 64)])
def test_dct_round_trip(env, rows, cols):
    """Forward then inverse on the GPU gives the image back."""
    x = synth.gray_real(rows, cols, seed=12)
    err = rel(gpu_dct(env, gpu_dct(env, x), inverse=True), x)
    print(f"[dct] round trip {rows}x{cols}: rel_l2={err:.3e}")
    assert err <= TOL, err


@pytest.mark.parametrize("rows,inverse", [(4096, False), (2048, True), (4096, True), (8192, False),
                                          (8192, True), (16384, False), (16384, True)])
def test_dct_withheld_load_times_out_cleanly(env, rows, inverse):
    """Failure path of the TMA-fed DCT column kernels: CTA 0 never issues the
    second load of its first tile, its bounded wait gives up, the host reads
    FFT2D_ERR_TIMEOUT, and the same plan then transforms correctly (8192
    rows: the CTA-pair kernel, both CTAs leave together; 16384 rows: the
    four-CTA kernel, all four leave together)."""
    torch, fft, orc = env
    cols = 64
    plan = fft.fft2d_plan(rows, cols, fft.FFT2D_R32_DCT2,
                          fft.FFT2D_INVERSE if inverse else fft.FFT2D_FORWARD)
    try:
        x = synth.gray_real(rows, cols, seed=rows) - np.float32(0.5)
        dx = torch.from_numpy(x).cuda()
        out = torch.empty_like(dx)
        fft.fft2d_sync_status(plan)
        fft.fft2d_selftest_withheld_load(plan, dx, out)
        with pytest.raises(fft.FFT2DError) as ei:
            fft.fft2d_sync_status(plan)
        assert ei.value.status == fft.FFT2D_ERR_TIMEOUT
        fft.fft2d_sync_status(plan)                      # cleared
        fft.fft2d_exec(plan, dx, out)
        fft.fft2d_sync_status(plan)
        assert rel(out.cpu().numpy(), orc.dct2d(x, inverse=inverse)) <= TOL
    finally:
        fft.fft2d_destroy(plan)


def test_dct_withheld_load_needs_a_tma_kernel(env):
    """Columns of 1024 points (plain kernel): the self-test is refused."""
    torch, fft, _ = env
    plan = fft.fft2d_plan(1024, 64, fft.FFT2D_R32_DCT2, fft.FFT2D_FORWARD)
    try:
        dx = torch.zeros((1024, 64), device="cuda")
        with pytest.raises(fft.FFT2DError) as ei:
            fft.fft2d_selftest_withheld_load(plan, dx, dx)
        assert ei.value.status == fft.FFT2D_ERR_ARG
    finally:
        fft.fft2d_destroy(plan)


def test_dct_host_pipeline_mixed(env):
    """fft2d_exec_host_many with DCT plans (forward, then the inverse of the
    same buffer in one call) mixed with a complex64 FFT plan."""
    torch, fft, orc = env
    x = synth.gray_real(256, 512, seed=21)
    z = synth.uniform_complex(128, 128, seed=22)
    pf = fft.fft2d_plan(256, 512, fft.FFT2D_R32_DCT2, fft.FFT2D_FORWARD)
    pi = fft.fft2d_plan(256, 512, fft.FFT2D_R32_DCT2, fft.FFT2D_INVERSE)
    pc = fft.fft2d_plan(128, 128, fft.FFT2D_C64, fft.FFT2D_FORWARD)
    try:
        hx = torch.from_numpy(x).pin_memory()
        hX = torch.empty_like(hx).pin_memory()
        hback = torch.empty_like(hx).pin_memory()
        hz = torch.from_numpy(z).pin_memory()
        hZ = torch.empty_like(hz).pin_memory()
        fft.fft2d_exec_host_many([pf, pc, pi], [hx, hz, hX], [hX, hZ, hback])
        assert rel(hX.numpy(), orc.dct2d(x)) <= TOL
        assert rel(hback.numpy(), x) <= TOL
        zc = np.asarray(hZ.numpy(), np.complex128)
        want = orc.fft2d(z)
        assert float(np.linalg.norm(zc - want) / np.linalg.norm(want)) <= TOL
    finally:
        for p in (pf, pi, pc):
            fft.fft2d_destroy(p)
