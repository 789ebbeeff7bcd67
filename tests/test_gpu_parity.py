"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Tolerance (the accuracy target for the FP32 complex64 path): relative L2
error <= 1e-5 against the FP64 oracle on the same seeded input.  Integer and
permutation work (scramble-only and exactly representable stages) must be
bit-exact.
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
    a = np.asarray(a, np.complex128)
    b = np.asarray(b, np.complex128)
    d = np.linalg.norm(b.ravel())
    return float(np.linalg.norm((a - b).ravel()) / (d if d > 0 else 1.0))


def gpu_fft(env, x, direction, inplace=False, stages=None):
    torch, fft, _ = env
    R, C = x.shape
    plan = fft.fft2d_plan(R, C, fft.FFT2D_C64, direction)
    try:
        dx = torch.from_numpy(np.ascontiguousarray(x)).cuda()
        out = dx if inplace else torch.empty_like(dx)
        if stages is None:
            fft.fft2d_exec(plan, dx, out)
        else:
            fft.fft2d_exec_stages(plan, dx, out, stages[0], stages[1])
        torch.cuda.synchronize()
        return out.cpu().numpy()
    finally:
        fft.fft2d_destroy(plan)


def report(name, err):
    print(f"[parity] {name}: rel_l2={err:.3e}")


# ------------------------------------------------------------------ configs
def test_256_gray_forward(env):
    """256x256, real part U[0,1), imaginary 0, forward, plain path."""
    _, _, orc = env
    x = synth.uniform_real(256, 256, seed=0)
    got = gpu_fft(env, x, -1)
    want = orc.fft2d(x)
    err = rel(got, want)
    report("256x256 fwd", err)
    assert err <= TOL
    # crops of the input through the direct double sum (eq. 1): the GPU's
    # 16x16 transform of the crop must match too
    for r0, c0 in ((0, 0), (120, 120)):
        crop = np.ascontiguousarray(x[r0:r0 + 16, c0:c0 + 16])
        assert rel(gpu_fft(env, crop, -1), orc.dft2d(crop)) <= TOL


@pytest.mark.parametrize("side", [1024, 4096, 8192])
def test_blob_forward_inverse(env, side):
    """Forward + inverse on the Gaussian-blob image at the paper's size, at
    4096x4096 (the benchmarked workload) and at 8192x8192 (columns on the
    CTA-pair kernel), whole outputs compared."""
    _, _, orc = env
    x = synth.blob_image(side, side, seed=0)
    X = gpu_fft(env, x, -1)
    Xo = orc.fft2d(x, threads=16)
    e_fwd = rel(X, Xo)
    y = gpu_fft(env, X, 1)
    e_inv = rel(y, orc.fft2d(X, inverse=True, threads=16))
    e_rt = rel(y, x)
    report(f"{side}^2 fwd", e_fwd)
    report(f"{side}^2 inv(of gpu fwd)", e_inv)
    report(f"{side}^2 round trip", e_rt)
    assert e_fwd <= TOL and e_inv <= TOL and e_rt <= TOL


SHAPES = [(1, 1), (1, 2), (2, 1), (2, 2), (4, 8), (8, 4), (16, 16), (32, 64), (64, 32),
          (128, 256), (256, 128), (512, 512), (2048, 128), (128, 2048), (256, 1024),
          (1024, 256), (2048, 2048), (16, 4096), (4096, 16), (64, 8192), (8192, 64),
          (16, 16384), (16384, 16), (1, 4096), (4096, 1), (2, 16384), (16384, 2)]


@pytest.mark.parametrize("shape", [(8192, 128), (16384, 64)], ids=lambda s: f"{s[0]}x{s[1]}")
def test_cluster_column_kernels_in_place(env, shape):
    """The CTA-pair and four-CTA column kernels with in == out, both
    directions (each CTA's output ranges are other CTAs' input rows)."""
    _, _, orc = env
    R, C = shape
    x = synth.uniform_complex(R, C, seed=R - C)
    for d, inv in ((-1, False), (1, True)):
        err = rel(gpu_fft(env, x, d, inplace=True), orc.fft2d(x, inverse=inv, threads=16))
        report(f"{R}x{C} in place {'inv' if inv else 'fwd'}", err)
        assert err <= TOL


@pytest.mark.parametrize("rows", [8192, 16384])
def test_l2_exchange_column_pass_on_concurrent_streams(env, rows):
    """The cluster column kernels that exchange through L2 take a scratch
    block per launch: the column passes of four images issued together on
    four streams with one plan give the same bits as one after another."""
    torch, fft, _ = env
    cols = 1024 if rows == 8192 else 512
    plan = fft.fft2d_plan(rows, cols, fft.FFT2D_C64, fft.FFT2D_FORWARD)
    try:
        assert "l2" in fft.fft2d_plan_describe(plan)
        dx = [torch.from_numpy(synth.uniform_complex(rows, cols, seed=rows + i)).cuda()
              for i in range(4)]
        want = []
        for d in dx:
            o = torch.empty_like(d)
            fft.fft2d_exec_pass(plan, fft.FFT2D_PASS_COLS, d, o)
            torch.cuda.synchronize()
            want.append(o.cpu().numpy())
        streams = [torch.cuda.Stream() for _ in range(4)]
        outs = [torch.empty_like(d) for d in dx]
        for _ in range(3):
            for o in outs:
                o.zero_()
            torch.cuda.synchronize()
            for st, d, o in zip(streams, dx, outs):
                fft.fft2d_exec_pass(plan, fft.FFT2D_PASS_COLS, d, o, st.cuda_stream)
            torch.cuda.synchronize()
            for i, (o, w) in enumerate(zip(outs, want)):
                assert np.array_equal(o.cpu().numpy(), w), f"image {i}"
        fft.fft2d_sync_status(plan)
    finally:
        fft.fft2d_destroy(plan)


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: f"{s[0]}x{s[1]}")
def test_shapes_both_directions(env, shape):
    _, _, orc = env
    R, C = shape
    x = synth.uniform_complex(R, C, seed=R * 7 + C)
    for d, inv in ((-1, False), (1, True)):
        err = rel(gpu_fft(env, x, d), orc.fft2d(x, inverse=inv, threads=8))
        report(f"{R}x{C} {'inv' if inv else 'fwd'}", err)
        assert err <= TOL


# ---------------------------------------------------------- bit-exact plumbing
@pytest.mark.parametrize("shape", [(8, 8), (64, 256), (512, 32), (4096, 4096), (16, 16384)],
                         ids=lambda s: f"{s[0]}x{s[1]}")
def test_scramble_only_is_exact_permutation(env, shape):
    """Zero butterfly stages: the fused scramble alone (Section 3.2) must equal
    the oracle's bit-reversal permutation bit for bit."""
    _, _, orc = env
    R, C = shape
    x = synth.uniform_complex(R, C, seed=5)
    got = gpu_fft(env, x, -1, stages=(0, 0))
    want = orc.fft2d(x, row_stages=0, col_stages=0).astype(np.complex64)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("shape,stages", [((16, 16), (2, 2)), ((256, 64), (1, 2)),
                                          ((1024, 1024), (2, 1)), ((64, 4096), (2, 2)),
                                          ((4096, 4096), (2, 2)), ((4, 4), (2, 2)),
                                          ((2, 4), (2, 1))])
def test_exact_stages_on_integers(env, shape, stages):
    """Stages 1-2 use only the rotation factors 1 and -i; on small-integer
    images every sum is exact in FP32, so the GPU must match the oracle bit
    for bit (this checks the scramble, the pairing of every butterfly, the
    stage order and the position order of partial results)."""
    _, _, orc = env
    R, C = shape
    x = synth.integer_image(R, C, seed=9)
    rs, cs = min(stages[0], C.bit_length() - 1), min(stages[1], R.bit_length() - 1)
    got = gpu_fft(env, x, -1, stages=(rs, cs))
    want = orc.fft2d(x, row_stages=rs, col_stages=cs)
    assert np.array_equal(got.astype(np.complex128), want)


@pytest.mark.parametrize("shape,stages", [((64, 128), (3, 5)), ((2048, 256), (7, 4)),
                                          ((4096, 4096), (9, 10)), ((32, 16384), (13, 2))])
def test_partial_stages_match_oracle(env, shape, stages):
    _, _, orc = env
    R, C = shape
    x = synth.uniform_complex(R, C, seed=3)
    got = gpu_fft(env, x, -1, stages=stages)
    want = orc.fft2d(x, row_stages=stages[0], col_stages=stages[1], threads=8)
    assert rel(got, want) <= TOL


# --------------------------------------------------------------- API plumbing
def test_inplace_equals_out_of_place(env):
    x = synth.uniform_complex(1024, 512, seed=1)
    a = gpu_fft(env, x, -1)
    b = gpu_fft(env, x, -1, inplace=True)
    assert np.array_equal(a, b)


def test_passes_compose_to_exec_and_runs_are_deterministic(env):
    torch, fft, _ = env
    x = torch.from_numpy(synth.blob_image(2048, 1024, seed=2)).cuda()
    plan = fft.fft2d_plan(2048, 1024, fft.FFT2D_C64, fft.FFT2D_INVERSE)
    try:
        a = torch.empty_like(x)
        b = torch.empty_like(x)
        fft.fft2d_exec(plan, x, a)
        fft.fft2d_exec_pass(plan, fft.FFT2D_PASS_ROWS, x, b)
        fft.fft2d_exec_pass(plan, fft.FFT2D_PASS_COLS, b, b)
        c = torch.empty_like(x)
        fft.fft2d_exec(plan, x, c)
        torch.cuda.synchronize()
        assert torch.equal(a, b)
        assert torch.equal(a, c)
    finally:
        fft.fft2d_destroy(plan)


def test_exec_host_matches_device_exec(env):
    torch, fft, _ = env
    x = synth.uniform_real(512, 2048, seed=4)
    want = gpu_fft(env, x, -1)
    plan = fft.fft2d_plan(512, 2048, fft.FFT2D_C64, fft.FFT2D_FORWARD)
    try:
        hin = torch.from_numpy(x).pin_memory()
        hout = torch.empty_like(hin).pin_memory()
        fft.fft2d_exec_host(plan, hin, hout)
        assert np.array_equal(hout.numpy(), want)
        # pageable numpy buffers, in place
        buf = x.copy()
        fft.fft2d_exec_host(plan, buf, buf)
        assert np.array_equal(buf, want)
    finally:
        fft.fft2d_destroy(plan)


def test_batched_uneven_equals_solo(env):
    torch, fft, _ = env
    shapes = synth.batch_shapes(12, seed=0)
    imgs = synth.batch_images(shapes, seed=0)
    plans = [fft.fft2d_plan(r, c, fft.FFT2D_C64, fft.FFT2D_FORWARD) for r, c in shapes]
    try:
        ins = [torch.from_numpy(im).cuda() for im in imgs]
        outs = [torch.empty_like(t) for t in ins]
        fft.fft2d_exec_batched(plans, ins, outs)
        torch.cuda.synchronize()
        for im, o in zip(imgs, outs):
            assert np.array_equal(o.cpu().numpy(), gpu_fft(env, im, -1))
        fft.fft2d_exec_batched([], [], [])
    finally:
        for p in plans:
            fft.fft2d_destroy(p)


def test_errors_are_reported_not_launched(env):
    torch, fft, _ = env
    plan = fft.fft2d_plan(64, 64, fft.FFT2D_C64, fft.FFT2D_FORWARD)
    try:
        x = torch.zeros(64, 64, dtype=torch.complex64, device="cuda")
        with pytest.raises(fft.FFT2DError):
            fft.fft2d_exec_stages(plan, x, x, 7, 0)          # 7 > log2(64)
        with pytest.raises(fft.FFT2DError):
            fft.fft2d_exec_pass(plan, 5, x, x)
        assert fft.fft2d_plan_info(plan) == (64, 64, 0, -1)
    finally:
        fft.fft2d_destroy(plan)


def rel_chunked(a, b, chunk=1 << 24):
    """rel() for images too large to widen whole (16384^2: 2 GiB complex64)."""
    a = np.asarray(a).reshape(-1)
    b = np.asarray(b).reshape(-1)
    num = den = 0.0
    for i in range(0, b.size, chunk):
        bb = b[i:i + chunk].astype(np.complex128)
        d = a[i:i + chunk].astype(np.complex128) - bb
        num += float(np.vdot(d, d).real)
        den += float(np.vdot(bb, bb).real)
    return float(np.sqrt(num / den))


def test_16384_square_whole_output(env):
    """16384x16384 (2 GiB per buffer, columns on the 16384-row kernel): the
    whole forward output against the FP64 oracle, the inverse of the GPU's
    spectrum against the oracle's inverse of it, and Parseval."""
    torch, fft, orc = env
    R = C = 16384
    xh = synth.uniform_complex(R, C, seed=8)
    x = torch.from_numpy(xh).cuda()
    pf = fft.fft2d_plan(R, C, fft.FFT2D_C64, fft.FFT2D_FORWARD)
    pi = fft.fft2d_plan(R, C, fft.FFT2D_C64, fft.FFT2D_INVERSE)
    try:
        X = torch.empty_like(x)
        fft.fft2d_exec(pf, x, X)
        px = (x.abs().double() ** 2).sum().item()
        pX = (X.abs().double() ** 2).sum().item() / (R * C)
        assert abs(px - pX) <= 1e-5 * px
        y = torch.empty_like(x)
        fft.fft2d_exec(pi, X, y)
        torch.cuda.synchronize()
        del x
        Xh = X.cpu().numpy()
        del X
        yh = y.cpu().numpy()
        del y
    finally:
        fft.fft2d_destroy(pf)
        fft.fft2d_destroy(pi)
    e_fwd = rel_chunked(Xh, orc.fft2d(xh, threads=16))
    e_rt = rel_chunked(yh, xh)
    e_inv = rel_chunked(yh, orc.fft2d(Xh, inverse=True, threads=16))
    report("16384^2 fwd", e_fwd)
    report("16384^2 inv(of gpu fwd)", e_inv)
    report("16384^2 round trip", e_rt)
    assert e_fwd <= TOL and e_inv <= TOL and e_rt <= TOL


def test_unaligned_buffers_take_the_plain_path(env):
    """A buffer that is only 8-byte aligned cannot feed TMA; the result must
    still match (the plain column kernel serves it)."""
    torch, fft, orc = env
    R = C = 1024
    x = synth.uniform_complex(R, C, seed=12)
    flat = torch.zeros(R * C + 1, dtype=torch.complex64, device="cuda")
    src = flat[1:].view(R, C)
    assert src.data_ptr() % 16 == 8
    src.copy_(torch.from_numpy(x))
    plan = fft.fft2d_plan(R, C, fft.FFT2D_C64, fft.FFT2D_FORWARD)
    try:
        fft.fft2d_exec(plan, src, src)
        fft.fft2d_sync_status(plan)
        assert rel(src.cpu().numpy(), orc.fft2d(x, threads=8)) <= TOL
    finally:
        fft.fft2d_destroy(plan)


@pytest.mark.parametrize("rows,variant", [(4096, "tma32"), (4096, "tmem"), (4096, "tma64"),
                                          (8192, "pair"),
                                          (16384, "quad"), (8192, "pairl2"), (16384, "quadl2")])
def test_withheld_tma_load_times_out_cleanly(env, rows, variant):
    """Failure path of the persistent TMA-fed column kernels: CTA 0 never
    issues one TMA load of its first tile, its bounded wait gives up, the
    kernel (for the CTA pair: both CTAs, agreeing at their cluster barrier)
    leaves cleanly, the host reads FFT2D_ERR_TIMEOUT, and the same plan then
    transforms correctly.  For the CTA pair and the four-CTA cluster every CTA
    learns of the loss at the tile's first cluster barrier and leaves."""
    torch, fft, orc = env
    cols = 256
    plan = fft.fft2d_plan(rows, cols, fft.FFT2D_C64, fft.FFT2D_FORWARD)
    try:
        L = rows.bit_length() - 1
        names = [fft.fft2d_variant_name(fft.FFT2D_PASS_COLS, L, v)
                 for v in range(fft.fft2d_variant_count(fft.FFT2D_PASS_COLS, L))]
        fft.fft2d_plan_set_variant(plan, fft.FFT2D_PASS_COLS, names.index(variant))
        x = synth.uniform_complex(rows, cols, seed=rows)
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
        assert rel(out.cpu().numpy(), orc.fft2d(x, threads=16)) <= TOL
    finally:
        fft.fft2d_destroy(plan)


def test_withheld_load_needs_a_tma_kernel(env):
    torch, fft, _ = env
    plan = fft.fft2d_plan(64, 64, fft.FFT2D_C64, fft.FFT2D_FORWARD)   # plain column kernel
    try:
        dx = torch.zeros((64, 64), dtype=torch.complex64, device="cuda")
        with pytest.raises(fft.FFT2DError) as ei:
            fft.fft2d_selftest_withheld_load(plan, dx, dx)
        assert ei.value.status == fft.FFT2D_ERR_ARG
    finally:
        fft.fft2d_destroy(plan)


def test_bounded_wait_reports_timeout_and_context_survives(env):
    """Failure path of the TMA pipeline: a wait on an mbarrier that nothing
    completes gives up (about 20 ms), the host reads FFT2D_ERR_TIMEOUT, the
    status clears, and the next transform is still correct."""
    torch, fft, orc = env
    plan = fft.fft2d_plan(256, 256, fft.FFT2D_C64, fft.FFT2D_FORWARD)
    try:
        fft.fft2d_sync_status(plan)                      # clean to start with
        fft.fft2d_selftest_timeout(plan)
        with pytest.raises(fft.FFT2DError) as ei:
            fft.fft2d_sync_status(plan)
        assert ei.value.status == fft.FFT2D_ERR_TIMEOUT
        fft.fft2d_sync_status(plan)                      # cleared
        x = synth.uniform_real(256, 256, seed=0)
        dx = torch.from_numpy(x).cuda()
        out = torch.empty_like(dx)
        fft.fft2d_exec(plan, dx, out)
        fft.fft2d_sync_status(plan)
        assert rel(out.cpu().numpy(), orc.fft2d(x)) <= TOL
    finally:
        fft.fft2d_destroy(plan)


def table1_rows():
    """Sizes and printed maximum errors of Table 1 (tests/golden/table1.txt)."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "table1.txt")
    rows = []
    with open(path) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                side, _, _, err = line.split()
                rows.append((int(side), float(err)))
    return rows


@pytest.mark.parametrize("side,paper_err", table1_rows())
def test_table1_sizes_max_error(env, side, paper_err):
    """At the sizes of Table 1, gray images in [0, 1): the largest error of
    the image recovered by forward + inverse (the reading of the paper's
    undefined "GPU maximum error" as an error in gray levels) stays far below
    the printed 0.007, and the forward spectrum matches the oracle."""
    _, _, orc = env
    x = synth.uniform_real(side, side, seed=side)
    X = gpu_fft(env, x, -1)
    assert rel(X, orc.fft2d(x)) <= TOL
    back = gpu_fft(env, X, 1)
    max_err = float(np.abs(back.astype(np.complex128) - x.astype(np.complex128)).max())
    print(f"[table1] {side}^2: max |ifft(fft(x)) - x| = {max_err:.2e} (paper: {paper_err})")
    assert max_err <= paper_err / 100


@pytest.mark.parametrize("side", [256, 4096, 8192])
def test_exec_in_a_cuda_graph(env, side):
    """Once a plan has run, fft2d_exec can be captured in a CUDA graph: the
    replayed forward + inverse give the same bits as the direct calls (at
    8192^2 the column pass's stream-ordered scratch becomes graph memory
    nodes)."""
    torch, fft, _ = env
    x = synth.uniform_complex(side, side, seed=side + 1)
    pf = fft.fft2d_plan(side, side, fft.FFT2D_C64, fft.FFT2D_FORWARD)
    pi = fft.fft2d_plan(side, side, fft.FFT2D_C64, fft.FFT2D_INVERSE)
    try:
        dx = torch.from_numpy(x).cuda()
        X = torch.empty_like(dx)
        Y = torch.empty_like(dx)
        fft.fft2d_exec(pf, dx, X)
        fft.fft2d_exec(pi, X, Y)
        torch.cuda.synchronize()
        want_X, want_Y = X.cpu().numpy(), Y.cpu().numpy()
        X.zero_()
        Y.zero_()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            fft.fft2d_exec(pf, dx, X, s.cuda_stream)
            fft.fft2d_exec(pi, X, Y, s.cuda_stream)
        g.replay()
        g.replay()
        torch.cuda.synchronize()
        fft.fft2d_sync_status(pf)
        assert np.array_equal(X.cpu().numpy(), want_X)
        assert np.array_equal(Y.cpu().numpy(), want_Y)
    finally:
        fft.fft2d_destroy(pf)
        fft.fft2d_destroy(pi)
