"""The serving loop on the GPU: a mix of forward and FFT -> low-pass -> inverse
requests of different shapes and storage types runs concurrently; every
result must equal the same request run alone (bit for bit: the kernels
compute the same bits in any batch) and match the FP64 oracle."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


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


def quantise_rows(x):
    """complex64 -> half2 [R, C, 2] with per-row exponents, by the storage
    format's definition (e = k - 14 for a row maximum f 2^k, f in [0.5, 1))."""
    m = np.maximum(np.abs(x.real), np.abs(x.imag)).max(axis=1).astype(np.float64)
    _, k = np.frexp(m)
    e = np.where(m > 0, k - 14, 0).astype(np.int32)
    f = np.ldexp(np.float32(1.0), -e).astype(np.float32)[:, None]
    q = np.empty(x.shape + (2,), np.float16)
    q[..., 0] = (x.real * f).astype(np.float16)
    q[..., 1] = (x.imag * f).astype(np.float16)
    return q, e


def dequantise_cols(q, e):
    s = np.ldexp(1.0, e.astype(np.int64))[None, :]
    return q[..., 0].astype(np.float64) * s + 1j * (q[..., 1].astype(np.float64) * s)


def test_results_same_alone_and_in_the_mix(env):
    torch, fft, orc = env
    g = np.random.default_rng(3)
    reqs = []
    for i in range(40):
        side = 1 << int(g.integers(6, 13))           # 64 .. 4096, as the served stream
        a = g.random()
        r, c = (side, side) if a < 0.5 else ((side, max(16, side // 4)) if a < 0.75
                                              else (max(16, side // 4), side))
        op = fft.FFT2D_OP_LOWPASS if g.random() < 0.5 else fft.FFT2D_OP_FORWARD
        dt = fft.FFT2D_C32H if g.random() < 0.3 else fft.FFT2D_C64
        img = synth.uniform_real(r, c, seed=i)
        if dt == fft.FFT2D_C32H:
            q, e = quantise_rows(img)
            x = (torch.from_numpy(q).pin_memory(), torch.from_numpy(e))
            y = (torch.empty_like(x[0]).pin_memory(), torch.zeros(c, dtype=torch.int32))
        else:
            x = (torch.from_numpy(img).pin_memory(), None)
            y = (torch.empty_like(x[0]).pin_memory(), None)
        reqs.append((op, r, c, dt, x, y))

    def submit(srv, op, r, c, dt, x, y):
        return fft.fft2d_serve_submit(srv, op, r, c, dt, x[0], y[0], x[1], y[1])

    def result(y):
        return (y[0].numpy().copy(), None if y[1] is None else y[1].numpy().copy())

    budget = 8 << 30
    srv = fft.fft2d_serve_create(budget, 4)
    try:
        tickets = [submit(srv, *rq) for rq in reqs]
        for t in tickets:
            fft.fft2d_serve_wait(srv, t, 120000)
        mixed = [result(y) for *_, y in reqs]
        st = fft.fft2d_serve_stats_get(srv)
        assert st["completed"] == len(reqs) and st["peak_device_bytes"] <= budget
        print(f"[serve] mix: batches={st['batches']} mean_batch={st['mean_batch_size']:.1f} "
              f"p50={st['p50_ms']:.2f}ms p99={st['p99_ms']:.2f}ms")
        for i, (op, r, c, dt, x, y) in enumerate(reqs):
            alone = (torch.empty_like(y[0]).pin_memory(),
                     None if y[1] is None else torch.zeros_like(y[1]))
            t = submit(srv, op, r, c, dt, x, alone)
            fft.fft2d_serve_wait(srv, t, 120000)
            a = result(alone)
            assert np.array_equal(a[0].view(np.uint8), mixed[i][0].view(np.uint8)), \
                f"request {i} differs alone"
            assert a[1] is None or np.array_equal(a[1], mixed[i][1])
    finally:
        fft.fft2d_serve_destroy(srv)
    for i, (op, r, c, dt, x, y) in enumerate(reqs):
        if dt == fft.FFT2D_C32H:
            q, e = x[0].numpy(), x[1].numpy()
            xin = (q[..., 0].astype(np.float64) + 1j * q[..., 1].astype(np.float64)) \
                * np.ldexp(1.0, e.astype(np.int64))[:, None]
            got = dequantise_cols(*mixed[i])
        else:
            xin, got = x[0].numpy(), mixed[i][0]
        want = (orc.filter_image(xin, threads=16) if op == fft.FFT2D_OP_LOWPASS
                else orc.fft2d(xin, threads=16))
        tol = 5e-3 if dt == fft.FFT2D_C32H else 1e-5
        err = rel(got, want)
        print(f"[serve] {r}x{c} op={op} dtype={dt}: rel_l2={err:.2e}")
        assert err <= tol


def test_lowpass_kernel_matches_oracle(env):
    torch, fft, orc = env
    x = synth.blob_image(512, 1024, seed=2)
    X = orc.fft2d(x)
    d = torch.from_numpy(X.astype(np.complex64)).cuda()
    fft.fft2d_lowpass(512, 1024, fft.FFT2D_C64, d, 64.0, 128.0)
    torch.cuda.synchronize()
    assert rel(d.cpu().numpy(), orc.lowpass(X, 64.0, 128.0)) <= 1e-6
