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
        x = torch.from_numpy(synth.uniform_real(r, c, seed=i)).pin_memory()
        y = torch.empty_like(x).pin_memory()
        reqs.append((op, r, c, dt, x, y))
    budget = 8 << 30
    srv = fft.fft2d_serve_create(budget, 4)
    try:
        tickets = [fft.fft2d_serve_submit(srv, op, r, c, dt, x, y) for op, r, c, dt, x, y in reqs]
        for t in tickets:
            fft.fft2d_serve_wait(srv, t, 120000)
        mixed = [y.numpy().copy() for *_, y in reqs]
        st = fft.fft2d_serve_stats_get(srv)
        assert st["completed"] == len(reqs) and st["peak_device_bytes"] <= budget
        print(f"[serve] mix: batches={st['batches']} mean_batch={st['mean_batch_size']:.1f} "
              f"p50={st['p50_ms']:.2f}ms p99={st['p99_ms']:.2f}ms")
        for i, (op, r, c, dt, x, y) in enumerate(reqs):
            alone = torch.empty_like(x).pin_memory()
            t = fft.fft2d_serve_submit(srv, op, r, c, dt, x, alone)
            fft.fft2d_serve_wait(srv, t, 120000)
            assert np.array_equal(alone.numpy(), mixed[i]), f"request {i} differs alone"
    finally:
        fft.fft2d_serve_destroy(srv)
    for i, (op, r, c, dt, x, y) in enumerate(reqs):
        xin = x.numpy()
        want = (orc.filter_image(xin, threads=16) if op == fft.FFT2D_OP_LOWPASS
                else orc.fft2d(xin, threads=16))
        tol = 5e-3 if dt == fft.FFT2D_C32H else 1e-5
        err = rel(mixed[i], want)
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
