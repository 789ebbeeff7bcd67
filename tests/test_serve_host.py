"""The serving loop's admission and continuous-batching logic, run in
simulation mode (no CUDA calls, modelled device time) so it needs no GPU."""
import time

import numpy as np
import pytest


@pytest.fixture(scope="module")
def fft():
    from conftest import build_lib
    build_lib()
    import paper_1505_08019_gb300 as fft
    return fft


def make(fft, budget, streams=4):
    return fft.fft2d_serve_create(budget, streams, fft.FFT2D_SERVE_SIMULATE)


def test_all_requests_complete_and_stats(fft):
    srv = make(fft, 1 << 30)
    buf = np.zeros(8, np.complex64)
    try:
        g = np.random.default_rng(0)
        tickets = []
        for i in range(200):
            r, c = 1 << int(g.integers(4, 11)), 1 << int(g.integers(4, 11))
            op = int(g.integers(0, 2))
            dt = fft.FFT2D_C32H if i % 3 == 0 else fft.FFT2D_C64
            ex = buf if dt == fft.FFT2D_C32H else None
            tickets.append(fft.fft2d_serve_submit(srv, op, r, c, dt, buf, buf, ex, ex))
        lats = [fft.fft2d_serve_wait(srv, t, 10000) for t in tickets]
        st = fft.fft2d_serve_stats_get(srv)
        assert st["completed"] == 200 and st["rejected"] == 0 and st["queued"] == 0
        assert 0 <= st["p50_ms"] <= st["p99_ms"] <= st["max_ms"]
        assert min(lats) > 0
        assert st["batches"] >= 1 and st["mean_batch_size"] >= 1
        assert 0 < st["peak_device_bytes"] <= 1 << 30
    finally:
        fft.fft2d_serve_destroy(srv)


def test_budget_bounds_device_memory(fft):
    """4 MiB requests under a 10 MiB budget: at most two in flight."""
    budget = 10 << 20
    srv = make(fft, budget)
    buf = np.zeros(8, np.complex64)
    try:
        tickets = [fft.fft2d_serve_submit(srv, 0, 512, 1024, fft.FFT2D_C64, buf, buf)
                   for _ in range(40)]
        for t in tickets:
            fft.fft2d_serve_wait(srv, t, 20000)
        st = fft.fft2d_serve_stats_get(srv)
        assert st["completed"] == 40
        assert st["peak_device_bytes"] <= budget
        assert st["batches"] >= 20          # memory admits at most two at a time
    finally:
        fft.fft2d_serve_destroy(srv)


def test_oversized_request_is_refused(fft):
    srv = make(fft, 1 << 20)
    buf = np.zeros(8, np.complex64)
    try:
        with pytest.raises(fft.FFT2DError) as ei:
            fft.fft2d_serve_submit(srv, 0, 1024, 1024, fft.FFT2D_C64, buf, buf)   # 8 MiB
        assert ei.value.status == fft.FFT2D_ERR_BUDGET
        t = fft.fft2d_serve_submit(srv, 0, 128, 128, fft.FFT2D_C64, buf, buf)    # 128 KiB
        fft.fft2d_serve_wait(srv, t, 10000)
        st = fft.fft2d_serve_stats_get(srv)
        assert st["rejected"] == 1 and st["completed"] == 1
    finally:
        fft.fft2d_serve_destroy(srv)


@pytest.mark.parametrize("args,status", [
    ((5, 64, 64, 0), "FFT2D_ERR_ARG"),           # bad op
    ((0, 48, 64, 0), "FFT2D_ERR_NOT_POW2"),
    ((0, 64, 1 << 15, 0), "FFT2D_ERR_TOO_LARGE"),
    ((0, 64, 64, 9), "FFT2D_ERR_ARG"),           # bad dtype
    ((0, 1, 64, 1), "FFT2D_ERR_UNSUPPORTED"),    # half2 needs sides >= 2
])
def test_submit_argument_errors(fft, args, status):
    srv = make(fft, 1 << 30)
    buf = np.zeros(8, np.complex64)
    try:
        with pytest.raises(fft.FFT2DError) as ei:
            fft.fft2d_serve_submit(srv, *args, buf, buf)
        assert ei.value.status == getattr(fft, status)
    finally:
        fft.fft2d_serve_destroy(srv)


def test_arrivals_during_work_are_batched(fft):
    """Continuous batching: requests that arrive while a batch is in flight are
    admitted together into later batches instead of one launch each."""
    srv = make(fft, 1 << 30, streams=1)
    buf = np.zeros(8, np.complex64)
    try:
        tickets = [fft.fft2d_serve_submit(srv, 0, 2048, 2048, fft.FFT2D_C64, buf, buf)]
        time.sleep(0.002)                          # first batch is now in flight
        tickets += [fft.fft2d_serve_submit(srv, 1, 256, 256, fft.FFT2D_C64, buf, buf)
                    for _ in range(30)]
        for t in tickets:
            fft.fft2d_serve_wait(srv, t, 20000)
        st = fft.fft2d_serve_stats_get(srv)
        assert st["completed"] == 31
        assert st["batches"] < 31 and st["mean_batch_size"] > 1.5
    finally:
        fft.fft2d_serve_destroy(srv)


def test_destroy_drains_queued_work(fft):
    srv = make(fft, 1 << 30)
    buf = np.zeros(8, np.complex64)
    for _ in range(50):
        fft.fft2d_serve_submit(srv, 1, 1024, 1024, fft.FFT2D_C64, buf, buf)
    t0 = time.time()
    fft.fft2d_serve_destroy(srv)
    assert time.time() - t0 < 30


def test_wait_timeout_and_unknown_ticket(fft):
    srv = make(fft, 1 << 34, streams=1)
    buf = np.zeros(8, np.complex64)
    try:
        t = fft.fft2d_serve_submit(srv, 1, 16384, 16384, fft.FFT2D_C64, buf, buf)  # ~2 s modelled
        with pytest.raises(fft.FFT2DError) as ei:
            fft.fft2d_serve_wait(srv, t, 1)
        assert ei.value.status == fft.FFT2D_ERR_TIMEOUT
        fft.fft2d_serve_wait(srv, t, 60000)
        with pytest.raises(fft.FFT2DError):
            fft.fft2d_serve_wait(srv, t, 1)        # each ticket is waited for once
    finally:
        fft.fft2d_serve_destroy(srv)


def test_oversized_pooled_buffer_does_not_stall_admission(fft):
    """A 128x128 complex64 request leaves a 128 KiB buffer in the pool.  The
    next request, a 128x128 half2 one, takes it for its 64 KiB half2 buffer
    (pooled buffers up to twice the size are reused) and would then find no
    room for its 1.5 KiB of exponents under a 132 000-byte budget, with
    nothing in flight to free memory.  The server must fall back to exact
    sizes instead of waiting for ever."""
    srv = make(fft, 132000, streams=1)
    buf = np.zeros(8, np.complex64)
    ex = np.zeros(512, np.int32)
    try:
        t = fft.fft2d_serve_submit(srv, 0, 128, 128, fft.FFT2D_C64, buf, buf)
        fft.fft2d_serve_wait(srv, t, 10000)
        t = fft.fft2d_serve_submit(srv, 1, 128, 128, fft.FFT2D_C32H, buf, buf, ex, ex)
        fft.fft2d_serve_wait(srv, t, 10000)
        st = fft.fft2d_serve_stats_get(srv)
        assert st["completed"] == 2 and st["peak_device_bytes"] <= 132000
    finally:
        fft.fft2d_serve_destroy(srv)


def test_half2_request_needs_its_exponent_vectors(fft):
    srv = make(fft, 1 << 30)
    buf = np.zeros(8, np.complex64)
    ex = np.zeros(64, np.int32)
    try:
        for a, b in ((None, ex), (ex, None)):
            with pytest.raises(fft.FFT2DError) as ei:
                fft.fft2d_serve_submit(srv, 0, 64, 64, fft.FFT2D_C32H, buf, buf, a, b)
            assert ei.value.status == fft.FFT2D_ERR_ARG
    finally:
        fft.fft2d_serve_destroy(srv)
