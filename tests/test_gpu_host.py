"""The pipelined host-buffer path (fft2d_exec_host_many) on the GPU.

Each image goes through the same two launches as fft2d_exec_host, only the
copies overlap, so every result must equal the one-at-a-time host call bit
for bit; a sample is also checked against the FP64 oracle.
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
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def test_many_host_images_equal_one_at_a_time(env):
    """Seven images (more than the three pipeline slots), mixed shapes and
    directions, pinned buffers; one of them in place."""
    torch, fft, orc = env
    shapes = [(512, 512), (1024, 256), (64, 4096), (2048, 2048), (1, 512), (256, 1), (4096, 4096)]
    dirs = [fft.FFT2D_FORWARD, fft.FFT2D_INVERSE] * 4
    imgs = synth.batch_images(shapes, seed=11)
    plans = [fft.fft2d_plan(r, c, fft.FFT2D_C64, d) for (r, c), d in zip(shapes, dirs)]
    try:
        want = []
        for p, im in zip(plans, imgs):
            h = torch.from_numpy(im).pin_memory()
            o = torch.empty_like(h).pin_memory()
            fft.fft2d_exec_host(p, h, o)
            want.append(o.numpy().copy())
        hin = [torch.from_numpy(im).pin_memory() for im in imgs]
        hout = [torch.empty_like(h).pin_memory() for h in hin]
        hout[3] = hin[3]                      # in place
        fft.fft2d_exec_host_many(plans, hin, hout)
        for i in range(len(shapes)):
            assert np.array_equal(hout[i].numpy(), want[i]), f"image {i} {shapes[i]}"
        for i in (0, 3):
            inv = dirs[i] == fft.FFT2D_INVERSE
            assert rel(hout[i].numpy(), orc.fft2d(imgs[i], inverse=inv, threads=8)) <= TOL
    finally:
        for p in plans:
            fft.fft2d_destroy(p)


def test_many_host_pageable_and_repeat(env):
    """Pageable numpy buffers work too, and a second call reuses the slots."""
    torch, fft, orc = env
    shapes = [(256, 512)] * 5
    imgs = synth.batch_images(shapes, seed=4)
    plan = fft.fft2d_plan(256, 512, fft.FFT2D_C64, fft.FFT2D_FORWARD)
    try:
        outs = [np.empty_like(im) for im in imgs]
        for _ in range(2):
            fft.fft2d_exec_host_many([plan] * 5, imgs, outs)
        for im, o in zip(imgs, outs):
            assert rel(o, orc.fft2d(im, threads=8)) <= TOL
    finally:
        fft.fft2d_destroy(plan)


def test_forward_and_inverse_in_one_call(env):
    """An image may read an earlier image's output in the same call: the
    inverse of each forward transform travels in the same call (its upload
    waits for the forward's download) and gives the same bits as two
    separate calls."""
    torch, fft, orc = env
    shapes = [(1024, 1024), (512, 2048), (2048, 512), (256, 256)]
    imgs = synth.batch_images(shapes, seed=21)
    fwd = [fft.fft2d_plan(r, c, fft.FFT2D_C64, fft.FFT2D_FORWARD) for r, c in shapes]
    inv = [fft.fft2d_plan(r, c, fft.FFT2D_C64, fft.FFT2D_INVERSE) for r, c in shapes]
    try:
        hin = [torch.from_numpy(im).pin_memory() for im in imgs]
        mid = [torch.empty_like(h).pin_memory() for h in hin]
        fft.fft2d_exec_host_many(fwd, hin, mid)
        want_fwd = [m.numpy().copy() for m in mid]
        back = [torch.empty_like(h).pin_memory() for h in hin]
        fft.fft2d_exec_host_many(inv, mid, back)
        want_rt = [b.numpy().copy() for b in back]

        mid2 = [torch.empty_like(h).pin_memory() for h in hin]
        back2 = [torch.empty_like(h).pin_memory() for h in hin]
        fft.fft2d_exec_host_many(fwd + inv, hin + mid2, mid2 + back2)
        for i in range(len(shapes)):
            assert np.array_equal(mid2[i].numpy(), want_fwd[i]), f"forward {shapes[i]}"
            assert np.array_equal(back2[i].numpy(), want_rt[i]), f"round trip {shapes[i]}"
            assert rel(back2[i].numpy(), imgs[i]) <= TOL
        # in place on the host: forward into the buffer, inverse back in it
        work = [torch.empty_like(h).pin_memory() for h in hin]
        fft.fft2d_exec_host_many(fwd + inv, hin + work, work + work)
        for i in range(len(shapes)):
            assert np.array_equal(work[i].numpy(), want_rt[i]), f"in place {shapes[i]}"
    finally:
        for p in fwd + inv:
            fft.fft2d_destroy(p)


def test_async_calls_back_to_back(env):
    """Several asynchronous calls queued back to back, one synchronisation:
    the same bits as synchronous calls, the host buffers reused across calls
    the way a repeated forward + inverse step reuses them."""
    torch, fft, _ = env
    shapes = [(2048, 2048)] * 3
    imgs = synth.batch_images(shapes, seed=5)
    pf = fft.fft2d_plan(2048, 2048, fft.FFT2D_C64, fft.FFT2D_FORWARD)
    pi = fft.fft2d_plan(2048, 2048, fft.FFT2D_C64, fft.FFT2D_INVERSE)
    try:
        hin = [torch.from_numpy(im).pin_memory() for im in imgs]
        ref = [torch.empty_like(h).pin_memory() for h in hin]
        fft.fft2d_exec_host_many([pf] * 3 + [pi] * 3, hin + ref, ref + ref)
        want = [r.numpy().copy() for r in ref]
        out = [torch.empty_like(h).pin_memory() for h in hin]
        stream = torch.cuda.current_stream()
        for _ in range(4):
            fft.fft2d_exec_host_many_async([pf] * 3 + [pi] * 3, hin + out, out + out,
                                           stream.cuda_stream)
        stream.synchronize()
        for i in range(3):
            assert np.array_equal(out[i].numpy(), want[i])
    finally:
        fft.fft2d_destroy(pf)
        fft.fft2d_destroy(pi)


def test_chained_images_skip_the_upload(env):
    """An image whose input is the previous image's output is transformed
    from the device copy of that output: the interleaved order (forward,
    its inverse, next forward, ...) and a chain of three give the same bits
    as separate calls, synchronous and asynchronous, with shapes that
    change along the call."""
    torch, fft, _ = env
    shapes = [(1024, 1024), (512, 2048), (2048, 512), (256, 256), (1024, 1024)]
    imgs = synth.batch_images(shapes, seed=33)
    fwd = [fft.fft2d_plan(r, c, fft.FFT2D_C64, fft.FFT2D_FORWARD) for r, c in shapes]
    inv = [fft.fft2d_plan(r, c, fft.FFT2D_C64, fft.FFT2D_INVERSE) for r, c in shapes]
    try:
        hin = [torch.from_numpy(im).pin_memory() for im in imgs]
        mid = [torch.empty_like(h).pin_memory() for h in hin]
        back = [torch.empty_like(h).pin_memory() for h in hin]
        fft.fft2d_exec_host_many(fwd, hin, mid)
        fft.fft2d_exec_host_many(inv, mid, back)
        want_fwd = [m.numpy().copy() for m in mid]
        want_rt = [b.numpy().copy() for b in back]
        again = [torch.empty_like(h).pin_memory() for h in hin]
        fft.fft2d_exec_host_many(fwd, back, again)
        want_again = [a.numpy().copy() for a in again]

        plans, ins, outs = [], [], []
        mid2 = [torch.empty_like(h).pin_memory() for h in hin]
        back2 = [torch.empty_like(h).pin_memory() for h in hin]
        for i in range(len(shapes)):
            plans += [fwd[i], inv[i]]
            ins += [hin[i], mid2[i]]
            outs += [mid2[i], back2[i]]
        fft.fft2d_exec_host_many(plans, ins, outs)
        for i in range(len(shapes)):
            assert np.array_equal(mid2[i].numpy(), want_fwd[i]), f"forward {shapes[i]}"
            assert np.array_equal(back2[i].numpy(), want_rt[i]), f"inverse {shapes[i]}"

        # forward and inverse into one host buffer: the overwritten forward
        # result is not copied back, the final content is the round trip
        one = [torch.empty_like(h).pin_memory() for h in hin]
        plans, ins, outs = [], [], []
        for i in range(len(shapes)):
            plans += [fwd[i], inv[i]]
            ins += [hin[i], one[i]]
            outs += [one[i], one[i]]
        fft.fft2d_exec_host_many(plans, ins, outs)
        for i in range(len(shapes)):
            assert np.array_equal(one[i].numpy(), want_rt[i]), f"same buffer {shapes[i]}"

        # in place on the host, chains of three, several asynchronous calls
        work = [torch.empty_like(h).pin_memory() for h in hin]
        plans, ins, outs = [], [], []
        for i in range(len(shapes)):
            plans += [fwd[i], inv[i], fwd[i]]
            ins += [hin[i], work[i], work[i]]
            outs += [work[i], work[i], work[i]]
        stream = torch.cuda.current_stream()
        for _ in range(3):
            fft.fft2d_exec_host_many_async(plans, ins, outs, stream.cuda_stream)
        stream.synchronize()
        for i in range(len(shapes)):
            assert np.array_equal(work[i].numpy(), want_again[i]), f"chain of three {shapes[i]}"
    finally:
        for p in fwd + inv:
            fft.fft2d_destroy(p)
