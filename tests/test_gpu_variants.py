"""Kernel variants, the autotuner and the grouped batch executor (GPU).

Every variant runs the same butterflies in the same order with the same
rounding, so all of them -- and the batched path -- must agree bit for bit;
the default variant is checked against the FP64 oracle elsewhere and here.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


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


def run(env, x, direction, row_variant=-1, col_variant=-1):
    torch, fft, _ = env
    R, C = x.shape
    plan = fft.fft2d_plan(R, C, fft.FFT2D_C64, direction)
    try:
        fft.fft2d_plan_set_variant(plan, fft.FFT2D_PASS_ROWS, row_variant)
        fft.fft2d_plan_set_variant(plan, fft.FFT2D_PASS_COLS, col_variant)
        dx = torch.from_numpy(x).cuda()
        out = torch.empty_like(dx)
        fft.fft2d_exec(plan, dx, out)
        fft.fft2d_sync_status(plan)
        return out.cpu().numpy()
    finally:
        fft.fft2d_destroy(plan)


SHAPES = [(64, 32), (512, 512), (1024, 2048), (2048, 4096), (4096, 4096), (8192, 256),
          (256, 8192), (16384, 64), (64, 16384), (1024, 8192), (512, 16384)]


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: f"{s[0]}x{s[1]}")
def test_every_variant_is_bit_identical(env, shape):
    torch, fft, orc = env
    R, C = shape
    x = synth.uniform_complex(R, C, seed=R + C)
    base = run(env, x, fft.FFT2D_FORWARD)
    assert rel(base, orc.fft2d(x, threads=8)) <= TOL
    Lr, Lc = R.bit_length() - 1, C.bit_length() - 1
    for v in range(fft.fft2d_variant_count(fft.FFT2D_PASS_ROWS, Lc)):
        got = run(env, x, fft.FFT2D_FORWARD, row_variant=v)
        name = fft.fft2d_variant_name(fft.FFT2D_PASS_ROWS, Lc, v)
        assert np.array_equal(got, base), f"row variant {name} differs"
    for v in range(fft.fft2d_variant_count(fft.FFT2D_PASS_COLS, Lr)):
        got = run(env, x, fft.FFT2D_FORWARD, col_variant=v)
        name = fft.fft2d_variant_name(fft.FFT2D_PASS_COLS, Lr, v)
        assert np.array_equal(got, base), f"column variant {name} differs"


def test_autotune_keeps_results_and_reports_choice(env):
    torch, fft, _ = env
    x = synth.blob_image(1024, 2048, seed=1)
    want = run(env, x, fft.FFT2D_INVERSE)
    plan = fft.fft2d_plan(1024, 2048, fft.FFT2D_C64, fft.FFT2D_INVERSE)
    try:
        assert "default" in fft.fft2d_plan_describe(plan)
        fft.fft2d_autotune(plan)
        desc = fft.fft2d_plan_describe(plan)
        print("[autotune] 1024x2048:", desc)
        assert desc.count("tuned") == 2
        dx = torch.from_numpy(x).cuda()
        out = torch.empty_like(dx)
        fft.fft2d_exec(plan, dx, out)
        fft.fft2d_sync_status(plan)
        assert np.array_equal(out.cpu().numpy(), want)
        # a new plan of the same shape starts from the tuned choice
        p2 = fft.fft2d_plan(1024, 2048, fft.FFT2D_C64, fft.FFT2D_INVERSE)
        assert fft.fft2d_plan_describe(p2) == desc
        fft.fft2d_destroy(p2)
    finally:
        fft.fft2d_destroy(plan)


def test_tune_cache_file_round_trip(env, tmp_path):
    cache = tmp_path / "tune.txt"
    code = ("import sys; sys.path.insert(0, %r); import paper_1505_08019_gb300 as f; "
            "p = f.fft2d_plan(512, 1024, 0, -1); %s; print(f.fft2d_plan_describe(p))")
    envv = dict(os.environ, FFT2D_TUNE_CACHE=str(cache))
    r1 = subprocess.run([sys.executable, "-c", code % (ROOT, "f.fft2d_autotune(p)")],
                        capture_output=True, text=True, env=envv, timeout=300)
    assert r1.returncode == 0, r1.stderr
    lines = cache.read_text().strip().splitlines()
    assert len(lines) == 2 and all(len(l.split("\t")) == 5 for l in lines)
    r2 = subprocess.run([sys.executable, "-c", code % (ROOT, "None")],
                        capture_output=True, text=True, env=envv, timeout=300)
    assert r2.returncode == 0, r2.stderr
    assert r2.stdout.strip() == r1.stdout.strip()
    assert r2.stdout.count("tuned") == 2


def test_batched_uneven_64_images_mixed_directions(env):
    """The batched workload: 64 images, sides log-uniform 128..2048 (both
    orientations), grouped launches; every image equals its solo transform
    bit for bit, and a sample matches the oracle."""
    torch, fft, orc = env
    shapes = synth.batch_shapes(64, seed=0)
    imgs = synth.batch_images(shapes, seed=0)
    dirs = [fft.FFT2D_FORWARD if i % 3 else fft.FFT2D_INVERSE for i in range(len(shapes))]
    plans = [fft.fft2d_plan(r, c, fft.FFT2D_C64, d) for (r, c), d in zip(shapes, dirs)]
    try:
        ins = [torch.from_numpy(im).cuda() for im in imgs]
        outs = [torch.empty_like(t) for t in ins]
        fft.fft2d_exec_batched(plans, ins, outs)
        torch.cuda.synchronize()
        for i, (im, o, d) in enumerate(zip(imgs, outs, dirs)):
            got = o.cpu().numpy()
            assert np.array_equal(got, run(env, im, d)), f"image {i} {im.shape}"
            if i % 16 == 0:
                want = orc.fft2d(im, inverse=(d == fft.FFT2D_INVERSE), threads=8)
                assert rel(got, want) <= TOL
    finally:
        for p in plans:
            fft.fft2d_destroy(p)


def test_batched_from_a_captured_cuda_graph(env):
    """The 64-image batch as one captured CUDA graph: after one direct call
    (the kernels' first-use set-up), fft2d_exec_batched is captured on a side
    stream -- its grouped launches on the internal streams join the capture
    through events -- and each replay gives the direct call's bits; every
    image also matches the oracle."""
    torch, fft, orc = env
    shapes = synth.batch_shapes(64, seed=0)
    imgs = synth.batch_images(shapes, seed=0)
    plans = [fft.fft2d_plan(r, c, fft.FFT2D_C64, fft.FFT2D_FORWARD) for r, c in shapes]
    try:
        ins = [torch.from_numpy(im).cuda() for im in imgs]
        outs = [torch.empty_like(t) for t in ins]
        fft.fft2d_exec_batched(plans, ins, outs)
        torch.cuda.synchronize()
        want = [o.cpu().numpy() for o in outs]
        for o in outs:
            o.zero_()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            fft.fft2d_exec_batched(plans, ins, outs, s.cuda_stream)
        for _ in range(2):
            g.replay()
            torch.cuda.synchronize()
            for i, (o, w) in enumerate(zip(outs, want)):
                assert np.array_equal(o.cpu().numpy(), w), f"image {i} {shapes[i]}"
        for p in plans:
            fft.fft2d_sync_status(p)
        errs = [rel(w, orc.fft2d(im, threads=16)) for w, im in zip(want, imgs)]
        print(f"[batched graph] 64 images, worst rel_l2 vs oracle {max(errs):.2e}")
        assert max(errs) <= TOL
    finally:
        for p in plans:
            fft.fft2d_destroy(p)


def test_batched_more_images_than_one_table(env):
    """More images than one launch's job table holds (128): split launches."""
    torch, fft, _ = env
    shapes = [(128, 256)] * 130 + [(256, 128)] * 3
    imgs = synth.batch_images(shapes, seed=7)
    plans = [fft.fft2d_plan(r, c, fft.FFT2D_C64, fft.FFT2D_FORWARD) for r, c in shapes]
    try:
        ins = [torch.from_numpy(im).cuda() for im in imgs]
        outs = [torch.empty_like(t) for t in ins]
        fft.fft2d_exec_batched(plans, ins, outs)
        torch.cuda.synchronize()
        for i in (0, 64, 127, 128, 129, 131):
            assert np.array_equal(outs[i].cpu().numpy(), run(env, imgs[i], fft.FFT2D_FORWARD))
    finally:
        for p in plans:
            fft.fft2d_destroy(p)


def _batch_case(env, shapes, seed):
    torch, fft, _ = env
    imgs = synth.batch_images(shapes, seed=seed)
    dirs = [fft.FFT2D_FORWARD if i % 2 else fft.FFT2D_INVERSE for i in range(len(shapes))]
    solo = [run(env, im, d) for im, d in zip(imgs, dirs)]
    plans = [fft.fft2d_plan(r, c, fft.FFT2D_C64, d) for (r, c), d in zip(shapes, dirs)]
    return imgs, dirs, solo, plans


def _run_batched(env, plans, imgs):
    torch, fft, _ = env
    ins = [torch.from_numpy(im).cuda() for im in imgs]
    outs = [torch.empty_like(t) for t in ins]
    fft.fft2d_exec_batched(plans, ins, outs)
    torch.cuda.synchronize()
    for p in plans[:1]:
        fft.fft2d_sync_status(p)
    return [o.cpu().numpy() for o in outs]


BATCH_SHAPES = [(512, 1024), (1024, 512), (4096, 512), (512, 4096), (2048, 2048), (128, 256),
                (256, 128), (1024, 1024), (64, 8192), (8192, 64), (16384, 32), (32, 16384)]


def test_batched_every_grouped_variant_is_bit_identical(env):
    """Each grouped row kernel x each grouped column kernel (plain, narrow
    tiles, persistent TMA-fed) gives every image its solo result bit for bit."""
    torch, fft, _ = env
    shapes = BATCH_SHAPES + synth.batch_shapes(12, seed=5)
    imgs, dirs, solo, plans = _batch_case(env, shapes, seed=5)
    R, C = fft.FFT2D_PASS_ROWS, fft.FFT2D_PASS_COLS
    try:
        assert fft.fft2d_batch_variant_count(R) >= 2
        assert fft.fft2d_batch_variant_count(C) >= 3
        for rv in range(fft.fft2d_batch_variant_count(R)):
            for cv in range(fft.fft2d_batch_variant_count(C)):
                for L in range(1, 15):
                    fft.fft2d_batch_set_variant(R, L, rv)
                    fft.fft2d_batch_set_variant(C, L, cv)
                assert fft.fft2d_batch_get_variant(C, 12) == cv
                got = _run_batched(env, plans, imgs)
                names = (fft.fft2d_batch_variant_name(R, rv), fft.fft2d_batch_variant_name(C, cv))
                for i, (g, w) in enumerate(zip(got, solo)):
                    assert np.array_equal(g, w), f"variants {names}: image {i} {shapes[i]}"
    finally:
        for L in range(1, 15):
            fft.fft2d_batch_set_variant(R, L, -1)
            fft.fft2d_batch_set_variant(C, L, -1)
        for p in plans:
            fft.fft2d_destroy(p)


def test_batch_variant_arguments(env):
    torch, fft, _ = env
    R, C = fft.FFT2D_PASS_ROWS, fft.FFT2D_PASS_COLS
    assert [fft.fft2d_batch_variant_name(C, v) for v in range(fft.fft2d_batch_variant_count(C))] \
        == ["plain", "narrow", "tma", "tmast", "tmah"]
    assert fft.fft2d_batch_variant_name(C, 99) == ""
    assert fft.fft2d_batch_get_variant(C, 12) == 4      # default for 4096-point columns: tmah
    assert fft.fft2d_batch_get_variant(R, 0) == -1
    with pytest.raises(fft.FFT2DError):
        fft.fft2d_batch_set_variant(C, 12, fft.fft2d_batch_variant_count(C))
    with pytest.raises(fft.FFT2DError):
        fft.fft2d_batch_set_variant(R, 15, 0)


def test_autotune_batched_then_batched_matches_solo(env):
    torch, fft, _ = env
    shapes = BATCH_SHAPES
    imgs, dirs, solo, plans = _batch_case(env, shapes, seed=9)
    R, C = fft.FFT2D_PASS_ROWS, fft.FFT2D_PASS_COLS
    try:
        ins = [torch.from_numpy(im).cuda() for im in imgs]
        outs = [torch.empty_like(t) for t in ins]
        fft.fft2d_autotune_batched(plans, ins, outs)
        chosen = {L: (fft.fft2d_batch_get_variant(R, L), fft.fft2d_batch_get_variant(C, L))
                  for L in (6, 7, 8, 9, 10, 11, 12, 13)}
        print("[autotune_batched]", chosen)
        for rv, cv in chosen.values():
            assert 0 <= rv < fft.fft2d_batch_variant_count(R)
            assert 0 <= cv < fft.fft2d_batch_variant_count(C)
        got = _run_batched(env, plans, imgs)
        for i, (g, w) in enumerate(zip(got, solo)):
            assert np.array_equal(g, w), f"image {i} {shapes[i]}"
    finally:
        for L in range(1, 15):
            fft.fft2d_batch_set_variant(R, L, -1)
            fft.fft2d_batch_set_variant(C, L, -1)
        for p in plans:
            fft.fft2d_destroy(p)
