#!/usr/bin/env python3
"""Benchmark of the 2D radix-2 DIT FFT on GB300: 4096x4096 complex64 images.

One step = R rounds (default 32) of forward 2D FFT then inverse 2D FFT of
each of B resident images (default 8, per rank).  ``value`` counts 2D transforms per second (a forward and an
inverse each count as one image transform), summed over ranks; inputs are
already in HBM when the timed region starts.  The working set (B images x
2 buffers x 128 MiB) is far larger than L2, so no image is L2-resident when
it is revisited.

Prints ONE JSON line on rank 0.  ``--impl reference`` times the FP64 CPU
oracle (the only other implementation of this path) on the host cores.
"""
from __future__ import annotations

import argparse
import csv
import hashlib
import io
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "2D FFT images/s & HBM GB/s vs peak at 4096²; serving p50/p99 latency"
UNIT = "images/s"
SIDE = 4096
BYTES_PER_PX_PASS = 16          # one read + one write of a complex64 pixel
FALLBACK_HBM_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--requests", type=int, default=20000, help="serving workload: requests")
    ap.add_argument("--rate", type=float, default=2000.0, help="serving workload: mean req/s")
    ap.add_argument("--workload", choices=["fft4096", "batched", "fp16", "serve", "dct", "sizes",
                                           "passes", "cpu"],
                    default="fft4096",
                    help="fft4096: the 4096x4096 forward+inverse benchmark (default); "
                         "batched: 64 uneven images through the grouped executor; "
                         "fp16: half2 storage vs complex64 at 8192^2 and 16384^2; "
                         "serve: Poisson stream of mixed requests through fft2d_serve_*; "
                         "dct: real 2D DCT-II at 4096^2 and 8192^2 beside the complex FFT; "
                         "sizes: forward+inverse at the paper's Table 1 image sizes; "
                         "passes: the default row and column kernels of one --shape image "
                         "(--dtype c64 or h16), timed one pass at a time (for profiling); "
                         "cpu: the CPU baseline (FP64 oracle, one thread and all cores) at "
                         "256^2, 1024^2, 4096^2 and 8192^2 beside the GPU's time")
    ap.add_argument("--shape", default="16384x512", help="passes workload: RxC")
    ap.add_argument("--dtype", choices=["c64", "h16"], default="c64",
                    help="passes workload: complex64 or half2 storage")
    ap.add_argument("--images", type=int, default=8, help="resident images per rank")
    ap.add_argument("--rounds", type=int, default=32,
                    help="one step = this many rounds of forward + inverse of every resident "
                         "image")
    ap.add_argument("--streams", type=int, default=0,
                    help="CUDA streams the resident images are spread over (0: one per image)")
    ap.add_argument("--fp16-sides", default="8192,16384",
                    help="fp16 workload: comma-separated square sides")
    ap.add_argument("--dct-sides", default="4096,8192",
                    help="dct workload: comma-separated sides (S or RxC)")
    ap.add_argument("--side", type=int, default=SIDE)
    ap.add_argument("--e2e-steps", type=int, default=12)
    ap.add_argument("--cpu-seconds", type=float, default=10.0,
                    help="bound on each CPU-baseline sample (wall seconds)")
    ap.add_argument("--no-sub", action="store_true",
                    help="default workload: leave out the serve / fp16 / batched sub-results")
    ap.add_argument("--serve-sample", type=int, default=4000,
                    help="default workload: requests of the serving sub-result")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-parity", action="store_true")
    return ap.parse_args()


# ------------------------------------------------------------------ helpers
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def init_dist(ws, backend):
    if ws <= 1:
        return None
    import torch.distributed as dist
    dist.init_process_group(backend=backend)
    return dist


def image_seeds(rank: int, images: int) -> list[int]:
    """Seeds of the images a rank keeps resident: disjoint across ranks, so N
    ranks transform N times the images (weak scaling, no data exchanged)."""
    return [rank * 1000 + i for i in range(images)]


def job_value(transforms_per_rank: int, world: int, ms_max: float) -> float:
    """Whole-job throughput: every rank's transforms over the slowest rank's time."""
    return transforms_per_rank * world / (ms_max * 1e-3)


def max_over_ranks(x: float, dist, device=None) -> float:
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def measured_hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            v = float(json.load(f)["hbm_gbs"])
        return v, "measured (MEASURED_PEAKS.json hbm_gbs)"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback 6.8 TB/s (MEASURED_PEAKS.json absent)"


# The translation units of the headline's row and column pass kernels and
# every header they include (the other units, such as the DCT and half2
# kernels, do not change them).
TIMED_KERNEL_SOURCES = ("async_copy.cuh", "col_group.cuh", "col_tmem.cuh", "kernels_col.cu",
                        "kernels_row.cu", "line_fft.cuh", "passes.h", "tmem.cuh")


def kernel_source_hash() -> str:
    """Hash of the CUDA sources the timed kernels are built from."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1505_08019_gb300", "csrc")
    for name in TIMED_KERNEL_SOURCES:
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(name.encode() + b"\0" + f.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, or
    None when the kernels changed since the counters were taken."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(p) as f:
            d = json.load(f)
    except Exception:
        return None
    if d.get("source_hash") != kernel_source_hash():
        return None
    v = d.get("kernels", {}).get(kernel, {}).get("dram_bytes_per_launch_full_size")
    return float(v) if v is not None else None


class ClockSampler:
    """nvidia-smi clock/throttle samples while the timed region runs."""

    FIELDS = ("uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid: str | None):
        self.uuid = uuid
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        rows = []
        for rec in csv.reader(io.StringIO(out)):
            rec = [r.strip() for r in rec]
            if len(rec) < 9:
                continue
            if self.uuid and rec[0] != self.uuid:
                continue
            try:
                rows.append((float(rec[1]), float(rec[2]), rec[5:9]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, fl in rows for i, v in enumerate(fl)
                          if v.lower().startswith("active")})
        sm = [r[0] for r in rows]
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(r[1] for r in rows),
                "samples": len(rows), "reasons": reasons}


# ------------------------------------------------------------- CPU oracle
def cpu_oracle_sample(side, seconds, threads):
    """Forward+inverse transforms of one side^2 blob image by the FP64 oracle
    on host threads, repeated while the wall-clock bound allows (at least
    one pair)."""
    import synth
    from oracle import oracle
    orc = oracle.get()
    x = synth.blob_image(side, side, seed=0).astype(np.complex128)
    n = 0
    t0 = time.perf_counter()
    while True:
        X = orc.fft2d(x, threads=threads)
        orc.fft2d(X, inverse=True, threads=threads)
        n += 2
        if time.perf_counter() - t0 >= seconds:
            break
    dt = time.perf_counter() - t0
    return n / dt, n, dt


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def cpu_model() -> str:
    """The host CPU's model name as lscpu reports it (else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part")):
                    return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def cpu_baseline(side, seconds):
    """The oracle on all host cores and on one thread, same workload."""
    th = host_cores()
    v, n, dt = cpu_oracle_sample(side, seconds, th)
    v1, n1, dt1 = cpu_oracle_sample(side, seconds, 1)
    return {"value": v, "unit": UNIT, "cores": th, "kind": "oracle",
            "cpu_model": cpu_model(),
            "sample": f"{n} transforms ({n // 2} forward+inverse pairs) of one "
                      f"{side}x{side} blob image, FP64 C oracle on {th} threads, {dt:.1f} s",
            "single_thread": {"value": v1, "unit": UNIT, "cores": 1,
                              "sample": f"{n1} transforms ({n1 // 2} pairs), one thread, "
                                        f"{dt1:.1f} s"}}


def rel_l2(a, b, chunk=1 << 24):
    """||a - b|| / ||b|| in float64 (b the reference), in chunks."""
    a = np.asarray(a).reshape(-1)
    b = np.asarray(b).reshape(-1)
    num = den = 0.0
    for i in range(0, b.size, chunk):
        bb = b[i:i + chunk].astype(np.complex128)
        d = a[i:i + chunk].astype(np.complex128) - bb
        num += float(np.vdot(d, d).real)
        den += float(np.vdot(bb, bb).real)
    return float(np.sqrt(num / den)) if den > 0 else float(np.sqrt(num))


# ------------------------------------------------- half2 storage, in numpy
def h16_quantise_rows(x):
    """complex64 image -> (half2 [R, C, 2], per-row exponents) by the storage
    format's definition: e = k - 14 for a row whose largest |component| is
    f 2^k (f in [0.5, 1)), q = x 2^-e rounded to half precision."""
    m = np.maximum(np.abs(x.real), np.abs(x.imag)).max(axis=1).astype(np.float64)
    _, k = np.frexp(m)
    e = np.where(m > 0, k - 14, 0).astype(np.int32)
    f = np.ldexp(np.float32(1.0), -e).astype(np.float32)[:, None]
    q = np.empty(x.shape + (2,), np.float16)
    q[..., 0] = (x.real * f).astype(np.float16)
    q[..., 1] = (x.imag * f).astype(np.float16)
    return q, e


def h16_dequantise(q, e, axis):
    """half2 [R, C, 2] with exponents per row (axis 0) or column (1) ->
    complex128 q * 2^e."""
    sc = np.ldexp(1.0, e.astype(np.int64))
    sc = sc[:, None] if axis == 0 else sc[None, :]
    return q[..., 0].astype(np.float64) * sc + 1j * (q[..., 1].astype(np.float64) * sc)


def cuda_timer(torch, stream):
    """fn, n -> mean ms per call over n calls after 3 warm-up calls, timed
    with CUDA events on `stream`."""
    def t(fn, n):
        for i in range(3):
            fn(i)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for i in range(n):
            fn(i)
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / n
    return t


def measure_fp16(fft, torch, orc, side, reps, check=True):
    """Forward 2D FFT of a side x side image (re, im ~ U[-1, 1)) with half2
    storage (fft2d_exec_h16) beside complex64 (fft2d_exec, autotuned), two
    input/output pairs in turn; relative L2 error of each against the FP64
    oracle of the input that path stored, with the half2 data quantised and
    dequantised in numpy from the format's definition."""
    import synth
    stream = torch.cuda.current_stream()
    sptr = stream.cuda_stream
    t = cuda_timer(torch, stream)
    peak, _ = measured_hbm_peak()
    th = host_cores()
    x = synth.uniform_complex(side, side, seed=side)
    p32 = fft.fft2d_plan(side, side, fft.FFT2D_C64, fft.FFT2D_FORWARD)
    p16 = fft.fft2d_plan(side, side, fft.FFT2D_C32H, fft.FFT2D_FORWARD)
    try:
        fft.fft2d_autotune(p32)
        dx = [torch.from_numpy(x).cuda() for _ in range(2)]
        dy = [torch.empty_like(dx[0]) for _ in range(2)]
        ms32 = t(lambda i: fft.fft2d_exec(p32, dx[i & 1], dy[i & 1], sptr), reps)
        ms32_rows = t(lambda i: fft.fft2d_exec_pass(p32, fft.FFT2D_PASS_ROWS, dx[i & 1],
                                                    dy[i & 1], sptr), reps)
        ms32_cols = t(lambda i: fft.fft2d_exec_pass(p32, fft.FFT2D_PASS_COLS, dy[i & 1],
                                                    dy[i & 1], sptr), reps)
        fft.fft2d_exec(p32, dx[0], dy[0], sptr)
        torch.cuda.synchronize()
        got32 = dy[0].cpu().numpy()
        del dx, dy
        q, e = h16_quantise_rows(x)
        dq = [torch.from_numpy(q).cuda() for _ in range(2)]
        de = torch.from_numpy(e).cuda()
        dqo = [torch.empty_like(dq[0]) for _ in range(2)]
        doe = [torch.empty(side, dtype=torch.int32, device="cuda") for _ in range(2)]
        ms16 = t(lambda i: fft.fft2d_exec_h16(p16, dq[i & 1], de, fft.FFT2D_PASS_ROWS,
                                              dqo[i & 1], doe[i & 1], sptr), reps)
        fft.fft2d_exec_h16(p16, dq[0], de, fft.FFT2D_PASS_ROWS, dqo[0], doe[0], sptr)
        torch.cuda.synchronize()
        q_out, e_out = dqo[0].cpu().numpy(), doe[0].cpu().numpy()
        del dq, dqo, doe
        desc32 = fft.fft2d_plan_describe(p32)
        desc16 = fft.fft2d_plan_describe(p16)
    finally:
        fft.fft2d_destroy(p32)
        fft.fft2d_destroy(p16)
    torch.cuda.empty_cache()
    e32 = e16 = None
    if check:
        want32 = orc.fft2d(x, threads=th)
        e32 = rel_l2(got32, want32)
        del want32, got32
        want16 = orc.fft2d(h16_dequantise(q, e, 0), threads=th)
        e16 = rel_l2(h16_dequantise(q_out, e_out, 1), want16)
        del want16
    px = side * side
    return {"fp16_ms": ms16, "fp32_ms": ms32, "speedup_fp16_vs_fp32": ms32 / ms16,
            "fp32_row_pass_ms": ms32_rows, "fp32_col_pass_ms": ms32_cols,
            "fp16_images_per_s": 1e3 / ms16, "fp32_images_per_s": 1e3 / ms32,
            "fp16_hbm_frac": (16.0 * px / (ms16 * 1e-3) / 1e9) / peak,
            "fp32_hbm_frac": (32.0 * px / (ms32 * 1e-3) / 1e9) / peak,
            "fp16_rel_l2_vs_fp64_oracle": e16, "fp32_rel_l2_vs_fp64_oracle": e32,
            "tolerance_fp16": 5e-3, "tolerance_fp32": 1e-5,
            "fp32_kernels": desc32, "fp16_kernels": desc16,
            "checking": "half2 input quantised and output dequantised in numpy"}


def measure_batched(fft, torch, orc, steps, tune_plans=False):
    """64 images with power-of-two sides log-uniform in 128..2048 (both
    orientations), real part U[0,1): one step transforms all of them forward
    through fft2d_exec_batched (grouped launches); the same images through
    one fft2d_exec per image give the single-image path's figure.  Every
    image of one batched step is checked against the FP64 oracle."""
    import synth
    shapes = synth.batch_shapes(64, seed=0)
    imgs = synth.batch_images(shapes, seed=0)
    if tune_plans:
        tuned = set()
        for r, c in shapes:
            if (r, c) not in tuned:
                p = fft.fft2d_plan(r, c, fft.FFT2D_C64, fft.FFT2D_FORWARD)
                fft.fft2d_autotune(p)
                fft.fft2d_destroy(p)
                tuned.add((r, c))
    plans = [fft.fft2d_plan(r, c, fft.FFT2D_C64, fft.FFT2D_FORWARD) for r, c in shapes]
    ins = [torch.from_numpy(im).cuda() for im in imgs]
    outs = [torch.empty_like(t) for t in ins]
    stream = torch.cuda.current_stream()
    sptr = stream.cuda_stream
    px = sum(r * c for r, c in shapes)
    t = cuda_timer(torch, stream)

    def batched(_i=0):
        fft.fft2d_exec_batched(plans, ins, outs, sptr)

    def single(_i=0):
        for p, x, o in zip(plans, ins, outs):
            fft.fft2d_exec(p, x, o, sptr)

    ms_default = t(batched, steps)
    fft.fft2d_autotune_batched(plans, ins, outs, sptr)
    R, C = fft.FFT2D_PASS_ROWS, fft.FFT2D_PASS_COLS
    chosen = {f"{1 << L}": [fft.fft2d_batch_variant_name(R, fft.fft2d_batch_get_variant(R, L)),
                            fft.fft2d_batch_variant_name(C, fft.fft2d_batch_get_variant(C, L))]
              for L in sorted({(r.bit_length() - 1) for r, _ in shapes}
                              | {(c.bit_length() - 1) for _, c in shapes})}
    ms_b = t(batched, steps)
    ms_s = t(single, steps)
    # the same grouped launches captured once in a CUDA graph and replayed
    gs = torch.cuda.Stream()
    gs.wait_stream(stream)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=gs):
        fft.fft2d_exec_batched(plans, ins, outs, gs.cuda_stream)
    ms_g = t(lambda _i: graph.replay(), steps)
    del graph
    peak, peak_src = measured_hbm_peak()
    gbs = 32.0 * px / (ms_b * 1e-3) / 1e9
    batched()
    torch.cuda.synchronize()
    th = host_cores()
    errs = [rel_l2(o.cpu().numpy(), orc.fft2d(im, threads=th)) for o, im in zip(outs, imgs)]
    for p in plans:
        fft.fft2d_destroy(p)
    return {"images_per_s": len(shapes) / (ms_b * 1e-3), "ms_per_step": ms_b,
            "pixels_per_step": px,
            "single_image_path": {"images_per_s": len(shapes) / (ms_s * 1e-3),
                                  "ms_per_step": ms_s,
                                  "call": "fft2d_exec per image"},
            "cuda_graph": {"images_per_s": len(shapes) / (ms_g * 1e-3), "ms_per_step": ms_g,
                           "call": "fft2d_exec_batched captured once in a CUDA graph, replayed"},
            "speedup_vs_single": ms_s / ms_b,
            "default_variants_ms_per_step": ms_default, "tuned_variants": chosen,
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s",
                         "frac": gbs / peak, "peak_source": peak_src,
                         "algorithmic_bytes_per_step": 32 * px},
            "rel_l2_max": max(errs), "rel_l2_median": float(np.median(errs)),
            "images_checked": len(errs), "tolerance": 1e-5,
            "gpu_launches_per_step": len({c for _, c in shapes}) + len({r for r, _ in shapes}),
            "gpu_launches_per_step_single": 2 * len(shapes)}


# ----------------------------------------------------------------- our arm
def run_ours(args):
    import torch
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = init_dist(ws, "nccl")

    import __graft_entry__
    __graft_entry__.build()          # no-op when the library is up to date
    import paper_1505_08019_gb300 as fft
    import synth

    side, B, R = args.side, args.images, max(1, args.rounds)
    imgs = [synth.blob_image(side, side, seed=sd) for sd in image_seeds(rank, B)]
    # B resident images, each with its own output buffer (B x 2 x 128 MiB,
    # far beyond L2); a step transforms every one R times, forward from its
    # input and back in place, so consecutive launches never find their
    # image in L2
    xs = [torch.from_numpy(im).to(dev) for im in imgs]
    Xs = [torch.empty_like(x) for x in xs]
    pf = fft.fft2d_plan(side, side, fft.FFT2D_C64, fft.FFT2D_FORWARD)
    pi = fft.fft2d_plan(side, side, fft.FFT2D_C64, fft.FFT2D_INVERSE)
    stream = torch.cuda.current_stream(dev)
    sptr = stream.cuda_stream
    ROWS, COLS = fft.FFT2D_PASS_ROWS, fft.FFT2D_PASS_COLS
    exec_pass = fft.fft2d_exec_pass

    # the resident images are independent: they are spread over several
    # streams, forked from and joined back into the timing stream, so one
    # image's launch tails overlap another's
    nstreams = min(args.streams if args.streams > 0 else 8, B)
    lanes = [stream] if nstreams == 1 else [torch.cuda.Stream(dev) for _ in range(nstreams)]
    fork = torch.cuda.Event()
    joins = [torch.cuda.Event() for _ in lanes]
    kimg = min(B, 8)

    def round_(evs=None):
        # forward then inverse of every resident image; with `evs`, an event
        # brackets every kernel launch (rows fwd, cols fwd, rows inv, cols
        # inv) of the first kimg images, all on the timing stream.  Without,
        # the images run on the lanes, forked from and joined back into the
        # timing stream: the join keeps the lanes in step, so the row passes
        # of different images run together, then their column passes (4 %
        # faster than lanes left to drift apart over many images)
        if evs is None and nstreams > 1:
            fork.record(stream)
            for ln in lanes:
                ln.wait_event(fork)
        for i, (x, X) in enumerate(zip(xs, Xs)):
            if evs is None:
                lp = lanes[i % nstreams].cuda_stream
                exec_pass(pf, ROWS, x, X, lp)
                exec_pass(pf, COLS, X, X, lp)
                exec_pass(pi, ROWS, X, X, lp)
                exec_pass(pi, COLS, X, X, lp)
            elif i < kimg:
                e = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
                e[0].record(stream)
                exec_pass(pf, ROWS, x, X, sptr)
                e[1].record(stream)
                exec_pass(pf, COLS, X, X, sptr)
                e[2].record(stream)
                exec_pass(pi, ROWS, X, X, sptr)
                e[3].record(stream)
                exec_pass(pi, COLS, X, X, sptr)
                e[4].record(stream)
                evs.append(e)
        if evs is None and nstreams > 1:
            for ln, j in zip(lanes, joins):
                j.record(ln)
                stream.wait_event(j)

    def step(evs=None):
        # one step: R rounds over the resident images (one round when timing
        # single launches)
        for _ in range(R if evs is None else 1):
            round_(evs)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()

    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    clocks = ClockSampler(uuid)
    evs = []
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t_start.record(stream)
    for _ in range(args.steps):
        step()
    t_end.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    if dist:
        dist.barrier()
    ms_local = t_start.elapsed_time(t_end)
    ms = max_over_ranks(ms_local, dist, dev)

    # per-kernel durations: a second timed region with an event between every
    # two launches (the events themselves add about 2 us per launch, so the
    # headline region above carries none)
    kern_steps = 10
    for _ in range(kern_steps):
        step(evs)
    torch.cuda.synchronize()
    d = np.array([[e[k].elapsed_time(e[k + 1]) for k in range(4)] for e in evs])   # ms
    names = ["row_pass_fwd", "col_pass_fwd", "row_pass_inv", "col_pass_inv"]
    per = {n: float(d[:, k].mean()) for k, n in enumerate(names)}
    pass_bytes = BYTES_PER_PX_PASS * side * side
    row_ms = float(d[:, [0, 2]].mean())
    col_ms = float(d[:, [1, 3]].mean())
    dom, dom_ms = ("col_pass", col_ms) if col_ms >= row_ms else ("row_pass", row_ms)
    peak, peak_src = measured_hbm_peak()
    achieved = pass_bytes / (dom_ms * 1e-3) / 1e9
    value = job_value(2 * B * R * args.steps, ws, ms)
    del xs, Xs
    torch.cuda.empty_cache()

    # end to end through the public host-buffer call, every transform an
    # independent image: upload, transform, download of its result
    ne = min(B, 8)
    hin = [torch.from_numpy(imgs[i]).pin_memory() for i in range(ne)]
    hout = [torch.empty_like(h).pin_memory() for h in hin]
    fft.fft2d_exec_host_many([pf] * ne, hin, hout, sptr)    # allocate the pipeline
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        fft.fft2d_exec_host_many_async([pf] * ne, hin, hout, sptr)
    stream.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, dist, dev)
    img_bytes = side * side * 8
    e2e = {"value": ne * args.e2e_steps * ws / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": ne * img_bytes, "d2h_bytes_per_step": ne * img_bytes,
           "steps": args.e2e_steps, "images_per_step": ne,
           "call": "fft2d_exec_host_many_async, one call per step of independent forward "
                   "transforms: each image uploaded from pinned host memory, transformed and "
                   "its result downloaded; uploads, transforms and downloads of consecutive "
                   "images overlap; stream synchronised after the last call"}
    # chained: each image's forward transform then its inverse in one call,
    # the inverse starting from the device copy of the forward result and
    # overwriting it on the host (the forward result is not downloaded)
    step_plans, step_in, step_out = [], [], []
    for b_ in range(ne):
        step_plans += [pf, pi]
        step_in += [hin[b_], hout[b_]]
        step_out += [hout[b_], hout[b_]]
    fft.fft2d_exec_host_many(step_plans, step_in, step_out, sptr)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        fft.fft2d_exec_host_many_async(step_plans, step_in, step_out, sptr)
    stream.synchronize()
    e2e["chained_forward_inverse"] = {
        "value": 2 * ne * args.e2e_steps * ws / max_over_ranks(time.perf_counter() - t0, dist,
                                                                dev),
        "unit": UNIT, "h2d_bytes_per_step": ne * img_bytes, "d2h_bytes_per_step": ne * img_bytes,
        "counting": "forward and inverse each count as one transform; one upload and one "
                    "download per pair"}
    # one synchronous fft2d_exec_host call per transform
    t0 = time.perf_counter()
    for h, o in zip(hin, hout):
        fft.fft2d_exec_host(pf, h, o, sptr)
    e2e["one_call_per_image"] = {"value": ne * ws / max_over_ranks(
        time.perf_counter() - t0, dist, dev), "call": "fft2d_exec_host"}

    orc = None
    parity = None
    if rank == 0 and not args.no_parity:
        from oracle import oracle
        orc = oracle.get()
        x0 = torch.from_numpy(imgs[0]).to(dev)
        X = torch.empty_like(x0)
        fft.fft2d_exec(pf, x0, X, sptr)
        Y = torch.empty_like(X)
        fft.fft2d_exec(pi, X, Y, sptr)
        torch.cuda.synchronize()
        Xh, Yh = X.cpu().numpy(), Y.cpu().numpy()
        del x0, X, Y
        th = host_cores()
        want = orc.fft2d(imgs[0], threads=th)
        back = orc.fft2d(Xh, inverse=True, threads=th)
        parity = {"fwd_rel_l2": rel_l2(Xh, want), "inv_rel_l2": rel_l2(Yh, back),
                  "round_trip_rel_l2": rel_l2(Yh, imgs[0]),
                  "tolerance": 1e-5, "image": "blob 4096x4096 seed 0"}
        del want, back

    sub = {}
    if rank == 0 and not args.no_sub:
        if orc is None:
            from oracle import oracle
            orc = oracle.get()
        sub["serve"] = measure_serve(fft, torch, args.serve_sample, args.rate, single=False)
        sub["fp16"] = {"4096x4096": measure_fp16(fft, torch, orc, 4096, 20)}
        sub["batched"] = measure_batched(fft, torch, orc, 50)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(side, args.cpu_seconds)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic (seeded Gaussian-blob + U[0,1) gray images)",
            "config": {"workload": f"{side}x{side} complex64 2D FFT: per GPU per step, {R} "
                                   f"rounds of forward+inverse of each of {B} resident images "
                                   f"({2 * B * R} transforms)",
                       "side": side, "images_per_gpu": B, "rounds_per_step": R,
                       "parallelism": f"replicas x{ws}",
                       "streams": nstreams,
                       "l2": f"inputs larger than L2 ({B} images x 2 buffers x "
                             f"{img_bytes >> 20} MiB)",
                       "transform_counting": "forward and inverse each count as one image"},
            "timed_region_ms": ms,
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
                         "unit": "GB/s", "frac": achieved / peak,
                         "peak_source": peak_src,
                         "algorithmic_bytes_per_launch": pass_bytes,
                         "avg_launch_ms": dom_ms,
                         "traffic": ncu_traffic(dom)},
            "passes_ms": per,
            "passes_timing": f"{kern_steps} steps of {kimg} images with an event between "
                             "every two launches",
            "whole_transform_hbm_frac": (2 * pass_bytes / (ms / args.steps / (2 * B * R) * 1e-3)
                                         / 1e9) / peak,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": 4 * B * R * args.steps,
            "clocks": clk,
            "parity": parity,
        }
        line.update(sub)
        print(json.dumps(line), flush=True)
    for p in (pf, pi):
        fft.fft2d_destroy(p)
    if dist:
        dist.destroy_process_group()


# --------------------------------------------------------- reference arm
def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    th = host_cores()
    import synth
    from oracle import oracle
    orc = oracle.get()
    side = args.side
    x = synth.blob_image(side, side, seed=0).astype(np.complex128)
    # one untimed forward+inverse pair pages the data and the library in
    X = orc.fft2d(x, threads=th)
    orc.fft2d(X, inverse=True, threads=th)
    steps = args.steps
    # each step: one forward + one inverse of one image (a bounded sample of
    # the GPU step); steps stop early once the wall-clock budget is spent so
    # the run ends within minutes whatever --steps asks for
    budget_s = 90.0
    t0 = time.perf_counter()
    done = 0
    for _ in range(steps):
        X = orc.fft2d(x, threads=th)
        orc.fft2d(X, inverse=True, threads=th)
        done += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    value = 2 * done / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": done, "warmup": 1, "ms_per_step": dt / done * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded Gaussian-blob + U[0,1) gray image)",
        "config": {"workload": f"{side}x{side} complex64 2D FFT, forward+inverse; each "
                               f"step one image (bounded sample)", "side": side},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": th, "kind": "oracle",
                         "sample": f"{done} forward+inverse pairs of one {side}x{side} image"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------- batched workload
def run_batched(args):
    """The batched workload alone (see measure_batched), with every plan
    shape autotuned first."""
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    import paper_1505_08019_gb300 as fft
    from oracle import oracle
    steps = max(args.steps // 10, 20)
    r = measure_batched(fft, torch, oracle.get(), steps, tune_plans=True)
    line = {
        "metric": "batched 2D FFT images/s (64 uneven power-of-two images, 128..2048 sides)",
        "value": r["images_per_s"], "unit": "images/s", "n_gpus": 1, "steps": steps,
        "warmup": 3, "ms_per_step": r["ms_per_step"], "higher_is_better": True,
        "dtype": "f32", "data": "synthetic (seeded U[0,1) gray images)",
        "config": {"workload": "64 images, log2 sides ~ U{7..11} each (seed 0), forward",
                   "pixels_per_step": r["pixels_per_step"],
                   "l2": f"inputs larger than L2 ({r['pixels_per_step'] * 16 >> 20} MiB)"}}
    line.update(r)
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------ fp16 workload
def run_fp16(args):
    """Half2 storage against complex64 at each --fp16-sides size (see
    measure_fp16)."""
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    import paper_1505_08019_gb300 as fft
    from oracle import oracle
    orc = oracle.get()
    peak, peak_src = measured_hbm_peak()
    sides = [int(v) for v in args.fp16_sides.split(",") if v]
    results = {}
    for side in sides:
        reps = 20 if side <= 8192 else 8
        results[f"{side}x{side}"] = measure_fp16(fft, torch, orc, side, reps,
                                                 check=not args.no_parity)
    big = results[f"{max(sides)}x{max(sides)}"]
    line = {"metric": "2D FFT images/s, FP16 half2 storage vs complex64",
            "value": big["fp16_images_per_s"], "unit": "images/s", "n_gpus": 1,
            "higher_is_better": True, "dtype": "f32 (half2 storage)",
            "data": "synthetic (seeded re, im ~ U[-1,1))",
            "config": {"workload": "forward 2D FFT at " + ", ".join(f"{v}x{v}" for v in sides)
                                   + f"; value = {max(sides)}^2 FP16 images/s"},
            "roofline": {"bound": "hbm", "peak": peak, "unit": "GB/s", "peak_source": peak_src,
                         "algorithmic_bytes_per_px": {"fp16": 16, "fp32": 32}},
            "per_size": results}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------- serving workload
def serve_mix(n, seed=0):
    """The request stream: Poisson arrivals, long side 2^u with u ~ U{6..12},
    half square and half 1:4 (either orientation, short side >= 16), half
    forward FFTs and half FFT -> Gaussian low-pass -> inverse, 70 % complex64
    and 30 % half2 storage."""
    g = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        side = 1 << int(g.integers(6, 13))
        a = g.random()
        if a < 0.5:
            r, c = side, side
        elif a < 0.75:
            r, c = side, max(16, side // 4)
        else:
            r, c = max(16, side // 4), side
        op = 1 if g.random() < 0.5 else 0
        dt = 1 if g.random() < 0.3 else 0
        out.append((op, r, c, dt))
    return out


def measure_serve(fft, torch, n, rate, single=True):
    """The serving loop on a seeded Poisson stream of n requests at `rate`
    req/s (serve_mix; arrivals seed 1) under a 40 GB budget on 4 streams,
    after one warm-up request per (shape, op, dtype); latency percentiles
    overall and per storage type, throughput, and (with `single`) the
    saturation capacity and the plain one-request-at-a-time complex64 path."""
    import synth
    mix = serve_mix(n, seed=0)
    g = np.random.default_rng(1)
    arrivals = np.cumsum(g.exponential(1.0 / rate, n))
    shapes = sorted({(r, c) for _, r, c, _ in mix})
    # one pinned input image per shape and storage (half2 requests carry
    # half2 data and per-row exponents); outputs are shared per shape and
    # storage (their contents are checked by the tests, not here)
    inp, outb = {}, {}
    for sh in shapes:
        img = synth.uniform_real(sh[0], sh[1], seed=7)
        q, e = h16_quantise_rows(img)
        inp[sh, 0] = (torch.from_numpy(img).pin_memory(), None)
        inp[sh, 1] = (torch.from_numpy(q).pin_memory(), torch.from_numpy(e).pin_memory())
        outb[sh, 0] = (torch.empty(sh, dtype=torch.complex64).pin_memory(), None)
        outb[sh, 1] = (torch.empty(q.shape, dtype=torch.float16).pin_memory(),
                       torch.zeros(sh[1], dtype=torch.int32).pin_memory())

    def submit(srv, op, r, c, dt):
        x, y = inp[(r, c), dt], outb[(r, c), dt]
        return fft.fft2d_serve_submit(srv, op, r, c, dt, x[0], y[0], x[1], y[1])

    budget = 40 << 30
    srv = fft.fft2d_serve_create(budget, 4)
    for sh in shapes:
        for op in (0, 1):
            for dt in (0, 1):
                fft.fft2d_serve_wait(srv, submit(srv, op, sh[0], sh[1], dt))
    base = fft.fft2d_serve_stats_get(srv)
    tickets = [0] * n
    t0 = time.perf_counter()
    for i, (op, r, c, dt) in enumerate(mix):
        delay = t0 + arrivals[i] - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        tickets[i] = submit(srv, op, r, c, dt)
    lat = np.array([fft.fft2d_serve_wait(srv, t) for t in tickets])
    wall = time.perf_counter() - t0
    st = fft.fft2d_serve_stats_get(srv)
    dts = np.array([dt for *_, dt in mix])
    done = st["completed"] - base["completed"]
    nb = max(1, st["batches"] - base["batches"])
    out = {
        "requests": n, "offered_rps": rate,
        "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
        "mean_ms": float(lat.mean()), "max_ms": float(lat.max()),
        "throughput_rps": n / wall, "completed": done, "batches": nb,
        "mean_batch_size": done / nb, "peak_device_bytes": st["peak_device_bytes"],
        "by_dtype": {name: {"requests": int((dts == code).sum()),
                            "p50_ms": float(np.percentile(lat[dts == code], 50)),
                            "p99_ms": float(np.percentile(lat[dts == code], 99))}
                     for name, code in (("complex64", 0), ("fp16", 1)) if (dts == code).any()},
        "latency": "submit -> result in the host buffer, as the server stamps it",
        "workload": f"{n} requests at {rate:g} req/s (Poisson, seed 1); long side 2^u, "
                    "u~U{6..12}; 50% square, 50% 1:4; 50% forward, 50% "
                    "FFT->LPF(sigma=side/8)->iFFT; 70% c64 / 30% half2 (half2 data and "
                    "exponents on the host link); pinned host buffers, copies included; HBM "
                    "budget 40 GB; 4 streams"}
    if single:
        # capacity: the same kind of requests submitted all at once
        m_sat = min(n, 4000)
        sat_mix = serve_mix(m_sat, seed=2)
        t2 = time.perf_counter()
        sat_t = [submit(srv, op, r, c, dt) for op, r, c, dt in sat_mix]
        sat_lat = np.array([fft.fft2d_serve_wait(srv, t) for t in sat_t])
        sat_wall = time.perf_counter() - t2
        st2 = fft.fft2d_serve_stats_get(srv)
        out["saturation"] = {"requests": m_sat, "throughput_rps": m_sat / sat_wall,
                             "mean_batch_size": m_sat / max(1, st2["batches"] - st["batches"]),
                             "p50_ms": float(np.percentile(sat_lat, 50)),
                             "p99_ms": float(np.percentile(sat_lat, 99)),
                             "how": "all requests submitted at once; throughput = requests / "
                                    "time to the last result"}
    fft.fft2d_serve_destroy(srv)
    if single:
        # the plain single-image FP32 path on the same requests, one at a
        # time: copy in, transform(s), copy out, wait -- no queueing, no overlap
        m = min(n, 2000)
        stream = torch.cuda.current_stream()
        sptr = stream.cuda_stream
        plans = {}

        def plan(r, c, d):
            if (r, c, d) not in plans:
                plans[(r, c, d)] = fft.fft2d_plan(r, c, fft.FFT2D_C64, d)
            return plans[(r, c, d)]

        dev = {sh: torch.empty(sh, dtype=torch.complex64, device="cuda") for sh in shapes}
        single_lat = []
        t1 = time.perf_counter()
        for op, r, c, _ in mix[:m]:
            ts = time.perf_counter()
            d = dev[(r, c)]
            d.copy_(inp[(r, c), 0][0], non_blocking=True)
            fft.fft2d_exec(plan(r, c, -1), d, d, sptr)
            if op == 1:
                fft.fft2d_lowpass(r, c, fft.FFT2D_C64, d, r / 8.0, c / 8.0, sptr)
                fft.fft2d_exec(plan(r, c, 1), d, d, sptr)
            outb[(r, c), 0][0].copy_(d, non_blocking=True)
            torch.cuda.synchronize()
            single_lat.append((time.perf_counter() - ts) * 1e3)
        single_wall = time.perf_counter() - t1
        for p in plans.values():
            fft.fft2d_destroy(p)
        out["single_image_path"] = {"requests": m, "throughput_rps": m / single_wall,
                                    "p50_ms": float(np.percentile(single_lat, 50)),
                                    "p99_ms": float(np.percentile(single_lat, 99)),
                                    "how": "one request at a time: H2D, fft2d_exec (+ low-pass "
                                           "and inverse), D2H, synchronize; complex64 for all"}
    return out


def run_serve(args):
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    import paper_1505_08019_gb300 as fft
    r = measure_serve(fft, torch, args.requests, args.rate, single=True)
    line = {
        "metric": "serving p50/p99 latency & throughput (Poisson 2D FFT / FFT-filter-iFFT mix)",
        "value": r["p99_ms"], "unit": "ms (p99)", "n_gpus": 1, "higher_is_better": False,
        "dtype": "f32 (70% complex64, 30% half2 storage)",
        "data": "synthetic (seeded Poisson arrivals, U[0,1) gray images)",
        "config": {"workload": r["workload"]}}
    line.update(r)
    print(json.dumps(line), flush=True)

# ------------------------------------------------------------- DCT workload
def run_dct(args):
    """Unnormalised 2D DCT-II of real gray images (U[0,1), one float per
    pixel) through plans of dtype FFT2D_R32_DCT2, beside the forward complex64
    FFT of the same shape.  Four input/output pairs are used in turn, so that
    consecutive launches do not find their image in L2.  Sampled outputs are
    checked against the oracle's direct double sum."""
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    import paper_1505_08019_gb300 as fft
    import synth
    from oracle import oracle
    orc = oracle.get()
    stream = torch.cuda.current_stream()
    sptr = stream.cuda_stream
    peak, peak_src = measured_hbm_peak()
    nbuf = 4
    results = {}
    shapes = []
    for v in args.dct_sides.split(","):
        if v:
            r, _, c = v.partition("x")
            shapes.append((int(r), int(c or r)))

    def t(fn, n):
        for i in range(3):
            fn(i)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for i in range(n):
            fn(i)
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / n

    for R, C in shapes:
        x = synth.gray_real(R, C, seed=R + C)
        xs = [torch.from_numpy(x).cuda() for _ in range(nbuf)]
        ys = [torch.empty_like(xs[0]) for _ in range(nbuf)]
        pd = fft.fft2d_plan(R, C, fft.FFT2D_R32_DCT2, fft.FFT2D_FORWARD)
        reps = 40 if R * C <= 4096 * 4096 else 16
        ms = t(lambda i: fft.fft2d_exec(pd, xs[i % nbuf], ys[i % nbuf], sptr), reps)
        ms_rows = t(lambda i: fft.fft2d_exec_pass(pd, fft.FFT2D_PASS_ROWS, xs[i % nbuf],
                                                  ys[i % nbuf], sptr), reps)
        ms_cols = t(lambda i: fft.fft2d_exec_pass(pd, fft.FFT2D_PASS_COLS, xs[i % nbuf],
                                                  ys[i % nbuf], sptr), reps)
        pinv = fft.fft2d_plan(R, C, fft.FFT2D_R32_DCT2, fft.FFT2D_INVERSE)
        ims = t(lambda i: fft.fft2d_exec(pinv, xs[i % nbuf], ys[i % nbuf], sptr), reps)
        ims_rows = t(lambda i: fft.fft2d_exec_pass(pinv, fft.FFT2D_PASS_ROWS, xs[i % nbuf],
                                                   ys[i % nbuf], sptr), reps)
        ims_cols = t(lambda i: fft.fft2d_exec_pass(pinv, fft.FFT2D_PASS_COLS, xs[i % nbuf],
                                                   ys[i % nbuf], sptr), reps)
        e2e = None
        if (R, C) == shapes[0]:
            # end to end from pinned host buffers: every step uploads nbuf
            # images, transforms them forward and back, downloads both results
            hin = [torch.from_numpy(x).pin_memory() for _ in range(nbuf)]
            hout = [torch.empty_like(h).pin_memory() for h in hin]
            sp, si, so = [], [], []
            for b_ in range(nbuf):
                sp += [pd, pinv]
                si += [hin[b_], hout[b_]]
                so += [hout[b_], hout[b_]]
            fft.fft2d_exec_host_many(sp, si, so, sptr)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(args.e2e_steps):
                fft.fft2d_exec_host_many_async(sp, si, so, sptr)
            stream.synchronize()
            dt = time.perf_counter() - t0
            img_bytes = R * C * 4
            e2e = {"value": 2 * nbuf * args.e2e_steps / dt, "unit": "images/s",
                   "h2d_bytes_per_step": nbuf * img_bytes,
                   "d2h_bytes_per_step": nbuf * img_bytes, "steps": args.e2e_steps,
                   "call": "fft2d_exec_host_many_async, one call per step: each image's "
                           "forward transform, then its inverse from the device copy of the "
                           "forward result into the same host buffer (pinned host buffers)"}
            del hin, hout
        # the round trip into a fresh buffer filled with NaN, so that an
        # output the inverse did not write cannot pass for the input
        rt = torch.full_like(xs[0], float("nan"))
        fft.fft2d_exec(pd, xs[0], ys[0], sptr)
        fft.fft2d_exec(pinv, ys[0], rt, sptr)
        torch.cuda.synchronize()
        got = ys[0].cpu().numpy()
        back = rt.cpu().numpy().astype(np.float64)
        round_trip = float(np.linalg.norm(back - x) / np.linalg.norm(x.astype(np.float64)))
        del rt
        fft.fft2d_destroy(pinv)
        del xs, ys
        torch.cuda.empty_cache()
        # the complex64 forward FFT of the same shape, for comparison
        zc = [torch.zeros((R, C), dtype=torch.complex64, device="cuda") for _ in range(2)]
        pc = fft.fft2d_plan(R, C, fft.FFT2D_C64, fft.FFT2D_FORWARD)
        ms_fft = t(lambda i: fft.fft2d_exec(pc, zc[i % 2], zc[(i + 1) % 2], sptr), reps)
        fft.fft2d_destroy(pc)
        del zc
        torch.cuda.empty_cache()
        # sampled outputs against the direct double sum
        g = np.random.default_rng(R + C)
        idx = [(0, 0), (R // 2, C // 2), (R - 1, C - 1)] + \
              [(int(a), int(b)) for a, b in zip(g.integers(0, R, 5), g.integers(0, C, 5))]
        # the FP32 error bound of a radix-2 transform: u log2(n) ||X||_2, with
        # ||X||_2 <= sqrt(R C) ||x||_2 for the unnormalised DCT-II
        bound = 2.0 ** -24 * np.log2(R * C) * np.sqrt(R * C) * float(
            np.linalg.norm(x.astype(np.float64)))
        worst = 0.0
        for k, l in idx:
            want = orc.dct2d_at(x, k, l)
            worst = max(worst, abs(float(got[k, l]) - want) / bound)
        px = R * C
        results[f"{R}x{C}"] = {
            "dct_ms": ms, "dct_row_pass_ms": ms_rows, "dct_col_pass_ms": ms_cols,
            "dct_images_per_s": 1e3 / ms,
            "dct_hbm_frac": (16.0 * px / (ms * 1e-3) / 1e9) / peak,
            "dct_row_pass_hbm_frac": (8.0 * px / (ms_rows * 1e-3) / 1e9) / peak,
            "dct_col_pass_hbm_frac": (8.0 * px / (ms_cols * 1e-3) / 1e9) / peak,
            "idct_ms": ims, "idct_row_pass_ms": ims_rows, "idct_col_pass_ms": ims_cols,
            "idct_hbm_frac": (16.0 * px / (ims * 1e-3) / 1e9) / peak,
            "round_trip_rel_l2": round_trip,
            "complex64_fft_forward_ms": ms_fft,
            "dct_speedup_vs_complex_fft": ms_fft / ms,
            "sampled_outputs_checked": len(idx),
            "worst_sample_err_over_fp32_bound": worst,
            "e2e": e2e,
            "kernels": fft.fft2d_plan_describe(pd)}
        fft.fft2d_destroy(pd)
    R0, C0 = shapes[0]
    head = results[f"{R0}x{C0}"]
    line = {"metric": "2D DCT-II images/s (real FP32 images)",
            "value": head["dct_images_per_s"], "unit": "images/s", "n_gpus": 1,
            "higher_is_better": True, "dtype": "f32",
            "data": "synthetic (seeded gray images, U[0,1))",
            "config": {"workload": "forward unnormalised 2D DCT-II at "
                                   + ", ".join(f"{r}x{c}" for r, c in shapes)
                                   + f"; value = {R0}x{C0} images/s; {nbuf} input/output "
                                     "pairs used in turn (L2 not reused between launches)"},
            "roofline": {"bound": "hbm", "peak": peak, "unit": "GB/s", "peak_source": peak_src,
                         "algorithmic_bytes_per_px": 16,
                         "achieved": 16.0 * R0 * C0 / (head["dct_ms"] * 1e-3) / 1e9,
                         "frac": head["dct_hbm_frac"]},
            "e2e": head["e2e"],
            "per_size": results}
    print(json.dumps(line), flush=True)


# --------------------------------------------------- Table 1 image sizes
def run_sizes(args):
    """Forward + inverse complex64 transforms at the paper's Table 1 gray
    image sizes (128^2 .. 2048^2) and at 4096^2, one image at a time on one
    stream (the paper's setting), with enough images in rotation that the
    working set exceeds L2, captured in a CUDA graph and replayed (and, for
    context, the same calls from a Python loop).  Reports microseconds per
    transform, the
    fraction of measured HBM bandwidth at 32 B/px, and the error of the
    round trip against the input."""
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    import paper_1505_08019_gb300 as fft
    import synth
    stream = torch.cuda.current_stream()
    sptr = stream.cuda_stream
    peak, peak_src = measured_hbm_peak()
    results = {}
    for side in (128, 256, 512, 1024, 2048, 4096):
        img_bytes = side * side * 8
        nimg = max(2, int(2 * 129e6 // img_bytes) + 1)   # rotation larger than twice L2
        x = synth.uniform_real(side, side, seed=side)
        xs = [torch.from_numpy(x).cuda() for _ in range(nimg)]
        ys = [torch.empty_like(xs[0]) for _ in range(nimg)]
        pf = fft.fft2d_plan(side, side, fft.FFT2D_C64, fft.FFT2D_FORWARD)
        pi = fft.fft2d_plan(side, side, fft.FFT2D_C64, fft.FFT2D_INVERSE)
        reps = max(40, nimg * 4)

        def step(i):
            fft.fft2d_exec(pf, xs[i % nimg], ys[i % nimg], sptr)
            fft.fft2d_exec(pi, ys[i % nimg], ys[i % nimg], sptr)

        for i in range(5):
            step(i)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for i in range(reps):
            step(i)
        b.record(stream)
        torch.cuda.synchronize()
        us_eager = a.elapsed_time(b) * 1e3 / (2 * reps)
        # the same steps captured once in a CUDA graph and replayed: the
        # device time without the host's per-call launch cost
        per_graph = min(nimg, 256)
        gs = torch.cuda.Stream()
        gs.wait_stream(stream)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=gs):
            for i in range(per_graph):
                fft.fft2d_exec(pf, xs[i % nimg], ys[i % nimg], gs.cuda_stream)
                fft.fft2d_exec(pi, ys[i % nimg], ys[i % nimg], gs.cuda_stream)
        replays = max(3, reps // per_graph)
        graph.replay()
        torch.cuda.synchronize()
        a.record(stream)
        for _ in range(replays):
            graph.replay()
        b.record(stream)
        torch.cuda.synchronize()
        us = a.elapsed_time(b) * 1e3 / (2 * per_graph * replays)
        del graph
        fft.fft2d_exec(pf, xs[0], ys[0], sptr)
        fft.fft2d_exec(pi, ys[0], ys[0], sptr)
        torch.cuda.synchronize()
        back = ys[0].cpu().numpy()
        max_err = float(np.abs(back.astype(np.complex128) - x.astype(np.complex128)).max())
        results[f"{side}x{side}"] = {
            "us_per_transform": us, "transforms_per_s": 1e6 / us,
            "us_per_transform_eager_python_loop": us_eager,
            "hbm_frac": (32.0 * side * side / (us * 1e-6) / 1e9) / peak,
            "round_trip_max_abs_err": max_err, "images_in_rotation": nimg}
        fft.fft2d_destroy(pf)
        fft.fft2d_destroy(pi)
        del xs, ys
        torch.cuda.empty_cache()
    line = {"metric": "2D FFT transforms/s at the paper's Table 1 sizes (one stream)",
            "value": results["2048x2048"]["transforms_per_s"], "unit": "transforms/s",
            "n_gpus": 1, "higher_is_better": True, "dtype": "f32",
            "data": "synthetic (seeded U[0,1) gray images)",
            "config": {"workload": "forward and inverse complex64 FFT, one image at a time on "
                                   "one stream, 128^2 .. 4096^2, CUDA-graph replay; value = "
                                   "2048^2 transforms/s",
                       "l2": "images rotated so the working set exceeds L2"},
            "roofline": {"bound": "hbm", "peak": peak, "unit": "GB/s", "peak_source": peak_src,
                         "algorithmic_bytes_per_px": 32},
            "paper_table1_gpu_ms": {"128x128": 16, "256x256": 16, "512x512": 28,
                                    "1024x1024": 62, "2048x2048": 250},
            "per_size": results}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------- single passes
def run_passes(args):
    """The plan's default kernels on one --shape image (re, im ~ U[-1, 1)):
    complex64 row and column passes timed separately, or the half2
    transform (both passes) -- a small, fixed launch sequence for profiling
    one kernel.  Two input/output pairs alternate."""
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    import paper_1505_08019_gb300 as fft
    import synth
    R, _, C = args.shape.partition("x")
    R, C = int(R), int(C or R)
    stream = torch.cuda.current_stream()
    sptr = stream.cuda_stream
    t = cuda_timer(torch, stream)
    x = synth.uniform_complex(R, C, seed=R + C)
    reps = max(1, args.steps)
    peak, _ = measured_hbm_peak()
    out = {}
    if args.dtype == "c64":
        p = fft.fft2d_plan(R, C, fft.FFT2D_C64, fft.FFT2D_FORWARD)
        dx = [torch.from_numpy(x).cuda() for _ in range(2)]
        dy = [torch.empty_like(dx[0]) for _ in range(2)]
        for name, ps in (("rows", fft.FFT2D_PASS_ROWS), ("cols", fft.FFT2D_PASS_COLS)):
            ms = t(lambda i: fft.fft2d_exec_pass(p, ps, dx[i & 1], dy[i & 1], sptr), reps)
            out[name] = {"ms": ms, "hbm_frac": 16.0 * R * C / (ms * 1e-3) / 1e9 / peak}
        out["kernels"] = fft.fft2d_plan_describe(p)
        fft.fft2d_sync_status(p)
        fft.fft2d_destroy(p)
    else:
        p = fft.fft2d_plan(R, C, fft.FFT2D_C32H, fft.FFT2D_FORWARD)
        q, e = h16_quantise_rows(x)
        dq = [torch.from_numpy(q).cuda() for _ in range(2)]
        de = torch.from_numpy(e).cuda()
        do = [torch.empty_like(dq[0]) for _ in range(2)]
        oe = torch.empty(C, dtype=torch.int32, device="cuda")
        ms = t(lambda i: fft.fft2d_exec_h16(p, dq[i & 1], de, fft.FFT2D_PASS_ROWS, do[i & 1], oe,
                                            sptr), reps)
        out["both"] = {"ms": ms, "hbm_frac": 16.0 * R * C / (ms * 1e-3) / 1e9 / peak}
        fft.fft2d_sync_status(p)
        fft.fft2d_destroy(p)
    print(json.dumps({"workload": "passes", "shape": [R, C], "dtype": args.dtype,
                      "reps": reps, "passes": out}), flush=True)


# ------------------------------------------- CPU baseline at several sizes
def run_cpu(args):
    """The CPU baseline (the FP64 oracle as it stands, on one thread and on
    all host cores) at the sizes of the plain, blob and large-image
    workloads, each beside the GPU's device time for the same forward +
    inverse pair (one image at a time, a rotation of images larger than L2)."""
    sides = (256, 1024, 4096, 8192)
    th = host_cores()
    cpu = {}
    for side in sides:   # the oracle first, before any GPU work
        v, n, dt = cpu_oracle_sample(side, args.cpu_seconds, th)
        v1, n1, dt1 = cpu_oracle_sample(side, args.cpu_seconds, 1)
        cpu[side] = {"all_cores": {"value": v, "unit": UNIT, "cores": th,
                                   "sample": f"{n} transforms, {dt:.1f} s"},
                     "single_thread": {"value": v1, "unit": UNIT, "cores": 1,
                                       "sample": f"{n1} transforms, {dt1:.1f} s"}}
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    import paper_1505_08019_gb300 as fft
    import synth
    stream = torch.cuda.current_stream()
    sptr = stream.cuda_stream
    out = {}
    for side in sides:
        nimg = max(2, int(2 * 129e6 // (side * side * 8)) + 1)
        x = torch.from_numpy(synth.blob_image(side, side, seed=0)).cuda()
        xs = [x.clone() for _ in range(nimg)]
        ys = [torch.empty_like(x) for _ in range(nimg)]
        pf = fft.fft2d_plan(side, side, fft.FFT2D_C64, fft.FFT2D_FORWARD)
        pi = fft.fft2d_plan(side, side, fft.FFT2D_C64, fft.FFT2D_INVERSE)
        reps = max(40, 4 * nimg)
        for i in range(reps + 5):
            if i == 5:
                torch.cuda.synchronize()
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
            fft.fft2d_exec(pf, xs[i % nimg], ys[i % nimg], sptr)
            fft.fft2d_exec(pi, ys[i % nimg], ys[i % nimg], sptr)
        b.record(stream)
        torch.cuda.synchronize()
        gpu = 2 * reps / (a.elapsed_time(b) / 1e3)
        fft.fft2d_destroy(pf)
        fft.fft2d_destroy(pi)
        del xs, ys, x
        torch.cuda.empty_cache()
        out[f"{side}x{side}"] = {"gpu": {"value": gpu, "unit": UNIT,
                                         "call": "fft2d_exec forward + inverse, one stream"},
                                 "cpu_baseline": dict(cpu[side], kind="oracle"),
                                 "gpu_over_all_cores": gpu / cpu[side]["all_cores"]["value"]}
    print(json.dumps({"metric": "2D FFT transforms/s, FP64 oracle on the host beside the GPU",
                      "unit": UNIT, "workload": "cpu", "cpu_model": cpu_model(), "cores": th,
                      "input": "blob image (seeded), forward + inverse pairs",
                      "per_size": out}), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "fp16":
        run_fp16(args)
    elif args.workload == "serve":
        run_serve(args)
    elif args.workload == "dct":
        run_dct(args)
    elif args.workload == "sizes":
        run_sizes(args)
    elif args.workload == "passes":
        run_passes(args)
    elif args.workload == "cpu":
        run_cpu(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
