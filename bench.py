"""Benchmark: Pilatus-6M-shape 1D azimuthal integration (2527 x 2463 uint32 frames, module-gap
mask, q in nm^-1, 1000 bins, full pixel split, dark/flat/solid-angle/polarisation), batched
FP32-compensated forward, frames/s.

A step integrates one batch of --frames frames that are already resident in HBM (the
batch, 3.2 GB at the default 128 frames, is far larger than the 129 MB L2, so every step
streams it from DRAM) against the detector's corrections, bound once beforehand like the
matrix (az_set_corrections).  Alongside the device-resident number the script reports:
  per_call_corrections  the same batches with the corrections formed again in every call;
  e2e          the same metric through az_integrate_batch_host (pinned host frames, copies
               inside the timed region; --e2e-frames frames per call, by default the step's);
  roofline     achieved HBM GB/s of the dominant kernel (phase-1 frames kernel), timed with
               CUDA events on its stream during the timed region;
  plain        the one-frame-per-launch FP64 form on the same GPU (the comparator: the faster
               of the tiled form and the look-up table), with its roofline fraction;
  parity       relative error per output (I, S, N, C) of frame 0: the FP32 batch and the FP64
               one-frame form against the oracle, and the two against each other;
  cpu_baseline the oracle (plain C, one thread) on a bounded sample of the same workload.

--impl reference times the oracle alone on the host cores (the reference arm).
Multi-GPU (torchrun): frames are independent, so each rank integrates its own batch on its
own GPU with no collective on the data path (weak scaling); only the timing is reduced.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Pilatus-6M-shape 1D integration frames/s & HBM GB/s vs plain, <=1e-5 rel err"
UNIT = "frames/s"


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--frames", type=int, default=128, help="frames per step (per GPU)")
    ap.add_argument("--e2e-frames", type=int, default=128,
                    help="frames per end-to-end call (at most --frames; default: the step's)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--autotune", action="store_true")
    ap.add_argument("--no-other-workloads", action="store_true",
                    help="skip the cake / batching / stream / adjoint measurements")
    ap.add_argument("--only-batching", action="store_true",
                    help="run only the many-instance launch (3 warm-up + --steps launches) "
                         "and print its figures")
    ap.add_argument("--only-cake", action="store_true",
                    help="run only the 2048 x 2048 cake batch (64 frames; 3 warm-up + --steps "
                         "calls) and print its rate")
    ap.add_argument("--only-single", action="store_true",
                    help="run only one Pilatus-6M frame per call (FP32, corrections; 3 warm-up "
                         "+ --steps calls) and print its time")
    ap.add_argument("--only-stream", action="store_true",
                    help="run only the 2167 x 2070 stream (--frames frames per call, 16 x 96 "
                         "tiles and 8 frames per pass, no autotuning; 1 warm-up + --steps calls) "
                         "and print its rate")
    ap.add_argument("--instances", type=int, default=64,
                    help="instances of the many-instance launch with --only-batching")
    return ap.parse_args(argv)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def frame_seeds(rank, n=8):
    """Seeds of the synthetic frames a rank cycles through (disjoint across ranks): each rank
    integrates its own frames, there is no exchange between ranks."""
    return [1000 * rank + k for k in range(n)]


def max_over_ranks(value, world):
    """The largest of every rank's `value` (the job's time is its slowest rank's)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" \
        else torch.device("cpu")
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(frames_per_rank_step, world, steps, ms):
    """Frames per second of the whole job: every rank's frames over the slowest rank's time."""
    return world * frames_per_rank_step * steps / (ms / 1e3)


def workload_inputs(w, og_positions):
    """Seeded synthetic inputs of the Pilatus workload shaped on centre q values."""
    from paper_1412_6367_gb300 import synth
    crad = og_positions
    mask = synth.pilatus_module_mask(w.ny, w.nx)
    dark, flat = synth.dark_flat(w.ny, w.nx, w.seed)
    return crad, mask, dark, flat


def algorithmic_bytes(nnz, n_unmasked, nrows, frames, dark=True):
    """Bytes the batched integration must move: the matrix once (8 B per entry: index +
    weight), the dark once, each frame's unmasked pixels (4 B) and 16 B of output per bin
    and frame; the frame-independent corrections and sums are counted separately."""
    return nnz * 8 + (n_unmasked * 4 if dark else 0) + frames * (n_unmasked * 4 + 16 * nrows)


def plain_fp64_bytes(nnz, n_unmasked, nrows):
    """Algorithmic bytes of one FP64 frame through the matrix: index and FP64 weight per entry,
    the image and the four correction arrays per pixel, the row pointers and four FP64
    outputs per row."""
    return nnz * 12 + n_unmasked * 4 * 5 + 4 * (nrows + 1) + 4 * 8 * nrows


def phase1_frames_bytes(nnz, n_unmasked, frames):
    """Algorithmic bytes of one phase-1 frames launch covering `frames` frames."""
    return nnz * 8 + n_unmasked * 4 + frames * n_unmasked * 4


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        fd, self.path = tempfile.mkstemp(prefix="azint_clocks_%d_" % index, suffix=".csv")
        os.close(fd)

    def start(self):
        try:
            fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index),
                 "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "50"], stdout=fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if not self.proc:
            try:
                os.remove(self.path)
            except OSError:
                pass
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    mx.append(float(f[2]))
                except ValueError:
                    continue
                for n, v in zip(names, f[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
        except OSError:
            return None
        finally:
            try:
                os.remove(self.path)
            except OSError:
                pass
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


FRAMES_SECTIONS = (("// frames pass with tile-resident entries", "// phase 2: per-row sums"),
                   ("// ---- frames kernel with tile-resident entries", "// flat * solid angle * polarisation per pixel"))


def frames_kernel_sha():
    """sha256 of the frames kernel's source: its device and launch sections of integrate.cu
    and the shared header (None if a section marker is missing)."""
    csrc = os.path.join(ROOT, "paper_1412_6367_gb300", "csrc")
    try:
        text = open(os.path.join(csrc, "integrate.cu")).read()
        common = open(os.path.join(csrc, "common.cuh")).read()
    except OSError:
        return None
    parts = []
    for a, b in FRAMES_SECTIONS:
        i, j = text.find(a), text.find(b)
        if i < 0 or j < i:
            return None
        parts.append(text[i:j])
    parts.append(common)
    return hashlib.sha256("".join(parts).encode()).hexdigest()


def ncu_traffic():
    """DRAM bytes per launch of the phase-1 frames kernel from the committed ncu summary,
    if that summary was taken on the current source of the kernel."""
    path = os.path.join(ROOT, "profiles", "frames_kernel_pilatus6m.txt")
    try:
        text = open(path).read()
    except OSError:
        return None
    sha = frames_kernel_sha()
    m = re.search(r"source_sha256:\s*([0-9a-f]+)", text)
    t = re.search(r"traffic_bytes_per_launch_full:\s*([0-9.e+]+)", text)
    f = re.search(r"capture_frames_per_launch:\s*([0-9]+)", text)
    if not m or not t or not f or m.group(1) != sha:
        return None
    return float(t.group(1)), int(f.group(1))


def cpu_baseline(w, seconds, check=None):
    """The oracle, as it stands, on a bounded sample of the workload: frames integrated one
    after the other on one host core for about `seconds` (matrix built beforehand, untimed).
    With check = (frame, I_gpu, solid_angle, polarisation) the oracle's matrix also gives the
    parity spot check of the GPU's I of that frame (its relative error, and both nnz)."""
    import oracle as O
    from paper_1412_6367_gb300 import synth
    og = O.Geometry(*w.geometry.astuple())
    t_build = time.perf_counter()
    rad, chi = O.corner_positions(og, w.ny, w.nx, w.unit)
    mask = synth.pilatus_module_mask(w.ny, w.nx)
    A = O.csr_build(w.ny, w.nx, rad, chi, mask, w.npt_rad, 0, w.split)
    t_build = time.perf_counter() - t_build
    crad, _ = O.centre_positions(og, w.ny, w.nx, w.unit)
    dark, flat = synth.dark_flat(w.ny, w.nx, w.seed)
    sa = O.solid_angle(og, w.ny, w.nx).astype(np.float32)
    pol = O.polarization(og, w.ny, w.nx, 0.99).astype(np.float32)
    frames = [synth.ring_image(crad, seed=1000 + k) for k in range(4)]
    n = 0
    t0 = time.perf_counter()
    while True:
        O.integrate(A, frames[n % 4], dark, flat, sa, pol)
        n += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    parity = None
    if check is not None:
        frame, got32, got64, sa_g, pol_g = check
        ref = O.integrate(A, frame, dark, flat, sa_g, pol_g)
        parity = {"nnz_oracle": int(A.nnz), "frame": "frame 0 of the timed batch",
                  "metric": "max |x - ref| / |ref| over bins with |ref| > 1e-3 max|ref|",
                  "fp32_batch_vs_oracle": {}, "fp64_one_frame_vs_oracle": {},
                  "fp32_batch_vs_fp64_one_frame": {}}
        for k, name in enumerate("ISNC"):
            parity["fp32_batch_vs_oracle"][name] = rel_max(got32[k], ref[k])
            parity["fp64_one_frame_vs_oracle"][name] = rel_max(got64[k], ref[k])
            parity["fp32_batch_vs_fp64_one_frame"][name] = rel_max(got32[k], got64[k])
        parity["max_rel_err_I"] = parity["fp32_batch_vs_oracle"]["I"]
    res = {"value": n / el, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": "%d Pilatus-6M frames integrated one by one by the C oracle (FP64, full "
                     "split, corrections) in %.1f s; matrix built beforehand" % (n, el),
           "matrix_build_s": t_build}
    # the multi-core CPU form of the paper (Sec. 3.4.1: per-thread histograms over the pixels,
    # OpenMP on every host core), FP64, on the oracle's matrix regrouped by pixel
    M = O.csc_of(A)
    ref = O.integrate(A, frames[0], dark, flat, sa, pol)
    got = O.omp_integrate(M, frames[0], dark, flat, sa, pol)
    m, t0 = 0, time.perf_counter()
    while True:
        _, _, _, _, used = O.omp_integrate(M, frames[m % 4], dark, flat, sa, pol)
        m += 1
        el2 = time.perf_counter() - t0
        if el2 >= seconds * 2 / 3:
            break
    res["multicore"] = {
        "value": m / el2, "unit": UNIT, "cores": int(used), "nproc": os.cpu_count(),
        "kind": "OpenMP per-thread histograms (oracle/azint_omp.c)",
        "sample": "%d Pilatus-6M frames one by one, FP64, in %.1f s" % (m, el2),
        "max_rel_err_vs_oracle": max(rel_max(g_, r_) for g_, r_ in zip(got[:4], ref))}
    return res, parity


def rel_max(got, ref, floor_frac=1e-3):
    """Largest relative error of `got` over the entries where |ref| > floor_frac max|ref|."""
    got = np.asarray(got, dtype=np.float64).ravel()
    ref = np.asarray(ref, dtype=np.float64).ravel()
    sel = np.abs(ref) > floor_frac * np.abs(ref).max()
    return float(np.max(np.abs(got[sel] - ref[sel]) / np.abs(ref[sel]))) if sel.any() else 0.0


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from paper_1412_6367_gb300 import synth
    w = synth.pilatus_workload()
    per_step = max(1.0, args.cpu_seconds / max(args.steps, 1))
    import oracle as O
    og = O.Geometry(*w.geometry.astuple())
    rad, chi = O.corner_positions(og, w.ny, w.nx, w.unit)
    mask = synth.pilatus_module_mask(w.ny, w.nx)
    A = O.csr_build(w.ny, w.nx, rad, chi, mask, w.npt_rad, 0, w.split)
    crad, _ = O.centre_positions(og, w.ny, w.nx, w.unit)
    dark, flat = synth.dark_flat(w.ny, w.nx, w.seed)
    sa = O.solid_angle(og, w.ny, w.nx).astype(np.float32)
    pol = O.polarization(og, w.ny, w.nx, 0.99).astype(np.float32)
    frames = [synth.ring_image(crad, seed=1000 + k) for k in range(4)]

    def step():
        n, t0 = 0, time.perf_counter()
        while True:
            O.integrate(A, frames[n % 4], dark, flat, sa, pol)
            n += 1
            if time.perf_counter() - t0 >= per_step:
                return n

    for _ in range(args.warmup):
        step()
    total_frames = 0
    t0 = time.perf_counter()
    for _ in range(args.steps):
        total_frames += step()
    el = time.perf_counter() - t0
    v = total_frames / el
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_dict(w, total_frames // max(args.steps, 1)),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": "%d frames over %d steps of ~%.1f s" % (total_frames, args.steps, per_step)},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def _event_ms(torch, fn, reps):
    """Mean device time of fn() over `reps` calls (CUDA events on the current stream)."""
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def stage_breakdown(torch, dev, reps=20):
    """Per-stage times of one Pilatus-1M int32 frame (1043 x 981, 1000 q bins, bounding-box
    split, corrections) integrated one frame per call from a pinned host buffer, the steps of
    the paper's table in Sec. 6.4: host-to-device copy of the image, the kernels by kind (the
    cast is fused into them), device-to-host copies of I, S and C, and the Python-level total
    of copy + integrate + copies back (wall clock, synchronised), for the tiled and the
    look-up-table layouts."""
    from paper_1412_6367_gb300 import api, synth
    w = synth.pilatus1m_workload()
    g = api.Geometry(*w.geometry.astuple())
    mask = synth.pilatus_module_mask(w.ny, w.nx)
    ig = api.Integrator.build(g, (w.ny, w.nx), w.npt_rad, 0, "q_nm^-1", "bbox", mask=mask, device=dev)
    crad, _ = g.positions(w.ny, w.nx, "q_nm^-1", "centres", chi=False, device=dev)
    img_h = torch.from_numpy(synth.ring_image(crad.cpu().numpy(), seed=5).view(np.int32)).pin_memory()
    dark, flat = (torch.from_numpy(a).to(dev) for a in synth.dark_flat(w.ny, w.nx, w.seed))
    sa, pol = g.solid_angle(w.ny, w.nx, device=dev), g.polarization(w.ny, w.nx, 0.99, device=dev)
    img_d = torch.empty_like(img_h, device=dev)
    outs = [torch.empty(ig.nrows, device=dev) for _ in range(3)]
    hosts = [torch.empty(ig.nrows).pin_memory() for _ in range(3)]
    res = {"workload": w.name, "nnz": ig.info["nnz"]}
    for layout in ("tiled", "lut"):
        ig.set_layout(layout)
        call = lambda: ig.integrate(img_d, dark, flat, sa, pol, precision="fp32")
        img_d.copy_(img_h, non_blocking=True)
        call()
        torch.cuda.synchronize()
        h2d = _event_ms(torch, lambda: img_d.copy_(img_h, non_blocking=True), reps)
        r = call()
        d2h = _event_ms(torch, lambda: [hh.copy_(t, non_blocking=True) for hh, t in
                                        zip(hosts, (r.I, r.sum_signal, r.count))], reps)
        ig.profile_read()
        ig.profile_enable(True)
        for _ in range(reps):
            call()
        ig.profile_enable(False)
        kinds = {k: v[1] / reps for k, v in ig.profile_read().items() if v[0]}
        t0 = time.perf_counter()
        for _ in range(reps):
            img_d.copy_(img_h, non_blocking=True)
            r = call()
            for hh, t in zip(hosts, (r.I, r.sum_signal, r.count)):
                hh.copy_(t, non_blocking=True)
            torch.cuda.synchronize()
        total = (time.perf_counter() - t0) / reps * 1e3
        res[layout] = {"python_total_ms": total, "h2d_image_ms": h2d, "d2h_3_outputs_ms": d2h,
                       "kernels_ms": kinds, "device_sum_ms": h2d + d2h + sum(kinds.values())}
    ig.set_layout("tiled")
    return res


def cake_workload(torch, dev, gen, reps=5):
    """2048 x 2048 float32 frames, 500 2theta x 360 chi bins, full split, corrections:
    64-frame batches and one frame per call."""
    from paper_1412_6367_gb300 import api, synth
    w = synth.cake_workload()
    g = api.Geometry(*w.geometry.astuple())
    ig = api.Integrator.build(g, (w.ny, w.nx), w.npt_rad, w.npt_azim, "2th_deg", "full", device=dev)
    dark = torch.rand((w.ny, w.nx), generator=gen, device=dev) + 10.0
    flat = 0.95 + 0.1 * torch.rand((w.ny, w.nx), generator=gen, device=dev)
    sa, pol = g.solid_angle(w.ny, w.nx, device=dev), g.polarization(w.ny, w.nx, 0.99, device=dev)
    frames = 1000.0 * torch.rand((64, w.ny, w.nx), generator=gen, device=dev)
    default = (ig.info["tile_h"], ig.info["tile_w"], ig.info["frames_per_pass"])
    ig.autotune(16)  # setup, untimed: tiles and frames per pass for this matrix
    for _ in range(3):
        ig.integrate_batch(frames, dark, flat, sa, pol)
    ms = _event_ms(torch, lambda: ig.integrate_batch(frames, dark, flat, sa, pol), reps)
    ms1 = _event_ms(torch, lambda: ig.integrate(frames[0], dark, flat, sa, pol, precision="fp32"), 10)
    res = {"batched_frames_per_s": 64 / (ms / 1e3), "single_frame_fp32_ms": ms1,
           "nnz": ig.info["nnz"], "default_tuning": default,
           "autotuned": (ig.info["tile_h"], ig.info["tile_w"], ig.info["frames_per_pass"])}
    del frames, ig
    return res


def stream_only(torch, dev, gen, reps, nframes):
    """The 2167 x 2070 / 2000-bin stream alone at a fixed tuning (16 x 96 tiles, 8 frames per
    pass: the frame-pair staging), nframes-frame device calls: frames/s and the frames pass."""
    from paper_1412_6367_gb300 import api, synth
    w = synth.stream_workload()
    g = api.Geometry(*w.geometry.astuple())
    ig = api.Integrator.build(g, (w.ny, w.nx), w.npt_rad, 0, "q_nm^-1", "full", device=dev)
    fr = torch.randint(0, 4000, (nframes, w.ny, w.nx), generator=gen, device=dev, dtype=torch.int32)
    fr = fr.view(torch.uint32)
    ig.set_tuning(16, 96, 0, 8)
    ig.integrate_batch(fr)
    ig.profile_read()
    ig.profile_enable(True)
    ms = _event_ms(torch, lambda: ig.integrate_batch(fr), reps)
    ig.profile_enable(False)
    n, k = ig.profile_read()["phase1_frames"]
    res = {"frames_per_s": nframes / (ms / 1e3), "frames_per_call": nframes, "tuning": [16, 96, 8],
           "nnz": ig.info["nnz"],
           "frames_pass_ms_per_64": k / max(n, 1)}
    del fr, ig
    return res


def single_frame_workload(torch, dev, reps=20):
    """One Pilatus-6M uint32 frame per call, FP32 compensated, with dark, flat, solid angle
    and polarisation: ms per frame."""
    from paper_1412_6367_gb300 import api, synth
    w = synth.pilatus_workload()
    g = api.Geometry(*w.geometry.astuple())
    mask = synth.pilatus_module_mask(w.ny, w.nx)
    ig = api.Integrator.build(g, (w.ny, w.nx), w.npt_rad, 0, "q_nm^-1", "full", mask=mask, device=dev)
    crad, _ = g.positions(w.ny, w.nx, "q_nm^-1", "centres", chi=False, device=dev)
    img = torch.from_numpy(synth.ring_image(crad.cpu().numpy(), seed=3).view(np.int32)).to(dev)
    img = img.view(torch.uint32)
    dark, flat = (torch.from_numpy(a).to(dev) for a in synth.dark_flat(w.ny, w.nx, w.seed))
    sa, pol = g.solid_angle(w.ny, w.nx, device=dev), g.polarization(w.ny, w.nx, 0.99, device=dev)
    for _ in range(3):
        ig.integrate(img, dark, flat, sa, pol, precision="fp32")
    ms = _event_ms(torch, lambda: ig.integrate(img, dark, flat, sa, pol, precision="fp32"), reps)
    return {"ms_per_frame": ms, "frames_per_s": 1e3 / ms}


def batching_workload(torch, dev, gen, reps=10, n=64):
    """n (default 64) heterogeneous instances (three detector shapes, 500 / 2000 / 5000 q
    bins, full split) in one graph-captured persistent launch: ms per launch and throughput."""
    from paper_1412_6367_gb300 import api, synth
    ws = synth.batch_instances()[:n]
    igs, imgs = [], []
    for wi in ws:
        gi = api.Geometry(*wi.geometry.astuple())
        igs.append(api.Integrator.build(gi, (wi.ny, wi.nx), wi.npt_rad, 0, "q_nm^-1", "full", device=dev))
        imgs.append(torch.randint(0, 4000, (wi.ny, wi.nx), generator=gen, device=dev, dtype=torch.int32))
    plan = api.MultiPlan(igs, imgs)
    for _ in range(3):
        plan.launch(use_graph=True)
    ms = _event_ms(torch, lambda: plan.launch(use_graph=True), reps)
    pix = sum(wi.ny * wi.nx for wi in ws)
    nnz = sum(gi.info["nnz"] for gi in igs)
    rows = sum(gi.nrows for gi in igs)
    # algorithmic bytes of the launch: every entry (2-byte location, 4-byte weight), every
    # image pixel, four outputs per row
    ab = 6 * nnz + 4 * pix + 16 * rows
    res = {"ms_per_launch": ms, "instances": len(ws), "instances_per_s": len(ws) / (ms / 1e3),
           "gpix_per_s": pix / (ms / 1e3) / 1e9, "nnz_total": nnz,
           "algorithmic_gbs": ab / (ms / 1e3) / 1e9}
    del plan, igs, imgs
    return res


def size_sweep(torch, dev, gen):
    """One int32 frame per call (tiled and look-up-table layouts, FP32) and 32-frame batches
    at the paper's benchmark sizes (1 to 16 Mpixel, bounding-box split, 1000 q bins):
    ms per frame and Mpixel/s."""
    from paper_1412_6367_gb300 import api, synth
    res = []
    for w in synth.size_sweep_workloads():
        g = api.Geometry(*w.geometry.astuple())
        ig = api.Integrator.build(g, (w.ny, w.nx), w.npt_rad, 0, "q_nm^-1", "bbox", device=dev)
        frames = torch.randint(0, 4000, (32, w.ny, w.nx), generator=gen, device=dev, dtype=torch.int32)
        row = {"shape": [w.ny, w.nx], "nnz": ig.info["nnz"]}
        for layout in ("tiled", "lut"):
            ig.set_layout(layout)
            for _ in range(3):
                ig.integrate(frames[0], precision="fp32")
            row[layout + "_single_ms"] = _event_ms(torch, lambda: ig.integrate(frames[0], precision="fp32"), 10)
        ig.set_layout("tiled")
        for _ in range(2):
            ig.integrate_batch(frames)
        row["batched_ms_per_frame"] = _event_ms(torch, lambda: ig.integrate_batch(frames), 3) / 32
        npix = w.ny * w.nx
        row["mpix_per_s"] = {k: npix / (row[k] / 1e3) / 1e6 for k in
                             ("tiled_single_ms", "lut_single_ms", "batched_ms_per_frame")}
        res.append(row)
        del frames, ig
    return res


def other_workloads(torch, dev, ig_pilatus, pilatus_inputs):
    """The other workloads' throughput (device-resident inputs, warm), reported beside the
    headline: the 2D cake, the 64-instance persistent launch, a 4096-frame stream through
    one matrix, and the adjoint on the Pilatus matrix."""
    from paper_1412_6367_gb300 import api, synth
    out = {}
    gen = torch.Generator(device=dev)
    gen.manual_seed(7)

    out["cake_2048x2048_500x360"] = cake_workload(torch, dev, gen)

    out["batching_64_instances"] = batching_workload(torch, dev, gen)

    # 4096 frames of 2167 x 2070 uint32 through one matrix (2000 q bins): a 256-frame device
    # buffer integrated 16 times
    w = synth.stream_workload()
    g = api.Geometry(*w.geometry.astuple())
    ig = api.Integrator.build(g, (w.ny, w.nx), w.npt_rad, 0, "q_nm^-1", "full", device=dev)
    buf = torch.randint(0, 4000, (256, w.ny, w.nx), generator=gen, device=dev, dtype=torch.int32)
    fr = buf.view(torch.uint32)
    ig.autotune(16)  # setup, untimed
    ig.integrate_batch(fr[:64])
    ms = _event_ms(torch, lambda: ig.integrate_batch(fr), 16)
    # beside it, the plain form: one frame per launch, FP64 (the faster of the tiled form and
    # the look-up table)
    plain = {}
    for form in ("tiled", "lut"):
        call = (lambda k: ig.integrate(fr[k], precision="fp64")) if form == "tiled" else \
            (lambda k: ig.integrate_lut(fr[k], precision="fp64"))
        for k in range(3):
            call(k)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for k in range(32):
            call(k)
        b.record()
        torch.cuda.synchronize()
        plain[form] = a.elapsed_time(b) / 32
    best = min(plain, key=plain.get)
    out["stream_4096x2167x2070"] = {"frames_per_s": 256 / (ms / 1e3), "ms_per_4096": 16 * ms,
                                     "autotuned": (ig.info["tile_h"], ig.info["tile_w"],
                                                   ig.info["frames_per_pass"]),
                                     "plain_fp64_one_frame_per_launch": {
                                         "frames_per_s": 1e3 / plain[best], "form": best,
                                         "ms_per_frame_by_form": plain},
                                     "speedup_vs_plain": (256 / (ms / 1e3)) / (1e3 / plain[best])}
    del buf, fr, ig

    # one Pilatus frame per call through the single-frame path (FP32 compensated)
    img, dark, flat, sa, pol = pilatus_inputs
    for _ in range(3):
        ig_pilatus.integrate(img, dark, flat, sa, pol, precision="fp32")
    ms = _event_ms(torch, lambda: ig_pilatus.integrate(img, dark, flat, sa, pol, precision="fp32"), 20)
    out["pilatus_single_frame_fp32"] = {"ms_per_frame": ms, "frames_per_s": 1e3 / ms}
    # the same frame through the corrections bound once (a batch of one)
    one = img.view(torch.int32).unsqueeze(0).view(torch.uint32)
    for _ in range(3):
        ig_pilatus.integrate_batch_bound(one)
    ms = _event_ms(torch, lambda: ig_pilatus.integrate_batch_bound(one), 20)
    out["pilatus_single_frame_fp32"]["bound_ms_per_frame"] = ms

    # the same frame through the look-up-table layout (Sec. 5.2), FP32 and FP64
    lut = {}
    for prec in ("fp32", "fp64"):
        ig_pilatus.integrate_lut(img, dark, flat, sa, pol, precision=prec)
        lut[prec + "_ms_per_frame"] = _event_ms(
            torch, lambda: ig_pilatus.integrate_lut(img, dark, flat, sa, pol, precision=prec), 10)
    info = ig_pilatus.refresh_info()
    lut["width"] = info["lut_width"]
    lut["slots_per_entry"] = info["lut_width"] * info["nrows"] / info["nnz"]
    lut["tiled_fp32_ms_per_frame"] = out["pilatus_single_frame_fp32"]["ms_per_frame"]
    out["pilatus_single_frame_lut"] = lut
    out["pilatus1m_stages"] = stage_breakdown(torch, dev)
    out["size_sweep_1_to_16_mpix"] = size_sweep(torch, dev, gen)

    # propagated Poisson variance of the bin sums, 64 Pilatus frames per call
    fr64 = img.view(torch.int32).unsqueeze(0).expand(64, -1, -1).contiguous().view(torch.uint32)
    ig_pilatus.variance(fr64)
    ms = _event_ms(torch, lambda: ig_pilatus.variance(fr64), 5)
    out["pilatus_variance_64_frames"] = {"us_per_frame": 1e3 * ms / 64}
    del fr64

    # adjoint (image and flat-field gradients) on the Pilatus matrix, FP32 and FP64
    for prec in ("fp32", "fp64"):
        res = ig_pilatus.integrate(img, dark, flat, sa, pol, precision=prec)
        gI = torch.ones_like(res.I)
        ig_pilatus.backward(gI, res.I, res.sum_norm, sa, pol, prec)
        ms = _event_ms(torch, lambda: ig_pilatus.backward(gI, res.I, res.sum_norm, sa, pol, prec), 10)
        out["backward_pilatus_" + prec] = {"ms_per_call": ms}
    return out


def config_dict(w, frames):
    return {"workload": "%s: %dx%d uint32, module-gap mask, q nm^-1, %d bins, full split, "
                        "dark/flat/solid-angle/polarisation" % (w.name, w.ny, w.nx, w.npt_rad),
            "frames_per_step": frames, "precision": "fp32-compensated (Kahan)",
            "corrections": "bound once per detector (az_set_corrections, setup like the matrix); "
                           "the per-call form is reported in per_call_corrections",
            "l2": "inputs larger than L2 (frame batch streamed from HBM every step)"}


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if args.only_cake:
        gen = torch.Generator(device=dev)
        gen.manual_seed(7)
        print(json.dumps({"cake_2048x2048_500x360": cake_workload(torch, dev, gen, args.steps)}))
        return
    if args.only_stream:
        gen = torch.Generator(device=dev)
        gen.manual_seed(7)
        print(json.dumps({"stream_2167x2070": stream_only(torch, dev, gen, args.steps, args.frames)}))
        return
    if args.only_single:
        print(json.dumps({"pilatus_single_frame_fp32": single_frame_workload(torch, dev, args.steps)}))
        return
    if args.only_batching:
        gen = torch.Generator(device=dev)
        gen.manual_seed(7)
        print(json.dumps({"batching_instances": batching_workload(torch, dev, gen, args.steps,
                                                                  args.instances)}))
        return

    from paper_1412_6367_gb300 import api, synth
    w = synth.pilatus_workload()
    g = api.Geometry(*w.geometry.astuple())
    t_build = time.perf_counter()
    mask = synth.pilatus_module_mask(w.ny, w.nx)
    ig = api.Integrator.build(g, (w.ny, w.nx), w.npt_rad, 0, "q_nm^-1", "full", mask=mask, device=dev)
    torch.cuda.synchronize()
    t_build = time.perf_counter() - t_build
    tuned = None
    if args.autotune:
        tuned = ig.autotune(32)
    info = ig.refresh_info()
    crad, _ = g.positions(w.ny, w.nx, "q_nm^-1", "centres", chi=False, device=dev)
    crad = crad.cpu().numpy()
    dark, flat = synth.dark_flat(w.ny, w.nx, w.seed)
    dark_d = torch.from_numpy(dark).to(dev)
    flat_d = torch.from_numpy(flat).to(dev)
    sa_d = g.solid_angle(w.ny, w.nx, device=dev)
    pol_d = g.polarization(w.ny, w.nx, w.polarization_factor, device=dev)
    B = args.frames
    base = np.stack([synth.ring_image(crad, seed=sd) for sd in frame_seeds(rank)])
    frames_i32 = torch.empty((B, w.ny, w.nx), dtype=torch.int32, device=dev)
    fb = torch.from_numpy(base.view(np.int32)).to(dev)
    for k in range(B):
        frames_i32[k].copy_(fb[k % 8])
    del fb
    frames = frames_i32.view(torch.uint32)  # the counts are uint32; moved as int32 bits
    fb0 = frames_i32[0].clone().view(torch.uint32)
    out = api.Result(torch.empty((B, ig.nrows), device=dev), torch.empty((B, ig.nrows), device=dev),
                     torch.empty(ig.nrows, device=dev), torch.empty(ig.nrows, device=dev))

    # the detector's corrections are bound once (setup, like the matrix): per-entry darks and
    # N, C per bin; every step then integrates its frames against them
    torch.cuda.synchronize()
    t_bind = time.perf_counter()
    ig.set_corrections(dark_d, flat_d, sa_d, pol_d)
    torch.cuda.synchronize()
    t_bind = time.perf_counter() - t_bind

    def step():
        ig.integrate_batch_bound(frames, out=out)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()

    # frame 0's four outputs (FP32 batch) and the FP64 one-frame form, for the parity check of
    # the CPU-baseline leg
    out32 = [out.I[0], out.sum_signal[0], out.sum_norm, out.count]
    out32 = [t.double().cpu().numpy() for t in out32]
    r64 = ig.integrate(frames[0], dark_d, flat_d, sa_d, pol_d, precision="fp64")
    out64 = [t.cpu().numpy() for t in r64]

    # timed region (device-resident inputs)
    clocks = Clocks(local)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    ig.profile_enable(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    ig.profile_enable(False)
    clk = clocks.stop()
    prof = ig.profile_read()
    ms = max_over_ranks(e0.elapsed_time(e1), world)
    ms_per_step = ms / args.steps
    value = whole_job_rate(B, world, args.steps, ms)

    # roofline of the dominant kernel (phase-1 frames): algorithmic bytes / mean duration
    peak, peak_kind = measured_peak()
    n_launch, tot_ms = prof["phase1_frames"]
    launches_per_step = sum(v[0] for v in prof.values()) / args.steps
    per_launch_frames = B * args.steps / max(n_launch, 1)
    ab = phase1_frames_bytes(info["nnz"], info["n_unmasked"], per_launch_frames)
    achieved = ab / (tot_ms / max(n_launch, 1) / 1e3) / 1e9 if n_launch else None
    # DRAM bytes of one launch from the committed capture; a capture of another launch size
    # is scaled by frames (approximate: the matrix part does not grow with the frames)
    cap = ncu_traffic()
    traffic_full = None
    if cap:
        traffic_full = cap[0] * (per_launch_frames / cap[1] if cap[1] != int(per_launch_frames) else 1.0)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": (achieved / peak) if achieved else None,
                "traffic": traffic_full,
                "kernel": "frames_kernel<G=%d,U32,dark> (frames pass, %d frames per launch)" % (
                    info["frames_per_pass"], int(per_launch_frames)),
                "duration_ms_per_launch": tot_ms / max(n_launch, 1),
                "algorithmic_bytes_per_launch": ab, "peak_source": peak_kind + " hbm_gbs",
                "kernel_share_of_step": tot_ms / ms if ms else None}
    step_bytes = algorithmic_bytes(info["nnz"], info["n_unmasked"], ig.nrows, B)

    # the same batches with the corrections passed on every call (per-entry darks, N and C
    # formed again in each call): az_integrate_batch
    def step_per_call():
        ig.integrate_batch(frames, dark_d, flat_d, sa_d, pol_d, out=out)

    step_per_call()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(args.steps):
        step_per_call()
    b.record()
    torch.cuda.synchronize()
    pc_ms = a.elapsed_time(b) / args.steps
    per_call = {"frames_per_s": B / (pc_ms / 1e3), "ms_per_step": pc_ms, "api": "az_integrate_batch",
                "bind_ms": t_bind * 1e3}

    # plain comparator: one frame per launch, FP64 accumulation, everything re-read; the
    # faster of the tiled single-pass form and the look-up table is kept
    plain = None
    if rank == 0:
        forms = {}
        for form in ("tiled", "lut"):
            call = (lambda k: ig.integrate(frames[k % B], dark_d, flat_d, sa_d, pol_d, precision="fp64")) \
                if form == "tiled" else \
                (lambda k: ig.integrate_lut(frames[k % B], dark_d, flat_d, sa_d, pol_d, precision="fp64"))
            for k in range(3):
                call(k)
            torch.cuda.synchronize()
            n_plain = 50
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            for k in range(n_plain):
                call(k)
            b.record()
            torch.cuda.synchronize()
            forms[form] = a.elapsed_time(b) / n_plain
        best = min(forms, key=forms.get)
        pms = forms[best]
        pbytes = plain_fp64_bytes(info["nnz"], info["n_unmasked"], ig.nrows)
        plain = {"value": 1e3 / pms, "unit": UNIT, "ms_per_frame": pms, "precision": "fp64",
                 "form": best, "ms_per_frame_by_form": forms,
                 "roofline": {"achieved": pbytes / (pms / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
                              "frac": pbytes / (pms / 1e3) / 1e9 / peak, "bytes_per_frame": pbytes},
                 "speedup_batched_fp32_vs_plain": value / world / (1e3 / pms)}

    # end to end through the host-buffer API (pinned frames, copies inside the timed region)
    e2e = None
    if rank == 0 or world > 1:
        Be = min(args.e2e_frames, B)
        host = torch.from_numpy(np.stack([base[k % 8] for k in range(Be)]).view(np.int32))
        host = host.pin_memory().view(torch.uint32)
        oI = torch.empty((Be, ig.nrows), dtype=torch.float32).pin_memory()
        oS = torch.empty((Be, ig.nrows), dtype=torch.float32).pin_memory()
        ig.integrate_batch_host(host, dark_d, flat_d, sa_d, pol_d, out_I=oI, out_S=oS)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ksteps = max(2, min(args.steps, 5))
        for _ in range(ksteps):
            ig.integrate_batch_host(host, dark_d, flat_d, sa_d, pol_d, out_I=oI, out_S=oS)
        el = time.perf_counter() - t0
        # the host link alone: one pinned host -> device copy of the same frames (the ceiling
        # of any end-to-end rate that uploads them)
        dbuf = torch.empty(host.numel(), dtype=torch.int32, device=dev)
        hsrc = host.view(torch.int32).reshape(-1)
        dbuf.copy_(hsrc, non_blocking=True)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(3):
            dbuf.copy_(hsrc, non_blocking=True)
        b.record()
        torch.cuda.synchronize()
        link_gbs = 3 * host.numel() * 4 / (a.elapsed_time(b) / 1e3) / 1e9
        del dbuf
        e2e = {"value": Be * ksteps / el * world, "unit": UNIT,
               "h2d_bytes_per_step": int(host.numel() * 4), "d2h_bytes_per_step": int(2 * oI.numel() * 4),
               "frames_per_step": Be, "api": "az_integrate_batch_host",
               "host_link": {"h2d_gbs": link_gbs, "frames_per_s_ceiling": link_gbs * 1e9 / (w.ny * w.nx * 4),
                             "how": "one pinned cudaMemcpyAsync of the step's frames, CUDA events"}}

    others = None
    if rank == 0 and not args.no_other_workloads:
        del frames_i32, frames, out
        torch.cuda.empty_cache()
        others = other_workloads(torch, dev, ig, (fb0, dark_d, flat_d, sa_d, pol_d))

    cpu = parity = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu, parity = cpu_baseline(w, args.cpu_seconds,
                                   check=(base[0], out32, out64, sa_d.cpu().numpy(), pol_d.cpu().numpy()))
        parity["nnz_gpu"] = int(info["nnz"])

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": max(args.warmup, 3), "ms_per_step": ms_per_step, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": config_dict(w, B), "e2e": e2e, "gpu_launches": int(round(launches_per_step * args.steps)),
                "roofline": roofline, "cpu_baseline": cpu, "clocks": clk,
                "gpix_per_s": value * w.ny * w.nx / 1e9,
                "step_algorithmic_gbs": step_bytes / (ms_per_step / 1e3) / 1e9,
                "plain_fp64_one_frame_per_launch": plain, "parity": parity,
                "per_call_corrections": per_call,
                "setup": {"csr_build_s": t_build, "nnz": info["nnz"], "n_unmasked": info["n_unmasked"],
                          "segments": info["n_segments"], "tile": [info["tile_h"], info["tile_w"]],
                          "rows_per_warp": info["rows_per_warp"],
                          "frames_per_pass": info["frames_per_pass"], "autotune_ms_per_frame": tuned},
                "kernel_ms": {k: v for k, v in prof.items()},
                "other_workloads": others}
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
