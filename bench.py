#!/usr/bin/env python3
"""OSEM throughput benchmark of libspect on the 128^3 x 120-angle workload.

One step = one full OSEM reconstruction of the workload (4 iterations x 8
subsets = 32 subiterations, attenuation and depth-dependent PSF on, FP32),
from f0 = 1, with the measured counts y and the attenuation cache already
resident in HBM.  The metric is subset-iterations per second over the whole
job (all ranks).  Each timed step is bracketed by CUDA events on the stream
the library launches on; L2 is flushed (256 MiB write) between steps, outside
the events.

Extra objects on the JSON line:
  e2e          the same metric through the C-ABI with host buffers: the
               copy of y from pinned host memory and the read-back of the
               image are inside the timed region;
  roofline     the dominant kernel's algorithmic bytes per launch over its
               CUDA-event duration (a second, profiled pass of the same
               steps), against the measured HBM copy bandwidth;
  cpu_baseline the FP64 CPU oracle on the whole 4 x 8 reconstruction of the
               workload (32 subiterations from the same y);
  accuracy_vs_fp64  relative L2 errors against that FP64 oracle of the
               reconstructed image and of the projections H f_true, for the
               FP32 form and the BF16-PSF form;
  bf16         the BF16-PSF form (tensor-core PSF GEMMs, FP64 attenuation
               sums) on the same workload and data, device and end to end;
  plan_time    plan creation (wall time) and the device time of the
               attenuation cache and subset sensitivities, per form;
  clocks       nvidia-smi SM clocks and throttle reasons sampled during the
               timed region.

--impl reference times the FP64 CPU oracle (the reference arm of this
benchmark) on the host cores, one OSEM subiteration per step.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "OSEM subset-iters/s at 128^3x120 angles vs plain FP32; serve p50/p99 latency"
UNIT = "subset-iters/s"
L2_FLUSH_BYTES = 256 << 20


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="libspect", choices=["libspect", "reference"])
    ap.add_argument("--workload", default="osem128")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--psf", default="fp32", choices=["fp32", "bf16"],
                    help="bf16: PSF as BF16 tensor-core GEMMs, FP64 attenuation sums")
    ap.add_argument("--serve-requests", type=int, default=256,
                    help="requests of the serving leg (0 skips it)")
    ap.add_argument("--serve-budget-gib", type=float, default=8.0)
    ap.add_argument("--no-map", action="store_true", help="skip the BSREM-RDP leg")
    ap.add_argument("--no-multipeak", action="store_true", help="skip the two-photopeak OSEM leg")
    ap.add_argument("--no-orbit", action="store_true", help="skip the non-circular orbit OSEM leg")
    ap.add_argument("--no-pet", action="store_true", help="skip the listmode PET leg")
    ap.add_argument("--no-autograd", action="store_true", help="skip the batch-of-4 192^3 gradient leg")
    ap.add_argument("--no-bf16", action="store_true", help="skip the BF16-PSF leg")
    ap.add_argument("--pet-only", action="store_true",
                    help="run only the listmode PET leg (one GPU) and print it as one JSON line")
    ap.add_argument("--pet-prompts", type=int, default=None, help="prompts of the PET leg (default 30 M)")
    ap.add_argument("--pet-workload", default="petlm204tof", choices=["petlm204tof", "petlm204"],
                    help="PET workload of --pet-only")
    return ap.parse_args()


def workload_desc(wl) -> dict:
    return {
        "workload": "%s: %dx%dx%d FP32 volume (%.2f cm voxels), %d angles over 360 deg, %dx%d bins, %d it x %d subsets, "
                    "attenuation (0.15/cm water, 0.25/cm bone) + PSF sigma=%.1f+%.2f*d, %.0e counts + %d%% scatter, "
                    "seed %d" % (wl.name, wl.n, wl.n, wl.nz, wl.voxel_cm, wl.n_angles, wl.n, wl.nz, wl.n_iters,
                                 wl.n_subsets, wl.sigma0, wl.slope, wl.counts, int(wl.scatter_frac * 100), wl.seed),
        "step": "one full %d x %d OSEM reconstruction (%d subiterations) from f0 = 1" % (
            wl.n_iters, wl.n_subsets, wl.n_iters * wl.n_subsets),
    }


# ---------------------------------------------------------------- helpers

def reduce_max(v: float, world: int, dist=None, device=None) -> float:
    """Maximum of v over the ranks (the job's time is its slowest rank's)."""
    if world == 1 or dist is None:
        return v
    import torch
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(world: int, steps: int, units_per_step: int, ms_max: float) -> float:
    """Whole-job units per second: every rank runs its own replica of the
    workload (weak scaling), the time is the slowest rank's."""
    return world * steps * units_per_step / (ms_max / 1e3)


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        # wait (at most 3 s) for the first sample so that every row that
        # follows falls inside the load the caller starts next
        t0 = time.time()
        while time.time() - t0 < 3.0 and self.proc.poll() is None:
            if os.path.getsize(self.path) > 0:
                break
            time.sleep(0.01)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def measured_peaks() -> dict:
    """HBM copy bandwidth and BF16 GEMM rate measured on this GPU type, and
    the FP32 FMA peak derived from the unit count and the maximum clock:
    SMs x 128 FP32 lanes x 2 flop x max SM clock."""
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        mhz = float(d.get("sm_max_mhz", 2070.0))
        return {"hbm_gbs": float(d["hbm_gbs"]), "bf16_tflops_sustained": float(d["bf16_tflops_sustained"]),
                "fp32_tflops": sms * 128 * 2 * mhz * 1e6 / 1e12, "source": "measured"}
    return {"hbm_gbs": 6800.0, "bf16_tflops_sustained": 1700.0, "fp32_tflops": sms * 128 * 2 * 2070e6 / 1e12,
            "source": "fallback"}


def psf_radii(wl) -> list:
    """Per-plane PSF radius R_i = ceil(nsigma * (sigma0 + slope * d_i)),
    d_i = n - i - 0.5 (as the plan builds its taps)."""
    return [int(math.ceil(wl.nsigma * (wl.sigma0 + wl.slope * (wl.n - i - 0.5)))) for i in range(wl.n)]


def algorithmic_flops(kernel: str, wl, n_sel: int) -> tuple:
    """(flops, pipe) of one launch.  FP32 per voxel and angle: forward 7
    (bilinear) + 1 (attenuation) + 2 (2R_i+1) (z blur) + 2 (2R_i+1) (y blur
    and depth sum); back blur 4 (2R_i+1) + 1; gather 2 per bilinear weight,
    4 weights per rotated sample, + 2 per voxel for the update.  BF16 path:
    per plane two 128 x n x n GEMMs, each as three BF16 products (hi/lo
    split of the taps and of the data), 2 flop per multiply-add, on the
    tensor pipe."""
    plane = float(wl.n) * wl.nz
    taps = [2 * r + 1 for r in psf_radii(wl)]
    if kernel == "forward":
        return n_sel * plane * sum(8 + 4 * t for t in taps), "fp32"
    if kernel == "blur_back":
        return n_sel * plane * sum(1 + 4 * t for t in taps), "fp32"
    if kernel in ("gather_update", "gather"):
        n3 = plane * wl.n
        return n_sel * n3 * 8 + 2 * n3, "fp32"
    if kernel in ("forward_bf16", "blur_back_bf16"):
        return n_sel * wl.n * 2 * 3 * 2.0 * 128 * wl.n * wl.n, "tensor"
    return 0.0, "fp32"


def algorithmic_bytes(kernel: str, wl, n_sel: int) -> float:
    """Algorithmic bytes of one launch of `kernel` in an OSEM subiteration.

    Per angle (FP32, attenuation cached): the forward reads the volume and
    A_a and writes a projection, (N^3 + N^3 + N^2) * 4; the back projection
    reads A_a and the projection ratio and writes its share of the volume,
    (N^3 + 2 N^2) * 4, split here between the blur (A_a, ratio) and the
    gather (the rotated-frame volume it reads, which replaces the second
    read of A_a); the fused update reads f and sens and writes f, 3 N^3 * 4.
    """
    n3 = float(wl.n) * wl.n * wl.nz
    n2 = float(wl.n) * wl.nz
    if kernel in ("forward", "forward_bf16"):
        return n_sel * (2 * n3 + n2) * 4
    if kernel in ("blur_back", "blur_back_bf16"):
        return n_sel * (n3 + n2) * 4
    if kernel in ("gather_update", "gather"):
        return (n_sel * n3 + 3 * n3) * 4
    return 0.0


def oracle_geom(wl, mu64):
    import oracle
    return oracle.Geom(n=wl.n, nz=wl.nz, n_angles=wl.n_angles, mu=mu64, voxel_cm=float(np.float32(wl.voxel_cm)),
                       sigma0=float(np.float32(wl.sigma0)), slope=float(np.float32(wl.slope)),
                       nsigma=float(np.float32(wl.nsigma)))


def cpu_baseline(wl, y, s, mu64, seconds: float, steps=None, full=False):
    """Time the FP64 oracle's OSEM on the host cores: whole subiterations until
    `seconds` have passed (or exactly `steps` of them; with full=True the
    whole n_iters x n_subsets reconstruction).  Returns the record and the
    oracle's image."""
    import oracle
    og = oracle_geom(wl, mu64)
    f = np.ones((wl.n, wl.n, wl.nz))
    done = 0
    total = wl.n_iters * wl.n_subsets
    t0 = time.perf_counter()
    while True:
        f, _ = oracle.osem(y, s, og, wl.n_subsets, done, 1, f)
        done += 1
        el = time.perf_counter() - t0
        if full:
            if done >= total:
                break
        elif steps is not None:
            if done >= steps:
                break
        elif el >= seconds:
            break
    what = ("the whole %dx%d OSEM (%d subiterations)" % (wl.n_iters, wl.n_subsets, done) if full and done == total
            else "first %d subiteration(s) of the %dx%d OSEM" % (done, wl.n_iters, wl.n_subsets))
    out = {"value": done / el, "unit": UNIT, "cores": oracle.n_threads(), "kind": "oracle",
           "sample": "%s on %s (FP64, %.1f s)" % (what, wl.name, el)}
    if steps is None:
        # the same oracle on one thread: one subiteration
        threads = oracle.n_threads()
        oracle.set_threads(1)
        try:
            t1 = time.perf_counter()
            oracle.osem(y, s, og, wl.n_subsets, 0, 1, np.ones((wl.n, wl.n, wl.nz)))
            out["one_thread_value"] = 1.0 / (time.perf_counter() - t1)
        finally:
            oracle.set_threads(threads)
    return out, f


def rel_l2(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def accuracy_vs_fp64(wl, mu64, f_true, ref_image, images: dict, projections: dict) -> dict:
    """Relative L2 errors of the GPU forms against the FP64 oracle: the
    4 x 8 OSEM image (against the oracle's image from the same y) and the
    projections H f_true of all angles (against the oracle's)."""
    import oracle
    t0 = time.perf_counter()
    ref_proj = oracle.forward(f_true.astype(np.float64), oracle_geom(wl, mu64))
    out = {"reference": "FP64 CPU oracle: the 4x8 OSEM image from the same y, and H f_true over all angles",
           "oracle_projection_s": round(time.perf_counter() - t0, 2)}
    for k, img in images.items():
        out["%s_image_rel_l2" % k] = rel_l2(img, ref_image)
    for k, prj in projections.items():
        out["%s_proj_rel_l2" % k] = rel_l2(prj, ref_proj)
    out["bars"] = {"fp32": "projections 1e-5, image 2e-5", "bf16": "1e-3"}
    return out


def make_inputs_host(wl):
    from paper_2309_01977_gb300 import phantom
    f_raw, mu = phantom.make_phantom(wl.n, wl.nz, wl.seed)
    return f_raw.astype(np.float32), mu.astype(np.float32)


# ---------------------------------------------------------------- reference arm

def run_reference(args):
    from paper_2309_01977_gb300 import phantom
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    wl = phantom.WORKLOADS[args.workload]
    f_raw, mu = make_inputs_host(wl)
    mu64 = mu.astype(np.float64)
    og = oracle.Geom(n=wl.n, nz=wl.nz, n_angles=wl.n_angles, mu=mu64, voxel_cm=float(np.float32(wl.voxel_cm)),
                     sigma0=float(np.float32(wl.sigma0)), slope=float(np.float32(wl.slope)),
                     nsigma=float(np.float32(wl.nsigma)))
    hf = oracle.forward(f_raw.astype(np.float64), og)
    _, y, s, _ = phantom.make_counts(f_raw.astype(np.float64), hf, wl.counts, wl.scatter_frac, wl.seed)
    s = float(np.float32(s))
    f = np.ones((wl.n, wl.n, wl.nz))
    t = 0
    for _ in range(args.warmup):
        f, _ = oracle.osem(y, s, og, wl.n_subsets, t, 1, f)
        t += 1
    t0 = time.perf_counter()
    for _ in range(args.steps):
        f, _ = oracle.osem(y, s, og, wl.n_subsets, t, 1, f)
        t += 1
    el = time.perf_counter() - t0
    value = args.steps / el
    desc = workload_desc(wl)
    desc["step"] = "one OSEM subiteration of the %dx%d reconstruction (FP64 CPU oracle)" % (wl.n_iters, wl.n_subsets)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": desc,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.n_threads(), "kind": "oracle",
                         "sample": "subiterations %d..%d of the %dx%d OSEM on %s" % (
                             args.warmup, args.warmup + args.steps - 1, wl.n_iters, wl.n_subsets, wl.name)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- serving leg

SERVE_CLASSES = [(64, 60), (96, 96), (128, 120)]


def make_serving_requests(spect, dev, count, seed0=1000):
    """Seeded request stream: size class uniform over 64^3/60, 96^3/96 and
    128^3/120 angles, 2-6 iterations x 8 subsets, counts log-uniform in
    [1e6, 1e7], a phantom and mu map per request; y ~ Poisson(H f + s) with H
    from the library (FP32)."""
    import torch

    from paper_2309_01977_gb300 import phantom
    rng = np.random.Generator(np.random.PCG64(seed0))
    reqs = []
    for r in range(count):
        n, na = SERVE_CLASSES[int(rng.integers(0, 3))]
        iters = int(rng.integers(2, 7))
        counts = float(10.0 ** rng.uniform(6.0, 7.0))
        f, mu = phantom.make_phantom(n, n, seed0 + r)
        g = spect.Geometry(n=n, nz=n, n_angles=na, n_subsets=8)
        plan = spect.Plan(g, torch.from_numpy(mu.astype(np.float32)).to(dev))
        hf = plan.forward(torch.from_numpy(f.astype(np.float32)).to(dev)).double().cpu().numpy()
        plan.close()
        _, y, s, _ = phantom.make_counts(f, hf, counts, 0.05, seed0 + r)
        reqs.append({"n": n, "na": na, "iters": iters, "mu": mu.astype(np.float32), "y": y.astype(np.float32),
                     "s": float(np.float32(s))})
    return reqs


def serve_stream(spect, reqs, bf16, budget, rate, seed=7):
    """Submit the requests with exponential inter-arrival times at `rate`
    (requests/s; None: all at once), wait for all; return stats and images."""
    sv = spect.Server(budget, max_slots=8, n_streams=8)
    rng = np.random.Generator(np.random.PCG64(seed))
    gaps = rng.exponential(1.0 / rate, size=len(reqs)) if rate else np.zeros(len(reqs))
    t0 = time.perf_counter()
    t_next = t0
    ids = []
    for q, gap in zip(reqs, gaps):
        t_next += gap
        delay = t_next - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        g = spect.Geometry(n=q["n"], nz=q["n"], n_angles=q["na"], n_subsets=8, psf_bf16=bf16, atten_f64=bf16)
        ids.append(sv.submit(g, q["mu"], q["y"], q["s"], q["iters"]))
    images = [sv.wait(i)[0] for i in ids]
    st = sv.stats()
    sv.close()
    return st, images


def run_serving(spect, dev, args):
    reqs = make_serving_requests(spect, dev, args.serve_requests)
    budget = int(args.serve_budget_gib * (1 << 30))
    out = {"requests": len(reqs), "hbm_budget_gib": args.serve_budget_gib, "max_slots": 8, "streams": 8,
           "classes": "64^3/60, 96^3/96, 128^3/120 angles; 2-6 it x 8 subsets; 1e6-1e7 counts; seeds 1000+i"}
    # saturation throughput of each form (all requests at once)
    cap = {}
    imgs = {}
    for form, bf16 in (("fp32", False), ("bf16", True)):
        st, im = serve_stream(spect, reqs, bf16, budget, None)
        cap[form] = st["recon_per_s"]
        imgs[form] = im
    # latency under Poisson arrivals at 80% of the FP32 saturation throughput,
    # repeated (the forms alternate) so that the spread between runs on the
    # shared host is reported next to the medians
    rate = 0.8 * cap["fp32"]
    out["arrival_rate_per_s"] = rate
    repeats = 3
    runs = {"fp32": [], "bf16": []}
    for _ in range(repeats):
        for form, bf16 in (("fp32", False), ("bf16", True)):
            st, _ = serve_stream(spect, reqs, bf16, budget, rate)
            runs[form].append(st)
    out["latency_repeats"] = repeats
    for form in ("fp32", "bf16"):
        rs = runs[form]
        p50 = [r["p50_ms"] for r in rs]
        p99 = [r["p99_ms"] for r in rs]
        out[form] = {"p50_ms": statistics.median(p50), "p99_ms": statistics.median(p99),
                     "p50_ms_runs": p50, "p99_ms_runs": p99,
                     "recon_per_s": statistics.median([r["recon_per_s"] for r in rs]),
                     "saturation_recon_per_s": cap[form], "peak_active": max(r["peak_active"] for r in rs),
                     "peak_gib": max(r["peak_bytes"] for r in rs) / (1 << 30)}
    diffs = [float(np.linalg.norm(a - b) / np.linalg.norm(b)) for a, b in zip(imgs["bf16"], imgs["fp32"])]
    out["bf16_vs_fp32_image_rel_l2_max"] = max(diffs)
    return out


# ---------------------------------------------------------------- libspect arm

def run_multipeak_leg(spect, torch, dev, wl, g, plan, f_raw, mu, y_dev, s, x, timed, max_over_ranks, world, k):
    """Two photopeaks on the same workload (extended system matrix): the
    second peak sees 1.25 x the attenuation map (a lower energy) through a
    wider collimator response (sigma = 0.7 + 0.04 d) with relative scale 0.6;
    its counts are drawn from the library's own forward projection of the
    same activity.  Timed: one 2-peak 4 x 8 OSEM reconstruction per step."""
    import dataclasses
    g2 = dataclasses.replace(g, psf_sigma0=0.7, psf_slope=0.04)
    mu2 = (1.25 * mu).astype(np.float32)
    plan2 = spect.Plan(g2, torch.from_numpy(mu2).to(dev))
    scale2 = 0.6
    hf1 = plan.forward(torch.from_numpy(f_raw).to(dev)).double().cpu().numpy()
    hf2 = plan2.forward(torch.from_numpy(f_raw).to(dev)).double().cpu().numpy()
    f_scale = wl.counts / float(hf1.sum())
    ybar2 = scale2 * hf2 * f_scale
    s2 = float(np.float32(wl.scatter_frac * ybar2.mean()))
    rng = np.random.Generator(np.random.PCG64(wl.seed + 104729))
    y2 = torch.from_numpy(rng.poisson(ybar2 + s2).astype(np.float32)).to(dev)
    n_sub = wl.n_iters * wl.n_subsets

    def step():
        x.fill_(1.0)
        spect.spect_multi_osem_run([plan, plan2], [1.0, scale2], [y_dev, y2], [s, s2], x, 0, n_sub)
    step()
    torch.cuda.synchronize()
    plan2.check()
    ms = max_over_ranks(timed(step, k))
    plan2.close()
    return {"peaks": "2 (scales 1, 0.6; mu x1, x1.25; sigma 0.5+0.03d, 0.7+0.04d)",
            "subset_iters_per_s": replica_throughput(world, k, n_sub, ms), "ms_per_recon": ms / k}


def run_orbit_leg(spect, torch, dev, wl, g, f_raw, mu, x, timed, max_over_ranks, world, k):
    """Non-circular (elliptical body-contour) orbit on the same workload: the
    detector face at radius r(t) = ab / sqrt((b cos t)^2 + (a sin t)^2) from
    the centre with a = n/2 + 4 and b = n/2 + 20 voxels, so the per-angle
    detector offset r(t) - n/2 runs from 4 to 20 voxels.  Counts from the
    library's forward projection.  Timed: one 4 x 8 OSEM reconstruction."""
    import dataclasses
    a, b = wl.n / 2 + 4.0, wl.n / 2 + 20.0
    t = 2.0 * np.pi * np.arange(wl.n_angles) / wl.n_angles
    r = a * b / np.sqrt((b * np.cos(t)) ** 2 + (a * np.sin(t)) ** 2)
    offs = [float(v) for v in (r - wl.n / 2)]
    go = dataclasses.replace(g, det_offsets=offs)
    po = spect.Plan(go, torch.from_numpy(mu).to(dev))
    hf = po.forward(torch.from_numpy(f_raw).to(dev)).double().cpu().numpy()
    from paper_2309_01977_gb300 import phantom
    _, y, s, _ = phantom.make_counts(f_raw.astype(np.float64), hf, wl.counts, wl.scatter_frac, wl.seed)
    s = float(np.float32(s))
    yd = torch.from_numpy(y.astype(np.float32)).to(dev)
    n_sub = wl.n_iters * wl.n_subsets

    def step():
        x.fill_(1.0)
        spect.spect_osem_run(po.handle, yd, s, x, 0, n_sub)
    step()
    torch.cuda.synchronize()
    po.check()
    ms = max_over_ranks(timed(step, k))
    po.close()
    return {"orbit": "ellipse, detector offsets %.1f to %.1f voxels" % (min(offs), max(offs)),
            "subset_iters_per_s": replica_throughput(world, k, n_sub, ms), "ms_per_recon": ms / k}


def run_pet_leg(torch, dev, timed, max_over_ranks, world, k, cpu_seconds: float, with_cpu: bool, prompts=None,
                workload: str = "petlm204tof"):
    """Listmode PET (Eq. PET_SM, Joseph projector, listmode OSEM) on the
    paper's PET grid: 204 x 204 x 154 voxels of 1.25 mm, a 338 mm scanner of
    64 rings x 448 crystals, 3 mm FWHM resolution model, 30 M prompts (10 %
    randoms) in 3 subsets; petlm204tof adds the paper's time of flight
    (550 ps, 21 bins over 30 cm).  The sensitivity image comes from the
    pairs of every 4th crystal of every 2nd ring, each weighted 64 (plan-time
    input, not timed).  Timed: one listmode OSEM iteration (3 subiterations
    over all 30 M events) per step."""
    from paper_2309_01977_gb300 import pet, pet_phantom as pp
    import dataclasses
    wl = pp.PET_WORKLOADS[workload]
    if prompts:
        wl = dataclasses.replace(wl, prompts=int(prompts))
    act, mu, semi = pp.head_phantom(wl.shape, wl.voxel, wl.seed, device=dev)
    lors, eta, s, n_true, tof_bin = pp.draw_events(wl, act, semi, device=dev)
    torch.cuda.empty_cache()
    g = pet.PetGeometry(wl.shape, wl.voxel, rr_sigma_mm=wl.rr_sigma_mm, n_subsets=wl.n_subsets,
                        n_tof_bins=wl.tof_bins, tof_bin_mm=wl.tof_bin_mm, tof_sigma_mm=wl.tof_sigma_mm)
    plan = pet.PetPlan(g, mu)
    mult = plan.mult(lors, eta)
    L_all, eta_all, w = pp.scanner_lors(wl.scanner, angle_step=4, ring_step=2, device=dev, eff_seed=wl.seed)
    sens = plan.back(plan.mult(L_all, eta_all) * w, L_all)
    del L_all, eta_all
    torch.cuda.empty_cache()
    x = torch.ones(wl.shape, device=dev)
    M = wl.n_subsets
    n_ev = lors.shape[0]

    def step():
        x.fill_(1.0)
        plan.lm_osem(lors, mult, s, sens, x, 0, M, tof_bin=tof_bin)
    step()
    torch.cuda.synchronize()
    ms = max_over_ranks(timed(step, k))
    plan.profile_enable(True)
    plan.profile_read(reset=True)
    timed(step, k)
    prof = plan.profile_read(reset=True)
    plan.profile_enable(False)
    em_name = "joseph_em_tof" if tof_bin is not None else "joseph_em"
    em = prof.get(em_name, (0, float("nan")))
    samples = float(sum(pet_sample_count(lors, wl)))  # Joseph planes per pass over all events
    leg = {"workload": "%s: 204x204x154 (1.25 mm), 64x448-crystal scanner (r 338 mm), %d prompts "
                       "(%d trues, 10%% randoms), 3 subsets, 3 mm FWHM T_rr, attenuation + normalisation%s" % (
                           wl.name, n_ev, n_true,
                           ", TOF %d bins of %.2f mm, sigma %.1f mm (%.0f ps)" % (
                               wl.tof_bins, wl.tof_bin_mm, wl.tof_sigma_mm, wl.tof_fwhm_ps) if wl.tof_bins else ""),
           "step": "one listmode OSEM iteration (3 subiterations over all events) from f0 = 1",
           "events_per_s": replica_throughput(world, k, n_ev, ms), "ms_per_iteration": ms / k,
           "kernel_avg_ms": {kk: round(v[1] / v[0], 3) for kk, v in prof.items()},
           # each launch walks one subset: 1/M of the events (planes of the
           # whole line; with time of flight only the window is visited)
           "em_kernel": em_name,
           "em_planes_per_s": samples * (em[0] / M) / (em[1] * 1e-3) if em[0] else None}
    l2 = os.path.join(ROOT, "profiles", "l2_petlm204.json")
    if os.path.exists(l2):
        with open(l2) as fh:
            prof_l2 = json.load(fh).get(em_name)
        # the walk gathers from and scatters into an image held in L2: its
        # bound is L2 throughput, measured by ncu as a fraction of L2 peak
        # (with time of flight the erf weights also keep the issue slots busy)
        if prof_l2:
            leg["roofline"] = {"bound": "l2", "kernel": em_name, "frac": prof_l2["lts_throughput_frac"],
                               "issue_active_frac": prof_l2["issue_active_frac"], "measured_in_run": False,
                               "source": "stored: ncu of the same kernel at 3 M prompts, read from "
                                         "profiles/l2_petlm204.json (profiles/pet_lm_em_petlm204.md); "
                                         "stale if the kernel has changed since"}
    if with_cpu:
        leg["cpu_baseline"] = pet_cpu_baseline(wl, act, mu, lors, mult, s, sens, cpu_seconds, tof_bin)
    plan.close()
    return leg


def pet_sample_count(lors, wl):
    """Joseph samples of each line (planes of its principal axis inside the
    image), counted on the host from the line ends: the work of one pass."""
    L = lors.double().cpu().numpy()
    v = np.asarray(wl.voxel)
    n = np.asarray(wl.shape)
    d = np.abs(L[:, 3:] - L[:, :3]) / v
    a = np.argmax(d, axis=1)
    org = -0.5 * (n - 1) * v
    s1 = (L[np.arange(len(L)), a] - org[a]) / v[a]
    s2 = (L[np.arange(len(L)), 3 + a] - org[a]) / v[a]
    lo = np.clip(np.ceil(np.minimum(s1, s2)), 0, None)
    hi = np.minimum(np.floor(np.maximum(s1, s2)), n[a] - 1)
    return [float(np.clip(hi - lo + 1, 0, None).sum())]


def pet_cpu_baseline(wl, act, mu, lors, mult, s, sens, seconds, tof_bin=None):
    """The FP64 oracle's listmode OSEM on the host cores for a bounded sample:
    one subiteration over the first events of subset 0, as many as fit in
    about `seconds` (measured on a small probe first), scaled to events/s."""
    from oracle import pet as opet
    og = opet.PetGeom(wl.shape, wl.voxel, rr_sigma_mm=float(np.float32(wl.rr_sigma_mm)), rr_nsigma=3.0)
    M = wl.n_subsets

    def tof(n):
        if tof_bin is None:
            return None
        return opet.Tof(n_bins=wl.tof_bins, bin_mm=float(np.float32(wl.tof_bin_mm)),
                        sigma_mm=float(np.float32(wl.tof_sigma_mm)), bins=tof_bin[:n].cpu().numpy())
    L = lors[:M * 20000].cpu().numpy()
    m = mult[:M * 20000].cpu().numpy()
    sv = s[:M * 20000].cpu().numpy()
    sn = sens.cpu().numpy()
    t0 = time.perf_counter()
    opet.lm_osem(L, m, sv, sn, og, M, count=1, tof=tof(M * 20000))
    el = time.perf_counter() - t0
    n = int(min(lors.shape[0], M * 20000 * max(1.0, seconds / max(el, 1e-3))))
    L = lors[:n].cpu().numpy()
    t0 = time.perf_counter()
    opet.lm_osem(L, mult[:n].cpu().numpy(), s[:n].cpu().numpy(), sn, og, M, count=1, tof=tof(n))
    el = time.perf_counter() - t0
    import oracle
    return {"value": (n // M) / el, "unit": "events/s", "cores": oracle.n_threads(), "kind": "oracle",
            "sample": "one listmode subiteration over %d events of %s (FP64, %.1f s)" % (n // M, wl.name, el)}


def run_autograd_leg(spect, torch, dev, timed, max_over_ranks, world, k):
    """The differentiable projector on the grad192 workload (batch of 4
    volumes of 192^3, 128 angles, 192 x 192 bins): one step is the Poisson
    log-likelihood of the batch and its gradient through torch.autograd
    (H x of all angles, L and dL/dp, H^T of all angles)."""
    from paper_2309_01977_gb300 import autograd, phantom
    wl = phantom.WORKLOADS["grad192"]
    f_raw, mu = phantom.make_phantom(wl.n, wl.nz, wl.seed)
    g = spect.Geometry(n=wl.n, nz=wl.nz, n_angles=wl.n_angles, n_subsets=1, voxel_cm=wl.voxel_cm,
                       psf_sigma0=wl.sigma0, psf_slope=wl.slope, psf_nsigma=wl.nsigma)
    plan = spect.Plan(g, torch.from_numpy(mu.astype(np.float32)).to(dev))
    batch = 4
    rng = np.random.Generator(np.random.PCG64(wl.seed))
    f0 = torch.from_numpy(f_raw.astype(np.float32)).to(dev)
    scales = torch.from_numpy(rng.uniform(0.5, 1.5, size=(batch, 1, 1, 1)).astype(np.float32)).to(dev)
    x = (f0[None] * scales).contiguous().requires_grad_(True)
    with torch.no_grad():
        p = autograd.SpectProjector.apply(x, plan, -1)
        counts = torch.poisson(p + 1.0).contiguous()
    s = 1.0

    def step():
        x.grad = None
        autograd.poisson_loss(x, counts, s, plan).backward()
    step()
    torch.cuda.synchronize()
    ms = max_over_ranks(timed(step, k))
    spect.spect_profile_enable(plan.handle, True)
    spect.spect_profile_read(plan.handle, reset=True)
    timed(step, k)
    prof = spect.spect_profile_read(plan.handle, reset=True)
    spect.spect_profile_enable(plan.handle, False)
    plan.close()
    return {"workload": "grad192: batch 4 x 192^3 (0.48 cm), 128 angles, 192 x 192 bins, attenuation + PSF",
            "step": "Poisson log-likelihood of the batch and its gradient through torch.autograd",
            "gradients_per_s": replica_throughput(world, k, batch, ms), "ms_per_step": ms / k,
            "kernel_avg_us": {kk: round(1e3 * v[1] / v[0], 1) for kk, v in prof.items()}}


def plan_time(spect, torch, dev, g, mu_dev) -> dict:
    """Plan-time costs (outside every timed step): a fresh plan's creation
    (wall time: tables, gather tables, the attenuation cache A_a of every
    angle, the subset sensitivities H_m^T 1, and the synchronisation), and
    the device time of rebuilding A_a and H_m^T 1 from a mu map
    (spect_plan_set_mu, CUDA events per kernel)."""
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    p = spect.Plan(g, mu_dev)
    create_ms = (time.perf_counter() - t0) * 1e3
    spect.spect_profile_enable(p.handle, True)
    spect.spect_profile_read(p.handle, reset=True)
    spect.spect_plan_set_mu(p.handle, mu_dev)
    prof = spect.spect_profile_read(p.handle, reset=True)
    p.close()
    att = sum(v[1] for k, v in prof.items() if k == "attenuation")
    sens = sum(v[1] for k, v in prof.items() if k != "attenuation")
    return {"create_ms": round(create_ms, 2), "attenuation_cache_ms": round(att, 3),
            "sensitivities_ms": round(sens, 3), "sensitivity_kernels": sorted(k for k in prof if k != "attenuation")}


def run_bf16_leg(spect, torch, dev, wl, mu_dev, f_dev, y_dev, y_host, s, timed, max_over_ranks, world, k):
    """The BF16-PSF form on the same workload and data: the PSF of every
    depth plane as banded-Toeplitz BF16 tensor-core GEMMs (FP32 accumulate),
    the attenuation prefix sums in FP64; the rest as in the FP32 form.  One
    step = one full 4 x 8 OSEM reconstruction from f0 = 1."""
    n_sub = wl.n_iters * wl.n_subsets
    g = spect.Geometry(n=wl.n, nz=wl.nz, n_angles=wl.n_angles, n_subsets=wl.n_subsets, voxel_cm=wl.voxel_cm,
                       psf_sigma0=wl.sigma0, psf_slope=wl.slope, psf_nsigma=wl.nsigma, psf_bf16=True,
                       atten_f64=True)
    pt = plan_time(spect, torch, dev, g, mu_dev)
    plan = spect.Plan(g, mu_dev)
    x = torch.empty((wl.n, wl.n, wl.nz), device=dev)
    x_host = torch.empty((wl.n, wl.n, wl.nz), dtype=torch.float32).pin_memory()

    def step():
        x.fill_(1.0)
        spect.spect_osem_run(plan.handle, y_dev, s, x, 0, n_sub)

    def step_e2e():
        y_dev.copy_(y_host, non_blocking=True)
        x.fill_(1.0)
        spect.spect_osem_run(plan.handle, y_dev, s, x, 0, n_sub)
        x_host.copy_(x, non_blocking=True)
    for _ in range(3):
        step()
    torch.cuda.synchronize()
    ms = max_over_ranks(timed(step, k))
    for _ in range(2):
        step_e2e()
    ms_e2e = max_over_ranks(timed(step_e2e, k))
    spect.spect_profile_enable(plan.handle, True)
    spect.spect_profile_read(plan.handle, reset=True)
    timed(step, k)
    prof = spect.spect_profile_read(plan.handle, reset=True)
    spect.spect_profile_enable(plan.handle, False)
    image = x.cpu().numpy()
    proj = plan.forward(f_dev).cpu().numpy()
    plan.check()
    plan.close()
    n_sel = -(-wl.n_angles // wl.n_subsets)
    peaks = measured_peaks()
    fwd = prof.get("forward_bf16")
    roof = None
    if fwd:
        avg_s = fwd[1] / fwd[0] / 1e3
        flops, _ = algorithmic_flops("forward_bf16", wl, n_sel)
        nbytes = algorithmic_bytes("forward_bf16", wl, n_sel)
        roof = {"kernel": "forward_bf16", "avg_launch_us": avg_s * 1e6,
                "tensor_frac": flops / avg_s / 1e12 / peaks["bf16_tflops_sustained"],
                "hbm_frac": nbytes / avg_s / 1e9 / peaks["hbm_gbs"],
                "tensor_flops_per_launch": flops, "algorithmic_bytes_per_launch": nbytes,
                "peaks": "BF16 sustained %.0f TF/s, HBM %.0f GB/s (%s)" % (
                    peaks["bf16_tflops_sustained"], peaks["hbm_gbs"], peaks["source"])}
    leg = {"form": "BF16 banded-Toeplitz PSF on tcgen05 (FP32 accumulate), FP64 attenuation sums",
           "subset_iters_per_s": replica_throughput(world, k, n_sub, ms), "ms_per_recon": ms / k,
           "e2e_subset_iters_per_s": replica_throughput(world, k, n_sub, ms_e2e),
           "kernel_avg_us": {kk: round(1e3 * v[1] / v[0], 2) for kk, v in prof.items()},
           "roofline": roof, "plan_time": pt}
    return leg, image, proj


def run_libspect(args):
    import torch
    import torch.distributed as dist

    from paper_2309_01977_gb300 import phantom, spect

    world, rank, local = dist_env()
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", torch.cuda.current_device())
    spect.load()  # fails loudly without the CUDA library

    wl = phantom.WORKLOADS[args.workload]
    f_raw, mu = make_inputs_host(wl)
    n_sub = wl.n_iters * wl.n_subsets
    bf16 = args.psf == "bf16"
    g = spect.Geometry(n=wl.n, nz=wl.nz, n_angles=wl.n_angles, n_subsets=wl.n_subsets, voxel_cm=wl.voxel_cm,
                       psf_sigma0=wl.sigma0, psf_slope=wl.slope, psf_nsigma=wl.nsigma,
                       psf_bf16=bf16, atten_f64=bf16)
    plan = spect.Plan(g, torch.from_numpy(mu).to(dev))
    # measured data: y ~ Poisson(H f_true + s), H from the library itself
    hf = plan.forward(torch.from_numpy(f_raw).to(dev)).double().cpu().numpy()
    _, y, s, _ = phantom.make_counts(f_raw.astype(np.float64), hf, wl.counts, wl.scatter_frac, wl.seed)
    s = float(np.float32(s))
    y_host = torch.from_numpy(y.astype(np.float32)).pin_memory()
    y_dev = y_host.to(dev)
    x = torch.empty((wl.n, wl.n, wl.nz), device=dev)
    x_host = torch.empty((wl.n, wl.n, wl.nz), dtype=torch.float32).pin_memory()
    flush = torch.empty(L2_FLUSH_BYTES // 4, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        x.fill_(1.0)
        spect.spect_osem_run(plan.handle, y_dev, s, x, 0, n_sub)

    def step_e2e():
        y_dev.copy_(y_host, non_blocking=True)
        x.fill_(1.0)
        spect.spect_osem_run(plan.handle, y_dev, s, x, 0, n_sub)
        x_host.copy_(x, non_blocking=True)

    def barrier():
        if world > 1:
            dist.barrier()

    def timed(fn, k):
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k)]
        barrier()
        torch.cuda.synchronize()
        for e0, e1 in evs:
            flush.zero_()
            e0.record(stream)
            fn()
            e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        return sum(e0.elapsed_time(e1) for e0, e1 in evs)

    def max_over_ranks(v: float) -> float:
        return reduce_max(v, world, dist, dev)

    clocks = ClockSampler(dev.index if world == 1 else local)
    clocks.start()
    for _ in range(max(args.warmup, 0)):
        step()
    torch.cuda.synchronize()

    launches0 = spect.spect_kernel_launches()
    ms = timed(step, args.steps)
    launches = spect.spect_kernel_launches() - launches0
    ms = max_over_ranks(ms)
    value = replica_throughput(world, args.steps, n_sub, ms)

    # end to end through the C ABI with host buffers
    for _ in range(2):
        step_e2e()
    ms_e2e = max_over_ranks(timed(step_e2e, args.steps))
    e2e = {"value": replica_throughput(world, args.steps, n_sub, ms_e2e), "unit": UNIT,
           "h2d_bytes_per_step": int(y_host.numel() * 4), "d2h_bytes_per_step": int(x_host.numel() * 4)}

    # profiled pass: per-kernel CUDA-event durations on the launch stream
    spect.spect_profile_enable(plan.handle, True)
    spect.spect_profile_read(plan.handle, reset=True)
    timed(step, args.steps)
    prof = spect.spect_profile_read(plan.handle, reset=True)
    spect.spect_profile_enable(plan.handle, False)
    clk = clocks.stop()  # samples span the timed, end-to-end and profiled passes
    top = max(prof.items(), key=lambda kv: kv[1][1])
    name, (n_launch, tot_ms) = top
    avg_s = tot_ms / n_launch / 1e3
    n_sel = -(-wl.n_angles // wl.n_subsets)
    nbytes = algorithmic_bytes(name, wl, n_sel)
    flops, pipe = algorithmic_flops(name, wl, n_sel)
    peaks = measured_peaks()
    traffic = None
    tpath = os.path.join(ROOT, "profiles", "traffic_%s%s.json" % (wl.name, "_bf16" if bf16 else ""))
    if os.path.exists(tpath):
        with open(tpath) as fh:
            traffic = json.load(fh).get(name)
    # the kernel's bound: the larger of its algorithmic HBM time and its
    # arithmetic time at the measured / derived peaks
    t_hbm = nbytes / (peaks["hbm_gbs"] * 1e9)
    fpeak = peaks["bf16_tflops_sustained"] if pipe == "tensor" else peaks["fp32_tflops"]
    t_alu = flops / (fpeak * 1e12)
    if t_hbm >= t_alu:
        roofline = {"bound": "hbm", "achieved": nbytes / avg_s / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s"}
    else:
        roofline = {"bound": "tensor" if pipe == "tensor" else "alu", "achieved": flops / avg_s / 1e12,
                    "peak": fpeak, "unit": "TFLOP/s"}
    roofline["frac"] = roofline["achieved"] / roofline["peak"]
    image_main = x.cpu().numpy()  # the last profiled step's 4 x 8 reconstruction
    f_dev = torch.from_numpy(f_raw).to(dev)
    proj_main = hf.astype(np.float32)
    plan_times = {"bf16" if bf16 else "fp32": plan_time(spect, torch, dev, g, torch.from_numpy(mu).to(dev))}
    roofline.update({
        "traffic": traffic, "kernel": name, "peak_source": peaks["source"] + (
            " (FP32: SMs x 128 lanes x 2 flop x max clock)" if roofline["bound"] == "alu" else
            " (BF16 sustained)" if roofline["bound"] == "tensor" else ""),
        "avg_launch_us": avg_s * 1e6, "algorithmic_bytes_per_launch": nbytes, "algorithmic_flops_per_launch": flops,
        "hbm_frac": nbytes / avg_s / 1e9 / peaks["hbm_gbs"], "alu_frac": flops / avg_s / 1e12 / fpeak,
        "t_bound_frac": max(t_hbm, t_alu) / avg_s,
        "kernel_share": {k: round(v[1] / sum(t[1] for t in prof.values()), 4) for k, v in prof.items()},
        "kernel_avg_us": {k: round(1e3 * v[1] / v[0], 2) for k, v in prof.items()},
        "plane_tiling": {k: plan.info()[k] for k in ("ztile", "n_ztiles", "threads", "smem_bytes")}})

    # MAP leg: BSREM with the relative difference prior (beta 0.3, gamma 2,
    # the paper's hyperparameters) on the same workload and data, 4 x 8
    legs = {}
    if not args.no_map:
        def step_map():
            x.fill_(1.0)
            plan.map(y_dev, s, x, 0, n_sub, "bsrem", "rdp", beta=0.3, gamma=2.0, alpha0=1.0)
        step_map()
        torch.cuda.synchronize()
        ms_map = max_over_ranks(timed(step_map, max(2, args.steps // 2)))
        k_map = max(2, args.steps // 2)
        legs["map"] = {"algorithm": "BSREM, relative difference prior (beta 0.3, gamma 2)",
                       "subset_iters_per_s": replica_throughput(world, k_map, n_sub, ms_map),
                       "ms_per_recon": ms_map / k_map}
    if not args.no_multipeak:
        legs["multipeak"] = run_multipeak_leg(spect, torch, dev, wl, g, plan, f_raw, mu, y_dev, s, x, timed,
                                              max_over_ranks, world, max(2, args.steps // 2))
    if not args.no_autograd:
        legs["autograd"] = run_autograd_leg(spect, torch, dev, timed, max_over_ranks, world, max(2, args.steps // 8))
        torch.cuda.empty_cache()
    if not args.no_orbit:
        legs["orbit"] = run_orbit_leg(spect, torch, dev, wl, g, f_raw, mu, x, timed, max_over_ranks, world,
                                      max(2, args.steps // 2))
    images = {"bf16" if bf16 else "fp32": image_main}
    projections = {"bf16" if bf16 else "fp32": proj_main}
    if not bf16 and not args.no_bf16:
        leg_b, img_b, proj_b = run_bf16_leg(spect, torch, dev, wl, torch.from_numpy(mu).to(dev), f_dev, y_dev,
                                            y_host, s, timed, max_over_ranks, world, args.steps)
        plan_times["bf16"] = leg_b.pop("plan_time")
        legs["bf16"] = leg_b
        images["bf16"], projections["bf16"] = img_b, proj_b

    serving = None
    if args.serve_requests > 0 and world == 1:
        serving = run_serving(spect, dev, args)

    cpu = None
    accuracy = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the oracle's whole 4 x 8 reconstruction from the same y: timed as the
        # CPU baseline, and the FP64 reference of the accuracy figures
        cpu, ref_image = cpu_baseline(wl, y, s, mu.astype(np.float64), args.cpu_seconds, full=True)
        accuracy = accuracy_vs_fp64(wl, mu.astype(np.float64), f_raw, ref_image, images, projections)

    # listmode PET last: its event lists are the largest allocations of the run
    if not args.no_pet:
        with_cpu = rank == 0 and world == 1 and not args.no_cpu_baseline
        legs["pet"] = run_pet_leg(torch, dev, timed, max_over_ranks, world, max(2, args.steps // 8),
                                  args.cpu_seconds / 2, with_cpu, workload="petlm204tof")
        torch.cuda.empty_cache()
        legs["pet_nontof"] = run_pet_leg(torch, dev, timed, max_over_ranks, world, max(2, args.steps // 8),
                                         args.cpu_seconds / 2, False, workload="petlm204")
        torch.cuda.empty_cache()

    if rank == 0:
        cfg = workload_desc(wl)
        cfg.update({"l2": "flushed between steps (256 MiB write), attenuation cache %.2f GB streamed"
                          % (plan.info()["atten_cache_bytes"] / 1e9),
                    "parallelism": "replicas" if world > 1 else "single GPU"})
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16 PSF, f32" if bf16 else "f32", "data": "synthetic",
            "config": cfg,
            "e2e": e2e, "roofline": roofline, "cpu_baseline": cpu, "gpu_launches": int(launches),
            "clocks": clk, "accuracy_vs_fp64": accuracy, "plan_time": plan_times, **legs, "serving": serving,
        }
        print(json.dumps(line), flush=True)
    plan.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_pet_only(args):
    """The listmode PET leg alone, on one GPU, timed like the main legs."""
    import torch

    from paper_2309_01977_gb300 import spect
    spect.load()
    dev = torch.device("cuda", torch.cuda.current_device())
    flush = torch.empty(L2_FLUSH_BYTES // 4, device=dev)
    stream = torch.cuda.current_stream()

    def timed(fn, k):
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k)]
        torch.cuda.synchronize()
        for e0, e1 in evs:
            flush.zero_()
            e0.record(stream)
            fn()
            e1.record(stream)
        torch.cuda.synchronize()
        return sum(e0.elapsed_time(e1) for e0, e1 in evs)

    leg = run_pet_leg(torch, dev, timed, lambda v: v, 1, max(2, args.steps // 8), args.cpu_seconds / 2,
                      not args.no_cpu_baseline, prompts=args.pet_prompts, workload=args.pet_workload)
    print(json.dumps({"pet": leg}), flush=True)
    return 0


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.pet_only:
        return run_pet_only(args)
    return run_libspect(args)


if __name__ == "__main__":
    sys.exit(main())
