"""Benchmark of the fastCAT CBCT hot path on GB300.

One step = the whole path over one synthetic scan: polyenergetic projection
with the fused energy integral, detector blur + scatter, Poisson noise, FDK
filter, FDK backprojection and HU (fc_project + fc_reconstruct).  The
workload is the Catphan-like kV case (256 x 256 x 10 voxels of 0.0625 cm,
360 projections on a 512 x 384 detector of 0.4 mm, 30 energy bins).

Metric: rays*bins/s = n_angles * n_v * n_u * n_E / step time (whole job,
summed over ranks); FDK voxel updates/s are reported beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank simulates its own scan (weak scaling, no
data-path collective); rank 0 prints one JSON line.  ``--impl reference``
times the FP64 CPU oracle as the reference arm.
"""
from __future__ import annotations

import argparse
import dataclasses
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2011_04736_gb300 import workloads as W  # noqa: E402

METRIC = "poly-projection rays·bins/s & FDK voxel-upd/s; surrogate vs plain @≤1e-3 err"
UNIT = "rays*bins/s"
WORKLOAD = "catphan_kv"
L2_FLUSH_BYTES = 256 << 20


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def _workload_desc(wl):
    g = wl.geom
    return {"workload": "%s: %dx%dx%d voxels of %.4g cm, %d projections, %dx%d detector of %.3g cm, "
                        "%d energy bins, SAD %g / SDD %g cm, noise seed %d"
                        % (wl.name, g.nx, g.ny, g.nz, g.dx, g.n_angles, g.n_u, g.n_v, g.du, wl.n_e,
                           g.sad, g.sdd, wl.seed),
            "rays_per_step": g.n_rays, "energy_bins": wl.n_e, "voxels": g.n_voxels,
            "n_angles": g.n_angles}


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons (200 ms period)."""

    FIELDS = ("pci.bus_id,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, bus_id=None):
        self.bus_id = (bus_id or "").lower()
        self.samples = []
        self.proc = None
        self.marks = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.th = threading.Thread(target=self._read, daemon=True)
        self.th.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            if self.bus_id and not parts[0].lower().endswith(self.bus_id[-12:]):
                continue
            self.samples.append((time.time(), parts))

    def mark(self):
        self.marks.append(time.time())

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self, t0, t1):
        sel = [p for (t, p) in self.samples if t0 <= t <= t1] or [p for (_, p) in self.samples]
        if not sel:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(p[1]) for p in sel if num(p[1]) is not None]
        mx = [num(p[2]) for p in sel if num(p[2]) is not None]
        reasons = set()
        for p in sel:
            for name, v in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                                "sw_power_cap"), p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sel)}


# ------------------------------------------------------------------ roofline
def _kernel_models(wl):
    """Algorithmic bytes and FLOPs per launch of each kernel for one step."""
    g = wl.geom
    px = g.n_angles * g.n_v * g.n_u
    rp = int(math.ceil(4 * wl.psf_sigma_px)) if wl.psf_sigma_px > 0 else 0
    rs = int(math.ceil(4 * wl.scatter_sigma_px)) if wl.scatter_sigma_px > 0 else 0
    taps = (2 * rp + 1) + (2 * rs + 1)
    zmax = (g.nz - 1) / 2 * g.dz
    rmax = math.hypot(g.nx * g.dx / 2, g.ny * g.dy / 2)
    vmax = zmax * g.sdd / (g.sad - rmax) / g.dv
    lo = max(0, int(math.floor((g.n_v - 1) / 2 - vmax)) - 2)
    hi = min(g.n_v - 1, int(math.ceil((g.n_v - 1) / 2 + vmax)) + 2)
    rows = hi - lo + 1
    fpx = g.n_angles * rows * g.n_u
    odd = g.n_u if (g.n_u - 1) % 2 == 1 else g.n_u - 1
    return {
        # labels once + T written once
        "project": {"bytes": g.n_voxels + 4 * px, "flops": None, "bound": "hbm"},
        # T read, two intermediates written (2 flops per tap per output of
        # direct convolution; on the tensor cores the MMA work is small next
        # to the traffic, so HBM is the roofline)
        "blur_rows": {"bytes": 12 * px, "flops": 2 * taps * px, "bound": "hbm"},
        # two intermediates read, counts written
        "blur_cols": {"bytes": 12 * px, "flops": 2 * taps * px, "bound": "hbm"},
        # reachable rows: counts read, filtered written; odd taps + centre
        "fdk_filter": {"bytes": 8 * fpx, "flops": 2 * (odd + 1) * fpx, "bound": "alu"},
        # filtered reachable rows read once, FP64 volume written once
        "backproject": {"bytes": 4 * fpx + 8 * g.n_voxels, "flops": None, "bound": "hbm"},
        "hu": {"bytes": 8 * 2 * g.n_voxels + 4 * g.n_voxels, "flops": None, "bound": "hbm"},
        # rates read, counts written
        "noise": {"bytes": 8 * px, "flops": None, "bound": "hbm"},
    }


def _traffic(kernel):
    """ncu DRAM bytes per launch from profiles/ncu_traffic.json, or None when
    absent or taken from a different source revision of the kernel."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    ent = d.get("kernels", {}).get(kernel)
    if not ent:
        return None
    src = os.path.join(ROOT, "paper_2011_04736_gb300", "csrc", ent.get("source", ""))
    if not os.path.exists(src):
        return None
    if hashlib.sha256(open(src, "rb").read()).hexdigest()[:16] != ent.get("source_sha"):
        return None
    return ent.get("dram_bytes_per_launch")


# ------------------------------------------------------------------ oracle arm
def _oracle_sample(wl, n_angles):
    """Oracle pipeline on the first n_angles projections of the workload:
    projection + energy sum, blur + scatter, Poisson noise and FDK over those
    projections.  Returns seconds."""
    import oracle
    oracle.build()
    g = dataclasses.replace(wl.geom, n_angles=n_angles,
                              arc=wl.geom.arc * n_angles / wl.geom.n_angles)
    lab = wl.make_phantom()
    w, d = wl.spectrum()
    mu = wl.mu()
    t0 = time.perf_counter()
    T = oracle.project_T(g, lab, w, d, mu)
    I = oracle.intensity(T, wl.psf_sigma_px, wl.scatter_sigma_px, wl.spr, wl.n0)
    K = oracle.poisson(I.astype(np.float32), wl.seed)
    oracle.fdk(g, K.astype(np.float64), oracle.i_flood(wl.n0, wl.spr))
    return time.perf_counter() - t0


def cpu_baseline(wl, n_angles):
    import oracle
    t = _oracle_sample(wl, n_angles)
    g = wl.geom
    units = n_angles * g.n_v * g.n_u * wl.n_e
    return {"value": units / t, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
            "sample": "%d of %d projections through the FP64 oracle (projection + energy sum, "
                      "blur + scatter, binary32 Poisson, FDK over those projections), %.2f s"
                      % (n_angles, g.n_angles, t)}


# ------------------------------------------------------------------ distributed
def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return 0, 1, None
    import torch
    import torch.distributed as dist
    backend = "nccl" if torch.cuda.is_available() else "gloo"
    dist.init_process_group(backend=backend)
    return dist.get_rank(), dist.get_world_size(), dist


def aggregate(dist, value, op="max"):
    """Max (or sum) of a host float over ranks; identity without a group."""
    if dist is None:
        return value
    import torch
    dev = "cuda" if torch.cuda.is_available() and dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def _barrier(dist):
    if dist is not None:
        dist.barrier()


# ------------------------------------------------------------------ main arms
def run_reference(args):
    rank, world, dist = _dist()
    if rank != 0:
        return 0
    wl = W.WORKLOADS[args.workload]
    g = wl.geom
    units = args.ref_angles * g.n_v * g.n_u * wl.n_e
    for _ in range(args.warmup):
        _oracle_sample(wl, max(1, args.ref_angles // 4))
    times = [_oracle_sample(wl, args.ref_angles) for _ in range(args.steps)]
    import oracle
    t = sum(times) / len(times)
    val = units / t
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": _workload_desc(wl),
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
                             "sample": "%d of %d projections per step through the FP64 oracle"
                                       % (args.ref_angles, g.n_angles)},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def _extra_adjoint(fc, torch):
    """Forward + adjoint of the CNR objective on the adjoint design case
    (128 x 128 x 32 voxels, 180 projections of 512 x 384, 30 bins)."""
    wl = W.WORKLOADS["adjoint_kv"]
    inp = W.adjoint_inputs(wl)
    sc = fc.Scanner(wl, labels=inp["labels"], noise=False)
    try:
        rho = torch.from_numpy(inp["rho"]).cuda()
        z = torch.from_numpy(inp["z"]).cuda()
        args = (sc.h, inp["logits"], inp["D"], inp["rho0"], rho, z, inp["rois"])
        fc.fc_cnr_grad(*args)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        reps = 3
        for _ in range(reps):
            J, gl, gd, gr = fc.fc_cnr_grad(*args)
        torch.cuda.synchronize()
        ms = (time.perf_counter() - t0) / reps * 1e3
        fc.fc_cnr_grad(*args, grads=False)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            fc.fc_cnr_grad(*args, grads=False)
        torch.cuda.synchronize()
        ms_fwd = (time.perf_counter() - t0) / reps * 1e3
        g = wl.geom
        return {"workload": "adjoint_kv: %dx%dx%d voxels, %d projections of %dx%d, %d bins"
                            % (g.nx, g.ny, g.nz, g.n_angles, g.n_u, g.n_v, wl.n_e),
                "J": J, "ms_forward": ms_fwd, "ms_forward_and_gradient": ms,
                "grad_norms": {"logits": float(np.linalg.norm(gl)), "D": float(np.linalg.norm(gd)),
                               "rho": float(torch.linalg.vector_norm(gr))}}
    finally:
        sc.close()


def _extra_paper_scale(fc, torch):
    """One simulate + reconstruct step of the paper-scale MV case (1024^2 x 10
    voxels, 720 projections of 1024 x 768, 60 bins) -- context for the
    paper's whole-pipeline wall times (different GPU, 18 energies, 180
    projections)."""
    wl = W.WORKLOADS["paper_mv"]
    g = wl.geom
    sc = fc.Scanner(wl, noise=False)
    try:
        vol = torch.empty((g.nz, g.ny, g.nx), dtype=torch.float64, device="cuda")
        fc.fc_project(sc.h, 0, g.n_angles, fc.FC_OUT_NONE, None)
        fc.fc_reconstruct(sc.h, None, vol_mu=vol)
        torch.cuda.synchronize()
        fc.fc_profile_enable(sc.h, True)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        fc.fc_project(sc.h, 0, g.n_angles, fc.FC_OUT_NONE, None)
        fc.fc_reconstruct(sc.h, None, vol_mu=vol)
        b.record()
        torch.cuda.synchronize()
        kern = fc.fc_profile_read(sc.h)
        ms = a.elapsed_time(b)
        return {"workload": "paper_mv: %dx%dx%d voxels, %d projections of %dx%d, %d MV bins"
                            % (g.nx, g.ny, g.nz, g.n_angles, g.n_u, g.n_v, wl.n_e),
                "ms_per_step": ms, "rays_bins_per_s": g.n_rays * wl.n_e / (ms / 1e3),
                "fdk_voxel_updates_per_s": g.n_voxels * g.n_angles / (ms / 1e3),
                "kernels_ms": {k: v[0] for k, v in kern.items() if v[1]},
                "paper_context_s": 61.0}
    finally:
        sc.close()


def _extra_dose(fc, torch):
    """Dose estimate per particle (D0(E), Dp) on the Catphan kV case: one
    projection, and every projection of the scan; plus the flood height that
    a 7 mGy scan of 360 projections implies."""
    wl = W.WORKLOADS["catphan_kv"]
    g = wl.geom
    sc = fc.Scanner(wl, noise=False)
    try:
        out = {"workload": "catphan_kv: %dx%dx%d voxels, projections of %dx%d, %d bins"
                           % (g.nx, g.ny, g.nz, g.n_u, g.n_v, wl.n_e)}
        e, m, r = wl.energies(), wl.muen_water(), wl.densities()
        for name, na in (("one_projection", 1), ("all_projections", g.n_angles)):
            fc.fc_dose_estimate(sc.h, 0, na, e, m, r)
            fc.fc_profile_enable(sc.h, True)
            reps = 5
            for _ in range(reps):
                d0, dp = fc.fc_dose_estimate(sc.h, 0, na, e, m, r)
            kern = fc.fc_profile_read(sc.h)
            fc.fc_profile_enable(sc.h, False)
            ms = kern["dose"][0] / reps
            out[name] = {"projections": na, "Dp_gy_per_particle": float(dp[0]),
                         "kernels_ms": ms, "rays_bins_per_s": na * g.n_u * g.n_v * wl.n_e / (ms / 1e3)}
        out["n0_for_7mGy_over_360"] = fc.fc_fluence_for_dose(
            sc.h, 7e-3 / 360, out["all_projections"]["Dp_gy_per_particle"])
        return out
    finally:
        sc.close()


def _extra_paper_timing(fc, torch):
    """The paper's timing scan (180 projections, 6 MV, 18 energies, noise
    before the optical spread) reconstructed to 512^2 x 10 and 1024^2 x 10:
    device time of simulate + reconstruct + HU, and wall time end to end
    through the C ABI from a host phantom to a host HU volume (phantom
    upload, brick map, all kernels, volume download; host-side phantom
    generation excluded).  The paper's 40 s / 61 s are context (another GPU,
    TIGRE, whole program)."""
    out = {}
    for name, paper_s in (("timing_mv_512", 40.0), ("timing_mv_1024", 61.0)):
        wl = W.WORKLOADS[name]
        g = wl.geom
        lab = wl.make_phantom()
        hu = np.empty((g.nz, g.ny, g.nx), np.float32)
        walls = []
        for rep in range(3):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            sc = fc.Scanner(wl, labels=lab, noise=True)
            try:
                fc.fc_set_noise_order(sc.h, fc.FC_NOISE_BEFORE_PSF)
                fc.fc_project(sc.h, 0, g.n_angles, fc.FC_OUT_NONE, None)
                fc.fc_reconstruct(sc.h, None, vol_hu=hu)
                walls.append(time.perf_counter() - t0)
                if rep == 2:
                    a = torch.cuda.Event(enable_timing=True)
                    b = torch.cuda.Event(enable_timing=True)
                    fc.fc_profile_enable(sc.h, True)
                    a.record()
                    fc.fc_project(sc.h, 0, g.n_angles, fc.FC_OUT_NONE, None)
                    fc.fc_reconstruct(sc.h, None, vol_hu=hu)
                    b.record()
                    torch.cuda.synchronize()
                    kern = fc.fc_profile_read(sc.h)
                    ms = a.elapsed_time(b)
            finally:
                sc.close()
        out[name] = {"workload": "%dx%dx%d voxels, %d projections of %dx%d, %d bins to %g keV"
                                 % (g.nx, g.ny, g.nz, g.n_angles, g.n_u, g.n_v, wl.n_e, wl.e_max),
                     "ms_device": ms, "s_wall_end_to_end": min(walls),
                     "kernels_ms": {k: v[0] for k, v in kern.items() if v[1]},
                     "paper_context_s": paper_s}
    return out


def _extra_groups(fc, torch):
    """One simulate + reconstruct step of the catphan_kv scan with the
    four-group detector model (per-group optical spread, fitted scatter
    profiles; W.energy_groups)."""
    wl = W.WORKLOADS["catphan_kv"]
    g = wl.geom
    sc = fc.Scanner(wl, noise=True)
    try:
        grp = W.energy_groups(wl, 4)
        fc.fc_set_energy_groups(sc.h, **grp)
        vol = torch.empty((g.nz, g.ny, g.nx), dtype=torch.float64, device="cuda")
        for _ in range(2):
            fc.fc_project(sc.h, 0, g.n_angles, fc.FC_OUT_NONE, None)
            fc.fc_reconstruct(sc.h, None, vol_mu=vol)
        torch.cuda.synchronize()
        fc.fc_profile_enable(sc.h, True)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        fc.fc_project(sc.h, 0, g.n_angles, fc.FC_OUT_NONE, None)
        fc.fc_reconstruct(sc.h, None, vol_mu=vol)
        b.record()
        torch.cuda.synchronize()
        kern = fc.fc_profile_read(sc.h)
        ms = a.elapsed_time(b)
        return {"workload": "catphan_kv with 4 energy groups", "ms_per_step": ms,
                "rays_bins_per_s": g.n_rays * wl.n_e / (ms / 1e3),
                "kernels_ms": {k: v[0] for k, v in kern.items() if v[1]}}
    finally:
        sc.close()


def _extra_deconv(fc, torch):
    """Richardson-Lucy deconvolution of the catphan_kv counts (10 iterations
    with the workload's PSF), per-iteration device time and the HBM rate of
    its algorithmic bytes (u and d read, u written: 12 B per pixel)."""
    wl = W.WORKLOADS["catphan_kv"]
    g = wl.geom
    sc = fc.Scanner(wl, noise=True)
    try:
        fc.fc_project(sc.h, 0, g.n_angles, fc.FC_OUT_NONE, None)
        fc.fc_deconvolve_rl(sc.h, 0, g.n_angles, wl.psf_sigma_px, 2)
        torch.cuda.synchronize()
        fc.fc_profile_enable(sc.h, True)
        n_iter = 10
        fc.fc_deconvolve_rl(sc.h, 0, g.n_angles, wl.psf_sigma_px, n_iter)
        kern = fc.fc_profile_read(sc.h)
        ms = kern["deconv"][0]
        per = ms / n_iter
        px = g.n_angles * g.n_v * g.n_u
        return {"workload": "catphan_kv counts, 360 x 512 x 384, PSF sigma %.1f px" % wl.psf_sigma_px,
                "iterations": n_iter, "ms_total": ms, "ms_per_iteration": per,
                "hbm_gbs_per_iteration": 12 * px / (per / 1e3) / 1e9}
    finally:
        sc.close()


def _extra_mtf(fc, torch):
    """Detector MTF by the slanted-slit method for the catphan_kv detector
    (single kernel) and its four-group model."""
    wl = W.WORKLOADS["catphan_kv"]
    sc = fc.Scanner(wl, noise=False)
    try:
        out = {}
        for name, grp in (("single_kernel", None), ("four_groups", W.energy_groups(wl, 4))):
            if grp is not None:
                fc.fc_set_energy_groups(sc.h, **grp)
            fc.fc_detector_mtf(sc.h)
            t0 = time.perf_counter()
            f, m = fc.fc_detector_mtf(sc.h)
            ms = (time.perf_counter() - t0) * 1e3
            f50 = float(np.interp(0.5, m[::-1], f[::-1]))
            out[name] = {"ms": ms, "f50_per_mm": f50, "mtf_at_1_per_mm": float(np.interp(1.0, f, m))}
        return out
    finally:
        sc.close()


def _extras(args, fc, torch):
    out = {}
    jobs = [("adjoint", lambda: _extra_adjoint(fc, torch)),
            ("dose", lambda: _extra_dose(fc, torch)),
            ("groups", lambda: _extra_groups(fc, torch)),
            ("deconv", lambda: _extra_deconv(fc, torch)),
            ("mtf", lambda: _extra_mtf(fc, torch)),
            ("paper_timing", lambda: _extra_paper_timing(fc, torch)),
            ("paper_scale", lambda: _extra_paper_scale(fc, torch))]
    if not args.no_surrogate and (not args.extra or "surrogate" in args.extra):
        from paper_2011_04736_gb300 import surrogate_study

        def sur():
            r = surrogate_study.run(steps=args.surrogate_steps, verbose=False)
            return {"workload": "head_surrogate: 256^3 voxels, 360 projections of 512x512, "
                                "120 bins, %d rays" % r["rays"],
                    "train": r["train"], "accuracy": r["accuracy"], "speed_ms": r["speed_ms"],
                    "crossover_bins": r["crossover_bins"]}
        jobs.append(("surrogate", sur))
    if args.extra:
        jobs = [j for j in jobs if j[0] in args.extra]
    for name, job in jobs:
        try:
            out[name] = job()
        except Exception as e:  # an extra never costs the main line
            out[name] = {"error": "%s: %s" % (type(e).__name__, str(e)[:300])}
        torch.cuda.synchronize()
    return out


def run_ours(args):
    rank, world, dist = _dist()
    import torch
    from paper_2011_04736_gb300 import fastcat as fc
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    fc.load()
    wl = W.WORKLOADS[args.workload]
    g = wl.geom
    lab = wl.make_phantom()
    stream = torch.cuda.Stream()
    sc = fc.Scanner(wl, labels=lab, device=local, noise=True, stream=stream)
    h = sc.h
    vol = torch.empty((g.nz, g.ny, g.nx), dtype=torch.float64, device="cuda")
    hu = torch.empty((g.nz, g.ny, g.nx), dtype=torch.float32, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def step():
        fc.fc_project(h, 0, g.n_angles, fc.FC_OUT_NONE, None, stream)
        fc.fc_reconstruct(h, None, vol_mu=vol, vol_hu=hu, stream=stream)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
    torch.cuda.synchronize()

    bus = None
    try:
        bus = torch.cuda.get_device_properties(local).pci_bus_id
    except Exception:
        pass
    clocks = ClockSampler(bus)
    clocks.start()
    time.sleep(0.3)
    fc.fc_profile_enable(h, True)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    _barrier(dist)
    torch.cuda.synchronize()
    t_wall0 = time.time()
    with torch.cuda.stream(stream):
        for i in range(args.steps):
            flush.fill_(float(i))           # evict L2 between timed steps (untimed)
            evs[i][0].record(stream)
            step()
            evs[i][1].record(stream)
    torch.cuda.synchronize()
    _barrier(dist)
    t_wall1 = time.time()
    dev_ms = sum(a.elapsed_time(b) for a, b in evs)
    kern = fc.fc_profile_read(h)
    fc.fc_profile_enable(h, False)
    ms_step = aggregate(dist, dev_ms / args.steps, "max")

    # e2e through the public API with host buffers (pinned)
    lab_h = torch.from_numpy(lab).pin_memory().numpy()
    vol_h = torch.empty((g.nz, g.ny, g.nx), dtype=torch.float64).pin_memory().numpy()
    for _ in range(2):
        fc.fc_set_phantom(h, lab_h, sc.n_mat, stream)
        fc.fc_project(h, 0, g.n_angles, fc.FC_OUT_NONE, None, stream)
        fc.fc_reconstruct(h, None, vol_mu=vol_h, stream=stream)
    _barrier(dist)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        fc.fc_set_phantom(h, lab_h, sc.n_mat, stream)          # H2D: labels
        fc.fc_project(h, 0, g.n_angles, fc.FC_OUT_NONE, None, stream)
        fc.fc_reconstruct(h, None, vol_mu=vol_h, stream=stream)  # D2H: volume (syncs)
    torch.cuda.synchronize()
    e2e_s = aggregate(dist, (time.perf_counter() - t0) / args.steps, "max")
    _barrier(dist)
    clocks.stop()

    units = g.n_rays * wl.n_e
    value = units * world / (ms_step / 1e3)
    vox_rate = g.n_voxels * g.n_angles * world / (ms_step / 1e3)
    peaks, peak_src = _peaks()
    models = _kernel_models(wl)
    kernels = {}
    for name, (ms, n) in kern.items():
        if n == 0 or name not in models:
            continue
        per = ms / args.steps
        m = models[name]
        ent = {"ms_per_step": per, "share": None, "launches_per_step": n / args.steps,
               "gbs": m["bytes"] / (per / 1e3) / 1e9}
        if m["flops"]:
            ent["gflops"] = m["flops"] / (per / 1e3) / 1e9
        kernels[name] = ent
    tot = sum(k["ms_per_step"] for k in kernels.values())
    for k in kernels.values():
        k["share"] = k["ms_per_step"] / tot if tot else None
    top = max(kernels, key=lambda k: kernels[k]["ms_per_step"])
    m = models[top]
    per_s = kernels[top]["ms_per_step"] / 1e3
    launches = kernels[top]["launches_per_step"]
    if m["bound"] == "alu":
        fmax = float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
        peak = 152 * 128 * 2 * fmax / 1e12  # FP32 FMA lanes x 2 flops x clock
        achieved = m["flops"] / per_s / 1e12
        unit = "TFLOP/s"
        peak_note = "FP32 FMA peak 152 SM x 128 lanes x 2 x %.0f MHz (derived)" % (fmax / 1e6)
    else:
        peak = float(peaks["hbm_gbs"])
        achieved = m["bytes"] / per_s / 1e9
        unit = "GB/s"
        peak_note = "HBM copy bandwidth (%s)" % peak_src
    traffic = _traffic(top)
    roof = {"kernel": top, "bound": m["bound"], "achieved": achieved, "peak": peak, "unit": unit,
            "frac": achieved / peak, "traffic": (traffic / launches if traffic else None),
            "peak_source": peak_note,
            "algorithmic": {"bytes_per_launch": m["bytes"] / launches,
                            "flops_per_launch": (m["flops"] / launches if m["flops"] else None)}}
    launches_total = int(sum(n for (_, n) in kern.values()))
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": dict(_workload_desc(wl), l2="flushed by a 256 MiB write between timed steps",
                       parallelism="replicas (one independent scan per GPU)"),
        "fdk_voxel_updates_per_s": vox_rate,
        "clocks": clocks.summary(t_wall0, t_wall1),
        "e2e": {"value": units * world / e2e_s, "unit": UNIT,
                "h2d_bytes_per_step": int(lab.nbytes), "d2h_bytes_per_step": int(vol_h.nbytes)},
        "gpu_launches": launches_total,
        "roofline": roof,
        "kernels": kernels,
    }
    sc.close()
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(wl, args.cpu_angles)
    if rank == 0 and world == 1 and not args.no_extras:
        line["extras"] = _extras(args, fc, torch)
    if rank == 0:
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default 300 for the GPU arm, so that the 200 ms "
                         "clock sampler sees the timed region several times; 50 for the "
                         "reference arm)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(W.WORKLOADS))
    ap.add_argument("--cpu-angles", type=int, default=96,
                    help="projections in the oracle CPU-baseline sample")
    ap.add_argument("--ref-angles", type=int, default=8,
                    help="projections per reference-arm step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the adjoint, paper-scale and surrogate measurements")
    ap.add_argument("--no-surrogate", action="store_true")
    ap.add_argument("--extra", action="append", default=[],
                    help="run only these extras (repeatable): adjoint, dose, groups, deconv, mtf, "
                         "paper_timing, paper_scale, surrogate")
    ap.add_argument("--surrogate-steps", type=int, default=20000)
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.steps is None:
        args.steps = 50 if args.impl == "reference" else 300
    if args.steps < 1:
        ap.error("--steps must be >= 1")
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
