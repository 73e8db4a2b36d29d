"""Benchmark of the fastCAT CBCT hot path on GB300.

One step = the whole path over one synthetic scan: polyenergetic projection
with the fused energy integral, detector blur + scatter (and Poisson noise
when the workload draws it), FDK filter, FDK backprojection and HU
(fc_project + fc_reconstruct).  The workload is the paper-scale MV case
(1024 x 1024 x 10 voxels of 0.015625 cm with the Catphan-like phantom, 720
projections on a 1024 x 768 detector of 0.392 mm, 60 energy bins of a
2.5 MV bremsstrahlung spectrum, noise-free), the largest configuration that
fits one GPU.

Metric: rays*bins/s = n_angles * n_v * n_u * n_E / step time (whole job,
summed over ranks); FDK voxel updates/s, rays traced/s and voxel crossings/s
are reported beside it.

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
WORKLOAD = "paper_mv"
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
def _hit_band(g):
    """Detector rows [lo, hi] whose rays can meet the voxel slab (the
    projector's traced band: |v| (SAD - r_max) / SDD <= nz dz / 2, two rows of
    margin), clipped to the detector; None when empty."""
    rmax = math.sqrt((0.5 * g.nx * g.dx) ** 2 + (0.5 * g.ny * g.dy) ** 2)
    vmax = 0.5 * g.nz * g.dz * g.sdd / (g.sad - rmax) / g.dv
    cv = 0.5 * (g.n_v - 1)
    lo = max(0, int(math.floor(cv - vmax)) - 2)
    hi = min(g.n_v - 1, int(math.ceil(cv + vmax)) + 2)
    return (lo, hi) if lo <= hi else None


def _reach_rows(g):
    """Detector rows the backprojector samples (conservative, two rows of
    margin): the rows of the filtered-projection buffer."""
    zmax = (g.nz - 1) / 2 * g.dz
    rmax = math.hypot(g.nx * g.dx / 2, g.ny * g.dy / 2)
    vmax = zmax * g.sdd / (g.sad - rmax) / g.dv
    lo = max(0, int(math.floor((g.n_v - 1) / 2 - vmax)) - 2)
    hi = min(g.n_v - 1, int(math.ceil((g.n_v - 1) / 2 + vmax)) + 2)
    return lo, hi


def _band_blur(wl):
    """Whether the detector blur of the workload's primary takes the band
    kernel (a traced band of at most 32 rows touching neither detector edge),
    and the band height."""
    g = wl.geom
    band = _hit_band(g)
    if band is None:
        return False, 0
    hb = band[1] - band[0] + 1
    return (hb <= 32 and band[0] >= 1 and band[1] + 1 <= g.n_v - 1), hb


def _blur_rows(wl):
    """(rows the row pass computes, output rows the column pass computes) on
    the tensor-core path for the projector's primary: the 64-row tiles
    holding the traced band, and the 128-row tiles from a multiple of 8
    covering the band widened by the larger blur radius."""
    g = wl.geom
    band = _hit_band(g)
    if band is None:
        return 0, 0
    lo, hi = band[0], band[1] + 1
    r_lo, r_hi = lo // 64 * 64, min(g.n_v, ((hi - 1) // 64 + 1) * 64)
    R = max(int(math.ceil(4 * wl.psf_sigma_px)), int(math.ceil(4 * wl.scatter_sigma_px)))
    clo, chi = max(0, lo - R), min(g.n_v, hi + R)
    m_off = clo // 8 * 8
    m_cnt = (chi - m_off + 127) // 128
    return r_hi - r_lo, min(g.n_v, m_off + 128 * m_cnt) - m_off


def ray_stats(g, rows=None):
    """Rays of detector rows `rows` (default: every row) that meet the voxel
    box, and the voxels they cross (Siddon segments: per axis the planes
    crossed inside the box, plus one), summed over every projection."""
    rows = np.arange(g.n_v) if rows is None else np.asarray(rows)
    u = (np.arange(g.n_u) - (g.n_u - 1) / 2) * g.du
    v = (rows - (g.n_v - 1) / 2) * g.dv
    uu, vv = np.meshgrid(u, v)
    uu, vv = uu.ravel(), vv.ravel()
    n = np.array([g.nx, g.ny, g.nz])
    d = np.array([g.dx, g.dy, g.dz])
    lo = -0.5 * n * d
    hits = 0
    cross = 0
    for th in g.angles():
        c, s_ = math.cos(th), math.sin(th)
        S = np.array([g.sad * c, g.sad * s_, 0.0])
        P = np.stack([-(g.sdd - g.sad) * c - uu * s_, -(g.sdd - g.sad) * s_ + uu * c, vv], 1)
        D = P - S
        with np.errstate(divide="ignore", invalid="ignore"):
            ta = (lo[None, :] - S[None, :]) / D
            tb = (-lo[None, :] - S[None, :]) / D
        tmin = np.where(D == 0, np.where((S[None, :] > lo) & (S[None, :] < -lo), -np.inf, np.inf),
                        np.minimum(ta, tb))
        tmax = np.where(D == 0, np.where((S[None, :] > lo) & (S[None, :] < -lo), np.inf, -np.inf),
                        np.maximum(ta, tb))
        t0 = np.maximum(0.0, tmin.max(1))
        t1 = np.minimum(1.0, tmax.min(1))
        h = t1 > t0
        if not h.any():
            continue
        E = S[None, :] + t0[h, None] * D[h]
        X = S[None, :] + t1[h, None] * D[h]
        iE = np.clip(np.floor((E - lo) / d), 0, n - 1)
        iX = np.clip(np.floor((X - lo) / d), 0, n - 1)
        hits += int(h.sum())
        cross += int(np.abs(iX - iE).sum() + h.sum())
    return hits, cross


def _kernel_models(wl):
    """Algorithmic bytes and FLOPs per step of each kernel: what the kernel
    must read and write at least, given what it computes in this design
    (the traced band, the blur tiles near it, the reachable filtered rows)."""
    g = wl.geom
    px = g.n_angles * g.n_v * g.n_u
    rp = int(math.ceil(4 * wl.psf_sigma_px)) if wl.psf_sigma_px > 0 else 0
    rs = int(math.ceil(4 * wl.scatter_sigma_px)) if wl.scatter_sigma_px > 0 else 0
    taps = (2 * rp + 1) + (2 * rs + 1)
    lo, hi = _reach_rows(g)
    rows = hi - lo + 1
    fpx = g.n_angles * rows * g.n_u
    fftl = 1 << max(1, int(math.ceil(math.log2(2 * g.n_u - 1)))) if g.n_u > 1 else 2
    row_rows, col_rows = _blur_rows(wl)
    bpx_r = g.n_angles * row_rows * g.n_u      # pixels the row pass computes
    bpx_c = g.n_angles * col_rows * g.n_u      # pixels the column pass computes
    band, hb = _band_blur(wl)
    bpx_b = g.n_angles * hb * g.n_u            # band pixels
    R = max(rp, rs)
    return {
        # labels once + T on the rows the blur reads (T = 1 fill included)
        "project": {"bytes": g.n_voxels + 4 * (bpx_b if band else bpx_r), "flops": None,
                    "bound": "hbm"},
        # band rows of T read, every output pixel written; row passes of the
        # band rows, column sums over the band rows near it
        "blur_band": {"bytes": 4 * bpx_b + 4 * px,
                      "flops": 2 * taps * bpx_b + 2 * 2 * hb * g.n_angles * g.n_u * min(g.n_v, hb + 2 * R),
                      "bound": "hbm"},
        # T read, two intermediates written on the computed tiles
        "blur_rows": {"bytes": 12 * bpx_r, "flops": 2 * taps * bpx_r, "bound": "hbm"},
        # intermediates read on the computed tiles, every output pixel written
        "blur_cols": {"bytes": 8 * bpx_c + 4 * px, "flops": 2 * taps * bpx_c, "bound": "hbm"},
        # reachable rows: counts read, filtered written; two rows per complex
        # FFT of length L (>= 2 n_u - 1): a forward and an inverse transform
        # of 5 L log2 L flops each and the spectrum product (2 L), per row pair
        "fdk_filter": {"bytes": 8 * fpx, "flops": (fpx // g.n_u) * (5 * fftl * int(math.log2(fftl)) + fftl),
                       "bound": "alu"},
        # filtered reachable rows read once, FP64 volume written once; per
        # voxel update 14 flops: v coordinate (fma), its fraction, three
        # linear interpolations (sub + fma each), the weighted sum (fma); the
        # per-(column, projection) set-up shared by the slices is not counted
        "backproject": {"bytes": 4 * fpx + 8 * g.n_voxels, "flops": 14 * g.n_voxels * g.n_angles,
                        "bound": "alu"},
        "hu": {"bytes": 8 * 2 * g.n_voxels + 4 * g.n_voxels, "flops": None, "bound": "hbm"},
        # rates read, counts written
        "noise": {"bytes": 8 * px, "flops": None, "bound": "hbm"},
    }


def _ncu_record(kernel):
    """ncu record of a kernel from profiles/ncu_traffic.json, or None when
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
    return ent


def _traffic(kernel, workload):
    """ncu DRAM bytes (read + write) of one launch of `kernel` on `workload`,
    or None when not recorded for this source and workload."""
    ent = _ncu_record(kernel)
    if not ent or not ent.get("dram") or ent["dram"].get("workload") != workload:
        return None
    return ent["dram"].get("bytes_per_launch")


# ------------------------------------------------------------------ oracle arm
def _oracle_sample(wl, n_angles):
    """Oracle pipeline on the first n_angles projections of the workload:
    projection + energy sum, blur + scatter, Poisson noise (when the
    workload draws it) and FDK over those projections.  Returns seconds."""
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
    K = oracle.poisson(I.astype(np.float32), wl.seed).astype(np.float64) if wl.noise else I
    oracle.fdk(g, K, oracle.i_flood(wl.n0, wl.spr))
    return time.perf_counter() - t0


def cpu_baseline(wl, n_angles):
    import oracle
    t = _oracle_sample(wl, n_angles)
    g = wl.geom
    units = n_angles * g.n_v * g.n_u * wl.n_e
    return {"value": units / t, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
            "sample": "%d of %d projections through the FP64 oracle (projection + energy sum, "
                      "blur + scatter%s, FDK over those projections) in %.2f s; every stage is "
                      "linear in the projections, so the full scan extrapolates linearly to "
                      "%.1f s at the same rate"
                      % (n_angles, g.n_angles, ", binary32 Poisson" if wl.noise else "", t,
                         t * g.n_angles / n_angles)}


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


def _extra_step(fc, torch, name, n_sm, mhz, steps=5, warmup=3, angle_stride=1):
    """One simulate + reconstruct step of another workload, timed like the
    headline (device time on the launching stream, L2 flushed between
    steps): ms per step, rays*bins/s, per-kernel times, the dominant
    kernel's roofline and the projector / backprojector rates."""
    wl = W.WORKLOADS[name]
    g = wl.geom
    stream = torch.cuda.Stream()
    sc = fc.Scanner(wl, noise=wl.noise, stream=stream)
    try:
        h = sc.h
        vol = torch.empty((g.nz, g.ny, g.nx), dtype=torch.float64, device="cuda")
        hu = torch.empty((g.nz, g.ny, g.nx), dtype=torch.float32, device="cuda")
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

        def step():
            fc.fc_project(h, 0, g.n_angles, fc.FC_OUT_NONE, None, stream)
            fc.fc_reconstruct(h, None, vol_mu=vol, vol_hu=hu, stream=stream)

        with torch.cuda.stream(stream):
            for _ in range(warmup):
                step()
        torch.cuda.synchronize()
        ms, kern, _, _ = _timed(fc, torch, h, step, steps, stream, flush)
        kernels = _kernel_table(wl, kern, steps)
        peaks, peak_src = _peaks()
        return dict(_workload_desc(wl), ms_per_step=ms,
                    rays_bins_per_s=g.n_rays * wl.n_e / (ms / 1e3),
                    fdk_voxel_updates_per_s=g.n_voxels * g.n_angles / (ms / 1e3),
                    kernels=kernels, roofline=_roofline(wl, kernels, peaks, peak_src, n_sm, mhz),
                    rates=_path_rates(fc, h, wl, kernels, n_sm, mhz, angle_stride))
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


def _extras(args, fc, torch, n_sm, mhz):
    out = {}
    jobs = [("catphan_kv", lambda: _extra_step(fc, torch, "catphan_kv", n_sm, mhz, steps=20)),
            ("head", lambda: _extra_step(fc, torch, "head_surrogate", n_sm, mhz, steps=5,
                                         angle_stride=8)),
            ("adjoint", lambda: _extra_adjoint(fc, torch)),
            ("dose", lambda: _extra_dose(fc, torch)),
            ("groups", lambda: _extra_groups(fc, torch)),
            ("deconv", lambda: _extra_deconv(fc, torch)),
            ("mtf", lambda: _extra_mtf(fc, torch)),
            ("paper_timing", lambda: _extra_paper_timing(fc, torch))]
    if not args.no_surrogate and (not args.extra or "surrogate" in args.extra):
        from paper_2011_04736_gb300 import surrogate_study

        def sur():
            r = surrogate_study.run(steps=args.surrogate_steps, verbose=False)
            return {"workload": "head_surrogate: 256^3 voxels, 360 projections of 512x512, "
                                "120 bins, %d rays" % r["rays"],
                    "train": r["train"], "accuracy": r["accuracy"], "guard": r["guard"],
                    "speed_ms": r["speed_ms"], "exact_ms_vs_bins": r["exact_ms_vs_bins"],
                    "surrogate_speedup_vs_bins": r["surrogate_speedup_vs_bins"],
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


def _timed(fc, torch, h, step, steps, stream, flush, dist=None):
    """Device time of `steps` calls of step() on `stream` (CUDA events on that
    stream, L2 flushed before each, barrier + synchronize around), with the
    library's per-kernel tracer on.  Returns (ms per step, tracer totals,
    wall-clock start, end)."""
    fc.fc_profile_enable(h, True)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(steps)]
    _barrier(dist)
    torch.cuda.synchronize()
    t0 = time.time()
    with torch.cuda.stream(stream):
        for i in range(steps):
            flush.fill_(float(i))           # evict L2 between timed steps (untimed)
            evs[i][0].record(stream)
            step()
            evs[i][1].record(stream)
    torch.cuda.synchronize()
    _barrier(dist)
    t1 = time.time()
    kern = fc.fc_profile_read(h)
    fc.fc_profile_enable(h, False)
    return sum(a.elapsed_time(b) for a, b in evs) / steps, kern, t0, t1


def _kernel_table(wl, kern, steps):
    models = _kernel_models(wl)
    kernels = {}
    for name, (ms, n) in kern.items():
        if n == 0 or name not in models:
            continue
        per = ms / steps
        m = models[name]
        ent = {"ms_per_step": per, "share": None, "launches_per_step": n / steps,
               "gbs": m["bytes"] / (per / 1e3) / 1e9}
        if m["flops"]:
            ent["gflops"] = m["flops"] / (per / 1e3) / 1e9
        kernels[name] = ent
    tot = sum(k["ms_per_step"] for k in kernels.values())
    for k in kernels.values():
        k["share"] = k["ms_per_step"] / tot if tot else None
    return kernels


def _issue(kernel, wl, units, seconds, n_sm, mhz):
    """Instruction-issue fraction of a kernel: its warp instructions per step
    (ncu record for the current source on this workload family, scaled by
    units of work) over n_SM x 4 schedulers x clock x time."""
    ent = _ncu_record(kernel)
    rec = ent.get("inst") if ent else None
    if not rec or not rec.get("warp_inst_per_launch") or not rec.get("units_per_launch"):
        return None
    if not rec.get("workload", "").startswith(wl.name):
        return None
    inst = rec["warp_inst_per_launch"] * units / rec["units_per_launch"]
    peak = n_sm * 4 * mhz * 1e6
    return {"warp_inst_per_step": inst, "achieved_warp_inst_per_s": inst / seconds,
            "peak_warp_inst_per_s": peak, "frac": inst / seconds / peak,
            "lanes_active_per_inst": rec.get("lanes_active_per_inst"),
            "source": "ncu smsp__inst_executed.sum on %s, scaled by %s" % (rec.get("workload"),
                                                                          rec.get("units"))}


def _roofline(wl, kernels, peaks, peak_src, n_sm, mhz):
    """Roofline of the kernel with the largest time share: achieved =
    algorithmic bytes (or FLOPs) per launch / its measured time."""
    models = _kernel_models(wl)
    top = max(kernels, key=lambda k: kernels[k]["ms_per_step"])
    m = models[top]
    per_s = kernels[top]["ms_per_step"] / 1e3
    launches = kernels[top]["launches_per_step"]
    if m["bound"] == "alu":
        fmax = float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
        peak = n_sm * 128 * 2 * fmax / 1e12  # FP32 FMA lanes x 2 flops x clock
        achieved = m["flops"] / per_s / 1e12
        unit = "TFLOP/s"
        peak_note = "FP32 FMA peak %d SM x 128 lanes x 2 x %.0f MHz (derived)" % (n_sm, fmax / 1e6)
    else:
        peak = float(peaks["hbm_gbs"])
        achieved = m["bytes"] / per_s / 1e9
        unit = "GB/s"
        peak_note = "HBM copy bandwidth (%s)" % peak_src
    traffic = _traffic(top, wl.name)
    return {"kernel": top, "bound": m["bound"], "achieved": achieved, "peak": peak, "unit": unit,
            "frac": achieved / peak, "traffic": traffic,
            "peak_source": peak_note,
            "algorithmic": {"bytes_per_launch": m["bytes"] / launches,
                            "flops_per_launch": (m["flops"] / launches if m["flops"] else None)}}


def _path_rates(fc, h, wl, kernels, n_sm, mhz, angle_stride=1):
    """Projector and backprojector rates beside the headline: rays traced,
    voxel crossings (Siddon segments of the rays that meet the voxels),
    exp2 evaluations against the MUFU rate (16 per SM per clock), voxel
    updates, and each kernel's issue fraction where an ncu record exists."""
    g = wl.geom
    band = _hit_band(g)
    out = {}
    if band is not None and "project" in kernels:
        gs = g if angle_stride == 1 else dataclasses.replace(g, n_angles=g.n_angles // angle_stride,
                                                             arc=g.arc * (g.n_angles // angle_stride)
                                                             * angle_stride / g.n_angles)
        hits, cross = ray_stats(gs, np.arange(band[0], band[1] + 1))
        hits, cross = hits * angle_stride, cross * angle_stride
        t = kernels["project"]["ms_per_step"] / 1e3
        exps = hits * wl.n_e
        mufu = n_sm * 16 * mhz * 1e6
        out["projector"] = {
            "band_rows": [band[0], band[1]], "rays_in_band": (band[1] - band[0] + 1) * g.n_u * g.n_angles,
            "rays_traced": hits, "rays_traced_per_s": hits / t,
            "voxel_crossings": cross, "voxel_crossings_per_s": cross / t,
            "exp2_per_s": exps / t, "mufu_peak_per_s": mufu, "mufu_frac": exps / t / mufu,
            "counted": "every projection" if angle_stride == 1 else "every %dth projection, scaled" % angle_stride,
            "issue": _issue("project", wl, (band[1] - band[0] + 1) * g.n_u * g.n_angles, t, n_sm, mhz)}
    if "backproject" in kernels:
        t = kernels["backproject"]["ms_per_step"] / 1e3
        upd = g.n_voxels * g.n_angles
        m = _kernel_models(wl)["backproject"]
        hbm = float(_peaks()[0]["hbm_gbs"])
        out["backprojector"] = {
            "variant": fc.FC_BP_NAMES.get(fc.fc_backprojector_in_use(h)),
            "voxel_updates_per_s": upd / t,
            # the algorithmic bytes against HBM (the filtered rows stay in L1 / L2)
            "hbm": {"achieved_gbs": m["bytes"] / t / 1e9, "peak_gbs": hbm, "frac": m["bytes"] / t / 1e9 / hbm},
            "issue": _issue("backproject", wl, upd, t, n_sm, mhz)}
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
    props = torch.cuda.get_device_properties(local)
    n_sm = props.multi_processor_count
    wl = W.WORKLOADS[args.workload]
    g = wl.geom
    lab = wl.make_phantom()
    stream = torch.cuda.Stream()
    sc = fc.Scanner(wl, labels=lab, device=local, noise=wl.noise, stream=stream)
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
        bus = props.pci_bus_id
    except Exception:
        pass
    clocks = ClockSampler(bus)
    clocks.start()
    time.sleep(0.3)
    ms_step, kern, t_wall0, t_wall1 = _timed(fc, torch, h, step, args.steps, stream, flush, dist)
    ms_step = aggregate(dist, ms_step, "max")

    # e2e through the public API with host buffers (page-locked): labels in,
    # volume out, every step.  The volume of step i is copied out
    # asynchronously (FC_HOST_ASYNC, the handle's copy stream) into one of
    # two host buffers while step i + 1 is simulated; the last copy is
    # waited for inside the timed region.
    lab_h = torch.from_numpy(lab).pin_memory().numpy()
    vol_h = [torch.empty((g.nz, g.ny, g.nx), dtype=torch.float64).pin_memory().numpy() for _ in range(2)]

    def e2e_step(i):
        fc.fc_set_phantom(h, lab_h, sc.n_mat, stream)          # H2D: labels
        fc.fc_project(h, 0, g.n_angles, fc.FC_OUT_NONE, None, stream)
        fc.fc_reconstruct(h, None, vol_mu=vol_h[i % 2], stream=stream, async_host=True)  # D2H: volume

    for i in range(2):
        e2e_step(i)
    fc.fc_wait_outputs(h)
    _barrier(dist)
    torch.cuda.synchronize()
    n_e2e = max(1, min(args.steps, 100))
    t0 = time.perf_counter()
    for i in range(n_e2e):
        e2e_step(i)
    fc.fc_wait_outputs(h)
    torch.cuda.synchronize()
    e2e_s = aggregate(dist, (time.perf_counter() - t0) / n_e2e, "max")
    _barrier(dist)
    clocks.stop()
    clk = clocks.summary(t_wall0, t_wall1)
    mhz = clk["sm_mhz"] or 2070.0

    units = g.n_rays * wl.n_e
    value = units * world / (ms_step / 1e3)
    vox_rate = g.n_voxels * g.n_angles * world / (ms_step / 1e3)
    peaks, peak_src = _peaks()
    kernels = _kernel_table(wl, kern, args.steps)
    roof = _roofline(wl, kernels, peaks, peak_src, n_sm, mhz)
    rates = _path_rates(fc, h, wl, kernels, n_sm, mhz)
    launches_total = int(sum(n for (_, n) in kern.values()))
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": dict(_workload_desc(wl), l2="flushed by a 256 MiB write between timed steps "
                                              "(the projection buffers are larger than L2 as well)",
                       parallelism="replicas (one independent scan per GPU)"),
        "fdk_voxel_updates_per_s": vox_rate,
        "rays_traced_per_s": (rates.get("projector", {}).get("rays_traced", 0) * world
                              / (ms_step / 1e3)),
        "clocks": clk,
        "e2e": {"value": units * world / e2e_s, "unit": UNIT,
                "h2d_bytes_per_step": int(lab.nbytes), "d2h_bytes_per_step": int(vol_h[0].nbytes),
                "steps": n_e2e,
                "note": "labels copied in from page-locked memory, the FP64 volume copied out "
                        "asynchronously (overlapping the next step's projector), every step"},
        "gpu_launches": launches_total,
        "roofline": roof,
        "rates": rates,
        "kernels": kernels,
    }
    sc.close()
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(wl, args.cpu_angles)
    if rank == 0 and world == 1 and not args.no_extras:
        line["extras"] = _extras(args, fc, torch, n_sm, mhz)
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
    ap.add_argument("--angles", type=int, default=None,
                    help="profile a smaller case: the workload's first N projections (same "
                         "angular step); the bench line then names the reduced workload")
    ap.add_argument("--coarse", type=int, default=None,
                    help="profile a smaller case: N projections spread over the workload's "
                         "whole arc (a full circle stays a full circle)")
    ap.add_argument("--cpu-angles", type=int, default=64,
                    help="projections in the oracle CPU-baseline sample")
    ap.add_argument("--ref-angles", type=int, default=8,
                    help="projections per reference-arm step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the adjoint, paper-scale and surrogate measurements")
    ap.add_argument("--no-surrogate", action="store_true")
    ap.add_argument("--extra", action="append", default=[],
                    help="run only these extras (repeatable): catphan_kv, head, adjoint, dose, "
                         "groups, deconv, mtf, paper_timing, surrogate")
    ap.add_argument("--surrogate-steps", type=int, default=20000)
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.steps is None:
        args.steps = 50 if args.impl == "reference" else 300
    if args.steps < 1:
        ap.error("--steps must be >= 1")
    if args.angles is not None:
        base = W.WORKLOADS[args.workload]
        if not 1 <= args.angles <= base.geom.n_angles:
            ap.error("--angles must be in [1, %d]" % base.geom.n_angles)
        name = "%s_%da" % (args.workload, args.angles)
        W.WORKLOADS[name] = dataclasses.replace(
            W.scaled(base, n_angles=args.angles, arc=base.geom.arc * args.angles / base.geom.n_angles),
            name=name)
        args.workload = name
    if args.coarse is not None:
        if args.angles is not None:
            ap.error("--coarse and --angles exclude each other")
        base = W.WORKLOADS[args.workload]
        if not 1 <= args.coarse <= base.geom.n_angles:
            ap.error("--coarse must be in [1, %d]" % base.geom.n_angles)
        name = "%s_%dc" % (args.workload, args.coarse)
        W.WORKLOADS[name] = dataclasses.replace(W.scaled(base, n_angles=args.coarse), name=name)
        args.workload = name
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
