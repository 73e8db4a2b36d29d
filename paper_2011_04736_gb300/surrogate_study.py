"""Learned-surrogate study on the head-like workload, through the C ABI.

Builds the head-like scan (256^3 voxels of 0.0625 cm, 360 projections of
512 x 512 pixels, 120 energy bins of 20-140 keV), emits the per-material path
lengths of every ray, draws the training set (2^24 rays without replacement,
seed 3) with exact ln T targets from the plain energy sum, trains the MLP with
Adam, then reports on all rays:

* accuracy: |ln T_surrogate - ln T_exact| (max, p99.9, p99, mean) and the
  number of rays that fell back to the exact sum;
* the per-ray guard: the baseline-attenuation threshold set from the
  training rays whose error exceeds 1e-3, the fraction of all rays it sends
  to the exact sum, and the error left on every ray;
* speed: energy stage alone (exact energy sum from L vs surrogate from L)
  and whole projection (projector with fused exact sum vs path-length
  emission + surrogate), CUDA events on the launching stream;
* the exact energy-sum time against the number of energy bins, the
  surrogate's speed-up at each, and the bin count at which the surrogate's
  constant cost equals it (interpolated between measured counts).

    python -m paper_2011_04736_gb300.surrogate_study [--steps 20000] [--batch 65536]
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import workloads as W


def run(steps=20000, batch=65536, n_train=1 << 24, lr=2e-3, workload="head_surrogate",
        chunk_angles=40, guard_tol=1e-3, verbose=True):
    import torch
    from . import fastcat as fc
    fc.load()
    wl = W.WORKLOADS[workload]
    g = wl.geom
    t0 = time.time()
    lab = wl.make_phantom()
    stream = torch.cuda.Stream()
    sc = fc.Scanner(wl, labels=lab, noise=False, stream=stream)
    h = sc.h
    n_mat = len(wl.labels)
    n = g.n_rays
    out = {"workload": workload, "rays": n, "energy_bins": wl.n_e}
    with torch.cuda.stream(stream):
        L = torch.empty((n, n_mat), dtype=torch.float32, device="cuda")
        per = g.n_v * g.n_u
        for a0 in range(0, g.n_angles, chunk_angles):
            na = min(chunk_angles, g.n_angles - a0)
            fc.fc_project_lengths(h, a0, na, L[a0 * per:(a0 + na) * per], stream)
        y = torch.empty(n, dtype=torch.float32, device="cuda")
        fc.fc_energy_sum_lengths(h, L, y, stream)
        torch.cuda.synchronize()
        idx = np.random.default_rng(3).choice(n, size=min(n_train, n), replace=False)
        idx_t = torch.from_numpy(np.sort(idx)).cuda()
        Lt = L.index_select(0, idx_t).contiguous()
        yt = y.index_select(0, idx_t).contiguous()
        torch.cuda.synchronize()
        out["setup_s"] = time.time() - t0
        fc.fc_surrogate_init(h, 3)
        t1 = time.time()
        hist = fc.fc_surrogate_train(h, Lt, yt, steps=steps, batch=batch, lr=lr, seed=3,
                                     stream=stream)
        torch.cuda.synchronize()
        out["train"] = {"steps": steps, "batch": batch, "samples": int(len(idx)), "lr": lr,
                        "seconds": time.time() - t1,
                        "mse_first": float(hist[:10].mean()) if steps else None,
                        "mse_last": float(hist[-10:].mean()) if steps else None}
        ys = torch.empty_like(y)
        nfb = fc.fc_surrogate_eval(h, L, ys, stream)
        torch.cuda.synchronize()
        err = (ys - y).abs()
        q = torch.quantile(err[torch.randperm(n, device="cuda")[:1 << 23]],
                           torch.tensor([0.99, 0.999], device="cuda")).tolist()
        out["accuracy"] = {"max_abs_dlnT": float(err.max()), "p999_abs_dlnT": q[1],
                           "p99_abs_dlnT": q[0], "mean_abs_dlnT": float(err.mean()),
                           "fallback_rays": int(nfb),
                           "rays_within_1e-3": float((err <= 1e-3).float().mean())}
        # per-ray guard judged by the exact sum: threshold from the training
        # set (rays whose error exceeds 1e-3 there), then every ray again
        thr = fc.fc_surrogate_guard(h, Lt, yt, guard_tol, stream)
        nfb_g = fc.fc_surrogate_eval(h, L, ys, stream)
        torch.cuda.synchronize()
        err_g = (ys - y).abs()
        out["guard"] = {"tol": guard_tol, "threshold_baseline_attenuation": thr,
                        "fallback_rays": int(nfb_g), "fallback_fraction": nfb_g / n,
                        "max_abs_dlnT": float(err_g.max()),
                        "rays_within_tol": float((err_g <= guard_tol).float().mean()),
                        "rays_beyond_tol": int((err_g > guard_tol).sum())}
        # speed (library CUDA-event tracer, per kernel): energy stage alone,
        # and projector with the fused exact sum vs path-length emission +
        # surrogate
        T = torch.empty((chunk_angles, g.n_v, g.n_u), dtype=torch.float32, device="cuda")
        reps = 3
        fc.fc_profile_enable(h, True)
        for _ in range(reps):
            fc.fc_surrogate_eval(h, L, ys, stream, count_fallback=False)
        t_guarded = fc.fc_profile_read(h)["surrogate_eval"][0] / reps
        fc.fc_surrogate_guard(h, Lt, yt, 0.0, stream)        # the network alone
        for _ in range(reps):
            fc.fc_energy_sum_lengths(h, L, y, stream)
            fc.fc_surrogate_eval(h, L, ys, stream, count_fallback=False)
            for a0 in range(0, g.n_angles, chunk_angles):
                na = min(chunk_angles, g.n_angles - a0)
                fc.fc_project(h, a0, na, fc.FC_OUT_PRIMARY, T[:na], stream)
                fc.fc_project_lengths(h, a0, na, L[a0 * per:(a0 + na) * per], stream)
        kt = fc.fc_profile_read(h)
        fc.fc_profile_enable(h, False)
        del T
        t_exact = kt["energy_sum"][0] / reps
        t_sur = kt["surrogate_eval"][0] / reps
        t_proj = kt["project"][0] / reps
        t_len = kt["lengths"][0] / reps
        out["speed_ms"] = {"energy_exact": t_exact, "energy_surrogate": t_sur,
                           "energy_speedup": t_exact / t_sur,
                           "energy_surrogate_guarded": t_guarded,
                           "energy_speedup_guarded": t_exact / t_guarded,
                           "project_exact_fused": t_proj, "project_lengths_only": t_len,
                           "project_surrogate": t_len + t_sur,
                           "project_speedup": t_proj / (t_len + t_sur)}
        # exact energy-sum cost versus number of bins
        curve = {}
        w_mu = wl.mu
        for ne in (15, 30, 60, 120, 240):
            e = W.energy_bins(wl.e_lo, wl.e_hi, ne)
            w = W.spectrum_kv(e, wl.e_max)
            d = W.detector_kv(e)
            fc.fc_set_spectrum_detector(h, w, d, W.mu_table(wl.labels, e), wl.psf_sigma_px,
                                        wl.scatter_sigma_px, wl.spr, wl.n0, wl.seed, 0)
            fc.fc_profile_enable(h, True)
            for _ in range(reps):
                fc.fc_energy_sum_lengths(h, L, y, stream)
            curve[ne] = fc.fc_profile_read(h)["energy_sum"][0] / reps
            fc.fc_profile_enable(h, False)
        del w_mu
        ks = sorted(curve)
        out["exact_ms_vs_bins"] = curve
        out["surrogate_speedup_vs_bins"] = {k: curve[k] / t_sur for k in ks}
        # bin count where the exact sum costs as much as the surrogate:
        # linear interpolation between the two measured counts around it
        cross = None
        for a, b in zip(ks, ks[1:]):
            if curve[a] <= t_sur < curve[b]:
                cross = a + (t_sur - curve[a]) * (b - a) / (curve[b] - curve[a])
        out["crossover_bins"] = cross
    sc.close()
    if verbose:
        print(json.dumps(out, indent=1))
    return out


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--batch", type=int, default=65536)
    ap.add_argument("--train", type=int, default=1 << 24)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--workload", default="head_surrogate")
    a = ap.parse_args(argv)
    run(a.steps, a.batch, a.train, a.lr, a.workload)


if __name__ == "__main__":
    main()
