"""Host logic of bench.py that needs no GPU: the algorithmic-traffic models
and the rule that an ncu traffic record counts only for the kernel source it
was captured from."""
import hashlib
import json
import os

import bench
from paper_2011_04736_gb300 import workloads as W


def test_kernel_models_cover_the_step_and_scale_with_the_workload():
    for name in ("catphan_kv", "paper_mv"):
        wl = W.WORKLOADS[name]
        m = bench._kernel_models(wl)
        assert set(m) == {"project", "blur_rows", "blur_cols", "blur_band", "fdk_filter",
                          "backproject", "hu", "noise"}
        g = wl.geom
        px = g.n_angles * g.n_v * g.n_u
        rows_r, rows_c = bench._blur_rows(wl)
        assert m["noise"]["bytes"] == 8 * px                  # rates in, counts out
        # labels once, T on the rows the blur reads (the band for both workloads)
        band, hb = bench._band_blur(wl)
        assert band
        assert m["project"]["bytes"] == g.n_voxels + 4 * g.n_angles * hb * g.n_u
        assert m["blur_cols"]["bytes"] >= 4 * px              # every output pixel written
        for k in m.values():
            assert k["bound"] in ("hbm", "alu") and k["bytes"] > 0
    # paper-scale MV: the traced band and the blur tiles are a small part of the detector
    wl = W.WORKLOADS["paper_mv"]
    lo, hi = bench._hit_band(wl.geom)
    assert (lo, hi) == (378, 389)
    assert bench._blur_rows(wl) == (128, 256)


def test_ray_stats_match_the_oracle_path_matrix(orc):
    """Rays that meet the voxels and the voxels they cross (the Siddon
    segments), counted by the host closed form, against the nonzeros of the
    oracle's ray x voxel path-length matrix."""
    import numpy as np
    wl = W.scaled(W.WORKLOADS["small_kv"], n_u=13, n_v=9, n_angles=7, nx=6, ny=5, nz=4,
                  dx=0.5, dy=0.4, dz=0.3, du=0.45, dv=0.3)
    g = wl.geom
    rowptr, col, val = orc.path_matrix(g)
    cs = np.concatenate([[0], np.cumsum(val > 0)])
    pos = cs[rowptr[1:]] - cs[rowptr[:-1]]          # voxels with positive length per ray
    # the closed form counts one voxel per plane crossed; where a ray crosses
    # two planes at one point (a voxel edge) Siddon has one segment fewer,
    # so the counts agree to a fraction of a percent, the hits exactly
    hits, cross = bench.ray_stats(g)
    assert hits == int((pos > 0).sum()) > 0
    assert abs(cross - int(pos.sum())) <= 0.005 * pos.sum()
    rows = np.arange(2, 7)
    sel = np.zeros((g.n_angles, g.n_v, g.n_u), bool)
    sel[:, rows, :] = True
    h2, c2 = bench.ray_stats(g, rows)
    assert h2 == int((pos.reshape(sel.shape)[sel] > 0).sum())
    assert abs(c2 - int(pos.reshape(sel.shape)[sel].sum())) <= 0.005 * c2


def test_traffic_record_is_ignored_once_the_source_changes(tmp_path, monkeypatch):
    src = tmp_path / "paper_2011_04736_gb300" / "csrc"
    src.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    (src / "k.cu").write_text("kernel v1\n")
    sha = hashlib.sha256(b"kernel v1\n").hexdigest()[:16]
    rec = {"kernels": {"noise": {"source": "k.cu", "source_sha": sha,
                                 "dram": {"workload": "catphan_kv", "bytes_per_launch": 123}}}}
    (tmp_path / "profiles" / "ncu_traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench._traffic("noise", "catphan_kv") == 123
    assert bench._traffic("noise", "paper_mv") is None        # another workload
    assert bench._traffic("project", "catphan_kv") is None
    (src / "k.cu").write_text("kernel v2\n")
    assert bench._traffic("noise", "catphan_kv") is None


def test_committed_traffic_record_names_existing_sources():
    rec = json.load(open(os.path.join(bench.ROOT, "profiles", "ncu_traffic.json")))
    for name, ent in rec["kernels"].items():
        assert os.path.exists(os.path.join(bench.ROOT, "paper_2011_04736_gb300", "csrc", ent["source"])), name
        assert ent["dram"]["bytes_per_launch"] > 0
        assert ent["inst"]["warp_inst_per_launch"] > 0 and ent["inst"]["units_per_launch"] > 0
