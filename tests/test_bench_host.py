"""Host logic of bench.py that needs no GPU: the algorithmic-traffic models
and the rule that an ncu traffic record counts only for the kernel source it
was captured from."""
import hashlib
import json
import os

import bench
from paper_2011_04736_gb300 import workloads as W


def test_kernel_models_cover_the_step_and_scale_with_the_workload():
    m = bench._kernel_models(W.WORKLOADS["catphan_kv"])
    assert set(m) == {"project", "blur_rows", "blur_cols", "fdk_filter", "backproject", "hu", "noise"}
    g = W.WORKLOADS["catphan_kv"].geom
    px = g.n_angles * g.n_v * g.n_u
    assert m["noise"]["bytes"] == 8 * px                  # rates in, counts out
    assert m["project"]["bytes"] == g.n_voxels + 4 * px   # labels once, T once
    for k in m.values():
        assert k["bound"] in ("hbm", "alu") and k["bytes"] > 0


def test_traffic_record_is_ignored_once_the_source_changes(tmp_path, monkeypatch):
    src = tmp_path / "paper_2011_04736_gb300" / "csrc"
    src.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    (src / "k.cu").write_text("kernel v1\n")
    sha = hashlib.sha256(b"kernel v1\n").hexdigest()[:16]
    rec = {"kernels": {"noise": {"source": "k.cu", "source_sha": sha, "dram_bytes_per_launch": 123}}}
    (tmp_path / "profiles" / "ncu_traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench._traffic("noise") == 123
    assert bench._traffic("project") is None
    (src / "k.cu").write_text("kernel v2\n")
    assert bench._traffic("noise") is None


def test_committed_traffic_record_names_existing_sources():
    rec = json.load(open(os.path.join(bench.ROOT, "profiles", "ncu_traffic.json")))
    for name, ent in rec["kernels"].items():
        assert os.path.exists(os.path.join(bench.ROOT, "paper_2011_04736_gb300", "csrc", ent["source"])), name
        assert ent["dram_bytes_per_launch"] > 0
