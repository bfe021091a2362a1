"""CPU checks of bench.py's host logic: both arms name the workload with the same
config, and the roofline traffic record is used only while the kernel sources it was
captured from are unchanged (else null)."""
import hashlib
import importlib.util
import json
import os
import shutil

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_config_names_the_workload_and_the_deviation_base():
    b = _bench()
    c = b._config(4096, "fp32", 1)
    assert set(c) == {"workload", "nx", "ny", "storage", "l2", "parallelism"}
    assert (c["nx"], c["ny"], c["storage"], c["parallelism"]) == (4096, 4096, "fp32", "single")
    assert "1.21 GB" in c["l2"]                    # 2 x 9 x 4096^2 x 4 B
    assert b._config(4096, "fp32", 8)["parallelism"] == "replicas"
    m = b._config(4096, "bf16", 1, "momentum")
    assert m["dev_base"] == "momentum" and "0.74 GB" in m["l2"]   # 2 x 11 planes x 2 B
    assert "dev_base" not in b._config(4096, "bf16", 1, "rest")


def test_traffic_record_follows_the_kernel_sources(tmp_path, monkeypatch):
    b = _bench()
    rec = json.load(open(os.path.join(ROOT, "profiles", "vanse_warp_fp32_channel_traffic.json")))
    root = tmp_path / "repo"
    (root / "profiles").mkdir(parents=True)
    csrc = root / "paper_2409_02964_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for f in rec["sources"]:
        shutil.copy(os.path.join(ROOT, "paper_2409_02964_gb300", "csrc", f), csrc / f)
    h = hashlib.sha256()
    for f in sorted(rec["sources"]):
        h.update((csrc / f).read_bytes())
    rec = dict(rec, source_sha256=h.hexdigest())
    (root / "profiles" / "vanse_warp_fp32_channel_traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(b, "ROOT", str(root))
    cells = 4096 * 4096
    assert b._kernel_traffic(cells) == round(rec["dram_bytes_per_cell"] * cells)
    # any change to a listed source makes the record stale
    src = csrc / rec["sources"][0]
    src.write_bytes(src.read_bytes() + b"\n")
    assert b._kernel_traffic(cells) is None
