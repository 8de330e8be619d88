"""Host-side logic of bench.py (no GPU): the algorithmic-byte model and the
lookup of a kernel's measured DRAM traffic, which must be reported only
while the sources it was measured on are unchanged."""
import hashlib
import os

import bench


def test_algorithmic_bytes_model():
    p = {"n_wedges": 10, "n_bloom_wedges": 4, "n_blooms": 2, "n_edges": 7,
         "link_visits": 8, "pair_slots": 5, "support_updates": 3}
    ab = bench.algorithmic_bytes(p)
    assert ab["count"] == 12 * 10 + 8 * 4 + 20 * 7
    assert ab["emit"] == 8 * 10 + 20 * 4 + 12 * 2
    assert ab["peel"] == 25 * 8 + 9 * 5 + 16 * 3


def _fake_root(tmp_path, traffic=123456789):
    root = tmp_path / "repo"
    csrc = root / "paper_2001_06111_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (root / "profiles").mkdir()
    (csrc / "peel.cu").write_text("// peel kernel\n")
    (csrc / "csr.cu").write_text("// csr build\n")
    h = {n: hashlib.sha256((csrc / n).read_bytes()).hexdigest() for n in ("peel.cu", "csr.cu")}
    (root / "profiles" / "k_peel-chunglu-2M.md").write_text(
        "| figure | value |\n|---|---|\n"
        f"| traffic_bytes_per_launch | {traffic} |\n"
        f"| kernel source sha256 (csrc/peel.cu) | {h['peel.cu']} |\n"
        f"| edge numbering sha256 (csrc/csr.cu) | {h['csr.cu']} |\n")
    return root, csrc


def test_traffic_reported_while_sources_match(tmp_path, monkeypatch):
    root, csrc = _fake_root(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench.measured_traffic("peel", "medium") == 123456789
    # no summary for this kernel or workload
    assert bench.measured_traffic("emit", "medium") is None
    assert bench.measured_traffic("peel", "small") is None


def test_traffic_withheld_after_a_source_change(tmp_path, monkeypatch):
    for name in ("peel.cu", "csr.cu"):
        root, csrc = _fake_root(tmp_path / name)
        monkeypatch.setattr(bench, "ROOT", str(root))
        (csrc / name).write_text((csrc / name).read_text() + "// changed\n")
        assert bench.measured_traffic("peel", "medium") is None


def test_committed_summary_names_both_sources():
    text = open(os.path.join(bench.ROOT, "profiles", "k_peel-chunglu-2M.md")).read()
    assert "sha256 (csrc/peel.cu)" in text and "sha256 (csrc/csr.cu)" in text
    assert "traffic_bytes_per_launch" in text
