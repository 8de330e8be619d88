"""Host-side logic of bench.py (no GPU): the algorithmic-byte model and the
lookup of a kernel's measured DRAM traffic, which must be reported only
while the sources it was measured on are unchanged."""
import hashlib
import os

import bench


def test_algorithmic_bytes_model():
    p = {"n_wedges": 10, "n_bloom_wedges": 4, "n_blooms": 2, "n_edges": 7,
         "link_visits": 8, "pair_slots": 5, "support_updates": 3, "scanned": 11}
    ab = bench.algorithmic_bytes(p)
    # pass A 4W + 12m, pass B 8W + 8 W2 + 8m
    assert ab["count"] == (4 * 10 + 12 * 7) + (8 * 10 + 8 * 4 + 8 * 7)
    # wedge ids and edge ids, twin pairs, links, bloom records
    assert ab["emit"] == 8 * 10 + 8 * 4 + 8 * 4 + 12 * 2
    # scanned entries, link visits, pair slots, support updates
    assert ab["peel"] == 9 * 11 + 8 * 8 + 10 * 5 + 8 * 3


def test_traffic_of_a_smaller_capture_scales_with_the_work(tmp_path, monkeypatch):
    root, csrc = _fake_root(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(root))
    h = {n: hashlib.sha256((csrc / n).read_bytes()).hexdigest() for n in ("peel.cu", "csr.cu")}
    (root / "profiles" / "k_peel-c3shape-3M.md").write_text(
        "captured on a smaller case of the same shape, scaled to the full workload\n"
        "| figure | value |\n|---|---|\n"
        "| traffic_bytes_per_launch | 1000 |\n| algorithmic_bytes_per_launch | 4000 |\n"
        f"| kernel source sha256 (csrc/peel.cu) | {h['peel.cu']} |\n"
        f"| edge numbering sha256 (csrc/csr.cu) | {h['csr.cu']} |\n")
    assert bench.measured_traffic("peel", "large", 40000) == 10000
    assert bench.measured_traffic("peel", "large", None) is None


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


def test_c3shape_workload_is_the_scaled_capture():
    # the 3M-edge workload whose capture is scaled to the 30M-edge graph: its
    # own traffic is the capture itself (ratio one), and it has the large
    # graph's generator parameters at a tenth of the edges
    w, big = bench.WORKLOADS["c3shape"], bench.WORKLOADS["large"]
    assert w["m"] * 10 == big["m"]
    for key in ("gammaU", "gammaL", "plant_lo", "plant_hi", "plant_p"):
        assert w[key] == big[key]
    assert bench.WORKLOAD_PROFILE_TAG["c3shape"] == bench.WORKLOAD_PROFILE_TAG["large"]
    text = open(os.path.join(bench.ROOT, "profiles", "k_peel-c3shape-3M.md")).read()
    assert "--workload c3shape" in text
