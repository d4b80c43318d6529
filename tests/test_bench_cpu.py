"""Host-side pieces of bench.py (no GPU): the ncu traffic figure is reported only for
the kernel source it was measured on, and the CPU baseline's single- and all-core
figures come out of the oracle on a small sample."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_traffic_is_tied_to_the_profiled_source(tmp_path, monkeypatch):
    src = "paper_2602_06991_b300/csrc/gs_blend.cu"
    digest = bench.source_digest(src)
    f = tmp_path / "traffic.txt"
    f.write_text(f"# comment\nk_blend_loss_group {digest} 1234\nk_blend_group 000000000000 99\n")
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(f))
    assert bench.measured_traffic("k_blend_loss_group", src) == 1234
    assert bench.measured_traffic("k_blend_group", src) is None          # measured on other source
    assert bench.measured_traffic("k_walk_bwd", src) is None             # never measured
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(tmp_path / "missing.txt"))
    assert bench.measured_traffic("k_blend_loss_group", src) is None


def test_committed_traffic_file_parses():
    with open(bench.TRAFFIC_FILE) as fh:
        rows = [l.split() for l in fh if l.strip() and not l.startswith("#")]
    assert rows and all(len(r) == 3 and len(r[1]) == 12 and int(r[2]) > 0 for r in rows)


def test_cpu_baseline_single_and_all_cores():
    cb = bench.cpu_baseline("small", budget_s=1.0)
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] > 0
    ac = cb["all_cores"]
    assert "unavailable" not in ac, ac
    assert ac["cores"] >= 1 and ac["value"] > 0
