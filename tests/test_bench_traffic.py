"""bench.py's DRAM-traffic entries: the per-event figure measured by ncu
stands for the kernel sources it was measured on, identified by a hash of
the sources without comments."""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_comments_and_whitespace_do_not_change_the_code_text():
    a = "int f(int x) {  // one\n  return x + 1; /* two\n three */ }\n"
    b = "int f(int x) {\n/* other */ return x + 1;   }  // trailing\n"
    assert bench._code_only(a) == bench._code_only(b)
    assert bench._code_only(a) != bench._code_only(a.replace("+ 1", "+ 2"))


def test_traffic_scales_with_events_while_the_sources_match(monkeypatch):
    wl, (b_ev, h1, h2) = next(iter(bench.TRAFFIC_B_PER_EVENT.items()))
    monkeypatch.setattr(bench, "kernel_sources_hash", lambda: (h1, h2))
    assert bench.measured_traffic(wl, 1000) == b_ev * 1000
    assert bench.measured_traffic(wl, 0) == 0
    assert bench.measured_traffic("no-such-workload", 1000) is None
    # a changed kernel invalidates the measured figure
    monkeypatch.setattr(bench, "kernel_sources_hash", lambda: (h1, "0" * 16))
    assert bench.measured_traffic(wl, 1000) is None


def test_measured_figures_are_near_the_record_bytes():
    # DRAM bytes per event: the record (12 or 8 B) plus a few percent of
    # index words, run-end sectors and ring-buffer reductions
    for wl, (b_ev, _, _) in bench.TRAFFIC_B_PER_EVENT.items():
        rec = 12.0 if "fp32" in wl else 8.0
        assert rec <= b_ev <= 1.25 * rec, wl


def test_hash_covers_the_two_kernel_sources():
    h = bench.kernel_sources_hash()
    assert len(h) == 2 and all(len(x) == 16 for x in h)
