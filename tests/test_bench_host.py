"""Host logic of bench.py's roofline bookkeeping (no GPU): the DRAM traffic
of a kernel comes from a stored ncu capture and is reported only while the
kernel's sources hash to the value recorded with the capture."""
import os

import pytest

import bench


def test_every_traffic_record_names_a_committed_summary():
    for key, rec in bench.PROFILED_TRAFFIC.items():
        per_walker, where, w_cap, files, digest = rec[:5]
        assert per_walker > 0 and w_cap > 0, key
        assert os.path.isfile(os.path.join(bench.ROOT, where)), (key, where)
        for f in files:
            assert os.path.isfile(os.path.join(bench.ROOT, "paper_2504_07948_gb300", "csrc", f)), (key, f)
        assert len(digest) == 16


def test_traffic_scales_with_walkers_and_keeps_fixed_bytes(monkeypatch):
    files = ("k_nlpp.cu",)
    digest = bench.sources_sha(files)
    monkeypatch.setitem(bench.PROFILED_TRAFFIC, ("demo", "k"), (100.0, "profiles/k_nlpp_water32_pp.md", 8, files,
                                                                 digest, 50.0))
    t, note = bench.profiled_traffic("demo", "k", 8)
    assert t == pytest.approx(850.0) and "scaled" not in note
    t, note = bench.profiled_traffic("demo", "k", 32)
    assert t == pytest.approx(3250.0) and "scaled by walker count to 32" in note


def test_traffic_is_withheld_once_the_sources_change(monkeypatch):
    monkeypatch.setitem(bench.PROFILED_TRAFFIC, ("demo", "k"), (100.0, "profiles/k_nlpp_water32_pp.md", 8,
                                                                 ("k_nlpp.cu",), "0000000000000000"))
    t, note = bench.profiled_traffic("demo", "k", 8)
    assert t is None and "changed" in note
    t, note = bench.profiled_traffic("no such workload", "k", 8)
    assert t is None
