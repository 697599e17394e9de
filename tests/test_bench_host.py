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


def test_rebuild_timing_amortises_over_the_period():
    import numpy as np
    from paper_2504_07948_gb300 import synth

    class FakeQ:
        @staticmethod
        def qmc_set_timing(h, on):
            pass

        @staticmethod
        def qmc_get_timing(h, family):
            assert family == "recompute"
            return 900.0, 2

    class FakeG:
        h = None

        def set_walkers(self, R):
            pass

    s = synth.water_system(2)
    R = np.zeros((16, s.n_elec, 3))
    r = bench.time_recompute(FakeQ, FakeG(), s, R, 100, 20, 0.09, live=0.5)
    assert r["ms_per_step_amortised"] == pytest.approx(9.0)
    assert r["step_ms_with_recompute_amortised"] == pytest.approx(99.0)
    dense = 16 * sum(n * 10.0 * n * s.n_basis + 2.0 * n ** 3 for n in (s.n_up, s.n_dn))
    assert r["achieved_fp64_tflops"] == pytest.approx(dense / 0.9 / 1e12)
    assert r["achieved_fp64_tflops_executed"] < r["achieved_fp64_tflops"]
    assert "live_basis_fraction" not in bench.time_recompute(FakeQ, FakeG(), s, R, 100, 20, 0.09)
    assert bench.time_recompute(FakeQ, FakeG(), s, R, 0, 20, 0.09) is None
