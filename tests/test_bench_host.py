"""Host-side logic of bench.py's roofline entry (no GPU): the dominant
kernel family is the one with the most device time per step summed over its
launches, its achieved rate uses the scope table's per-atom-step operation
counts, and a DRAM profile taken on other kernel sources is never reused."""
import pytest


def test_roofline_picks_the_kernel_with_most_time_per_step(monkeypatch):
    import bench
    monkeypatch.setattr(bench, "measured_peaks", lambda: {"hbm_gbs": 6000.0})
    # spin half-ops 0.3 + 0.3 ms (30 colour passes) against forces 0.5 ms
    phases = {"kick": (0.1, 10), "spin_half_op_1": (3.0, 10), "drift_rebuild": (0.6, 10),
              "exchange_table": (1.0, 10), "spin_half_op_2": (3.0, 10), "force_kick": (5.0, 10)}
    n = 2_000_000
    r = bench.kernel_roofline(phases, n, "fe_bcc_100x100x100_nve", 1.2, peak=4.0)
    assert r["kernel"] == "k_sweep_pass"
    assert r["ops_per_atom_step"] == 4 * (14 * 3 + 60)
    assert r["achieved"] == pytest.approx(408 * n / 0.6e-3 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / 4.0)
    assert r["ms_per_launch"] == pytest.approx(0.6 / 30)
    # the committed profile of this kernel and workload, if its sources are current
    prof = bench.profiled("fe_bcc_100x100x100_nve", "k_sweep_pass")
    assert r["traffic"] == (prof["dram_bytes_per_launch"] if prof else None)
    assert r["hbm_frac_state_traffic"] == pytest.approx(144.0 * n / 1.2e-3 / 1e9 / 6000.0)
    phases["force_kick"] = (7.0, 10)
    assert bench.kernel_roofline(phases, n, "x", 1.2, peak=4.0)["kernel"] == "k_force"


def test_stale_profiles_are_not_used(monkeypatch):
    import bench
    monkeypatch.setattr(bench, "measured_peaks", lambda: {"hbm_gbs": 6000.0})
    phases = {"kick": (0.1, 1), "spin_half_op_1": (0.3, 1), "drift_rebuild": (0.06, 1),
              "exchange_table": (0.1, 1), "spin_half_op_2": (0.3, 1), "force_kick": (0.5, 1)}
    key = ("w", "k_sweep_pass")
    monkeypatch.setitem(bench.PROFILED_DRAM, key, {"dram_bytes_per_launch": 1e6, "sources_sha": "0" * 16,
                                                   "profile": "p.md"})
    assert bench.kernel_roofline(phases, 1000, "w", 1.0, peak=4.0)["traffic"] is None
    monkeypatch.setitem(bench.PROFILED_DRAM, key, {"dram_bytes_per_launch": 1e6,
                                                   "sources_sha": bench.kernel_sources_sha(), "profile": "p.md"})
    r = bench.kernel_roofline(phases, 1000, "w", 1.0, peak=4.0)
    assert r["traffic"] == 1e6 and r["traffic_profile"] == "p.md"
