"""Host-side logic of bench.py on CPU: the clock-sample summary that decides
whether a run was throttled, the node ranges its work model uses (against the
oracle's tree), the per-phase roofline arithmetic and the rounding of the one-line summary."""
import numpy as np

import bench
import oracle


def _row(idx, sm, smax, reasons=("Not Active",) * 4):
    return [str(idx), str(sm), str(smax), "900.00", "0x0", *reasons]


def test_clock_summary_median_max_and_reasons():
    rows = [_row(0, 2070, 2070), _row(0, 1980, 2070), _row(0, 2070, 2070),
            _row(1, 500, 2070, ("Active", "Not Active", "Not Active", "Not Active")),  # another GPU
            _row(0, 1500, 2070, ("Not Active", "Not Active", "Not Active", "Active")),
            ["0", "[N/A]"]]                                                          # a short row
    out = bench.summarize_clocks(rows, 0)
    assert out["samples"] == 4
    assert out["sm_mhz"] == 2025.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]
    hot = bench.summarize_clocks([_row(0, 1400, 2070, ("Not Active", "Active", "Not Active", "Not Active"))], 0)
    assert hot["reasons"] == ["hw_thermal_slowdown"]
    assert bench.summarize_clocks([], 0) == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}


def test_work_model_node_ranges_equal_the_oracle_tree():
    for N, m in ((4096, 256), (5000, 300), (777, 50), (3, 1), (100, 1000), (70001, 1024)):
        D, lo, hi = bench.tree_ranges(N, m)
        o = oracle.Oracle(np.random.default_rng(N).random((N, 2)), m)
        assert D == o.D
        for a in range(1, o.nnodes + 1):
            assert (lo[a], hi[a]) == o.node_range(a)


def test_phase_roofline_arithmetic():
    peaks = {"hbm_gbs": 5000.0, "bf16_tflops": 2000.0}
    work = {"solve_leaf": ("hbm", 1e9, "sweep"), "z_lu": ("fp64", 2.5e11, "step"), "zoff": ("tf32", 0.0, "step")}
    ms = {"solve_leaf": 10.0, "z_lu": 400.0, "zoff": 5.0}
    launches = {"solve_leaf": 20, "matvec_leaf": 0}
    out = bench.phase_rooflines(work, ms, launches, 2, peaks)
    # 10 sweeps per step x 2 steps x 1 GB in 10 ms = 2000 GB/s of 5000
    assert out["solve_leaf"]["achieved"] == 2000.0 and out["solve_leaf"]["frac"] == 0.4
    assert out["solve_leaf"]["per_step"] == 10.0
    # 2 x 2.5e11 flops in 0.4 s = 1.25 TFLOP/s, the nominal FP64 rate
    assert out["z_lu"]["achieved"] == 1.25 and out["z_lu"]["frac"] == 1.0
    assert "zoff" not in out                        # no work: no rate


def test_error_rounding_reaches_nested_groups():
    line = {"value": 1.0891234, "mixed_rel_err_vs_oracle": 2.21234e-10,
            "near_field": {"richardson_rel_err": 3.466450935e-07, "factorize_s": [1.4957, 4.7189],
                           "block16_rhs_per_s": {"mixed_tc": 141.3612}},
            "batched": None}
    out = bench.round_errors(line)
    assert out["value"] == 1.0891234 and out["mixed_rel_err_vs_oracle"] == 2.21e-10
    assert out["near_field"]["richardson_rel_err"] == 3.47e-07
    assert out["near_field"]["factorize_s"] == [1.4957, 4.7189]
    assert out["near_field"]["block16_rhs_per_s"]["mixed_tc"] == 141.3612 and out["batched"] is None
