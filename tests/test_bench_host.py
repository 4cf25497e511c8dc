"""Host-side pieces of bench.py (no GPU): the nvidia-smi clock summary that
decides whether a bench line is valid (median SM clock, throttle reasons),
the roofline record of a kernel class, and the oracle's work count."""
import bench


def test_clock_rows_median_max_and_reasons():
    lines = [
        "0, 2070, 2070, 900.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n",
        "0, 2055, 2070, 1350.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active\n",
        "0, 2070, 2070, 1390.2, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n",
        "garbage line\n",
    ]
    c = bench.parse_clock_rows(lines)
    assert c["samples"] == 3
    assert c["sm_mhz"] == 2070.0 and c["sm_max_mhz"] == 2070.0
    assert c["reasons"] == ["sw_power_cap"]
    lines.append("0, 1800, 2070, 800.0, 0x0000000000000040, Not Active, Active, Not Active, Not Active\n")
    c = bench.parse_clock_rows(lines)
    assert c["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]
    assert bench.parse_clock_rows(["x\n"]) is None


def test_roofline_record_of_the_dominant_class():
    prof = {"coarse": {"launches": 10, "ms": 20.0, "alg_bytes": 100e9},
            "inner": {"launches": 70, "ms": 60.0, "alg_bytes": 360e9},
            "qoi": {"launches": 1, "ms": 0.1, "alg_bytes": 1e6}}
    r = bench._roofline(prof, ("coarse", "inner"), {"coarse": "k_coarse", "inner": "k_inner"})
    assert r["kernel"] == "k_inner"
    assert r["achieved"] == round(360e9 / 0.060 / 1e9, 1)
    assert r["frac"] == round(r["achieved"] / r["peak"], 4)
    assert r["alg_bytes_per_launch"] == 360e9 / 70
    assert abs(r["share_of_kernel_time"] - round(60.0 / 80.1, 4)) < 1e-12
    j = bench._classes_json(prof)
    assert j["inner"]["alg_GBps"] == round(360e9 / 0.060 / 1e9, 1)


def test_oracle_work_count_matches_the_metric():
    """N_steps (n_free + p |R|) with R the vertices of elements touching P:
    the unit of the benchmark's metric, counted on the host."""
    cfg = bench._cfg("plain")
    units = bench.oracle_units_per_sample(cfg, 0)
    from workload import level_problem
    lev = level_problem(cfg, 0)
    m = lev["mesh"]
    free = ~m.dirichlet.astype(bool)
    assert units > lev["n_steps"] * int(free.sum())
    assert units < lev["n_steps"] * (1 + cfg.p) * int(free.sum())


def test_slices_cover_every_outer_step_once():
    """The bench step is one time slice; n consecutive slices run every outer
    step of a batch exactly once (the library's floor(N k / n) rule)."""
    for N in (1, 7, 432, 1727, 6907):
        for n in (1, 3, 20, 64):
            st = bench.slice_steps(N, n)
            assert sum(st) == N and len(st) == n
            assert max(st) - min(st) <= 1


def test_roofline_traffic_from_the_capture_of_the_current_kernels():
    """traffic = captured DRAM/algorithmic ratio x algorithmic bytes per
    launch while the kernel source is the captured one; null otherwise."""
    prof = {"coarse": {"launches": 10, "ms": 20.0, "alg_bytes": 100e9},
            "inner": {"launches": 70, "ms": 60.0, "alg_bytes": 360e9}}
    names = {"coarse": "k_coarse", "inner": "k_inner"}
    r = bench._roofline(prof, ("coarse", "inner"), names)
    cap = bench.CAPTURED["inner"]
    assert abs(r["traffic"] - cap["dram_bytes"] / cap["alg_bytes"] * 360e9 / 70) < 1.0
    assert 1.0 < r["traffic_over_alg"] < 2.0
    # the DRAM rate: that traffic over the average launch time (60 ms / 70)
    assert r["dram_achieved"] == round(r["traffic"] / (0.060 / 70) / 1e9, 1)
    assert r["dram_frac"] == round(r["dram_achieved"] / r["peak"], 4)
    assert r["dram_frac"] > r["frac"]
    saved = cap["sha16"]
    try:
        cap["sha16"] = "0" * 16
        r0 = bench._roofline(prof, ("coarse", "inner"), names)
        assert r0["traffic"] is None and r0["dram_achieved"] is None and r0["dram_frac"] is None
    finally:
        cap["sha16"] = saved


def test_captured_traffic_matches_the_current_kernel_sources():
    """Every captured figure names the sources it was taken with; the record
    uses it only while their hash is unchanged."""
    for cls, cap in bench.CAPTURED.items():
        assert cap["src"] and len(cap["sha16"]) == 16, cls
        assert 1.0 < cap["dram_bytes"] / cap["alg_bytes"] < 4.0, cls
