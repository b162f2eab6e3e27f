"""Host logic of the benchmark, without a GPU: the clock record taken during
the timed region (which decides whether a run is rejected), the traffic pin
of a profiled kernel (reported only for the profiled source and workload),
and the multiply-add count of the blocked triangular solve."""
import os

import bench
import workloads


def row(sm, mx, reasons=("Not Active",) * 4):
    # index, clocks.sm, clocks.max.sm, power.draw, reasons.active, hw_slowdown,
    # hw_thermal_slowdown, sw_thermal_slowdown, sw_power_cap
    return ["0", str(sm), str(mx), "900.0", "0x0", *reasons]


def sampler(rows, t0, t1):
    s = bench.ClockSampler(0)
    s.rows = rows
    s.t0, s.t1 = t0, t1
    return s


def test_clock_summary_inside_the_timed_region():
    rows = [(0.9, row(1500, 2070)), (1.0, row(2070, 2070)), (1.05, row(2055, 2070)), (1.1, row(2070, 2070)),
            (2.0, row(1200, 2070))]
    s = sampler(rows, 1.0, 1.1).summary()
    assert s["samples"] == 3
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == []


def test_clock_summary_names_active_throttle_reasons():
    hot = ("Not Active", "Active", "Not Active", "Active")  # hw_thermal_slowdown, sw_power_cap
    rows = [(1.0, row(1800, 2070, hot)), (1.02, row(1900, 2070))]
    s = sampler(rows, 1.0, 1.02).summary()
    assert s["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]
    assert s["sm_mhz"] == 1850.0


def test_clock_summary_short_region_takes_the_nearest_sample():
    rows = [(0.5, row(1000, 2070)), (1.2, row(2040, 2070))]
    s = sampler(rows, 1.001, 1.002).summary()   # no sample arrived inside the region
    assert s["samples"] == 1 and s["sm_mhz"] == 2040.0


def test_clock_summary_ignores_unparsable_rows_and_no_samples():
    rows = [(1.0, ["0", "[N/A]", "2070", "", "", "", "", "", ""]), (1.0, ["garbage"])]
    s = sampler(rows, 0.9, 1.1).summary()
    assert s["samples"] == 0 and s["sm_mhz"] is None and s["reasons"] == []


def test_traffic_pin_only_for_the_profiled_source_and_workload(monkeypatch):
    import hashlib
    by_name = {w.name: w for w in workloads.WORKLOADS.values()}
    # pin the recorded hashes to the sources as they stand, so that only the workload decides here
    def current(fname):
        with open(os.path.join(bench.ROOT, "paper_1111_6900_gb300", "csrc", fname), "rb") as fh:
            return fname, hashlib.sha256(fh.read()).hexdigest()

    for key, pins in list(bench.PROFILED_SOURCES.items()):
        monkeypatch.setitem(bench.PROFILED_SOURCES, key, tuple(current(f) for f, _ in pins))
    monkeypatch.setattr(bench, "WORKLOAD", by_name["gf16_4096_mul"])
    t = bench.TRAFFIC["tc_f4/karatsuba"]["bytes"]
    assert bench.kernel_traffic("tc_f4/karatsuba") == t
    assert bench.kernel_traffic("newton_john/alpha_b") is None     # profiled on another workload
    assert bench.kernel_traffic("tc_f8/alpha_b") is None           # never profiled
    monkeypatch.setattr(bench, "WORKLOAD", by_name["gf256_8192x64x8192_addmul"])
    assert bench.kernel_traffic("newton_john/alpha_b") == bench.TRAFFIC["newton_john/alpha_b"]["bytes"]
    assert bench.kernel_traffic("tc_f4/karatsuba") is None
    # a changed source voids the pin
    monkeypatch.setitem(bench.PROFILED_SOURCES, "newton_john/alpha_b", (("nj_kernel.cuh", "0" * 64),))
    assert bench.kernel_traffic("newton_john/alpha_b") is None
    # so does a change to any one of several pinned sources (the launching host code)
    monkeypatch.setattr(bench, "WORKLOAD", by_name["gf16_4096_mul"])
    monkeypatch.setitem(bench.PROFILED_SOURCES, "tc_f4/karatsuba",
                        (current("gemm_tc.cu"), ("api.cu", "0" * 64)))
    assert bench.kernel_traffic("tc_f4/karatsuba") is None


def test_recorded_traffic_pins_match_the_sources():
    """The committed pins hold for the sources as committed: a kernel or
    launch change without a new capture must show up here."""
    import hashlib
    for key, pins in bench.PROFILED_SOURCES.items():
        for fname, sha in pins:
            with open(os.path.join(bench.ROOT, "paper_1111_6900_gb300", "csrc", fname), "rb") as fh:
                assert hashlib.sha256(fh.read()).hexdigest() == sha, (key, fname)


def test_triangular_solve_multiply_adds():
    # one leaf: the whole triangle times n columns
    assert bench.trsm_macs(100, 7) == 100 * 100 * 7
    # m a power-of-two multiple of the block: leaves nb^2 n each, updates (m^2 - m nb) n / 2
    for m in (256, 1024, 4096):
        assert bench.trsm_macs(m, 3) == (m * m + 128 * m) * 3 // 2
    # ragged m: leaves and updates still cover every (row, column) pair of the triangle once
    m, n = 1000, 1
    leaves = bench.trsm_macs(m, n) - (m * m - sum(b * b for b in blocks(m))) // 2
    assert leaves == sum(b * b for b in blocks(m))


def blocks(m, nb=128):
    if m <= nb:
        return [m]
    m1 = -(-((m + 1) // 2) // nb) * nb
    return blocks(m1, nb) + blocks(m - m1, nb)


def test_replica_throughput_of_one_process():
    assert bench.replica_throughput(3.0e9, 1.5) == (2.0e9, 1.5)
