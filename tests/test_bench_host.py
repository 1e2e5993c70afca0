"""Host-side pieces of bench.py (no GPU): the workload it times, the peak it
divides by, and the choice of roofline for the 16-bit variant."""
import bench


def test_benchmark_workload_is_the_512cube_forced_thermal_box():
    w = bench.workload_config("f32", 512)
    assert (w["nx"], w["ny"], w["nz"]) == (512, 512, 512)
    assert w["pattern"] == "aa" and w["store"] == "f32" and w["lattice"] == "d3q19"
    assert (w["kT"], w["gamma_shear"], w["gamma_bulk"], w["gamma_ghost"], w["seed"], w["force_amp"]) == \
        (1e-4, 0.3, 0.2, 0.0, 3, 1e-5)
    cfg = bench.arm_config("f32", 512, 1)
    assert cfg["sites"] == 512 ** 3 and cfg["pattern"] == "AA" and "512^3" in cfg["workload"]


def test_peak_is_positive_and_labelled():
    peak, kind = bench.measured_peaks()
    assert peak > 1000 and kind in ("measured", "fallback")


def test_the_nearer_roofline_is_reported_as_the_bound():
    P = 152 * 4 * 32 * 2070e6
    # HBM nearer: 4.9 TB/s of 6.8 against 0.6 of the issue peak
    r = bench.f16_roofline(0.6 * P, 400.0, 4900.0, 6800.0, P, "test")
    assert r["bound"] == "hbm" and abs(r["frac"] - 4900 / 6800) < 1e-12
    assert r["other"]["bound"] == "alu" and abs(r["other"]["frac"] - 0.6) < 1e-12
    # issue nearer
    r = bench.f16_roofline(0.8 * P, 500.0, 4000.0, 6800.0, P, "test")
    assert r["bound"] == "alu" and r["other"]["bound"] == "hbm"
    # no instruction count on record: the HBM roofline alone decides
    r = bench.f16_roofline(None, None, 3000.0, 6800.0, P, "test")
    assert r["bound"] == "hbm" and r["other"]["frac"] is None


class _FakeProps:
    multi_processor_count = 150


class _FakeCuda:
    @staticmethod
    def current_device():
        return 0

    @staticmethod
    def get_device_properties(i):
        return _FakeProps()


class _FakeTorch:
    cuda = _FakeCuda()


def test_issue_peak_uses_the_device_sm_count_and_the_sampled_clock():
    peak, src = bench.issue_peak(_FakeTorch(), 1900.0)
    assert peak == 150 * 4 * 32 * 1900e6 and "150 SMs" in src and "sampled" in src
    peak, src = bench.issue_peak(_FakeTorch(), None)      # no sample: the maximum clock
    assert peak > 0 and "150 SMs" in src and "maximum" in src


def test_ensemble_workload_is_the_batched_replicas_and_mixed_cubes():
    edges, gammas = bench.ensemble_boxes()
    assert edges[:64] == [64] * 64 and len(edges) == 80
    assert edges[64:] == [32, 40, 48, 48, 56, 64, 72, 80, 80, 88, 96, 104, 112, 112, 120, 128]
    assert sum(e ** 3 for e in edges) == 28_256_256
    assert all(0.0 <= g <= 0.8 for g in gammas) and len(gammas) == 80


class _FakeNvml:
    """Stands in for the NVML reader: a clock sequence and reason bits."""

    def __init__(self, clocks, bits):
        self.clocks, self.bits, self.k = list(clocks), list(bits), 0

    def sm_mhz(self):
        v = self.clocks[min(self.k, len(self.clocks) - 1)]
        return v

    def reasons(self):
        v = self.bits[min(self.k, len(self.bits) - 1)]
        self.k += 1
        return v

    def max_sm_mhz(self):
        return 2070.0


def test_clock_sampler_reads_nvml_during_the_region_and_names_the_reasons():
    import time
    fake = _FakeNvml([2070.0, 2070.0, 1980.0], [0, 0x4, 0x4 | 0x40])
    with bench.ClockSampler(0, reader=fake) as s:
        time.sleep(0.05)
    out = s.summary()
    assert out["source"] == "nvml" and out["samples"] >= 3
    assert out["sm_max_mhz"] == 2070.0 and out["sm_mhz"] in (2070.0, 1980.0)
    # power cap (kept, noted) and hardware thermal slowdown (rejecting) both named
    assert out["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]
    quiet = _FakeNvml([2070.0], [0])
    with bench.ClockSampler(0, reader=quiet) as s:
        time.sleep(0.01)
    assert s.summary()["reasons"] == [] and s.summary()["sm_mhz"] == 2070.0


def test_ensemble_traffic_needs_the_recorded_pattern(monkeypatch):
    rec = {"kernel_hash": "x", "sites": 10, "dram_bytes_per_step": 1234.0, "pattern": "ab"}
    monkeypatch.setattr(bench, "ncu_record", lambda store: rec if store == "ensemble_f32" else None)
    assert bench.ensemble_traffic("f32", "ab") == 1234.0
    assert bench.ensemble_traffic("f32", "aa") is None          # another pattern moves other bytes
    assert bench.ensemble_traffic("f16dev", "ab") is None       # no record
