"""Host logic of bench.py that needs no GPU: the DRAM traffic recorded under
profiles/ is reported only while the stage-kernel sources hash to the value
recorded with it (else null), and the clock summary flags throttling."""
import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def test_traffic_reported_only_for_matching_sources(tmp_path):
    b = _bench()
    sha = b.kernel_sources_sha1()
    f = tmp_path / "t.md"
    f.write_text(f"# x\nkernel_sources_sha1: {sha}\nlocal_f16_C3_bytes_per_application: 812.5e6\n")
    b.TRAFFIC_FILE = str(f)
    assert b.recorded_traffic("local_f16_C3_bytes_per_application") == 812.5e6
    assert b.recorded_traffic("global_f32_C3_bytes_per_application") is None
    f.write_text("kernel_sources_sha1: 000000000000\nlocal_f16_C3_bytes_per_application: 812.5e6\n")
    assert b.recorded_traffic("local_f16_C3_bytes_per_application") is None


def test_clock_summary_flags_throttling(tmp_path):
    b = _bench()
    c = b.ClockSampler(0)
    c.proc = object()  # samples already on disk
    c.path = str(tmp_path / "c.csv")
    with open(c.path, "w") as f:
        f.write("0, 2070, 2070, 900, 0x0, Not Active, Not Active, Not Active, Not Active\n")
        f.write("0, 1800, 2070, 1400, 0x4, Not Active, Not Active, Not Active, Active\n")
        f.write("0, 1500, 2070, 1400, 0x8, Not Active, Active, Not Active, Not Active\n")
    s = c.summary()
    assert s["sm_max_mhz"] == 2070 and s["sm_mhz"] == 1800
    assert set(s["reasons"]) == {"sw_power_cap", "hw_thermal_slowdown"}
