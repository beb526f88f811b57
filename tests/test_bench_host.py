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


def test_algorithmic_bytes_follow_the_stage_count():
    """Per output 5D site a hop stage moves 24 w in + 24 w out + 8 * 12 * w / Ls
    of links (+ 8 / Ls of FP32 scales for the scaled 16-bit formats): 113 B in
    FP16 and 224 B in FP32 at Ls = 12.  One global D^+D is four stages over
    the even sites (896 B per even 5D site in FP32); one local operator is the
    four stages over O1, E2, O1 and the block interior."""
    b = _bench()
    assert abs(b.stage_bytes(12, "f16") - 113.0) < 0.5
    assert b.stage_bytes(12, "bf16") == 112.0
    assert b.stage_bytes(12, "f32") == 224.0
    assert b.stage_bytes(8, "bf16") == 120.0
    geo = {"blocks": 32, "block_sites": 2048, "o1_sites": 4096, "e2_sites": 6912, "even_sites": 65536}
    assert b.global_op_bytes(geo, 12, "f32") == 896 * 65536 * 12
    assert b.local_stage_sites(geo, 12) == 32 * (4096 + 6912 + 4096 + 2048) * 12
    assert abs(b.local_op_bytes(geo, 12, "f16") / 6586368 - b.stage_bytes(12, "f16")) < 1e-9
