"""Host logic of the benchmark that needs no GPU: the clock-sample parser
(throttle reasons decide whether a run is kept) and the lookup of the
committed per-launch DRAM traffic."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


class _Done:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _clocks(tmp_path, rows):
    path = tmp_path / "clocks.csv"
    path.write_text("\n".join(rows) + "\n")
    c = bench.Clocks.__new__(bench.Clocks)
    c.proc, c.path = _Done(), str(path)
    return c.stop()


def test_clock_samples_and_reasons(tmp_path):
    ok = "0, 2070, 2070, 812.40, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active"
    capped = "0, 1980, 2070, 1400.00, 0x0000000000000004, Not Active, Not Active, Not Active, Active"
    hot = "0, 1500, 2070, 1100.00, 0x0000000000000040, Not Active, Active, Not Active, Not Active"
    r = _clocks(tmp_path, [ok, ok, capped])
    assert r == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    r = _clocks(tmp_path, [ok, hot, hot, "garbage line"])
    assert r["reasons"] == ["hw_thermal_slowdown"] and r["samples"] == 3 and r["sm_mhz"] == 1500.0
    assert _clocks(tmp_path, []) is None


def test_no_sampler_no_clocks():
    c = bench.Clocks.__new__(bench.Clocks)
    c.proc = None
    assert c.stop() is None


def test_traffic_only_for_the_profiled_kernel(tmp_path, monkeypatch):
    """The DRAM bytes are taken only from a summary of this kernel version
    and record layout (the tile does not change them)."""
    f = tmp_path / "traffic.md"
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(f))
    assert bench.measured_traffic(1, (4, 8)) is None            # no summary
    f.write_text(f"# x\n\n- kernel_version: {bench.KERNEL_VERSION}\n- layout: aos16\n- tile: 8x4\n"
                 "- dram_bytes_per_launch: 647810560\n")
    assert bench.measured_traffic(1, (4, 8)) == 647810560
    assert bench.measured_traffic(1, (8, 4)) == 647810560
    assert bench.measured_traffic(0, (4, 8)) is None            # other layout
    f.write_text("- kernel_version: render-v0\n- layout: aos16\n- dram_bytes_per_launch: 1\n")
    assert bench.measured_traffic(1, (4, 8)) is None            # other kernel version
    f.write_text(f"- kernel_version: {bench.KERNEL_VERSION}\n- layout: aos16\n- dram_bytes_per_launch: n/a\n")
    assert bench.measured_traffic(1, (4, 8)) is None


def test_job_throughput_counts_every_rank():
    # 2 ranks, 1000 rays per step, 10 steps in 20 ms -> 1.0 Mrays/s
    assert abs(bench.job_throughput(2, 1000, 10, 20.0) - 1.0) < 1e-12
