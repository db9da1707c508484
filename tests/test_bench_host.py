"""Host logic of bench.py that decides what a measurement reports, without a GPU: the
parser of the nvidia-smi clock samples (median SM clock, maximum, throttle reasons seen) and
the rule that the ncu DRAM traffic of the frame kernel is reported only for the kernel
source it was captured on."""
from __future__ import annotations

import hashlib
import os

import pytest

import bench


class _FakeProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0

    def kill(self):
        pass


def _sampler_over(tmp_path, lines):
    cs = bench.ClockSampler(0, enabled=False)
    path = tmp_path / "clocks.csv"
    path.write_text("\n".join(lines) + "\n")
    cs.path = str(path)
    cs.f = open(os.devnull, "w")
    cs.proc = _FakeProc()
    return cs


def test_clock_samples_median_max_and_reasons(tmp_path):
    cs = _sampler_over(tmp_path, [
        "0, 2070, 2070, 812.3, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
        "0, [N/A], 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ])
    out = cs.stop()
    assert out == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}


def test_clock_samples_thermal_and_hw_slowdown_are_reported(tmp_path):
    cs = _sampler_over(tmp_path, [
        "0, 1500, 2070, 1400.0, 0x48, Active, Active, Not Active, Not Active",
        "0, 1600, 2070, 1400.0, 0x20, Not Active, Not Active, Active, Not Active",
    ])
    out = cs.stop()
    assert out["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]
    assert out["sm_mhz"] == 1550.0


def test_clock_samples_absent():
    assert bench.ClockSampler(0, enabled=False).stop() is None


def test_frame_traffic_only_for_the_captured_source(monkeypatch):
    src = os.path.join(bench.ROOT, "paper_1609_04104_gb300", "csrc", "tts_frame.cu")
    h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    monkeypatch.setattr(bench, "FRAME_TRAFFIC_SRC_SHA", h)
    assert bench.frame_traffic() == bench.FRAME_TRAFFIC_BYTES
    monkeypatch.setattr(bench, "FRAME_TRAFFIC_SRC_SHA", "0" * 16)
    assert bench.frame_traffic() is None


@pytest.mark.parametrize("s", [1, 32, 256])
def test_frame_flops_grow_with_the_line_count(s):
    """More acquired lines, more work; the K MM iterations scale the per-iteration part."""
    a = bench.frame_flops(256, 256, 32, 3, s)
    b = bench.frame_flops(256, 256, 32, 3, s + 1)
    k1, k2 = bench.frame_flops(256, 256, 32, 1, s), bench.frame_flops(256, 256, 32, 2, s)
    assert b > a > 0
    assert abs((a - k2) - (k2 - k1)) < 1e-6 * a


def _profile_bench_commands():
    """(summary, bench.py arguments) pairs from profiles/commands.txt."""
    cmds = []
    for line in open(os.path.join(bench.ROOT, "profiles", "commands.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        name, args = (x.strip() for x in line.split("|", 1))
        cmds.append((name, args))
    return cmds


def test_profile_commands_parse_with_the_bench(monkeypatch):
    """Every bench command listed for the summaries in profiles/ is accepted by bench.py's own
    argument parser (a renamed or removed flag would leave a summary that cannot be re-run),
    and every summary has its command listed."""
    import glob
    import shlex
    cmds = _profile_bench_commands()
    summaries = {os.path.basename(p) for p in glob.glob(os.path.join(bench.ROOT, "profiles", "*.md"))}
    assert summaries and summaries <= {name for name, _ in cmds}
    for name, args in cmds:
        assert name in summaries, name
        monkeypatch.setattr("sys.argv", ["bench.py", *shlex.split(args)])
        bench.parse()


def test_oracle_single_thread_timing_runs_in_its_own_process():
    """The one-core oracle timing of the cpu_baseline leg: a fresh interpreter with BLAS on
    one thread, no CUDA; one fully sampled frame gives a positive rate."""
    v = bench.oracle_single_thread(1)
    assert 0.0 < v < 100.0
