"""Host logic of bench.py that decides whether a measurement is kept: the
clock record sampled during the timed region (throttle reasons, medians) and
the source-hash gate on the committed DRAM-traffic figure.  No GPU needed."""
import os
import shutil
import types

import bench

HASHED = ("step_kernel.cuh", "step_wide.cuh", "step_staged.cuh", "step_window.cuh", "async_copy.cuh",
          "step_launch.cuh", "cld_internal.cuh")


def _sampler(tmp_path, lines):
    s = bench.ClockSampler(name="clocks_test.csv")
    s.path = str(tmp_path / "clocks_test.csv")
    with open(s.path, "w") as f:
        f.write("\n".join(lines) + "\n")
    s.proc = object()  # stands for a sampler that ran
    return s


def test_clock_summary_medians_and_power_cap(tmp_path):
    na = "Not Active"
    rows = ["0, %d, 2070, %d, 0x0000000000000004, %s, %s, %s, %s" % (mhz, w, na, na, na, cap)
            for mhz, w, cap in ((2070, 900, na), (2055, 1350, "Active"), (2070, 910, na))]
    s = _sampler(tmp_path, ["garbage line", "0, [N/A], 2070, 1, x, a, b, c, d"] + rows)
    r = s.summary()
    assert r["sm_mhz"] == 2070.0 and r["sm_min_mhz"] == 2055.0 and r["sm_max_mhz"] == 2070.0
    assert r["samples"] == 3 and r["power_w"] == 910.0
    assert r["reasons"] == ["sw_power_cap"]


def test_clock_summary_flags_every_slowdown(tmp_path):
    s = _sampler(tmp_path, ["0, 1200, 2070, 700, 0x68, Active, Active, Active, Not Active"])
    assert s.summary()["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]


def test_clock_summary_without_samples_or_sampler(tmp_path):
    assert _sampler(tmp_path, ["header only"]).summary()["reasons"] == ["no samples"]
    s = bench.ClockSampler(name="clocks_none.csv")
    s.failure = "nvidia-smi unavailable: not found"
    r = s.summary()
    assert r["sm_mhz"] is None and r["reasons"] == ["nvidia-smi unavailable: not found"]


def _tree(tmp_path, traffic_hash):
    csrc = tmp_path / "paper_1503_06394_gb300" / "csrc"
    csrc.mkdir(parents=True)
    src = os.path.join(bench.ROOT, "paper_1503_06394_gb300", "csrc")
    for name in HASHED:
        shutil.copy(os.path.join(src, name), csrc / name)
    (tmp_path / "profiles").mkdir()
    with open(tmp_path / "profiles" / "step_kernel_config2_traffic.md", "w") as f:
        f.write("# traffic\n\nstep_kernels_sha256: %s\ntraffic_bytes_per_launch_v6: 123456\n" % traffic_hash)
    return csrc


def test_traffic_is_reported_only_for_the_captured_sources(tmp_path, monkeypatch):
    want = bench.step_sources_sha256(os.path.join(bench.ROOT, "paper_1503_06394_gb300", "csrc"))
    csrc = _tree(tmp_path, want)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    args = types.SimpleNamespace(config=2, d=None, dtype="f32")
    assert bench.profiled_traffic(args, None, 6) == 123456.0
    assert bench.profiled_traffic(args, None, 5) is None  # no figure for that variant
    for other in (dict(config=1), dict(d=1000), dict(dtype="bf16")):
        assert bench.profiled_traffic(types.SimpleNamespace(**{**vars(args), **other}), None, 6) is None
    # a change outside the StepArgs block of the internal header keeps the figure
    with open(csrc / "cld_internal.cuh", "a") as f:
        f.write("\n// trailing comment\n")
    assert bench.profiled_traffic(args, None, 6) == 123456.0
    # a change to a step kernel's source drops it
    with open(csrc / "step_staged.cuh", "a") as f:
        f.write("\n// edited\n")
    assert bench.profiled_traffic(args, None, 6) is None
