"""Host-side logic of the benchmark, on the CPU with fakes: the clock sampler's reduction of
nvidia-smi lines and of NVML samples (median SM clock, maximum, active slowdown reasons), the
algorithmic bytes of the field clearing, and the kernels-per-step count the step graph is checked
against on the GPU."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


class _Proc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0

    def kill(self):
        pass


class _Thread:
    def join(self, timeout=None):
        pass


def _smi_line(sm, smax, hw="Not Active", hw_th="Not Active", sw_th="Not Active", cap="Not Active"):
    return "0, %s, %s, 900.5, 0x0, %s, %s, %s, %s" % (sm, smax, hw, hw_th, sw_th, cap)


def test_nvidia_smi_lines_reduce_to_median_max_and_reasons():
    s = bench.ClockSampler(0)
    s.proc, s.t = _Proc(), _Thread()
    s.lines = [_smi_line(2070, 2070), _smi_line(1980, 2070, cap="Active"), _smi_line(2070, 2070),
               "garbage line", "0, [N/A], 2070, 1, 0x0, a, b, c, d", _smi_line(2055, 2070)]
    r = s.stop()
    # median of 2070, 1980, 2070, 2055 (the unparsable lines are skipped)
    assert r["sm_mhz"] == 2062.5 and r["sm_max_mhz"] == 2070.0 and r["samples"] == 4
    assert r["reasons"] == ["sw_power_cap"]
    assert "nvidia-smi" in r["source"]


def test_nvidia_smi_thermal_and_hw_slowdowns_are_reported():
    s = bench.ClockSampler(0)
    s.proc, s.t = _Proc(), _Thread()
    s.lines = [_smi_line(1500, 2070, hw="Active"), _smi_line(1400, 2070, hw_th="Active", sw_th="Active")]
    r = s.stop()
    assert r["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]
    assert r["sm_mhz"] == 1450.0


def test_no_sampler_reports_unavailable():
    s = bench.ClockSampler(0)
    r = s.stop()
    assert r["sm_mhz"] is None and r["reasons"] == ["nvidia-smi unavailable"]


class _FakeNvml:
    max_mhz = 2070.0

    def close(self):
        self.closed = True


def test_nvml_samples_reduce_to_median_and_decoded_reasons():
    s = bench.ClockSampler(0)
    s.nvml, s.t = _FakeNvml(), _Thread()
    bits = dict(bench._Nvml.REASONS)
    # the event-reason mask's other bits (idle, applications clocks, ...) are not slowdowns
    s.samples = [(2070.0, 0x1), (2070.0, bits["sw_power_cap"]), (1995.0, 0x2), (2070.0, 0)]
    r = s.stop()
    assert r["sm_mhz"] == 2070.0 and r["sm_max_mhz"] == 2070.0 and r["samples"] == 4
    assert r["reasons"] == ["sw_power_cap"]
    assert s.nvml.closed
    s = bench.ClockSampler(0)
    s.nvml, s.t = _FakeNvml(), _Thread()
    s.samples = [(1200.0, bits["hw_thermal_slowdown"] | bits["hw_slowdown"])]
    assert s.stop()["reasons"] == ["hw_slowdown", "hw_thermal_slowdown"]


def test_nvml_reason_bits_are_distinct_single_bits():
    vals = [b for _, b in bench._Nvml.REASONS]
    assert len(set(vals)) == len(vals) and all(v & (v - 1) == 0 for v in vals)


def test_clear_bytes_counts_the_projected_fields():
    # two interface fields of nz + 1 levels and seven centre fields of nz levels, FP64; with the
    # potential-temperature flux two more centre fields
    nx, ny, nz = 7, 5, 11
    cells = nx * ny
    assert bench.clear_bytes(nx, ny, nz) == 8 * cells * (2 * (nz + 1) + 7 * nz)
    assert bench.clear_bytes(nx, ny, nz, theta=True) - bench.clear_bytes(nx, ny, nz) == 8 * cells * 2 * nz
    # the 256 x 128 x 90 sphere: 213 MB a step; the 128 x 64 x 90 capture case: 53.2 MB
    assert abs(bench.clear_bytes(256, 128, 90) / 1e6 - 212.86) < 0.01
    assert abs(bench.clear_bytes(128, 64, 90) / 1e6 - 53.22) < 0.01


def test_launches_per_step_counts_each_optional_phase_once():
    base = dict(cap_per_column=0, saturation=0, smoothing=0)
    n0 = bench.launches_per_step(base)
    assert bench.launches_per_step(dict(base, cap_per_column=12)) == n0 + 4
    assert bench.launches_per_step(dict(base, saturation=1)) == n0 + 2
    full = dict(cap_per_column=12, saturation=1, smoothing=1)
    # either form: one grid-phase kernel besides the divergence (the smoothing, or the field split
    # / narrowing without it), so both forms launch the same count
    assert bench.launches_per_step(full) == bench.launches_per_step(full, fp32=True) == n0 + 6
    assert bench.launches_per_step(dict(full, smoothing=0)) == bench.launches_per_step(full)
