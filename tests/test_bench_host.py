"""Host-side pieces of bench.py that decide whether a measurement stands: the
clock and throttle-reason summary of the nvidia-smi samples, the whole-job
rate, and the per-step units of the metric."""
import importlib.util
import os

import pytest

from paper_1804_02883_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def test_clock_summary_reads_samples_and_reasons(tmp_path):
    b = _bench()
    f = tmp_path / "clocks.csv"
    f.write_text("0, 2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n"
                 "0, 1965, 2070, 1400.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active\n"
                 "[N/A]\n"
                 "0, 2070, 2070, 950.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n")
    c = b.Clocks(0)
    c.proc, c.path = object(), str(f)
    s = c.summary()
    assert s == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    assert not f.exists()  # the sample file is removed


def test_clock_summary_flags_thermal_slowdown(tmp_path):
    b = _bench()
    f = tmp_path / "clocks.csv"
    f.write_text("0, 1500, 2070, 1200.0, 0x0000000000000040, Not Active, Active, Not Active, Not Active\n")
    c = b.Clocks(0)
    c.proc, c.path = object(), str(f)
    assert c.summary()["reasons"] == ["hw_thermal_slowdown"]


def test_clock_summary_without_nvidia_smi():
    b = _bench()
    assert b.Clocks(0).summary()["reasons"] == ["nvidia-smi unavailable"]


def test_units_and_whole_job_rate():
    b = _bench()
    runs = W.channel_256x512()
    # site.contour-step updates of one step: 2 chains x 2 solves per run
    assert b.units_per_step(runs) == 4 * 512 * 256 * 64 * 4
    assert b.sites_per_step(runs) == 4 * 512 * 256
    # K steps on each of N ranks in T seconds (the slowest rank's time)
    assert b.job_rate(100.0, 10, 2, 0.5) == pytest.approx(100.0 * 10 * 2 / 0.5)
    assert b.max_over_ranks(3.5) == 3.5  # no process group: the value itself


def test_precision_errors_of_the_mixed_path():
    import numpy as np

    b = _bench()
    rng = np.random.default_rng(0)
    ref_phi = [0.2 + 1e-3 * rng.standard_normal((3, 4, 8)) for _ in range(2)]
    ref_vel = [np.zeros((2, 4, 8)), 1e-2 * rng.standard_normal((2, 4, 8))]

    class H:
        def __init__(self, dphi, dvel):
            self.dphi, self.dvel = dphi, dvel

        def densities(self, k):
            return ref_phi[k] + self.dphi, None

        def velocity(self, k):
            return ref_vel[k] + self.dvel

    e = b.precision_errors(H(2e-7, 1e-6), H(0.0, 0.0), 2, np)
    for k in range(2):
        assert e["phi_rel"][k] == pytest.approx(2e-7 / np.abs(ref_phi[k]).max(), rel=1e-6)
        fl = max(np.abs(ref_phi[k][i] - ref_phi[k][i].mean()).max() for i in range(3))
        assert e["phi_rel_fluctuation"][k] == pytest.approx(2e-7 / fl, rel=1e-6)
    assert e["velocity_rel"][0] is None  # no flow in the reference: no relative error
    assert e["velocity_rel"][1] == pytest.approx(1e-6 / np.abs(ref_vel[1]).max(), rel=1e-6)
