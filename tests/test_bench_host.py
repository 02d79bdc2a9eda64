"""Host-side logic of bench.py that needs no GPU: the clock record taken during the
timed region, the whole-job throughput and the workload description."""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def row(sm, mx, hw="Not Active", hwt="Not Active", swt="Not Active", cap="Not Active"):
    return "0, %s, %s, 812.50, 0x0000000000000000, %s, %s, %s, %s\n" % (sm, mx, hw, hwt, swt, cap)


def test_clock_summary_median_max_and_no_reasons():
    c = bench.clock_summary([row(2070, 2070), row(2055, 2070), row(1980, 2070)])
    assert c == {"sm_mhz": 2055.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 3}


def test_clock_summary_collects_every_active_reason():
    c = bench.clock_summary([row(2070, 2070, cap="Active"), row(1500, 2070, hwt="Active"),
                             row(2070, 2070)])
    assert c["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]
    assert c["sm_mhz"] == 2070.0


def test_clock_summary_skips_unavailable_fields_and_short_lines():
    c = bench.clock_summary(["garbage\n", row("[N/A]", 2070), row(1900, "[N/A]"), "\n"])
    assert c["samples"] == 2
    assert c["sm_mhz"] == 1900.0 and c["sm_max_mhz"] == 2070.0


def test_clock_summary_without_samples():
    assert bench.clock_summary([]) == {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}


@pytest.mark.parametrize("ws", [1, 2, 8])
def test_job_throughput_counts_every_rank(ws):
    """value = the solves of all ranks / the slowest rank's time (weak scaling)."""
    assert bench.job_throughput(ws, 1000, 10, 5.0) == pytest.approx(ws * 1000 * 10 / 5e-3)


def test_workload_config_names_the_workload():
    cfg = bench.workload_config()
    assert "64^3" in cfg["workload"] and "LQ_8" in cfg["workload"]


def test_clocks_stop_reads_the_sampler_output_and_cleans_up():
    """Clocks.stop with a stand-in sampler process (no nvidia-smi here): the rows it
    wrote are summarised and the temporary file is removed; without a sampler the
    record says so."""
    import subprocess
    c = bench.Clocks(0)
    line = row(2070, 2070, cap="Active").strip()
    c.p = subprocess.Popen([sys.executable, "-c", "import time; print(%r, flush=True); time.sleep(30)" % line],
                           stdout=c.f)
    name = c.f.name
    for _ in range(100):
        if os.path.getsize(name) > 0:
            break
        import time
        time.sleep(0.05)
    got = c.stop()
    assert got["reasons"] == ["sw_power_cap"] and got["samples"] == 1
    assert not os.path.exists(name)
    c = bench.Clocks(0)
    name = c.f.name
    assert c.stop()["reasons"] == ["nvidia-smi unavailable"]
    assert not os.path.exists(name)


def test_a_failing_secondary_report_keeps_the_line():
    def boom(x):
        raise RuntimeError("no network (%d)" % x)
    assert bench.guarded(boom, 3) == {"error": "RuntimeError: no network (3)"}
    assert bench.guarded(lambda a, b: {"v": a + b}, 1, 2) == {"v": 3}


def test_parity_report_on_known_arrays():
    """The parity object of the bench line: a planted error of 1e-6 on a node of
    value 1 (group max 1) and of 1e-12 on a node of value 1e-9 (group max 2)."""
    import numpy as np
    ref = np.ones((2, 3, 8))
    ref[1] *= 2.0
    ref[1, 0, 0] = 1e-9
    phi = ref.copy()
    phi[0, 1, 2] += 1e-6
    phi[1, 0, 0] += 1e-12
    r = bench.parity_report(phi, ref)
    assert r["maxnorm_rel"] == pytest.approx(1e-6)
    assert r["point_rel_at_1pct"] == pytest.approx(1e-6)
    # the tiny node: 1e-12 / (1e-9 + 2e-8) under the 1e-8 floor (larger than the other
    # node's 1e-6), 1e-12 / (1e-9 + 2e-6) under 1e-6 (smaller)
    assert r["point_rel_floored_1e-8max"] == pytest.approx(1e-12 / 2.1e-8)
    assert r["point_rel_floored_1e-6max"] == pytest.approx(1e-6 / (1 + 1e-6))
    assert r["mean_rel_floored_1e-8max"] == pytest.approx(0.5 * (1e-6 / (1 + 1e-8) / 24 + 1e-12 / 2.1e-8 / 24))
