"""Host-side logic of bench.py (no GPU): the roofline arithmetic, the whole-job rate of replicas, the peak
source, the choice of the oracle sample and the parsing of the clock samples taken during the timed
region."""
import json
import os

import bench


def test_roofline_fraction_is_achieved_over_measured_peak():
    pk = {"hbm_gbs": 6780.0, "source": "measured (MEASURED_PEAKS.json)"}
    r = bench.roofline("k", 6.78e9, 1000.0, 3, pk, alg_flops=2.0e12)
    assert abs(r["achieved"] - 6.78) < 1e-12  # 6.78 GB in one second
    assert abs(r["frac"] - 6.78 / 6780.0) < 1e-15
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["peak"] == 6780.0
    assert r["launches_per_step"] == 3 and r["traffic"] is None
    assert abs(r["flop_view"]["alg_tflops"] - 2.0) < 1e-12


def test_replica_rate_is_the_whole_job_over_the_slowest_rank():
    # four replicas of 1 M cells each, the slowest step 10 ms: 400 M cells/s for the job
    assert abs(bench.replica_rate(1.0e6, 10.0, 4) - 400.0) < 1e-9
    assert bench.max_over_ranks([3.0, 5.0], 1) == [3.0, 5.0]


def test_peaks_come_from_the_measured_file_else_the_stated_fallback(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    pk = bench.peaks()
    assert pk["hbm_gbs"] == 6800.0 and pk["source"].startswith("fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6123.0, "bf16_tflops": 1800.0}))
    pk = bench.peaks()
    assert pk["hbm_gbs"] == 6123.0 and pk["source"].startswith("measured")


def test_oracle_sample_is_the_smallest_instance_of_each_level_count():
    params = [{"levels": k} for k in (1, 2, 3, 3, 1, 2, 3, 3)]
    cells = [50, 40, 300, 200, 10, 90, 100, 400]
    # level 1: instance 4 (10 cells); level 2: instance 1 (40); level 3: instances 6 and 3 (100, 200)
    assert bench.batch_sample(params, cells) == [1, 3, 4, 6]


class _Done:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def test_clock_summary_reports_median_clock_and_throttle_reasons(tmp_path):
    cs = bench.ClockSampler(0)
    cs.path = str(tmp_path / "clocks.csv")
    rows = [
        "0, 2070, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 2070, 2070, 1100.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 1980, 2070, 1300.0, 0x8, Active, Not Active, Not Active, Not Active",
    ]
    with open(cs.path, "w") as fh:
        fh.write("\n".join(rows) + "\n")
    cs.proc = _Done()
    s = cs.summary()
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["hw_slowdown", "sw_power_cap"]
    os.remove(cs.path)
