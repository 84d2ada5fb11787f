"""Host logic of the benchmark on CPU: its per-kernel byte model agrees with
the oracle's access model (Table 2, Sec. 5.1) for every stencil and storage,
the clock sampler turns nvidia-smi rows into the median clock and the active
throttle reasons, a stale ncu traffic record is dropped, and odd step counts
are refused."""
import sys

import pytest

import bench
import oracle as O


@pytest.mark.parametrize("q", [19, 27])
@pytest.mark.parametrize("b_pdf", [4, 2])
def test_pair_bytes_equal_the_access_model(q, b_pdf):
    nf = 1000
    pair = bench.algorithmic_bytes(nf, b_pdf, q, 0) + bench.algorithmic_bytes(nf, b_pdf, q, 1)
    assert pair / (2 * nf) == O.access_bytes(q, b_pdf, bench.B_IDX, "aa", "sparse", "gpu")
    # even step: a read and a write of every population, no index
    assert bench.algorithmic_bytes(nf, b_pdf, q, 0) == nf * 2 * q * b_pdf
    # odd step: the same plus one index per non-rest direction
    assert bench.algorithmic_bytes(nf, b_pdf, q, 1) - bench.algorithmic_bytes(nf, b_pdf, q, 0) == nf * (q - 1) * 4


def test_headline_ceiling_matches_the_paper_byte_count():
    # D3Q19 FP32 with int32 indices: 188 B per fluid update
    assert bench.algorithmic_bytes(1, 4, 19, 0) + bench.algorithmic_bytes(1, 4, 19, 1) == 2 * 188


class _FakeProc:
    def __init__(self, text):
        self.text = text
        self.terminated = False

    def terminate(self):
        self.terminated = True

    def communicate(self, timeout=None):
        return self.text, ""


def _row(sm, smax=2070, power=900.5, hw="Not Active", sw_power="Not Active"):
    return f"0, {sm}, {smax}, {power}, 0x0, {hw}, Not Active, Not Active, {sw_power}"


def test_clock_sampler_median_and_reasons():
    s = bench.ClockSampler(0)
    s.proc = _FakeProc("\n".join([_row(2070), _row(2055, sw_power="Active"), _row(1980), "garbage"]) + "\n")
    out = s.stop()
    assert s.proc.terminated
    assert out["sm_mhz"] == 2055.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"] and out["samples"] == 3
    assert out["power_w_max"] == 900.5


def test_clock_sampler_reports_hardware_slowdown():
    s = bench.ClockSampler(0)
    s.proc = _FakeProc(_row(1500, hw="Active") + "\n" + _row(2070) + "\n")
    assert s.stop()["reasons"] == ["hw_slowdown"]


def test_clock_sampler_without_samples():
    s = bench.ClockSampler(0)
    assert s.stop() is None                     # never started
    s.proc = _FakeProc("")
    assert s.stop()["reasons"] == ["no samples"]


class _Dom:
    def __init__(self, nf):
        self.n_fluid = nf


def test_stale_traffic_record_is_dropped(monkeypatch):
    doms = [(0.5, None, _Dom(1000)), (0.7, None, _Dom(3000))]
    monkeypatch.setattr(bench, "kernel_digest", lambda: "not-the-recorded-digest")
    assert bench.traffic_for("aa_odd", doms) is None


def test_current_traffic_record_scales_by_mean_cells(monkeypatch, tmp_path):
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "ncu_traffic.json").write_text(
        '{"source_digest": "d1", "kernels": {"aa_odd": {"dram_bytes_per_cell": 210.5}}}')
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_digest", lambda: "d1")
    doms = [(0.5, None, _Dom(1000)), (0.7, None, _Dom(3000))]
    assert bench.traffic_for("aa_odd", doms) == round(210.5 * 2000)
    assert bench.traffic_for("aa_even", doms) is None


def test_traffic_record_follows_the_storage(monkeypatch, tmp_path):
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "ncu_traffic.json").write_text(
        '{"source_digest": "d1", "kernels": {"aa_odd_kernel": {"dram_bytes_per_cell": 200.0},'
        ' "fp16_aa_odd_kernel": {"dram_bytes_per_cell": 130.0}}}')
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_digest", lambda: "d1")
    doms = [(0.5, None, _Dom(1000))]
    assert bench.traffic_for(bench.traffic_key("fp32", "aa_odd_kernel"), doms) == 200000
    assert bench.traffic_for(bench.traffic_key("fp16", "aa_odd_kernel"), doms) == 130000
    assert bench.traffic_key("bf16", "aa_odd_kernel") is None
    assert bench.traffic_for(bench.traffic_key("bf16", "aa_odd_kernel"), doms) is None


def test_committed_traffic_record_names_the_benchmarked_kernels():
    import json
    with open(bench.os.path.join(bench.ROOT, "profiles", "ncu_traffic.json")) as f:
        rec = json.load(f)
    for storage in ("fp32", "fp16"):
        for k in ("aa_even_kernel", "aa_odd_kernel"):
            assert bench.traffic_key(storage, k) in rec["kernels"]


def test_odd_lbm_step_count_is_refused(monkeypatch):
    monkeypatch.setattr(sys, "argv", ["bench.py", "--lbm-steps", "7"])
    with pytest.raises(SystemExit):
        bench.parse()
    monkeypatch.setattr(sys, "argv", ["bench.py", "--porosities", "0.3,0.9"])
    a = bench.parse()
    assert a.porosities == (0.3, 0.9) and a.gpus == 1 and a.warmup >= 3


def test_reference_arm_samples_every_domain_of_the_workload(monkeypatch):
    # a tiny sweep: the reference line carries our arm's workload and metric,
    # and its steps cycle through every porosity of the sweep
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--size", "16", "--porosities", "0.5,0.7",
                                      "--steps", "2", "--warmup", "1"])
    a = bench.parse()
    out = bench.run_reference(a)
    assert out["impl"] == "reference" and out["metric"] == bench.METRIC and out["unit"] == bench.UNIT
    assert out["config"]["workload"] == bench.workload_name(a)
    assert "blocks of 1/1" in out["config"]["sample"] and "0.5/0.7" in out["config"]["sample"]
    assert out["value"] > 0
    assert out["e2e"]["h2d_bytes_per_step"] == 0 and out["cpu_baseline"]["kind"] == "oracle"


def test_cpu_baseline_covers_every_domain(monkeypatch):
    monkeypatch.setattr(sys, "argv", ["bench.py", "--size", "16", "--porosities", "0.5,0.7", "--cpu-seconds", "0"])
    a = bench.parse()
    out = bench.cpu_baseline(a)
    assert out["kind"] == "oracle" and out["value"] > 0 and out["cores"] >= 1
    assert "4 LBM steps" in out["sample"] and "0.5/0.7" in out["sample"]     # one 2-step run per domain
