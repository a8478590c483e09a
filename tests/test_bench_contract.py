"""bench.py's JSON helpers on synthetic profile counters (no GPU): roofline fields and arithmetic."""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def fake_profile(**kw):
    p = dict(launches=100, n_factor=2, ms_factor=10.0, flops_factor=4.0e9, n_sweep=8, ms_sweep=2.0,
             flops_sweep=3.0e8, n_resid=4, ms_resid=0.4, bytes_resid=8.0e7, n_resid32=2, ms_resid32=0.1,
             bytes_resid32=4.0e8)
    p.update(kw)
    return p


def test_dominant_roofline_picks_the_larger_class_and_divides_by_the_peak(bench):
    w = bench.workload("2d")
    r = bench.dominant_roofline(fake_profile(), w, 0, ms_total=20.0, traffic_ok=True)
    assert r["kernel"].startswith("k_factor")
    assert r["achieved"] == pytest.approx(4.0e9 / 5e-3 / 1e12, rel=1e-3)
    assert r["frac"] == pytest.approx(r["achieved"] / bench.FP64_PEAK_TFLOPS, rel=1e-3)
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["traffic"] == round(bench.NCU_BYTES_PER_SUBVOLUME[("factor", 0)] * 4096)
    # sweep dominant: the counters hold whole sweeps (all colours); FP64 against the FP64 pipe
    r = bench.dominant_roofline(fake_profile(ms_sweep=40.0), w, 0, ms_total=60.0, traffic_ok=False)
    assert r["kernel"].startswith("k_sweep_fine")
    assert r["achieved"] == pytest.approx(3.0e8 / 5e-3 / 1e12, rel=1e-3)
    assert r["peak"] == pytest.approx(bench.FP64_PEAK_TFLOPS, rel=1e-4)
    assert r["traffic"] is None
    # the complex64 sweep against HBM: every factor once (4096 x 21 blocks x 256 x 8 B at NPAD 96),
    # c in and out and f (8 B per unknown each), V0 (8 B per point)
    r = bench.dominant_roofline(fake_profile(ms_sweep=40.0), w, 1, ms_total=60.0, traffic_ok=False)
    algo = 4096 * 21 * 256 * 8 + 256 * 256 * 6 * 24 + 256 * 256 * 8
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["algorithmic_bytes"] == algo
    assert r["achieved"] == pytest.approx(algo / 5e-3 / 1e9, rel=1e-3)
    assert r["frac"] == pytest.approx(r["achieved"] / bench.hbm_peak()[0], abs=1e-4)


def test_stencil_roofline_is_bytes_over_event_time_against_hbm(bench):
    s = bench.stencil_roofline(fake_profile(), 0)
    peak, note = bench.hbm_peak()
    assert s["bound"] == "hbm" and s["unit"] == "GB/s" and s["peak"] == peak
    assert s["achieved"] == pytest.approx(8.0e7 / 0.4e-3 / 1e9, rel=1e-3)
    assert s["us_per_launch"] == pytest.approx(100.0)
    assert bench.stencil_roofline(fake_profile(n_resid=0), 0) is None
    c = bench.stencil_roofline(fake_profile(), 1, c64=True)
    assert c["achieved"] == pytest.approx(4.0e8 / 0.1e-3 / 1e9, rel=1e-3) and c["launches"] == 2
    assert bench.stencil_roofline(fake_profile(n_resid32=0), 1, c64=True) is None


def test_workloads_named_by_the_bench(bench):
    w = bench.workload("2d")
    assert w.n[:2] == (256, 256) and w.nt == 6 and w.levels == 4 and w.sub[:2] == (4, 4)
    assert (w.nu1, w.nu2, w.trial) == (1, 2, 3)
    assert bench.workload("2d-small").n[:2] == (128, 128)
    for name, n in (("3d", 128), ("3d-mid", 64), ("3d-small", 32)):
        w = bench.workload(name)
        assert w.n == (n, n, n) and w.nt == 4 and w.sub == (4, 4, 4) and bench.default_precision(name) == 1


def test_factor_store_and_l2_note(bench):
    """The factor store the finest sweeps stream: 4096 subvolumes of 21 packed 16 x 16 blocks
    (86 KB complex128, 43 KB complex64) at 256^2 x 6, larger than L2; the dense LU of the square
    form is 96^2 entries; the 1D workload fits in L2 and the line says it is not flushed."""
    w = bench.workload("2d")
    assert bench.finest_factor_store(w, 0) == (4096, 21 * 256 * 16)
    assert bench.finest_factor_store(w, 1) == (4096, 21 * 256 * 8)
    assert bench.finest_factor_store(bench.workload("2d-square"), 0) == (4096, 96 * 96 * 16)
    assert "352 MB" in bench.l2_note(w, 0) and "(> L2)" in bench.l2_note(w, 0)
    assert "fits in L2" in bench.l2_note(bench.workload("1d"), 0)


def test_reference_arm_line(bench):
    """`--impl reference` (the CPU oracle, run here on the 1D workload) prints one JSON line with the
    contract's keys and the same config object as the GPU arm."""
    import json
    import subprocess
    import sys
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "1d",
                          "--steps", "2", "--warmup", "1"], capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "unknowns/s"
    assert d["value"] > 0 and d["higher_is_better"] is True and d["n_gpus"] == 1
    assert d["steps"] == 2 and d["warmup"] == 1
    assert d["config"] == bench.workload_config(bench.workload("1d"), 0, 1)
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_default_line_is_the_3d_workload(bench):
    """No flags: the 3D workload (128^3, K = 4, 4x4x4 subvolumes of 256 unknowns, 2x2x2 on the Galerkin
    levels, 4 levels) in its own arithmetic (FP64 with complex64 local solves); its factor store is
    32768 subvolumes of 136 packed blocks; the oracle times a 32^3 sample of it."""
    w = bench.workload("3d")
    assert w.n == (128, 128, 128) and w.nt == 4 and w.sub == (4, 4, 4) and w.coarse_sub == (2, 2, 2)
    assert w.levels == 4 and (w.nu1, w.nu2, w.coarse_nu, w.trial) == (1, 2, (1, 0), 3)
    assert bench.default_precision("3d") == 1 and bench.default_precision("2d") == 0
    assert bench.finest_factor_store(w, 1) == (32768, 136 * 256 * 8)
    sample, extrap = bench.oracle_sample(w)
    assert extrap and sample.n == (32, 32, 32) and sample.sub == w.sub and sample.nt == w.nt
    assert bench.oracle_sample(bench.workload("2d")) == (bench.workload("2d"), False)


def test_wide_factor_roofline_against_the_measured_peak(bench):
    """The wide complex64 factorisation dominates: alu-bound against the FP32 peak measured in the run."""
    w = bench.workload("3d")
    r = bench.dominant_roofline(fake_profile(), w, 1, ms_total=20.0, traffic_ok=False, peaks=(1.2, 75.0, 152))
    assert r["kernel"].startswith("k_factor_wide") and r["bound"] == "alu"
    assert r["peak"] == pytest.approx(75.0) and "measured" in r["peak_note"] and "152 SMs" in r["peak_note"]
    assert r["frac"] == pytest.approx(4.0e9 / 5e-3 / 1e12 / 75.0, abs=1e-4)


def test_transfer_roofline_is_bytes_over_event_time(bench):
    p = fake_profile(n_restrict=4, ms_restrict=0.2, bytes_restrict=6.0e8, n_prolong=4, ms_prolong=0.4,
                     bytes_prolong=1.0e9)
    t = bench.transfer_roofline(p)
    peak, _ = bench.hbm_peak()
    assert t["bound"] == "hbm" and t["peak"] == peak
    assert t["restrict"]["achieved"] == pytest.approx(6.0e8 / 0.2e-3 / 1e9, rel=1e-3)
    assert t["prolong_add"]["us_per_launch"] == pytest.approx(100.0)
    assert bench.transfer_roofline(fake_profile(n_restrict=0)) is None
