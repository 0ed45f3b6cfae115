"""The benchmark's roofline arithmetic (host only).

The bench line's `roofline` and `mixed.roofline` objects divide an
algorithmic count by a live event time.  These checks pin that arithmetic
against hand-written closed forms for the 1024-walker 2^21 step, so a
changed flop model, a dropped factor of two or a swapped unit shows up
without a GPU.
"""
import json
import os

import pytest

import bench


def test_flop_model_counts():
    # 24 per harmonic (rotation 6, three quadratic amplitudes 12, three
    # accumulations 6) and 172 per sample
    assert bench.flop_model(20) == 24 * 20 + 172 == 652
    assert bench.flop_model(10) == 412
    assert bench.flop_model(1) - bench.flop_model(0) == 24


def test_derived_peaks():
    # 152 SMs x (2 FP64 | 128 FP32) FMA per clock x 2 flops x 2.07 GHz
    assert bench.FP64_PEAK_TFLOPS == pytest.approx(1.258560, rel=1e-12)
    assert bench.FP32_PEAK_TFLOPS == pytest.approx(80.54784, rel=1e-12)


def test_mixed_roofline_arithmetic(monkeypatch):
    monkeypatch.setattr(bench, "hbm_peak_gbs", lambda: (6687.1, "measured"))
    steps, walkers, n, n_max = 5, 1024, 1 << 21, 20
    kt = {"wave": (26.4 * steps, steps), "fft_pass1": (7.84 * steps, steps), "fft_pass2_ip": (6.68 * steps, steps),
          "orbit": (3.7 * steps, 2 * steps)}
    r = bench.mixed_roofline(kt, walkers, n, n_max, steps)
    samples = walkers * n
    wave = r["k2_wave_mixed"]
    assert wave["achieved"] == pytest.approx(652 * samples / 26.4e-3 / 1e12, rel=1e-12)
    assert wave["frac"] == pytest.approx(wave["achieved"] / 80.54784, rel=1e-12)
    assert 0.6 < wave["frac"] < 0.7
    p1, p2 = r["k3_pass1<float2>"], r["k4_pass2_ip_r8"]
    # pass 1 reads and writes the 8-byte series, pass 2 reads it once
    assert p1["achieved"] == pytest.approx(16 * samples / 7.84e-3 / 1e9, rel=1e-12)
    assert p2["achieved"] == pytest.approx(8 * samples / 6.68e-3 / 1e9, rel=1e-12)
    assert p1["frac"] == pytest.approx(p1["achieved"] / 6687.1, rel=1e-12)
    assert (p1["unit"], p2["unit"], wave["unit"]) == ("GB/s", "GB/s", "TFLOP/s")
    assert p1["ms_per_step"] == pytest.approx(7.84)
    # kernels that did not run are left out
    assert bench.mixed_roofline({"wave": (0.0, 0)}, walkers, n, n_max, steps) == {}


def test_hbm_peak_source(tmp_path, monkeypatch):
    f = tmp_path / "peaks.json"
    f.write_text(json.dumps({"hbm_gbs": 6687.1}))
    monkeypatch.setattr(bench, "MEASURED_PEAKS", str(f))
    assert bench.hbm_peak_gbs() == (6687.1, "measured")
    monkeypatch.setattr(bench, "MEASURED_PEAKS", os.path.join(str(tmp_path), "missing.json"))
    assert bench.hbm_peak_gbs() == (6800.0, "fallback")


def test_fp64_traffic_per_sample():
    # ncu DRAM bytes of the 64-walker 2^20 capture, per sample: the 16-byte
    # FP64 series it writes plus per-segment records
    per = bench.K2_F64_DRAM_BYTES_PER_SAMPLE
    assert 16.0 < per < 16.2
