"""Host-side pieces of bench.py's roofline that need no GPU: the algorithmic
byte table, the derived FP32 peak (SM count read from the device), and the committed ncu summaries the bench
reads its DRAM traffic from (each names the command that made it, runs only
committed entry points and leaves the GPU clocks alone)."""

import os
import re
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

FP32, DF, MASK = 4.0, 8.0, 0.125


def test_algorithmic_bytes_follow_from_the_vectors_each_class_moves():
    b = bench.ALGO_BYTES_PER_VALUE
    assert b["oras_fine"] == FP32 + FP32 + MASK + FP32             # read x, b, mask; write x
    assert b["residual_fine"] == DF + FP32 + MASK + DF + FP32      # read u, e, mask; write u, r
    assert b["prolong_fine"] == FP32 + FP32 + FP32 / 4 + MASK + FP32   # read x, b, e_H; write x
    assert b["restrict_fine"] == FP32 + FP32 + MASK + FP32 / 4     # read x, b, mask; write b_H


def test_derived_fp32_peak(monkeypatch):
    """SMs from the device attribute x 128 FP32 lanes x 2 flop/FMA x the
    maximum SM clock (a stand-in device reports 148 SMs)."""
    import types
    torch = __import__("torch")
    props = types.SimpleNamespace(multi_processor_count=148)
    monkeypatch.setattr(torch.cuda, "get_device_properties", lambda d: props)
    peak, src = bench.fp32_peak_tflops(0, {"sm_max_mhz": 2032.0})
    assert abs(peak - 148 * 128 * 2 * 2.032e9 / 1e12) < 1e-9
    assert 76.9 < peak < 77.1
    assert "148 SMs" in src and "2032 MHz" in src
    peak, src = bench.fp32_peak_tflops(0, {})
    assert 76.9 < peak < 77.1 and "fallback" in src


def test_profile_summaries_carry_traffic_and_their_commands():
    prof = os.path.join(ROOT, "profiles")
    for name in bench.ALGO_BYTES_PER_VALUE:
        path = os.path.join(prof, f"{name}_4k_rgb.md")
        assert os.path.exists(path), path
        text = open(path).read()
        m = re.search(r"^traffic_bytes_per_launch: (\d+)$", text, re.M)
        assert m, path
        traffic = int(m.group(1))
        # within a factor of two of the algorithmic bytes of one 4K RGB launch
        algo = bench.ALGO_BYTES_PER_VALUE[name] * bench.H4K * bench.W4K * 3
        assert 0.5 * algo < traffic < 2.0 * algo, (name, traffic, algo)
    for fn in sorted(os.listdir(prof)):
        text = open(os.path.join(prof, fn)).read()
        cmds = [ln for ln in text.splitlines() if ln.startswith("ncu ")]
        assert cmds, fn
        for ln in cmds:
            assert "--clock-control none" in ln, fn
        for mod in re.findall(r"python -m ([\w.]+)", text):
            assert os.path.exists(os.path.join(ROOT, *mod.split(".")) + ".py"), (fn, mod)
        for script in re.findall(r"python (\w+\.py)", text):
            assert os.path.exists(os.path.join(ROOT, script)), (fn, script)
