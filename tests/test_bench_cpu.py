"""Host logic of bench.py that needs no GPU: the clock record keeps only the
nvidia-smi samples taken inside the timed region, and every workload names its
default step count."""

import datetime
import importlib.util
import os
import time

from tests.conftest import ROOT


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _line(t, mhz, cap):
    ts = datetime.datetime.fromtimestamp(t).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    return (f"{ts}, 0, GPU-test, {mhz}, 2070, 1200.0, 0x4, Not Active, Not Active, Not Active, "
            f"{'Active' if cap else 'Not Active'}\n")


def test_clock_record_keeps_samples_inside_the_timed_region():
    b = _bench()
    c = b.ClockSampler("GPU-test")
    now = time.time()
    c.t0, c.t1 = now - 1.0, now
    for t, mhz, cap in ((now - 1.4, 2070, False), (now - 0.7, 1600, True), (now - 0.3, 1500, True),
                        (now + 0.2, 2070, False)):
        c.tmp.write(_line(t, mhz, cap))
    out = c.summary()
    assert out["samples"] == 2 and out["sm_mhz"] == 1550 and out["reasons"] == ["sw_power_cap"]
    assert out["sm_max_mhz"] == 2070 and "note" not in out


def test_clock_record_of_a_region_shorter_than_the_interval():
    b = _bench()
    c = b.ClockSampler("GPU-test")
    now = time.time()
    c.t0, c.t1 = now - 0.05, now
    c.tmp.write(_line(now - 0.5, 2070, False))
    c.tmp.write(_line(now + 0.2, 1900, False))
    out = c.summary()
    assert out["samples"] == 2 and "note" in out and out["reasons"] == []


def test_every_workload_has_default_steps():
    b = _bench()
    for name, wl in b.WORKLOADS.items():
        assert isinstance(wl.get("steps"), int) and wl["steps"] >= 3, name


def test_traffic_key_ignores_comments_only():
    b = _bench()
    code = "int f(int x) {  // doubles\n  /* block\n     comment */\n  return 2 * x;\n}\n"
    same = "// header\nint f(int x) {\n\n  return 2 * x;  // changed comment\n}\n"
    other = "int f(int x) {\n  return 3 * x;\n}\n"
    assert b._code_only(code) == b._code_only(same)
    assert b._code_only(code) != b._code_only(other)


def test_vs_fp32_compares_each_split_form_with_the_fp32_path():
    """The default line's FP32 comparison: speedups over the plain FP32 path and
    each form's error against the oracle, from the extras' own keys."""
    b = _bench()
    assert b.vs_fp32({"value": 30.0}) is None  # no FP32 extra (--no-extras)
    line = {"value": 30.0, "vs_oracle": {"rel_fro": 1e-3},
            "precise": {"value": 20.0, "vs_oracle": {"rel_fro": 8e-5}},
            "fp32": {"value": 3.0, "vs_oracle": {"rel_fro": 5e-6}}}
    v = b.vs_fp32(line)
    assert v["speedup_split"] == 10.0 and v["speedup_precise"] == 20.0 / 3.0
    assert (v["split_rel_fro"], v["precise_rel_fro"], v["fp32_rel_fro"]) == (1e-3, 8e-5, 5e-6)
    assert any(name == "plain-r15-fp32-n8192-k3375" for _, name, _ in b.EXTRAS)
    assert b.WORKLOADS["plain-r15-fp32-n8192-k3375"]["n"] == b.WORKLOADS[b.DEFAULT_WORKLOAD]["n"]
