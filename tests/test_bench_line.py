"""bench.py on CPU: its JSON line from fake measurements, and no undefined names.

The GPU legs of bench.py cannot run here, so the line they print is assembled by a pure
function (bench.assemble_line) that this test drives with made-up timings, checking every
key the bench contract asks for.  A static pass over bench.py (symtable) then checks that
every global name read inside a function is defined at module level or is a builtin, which
catches the class of error (a renamed variable left behind in one leg) that no CPU run of
the bench would reach.
"""
import builtins
import json
import os
import symtable

import bench
import workloads

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def fake_measurements(extras=True):
    w = workloads.workload("cfg3")
    m = {"ms": 1000.0, "launches": 4 * 170, "clocks": {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0,
                                                      "reasons": [], "samples": 5},
         "N": w.ndof, "nvec": w.nvec, "degree": w.degree, "l2_gb": 32.8, "peak": (6802.0, "measured"),
         "traffic": {"bytes_per_launch_full_block": 1.7e10},
         "variants_ms": {"df_residual": 720.0, "fp16_storage": 870.0, "bf16_storage": 900.0,
                         "bfp12_residual": 950.0},
         "kernel": {"blk": 256, "k_ms": 3.5, "step_ms": 4.0, "k16_ms": 4.4, "kbfp_ms": 3.3},
         "residual": {"fp64_ms": 88.0, "df_ms": 17.8}}
    if extras:
        m.update({"fp64_chfsi": {"blk": 256, "f64_ms": 3500.0, "mix_ms": 250.0},
                  "e2e": {"ms": 1200.0, "ne": w.nvec, "h2d": w.nvec * w.ndof * 16, "d2h": w.nvec * w.ndof * 16,
                          "sample": "full workload", "link": {"h2d_gbs": 200.0, "d2h_gbs": 190.0}},
                  "adjoint": {"fp64": {"forward_ms": 1.0, "adjoint_ms": 3.0, "ratio": 3.0}},
                  "bfp_codec": {"12": {"encode_ms": 1.0}},
                  "cpu_baseline": {"value": 3.2e7, "dt": 8.0}})
    return w, m


def test_assembled_line_has_every_key():
    w, m = fake_measurements()
    line = bench.assemble_line(w, 1, 20, 5, m)
    json.dumps(line)                                     # serialisable
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "gpu_launches", "clocks", "roofline",
              "cpu_baseline", "e2e", "variants", "residual", "fp64_chfsi"):
        assert k in line, k
    units = w.ndof * w.nvec * w.degree
    assert abs(line["value"] - units / 1.0) < 1e-6 * line["value"]
    assert line["ms_per_step"] == 1000.0 and line["steps"] == 20 and line["warmup"] == 5
    assert line["higher_is_better"] is True and line["scaling"] == "weak" and line["vs_baseline"] is None
    assert "workload" in line["config"] and "cfg3" in line["config"]["workload"]
    assert "RCF_FP32" in line["config"]["precision"] and "FP64" in line["config"]["precision"]
    rf = line["roofline"]
    assert rf["bound"] == "hbm" and rf["unit"] == "GB/s" and rf["peak_source"] == "measured"
    alg = 32.0 * w.ndof * 256
    assert abs(rf["achieved"] - alg / 3.5e-3 / 1e9) < 1e-6 * rf["achieved"]
    assert abs(rf["frac"] - rf["achieved"] / 6802.0) < 1e-12
    assert rf["traffic"] == 1.7e10
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == 3.2e7 and cb["sample"]
    e = line["e2e"]
    assert e["h2d_bytes_per_step"] == w.nvec * w.ndof * 16 and e["d2h_bytes_per_step"] > 0
    assert abs(e["value"] - units / 1.2) < 1e-6 * e["value"]
    assert line["fp64_chfsi"]["speedup_mixed_over_fp64"] == 14.0
    assert set(line["variants"]) == {"df_residual", "fp16_storage", "bf16_storage", "bfp12_residual"}
    rb = line["roofline_bfp12_step"]
    assert abs(rb["achieved"] - 27.0 * w.ndof * 256 / 3.3e-3 / 1e9) < 1e-6 * rb["achieved"]
    assert abs(rb["frac"] - rb["achieved"] / 6802.0) < 1e-12


def test_assembled_line_scales_with_ranks_and_nulls_stale_traffic():
    w, m = fake_measurements(extras=False)
    m["traffic"] = None
    m["peak"] = (6800.0, "fallback")
    one = bench.assemble_line(w, 1, 3, 3, m)
    two = bench.assemble_line(w, 2, 3, 3, m)
    assert abs(two["value"] - 2 * one["value"]) < 1e-9 * two["value"]
    assert two["config"]["parallelism"] != one["config"]["parallelism"]
    assert one["roofline"]["traffic"] is None and one["roofline"]["peak_source"] == "fallback"
    assert "e2e" not in one and "cpu_baseline" not in one


def test_measured_peak_source():
    v, src = bench.measured_hbm_peak()
    if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")):
        assert src == "measured" and v == json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]
    else:
        assert src == "fallback"


def _undefined_globals(path):
    src = open(path).read()
    top = symtable.symtable(src, path, "exec")
    defined = {s.get_name() for s in top.get_symbols() if s.is_assigned() or s.is_imported()}
    known = defined | set(dir(builtins))
    bad = []

    def walk(tab):
        for ch in tab.get_children():
            if ch.get_type() in ("function", "class"):
                for s in ch.get_symbols():
                    if s.is_referenced() and s.is_global() and s.get_name() not in known:
                        bad.append((ch.get_name(), s.get_name()))
            walk(ch)
    walk(top)
    return bad


def test_bench_reads_no_undefined_name():
    assert _undefined_globals(os.path.join(ROOT, "bench.py")) == []
    assert _undefined_globals(os.path.join(ROOT, "__graft_entry__.py")) == []


def test_undefined_name_check_catches_a_stray_name(tmp_path):
    p = tmp_path / "m.py"
    p.write_text("peak = 1\n\ndef f():\n    return peaks\n")
    assert _undefined_globals(str(p)) == [("f", "peaks")]
