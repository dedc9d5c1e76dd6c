"""The benchmark's reference arm (the oracle on the host cores) runs on CPU
and prints one JSON line with the contract's keys."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--cpu-n", "16", "--steps", "1", "--warmup", "3"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]


def test_traffic_figure_is_tied_to_the_pass_source_and_flags(monkeypatch):
    """`roofline.traffic` comes from the committed ncu figures only while the
    pass source and its nvcc flags are those they were taken on."""
    sys.path.insert(0, ROOT)
    import importlib
    import bench
    b = importlib.import_module("paper_1810_13416_gb300.build")
    with open(bench.TRAFFIC_JSON) as f:
        committed = json.load(f)["f32"]["src_sha256_16"]
    current = bench._src_hash()
    march, tile = (0, 0, 0), (1, 0, 0)
    assert (bench._traffic_per_cell("f32", march) is not None) == (current == committed)
    if current == committed:
        # the figure follows the design of each axis
        assert bench._traffic_per_cell("f32", march) != bench._traffic_per_cell("f32", tile)
    for unit in ("sweep_f32", "tile_f32"):
        flags = dict(b.UNIT_FLAGS)
        flags[unit] = [f for f in flags[unit] if f != "-ftz=true"]
        monkeypatch.setattr(b, "UNIT_FLAGS", flags)
        assert bench._src_hash() != current
        if current == committed:
            assert bench._traffic_per_cell("f32", march) is None
