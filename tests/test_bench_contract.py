"""bench.py's reference arm (the FP64 oracle on the host cores) prints one JSON line with the
benchmark contract's keys, on the same metric, unit and workload as the GPU arm (no GPU needed)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    sys.path.insert(0, ROOT)
    import bench
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2", "--warmup", "1"],
                         cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, out.stdout
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["config"]["workload"] == bench.WORKLOAD
    # fewer than 3 warm-up steps are raised to 3 (the timing rules' minimum), and the line says so
    assert d["n_gpus"] == 1 and d["steps"] == 2 and d["warmup"] == 3 and d["higher_is_better"] is True
    # a step is one bounded sample: ms_per_step is its measured time; value is the full iteration's
    # rate, from the pixel-independent part plus the per-tile time scaled to the whole image
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert abs(d["full_iteration_s"] * d["value"] - 1.0) < 1e-9
    assert d["full_iteration_s"] > d["ms_per_step"] / 1000.0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_full_iteration_from_fixed_part_and_tiles():
    """t_fixed + (t_sample - t_fixed) / n x (W H / 256): a sample of n tiles that costs t_sample,
    of which t_fixed does not depend on the pixels."""
    sys.path.insert(0, ROOT)
    import bench
    tiles = bench.W * bench.H / 256.0
    assert bench.oracle_full_iteration_s(2.0, 6.0, 4) == 2.0 + 1.0 * tiles
    assert bench.oracle_full_iteration_s(2.0, 1.0, 4) == 2.0      # noise below the fixed part


def test_sample_tiles_cover_the_image():
    """The CPU-oracle samples take their 16x16 tiles from one list of 128 inside the image, any
    prefix of which is spread over it (each quadrant holds a quarter of the first 32)."""
    sys.path.insert(0, ROOT)
    import bench
    t = bench.sample_tiles()
    assert len(t) == 128 and len(set(t)) == 128
    assert all(0 <= x <= bench.W - 16 and 0 <= y <= bench.H - 16 for x, y in t)
    quad = [(x >= (bench.W - 16) / 2, y >= (bench.H - 16) / 2) for x, y in t[:32]]
    assert all(quad.count(q) == 8 for q in set(quad)) and len(set(quad)) == 4


def test_traffic_is_reported_only_for_the_captured_source_and_layout():
    """The DRAM traffic on the bench line comes from an ncu capture of one kernel source and
    layout; it is reported while the source's sha256 and the layout still match, else null."""
    sys.path.insert(0, ROOT)
    import hashlib
    import bench
    for kernel, entry in bench.NCU_TRAFFIC.items():
        src = os.path.join(ROOT, entry["source"])
        matches = hashlib.sha256(open(src, "rb").read()).hexdigest() == entry["sha256"]
        got = bench._ncu_traffic(kernel, entry["tile"], entry["ppt"])
        assert got == (entry["bytes"] if matches else None)
        # another layout never borrows the figure
        assert bench._ncu_traffic(kernel, entry["tile"], entry["ppt"] + 8) is None
    assert bench._ncu_traffic("no_such_kernel", 16, 2) is None
    saved = dict(bench.NCU_TRAFFIC["raster_fused"])
    try:
        bench.NCU_TRAFFIC["raster_fused"]["sha256"] = "0" * 64
        assert bench._ncu_traffic("raster_fused", saved["tile"], saved["ppt"]) is None
    finally:
        bench.NCU_TRAFFIC["raster_fused"].update(saved)
