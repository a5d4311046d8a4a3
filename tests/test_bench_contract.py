"""The benchmark's command-line contract on CPU: the reference arm (the FP64 oracle timed
on the host cores) prints one JSON line with the same metric, unit and direction as the
GPU arm, and the timing rules are enforced before anything runs."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench(*args, timeout=600):
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT, capture_output=True,
                          text=True, timeout=timeout)


def test_reference_arm_prints_one_json_line():
    sys.path.insert(0, ROOT)
    import bench
    r = _bench("--impl", "reference", "--steps", "1", "--warmup", "3")
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [x for x in r.stdout.splitlines() if x.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert (d["metric"], d["unit"], d["higher_is_better"]) == (bench.METRIC, bench.UNIT, True)
    assert (d["n_gpus"], d["steps"], d["warmup"], d["dtype"]) == (1, 1, 3, "f64")
    assert d["value"] > 0 and abs(d["value"] - 1000.0 / d["ms_per_step"]) <= 1e-9 * d["value"]
    assert d["config"]["workload"] == bench.WORKLOAD
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": bench.UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_fewer_than_three_warmup_steps_are_refused():
    r = _bench("--warmup", "2", timeout=120)
    assert r.returncode != 0 and "--warmup must be >= 3" in r.stderr


def test_pixel_iterations_per_field_of_the_workloads():
    # n * sum_l N_l with N_l = ceil(H / 2^l) * ceil(W / 2^l): the unit of the reported
    # Mpix*iter/s, for the 256^2 (2 levels, 4 iterations), 1024^2 (3, 5) and 2048^2 (4, 6)
    # workloads, and a ragged size whose levels round up
    sys.path.insert(0, ROOT)
    import bench
    assert bench.pixel_iterations(256, 256, 2, 4) == 327_680
    assert bench.pixel_iterations(1024, 1024, 3, 5) == 6_881_280
    assert bench.pixel_iterations(2048, 2048, 4, 6) == 33_423_360
    assert bench.pixel_iterations(383, 1791, 3, 1) == 383 * 1791 + 192 * 896 + 96 * 448


def test_algorithmic_bytes_of_the_headline_workload():
    # 1024^2, 12-bit camera counts (2 B), FP16 reduced levels, L = 3, n = 5, counted by hand:
    # levels of 1,048,576, 262,144 and 65,536 px; per pixel-iteration I1 + I2 (2 x 2 B) and
    # the estimate in and out (8 + 8 B), except that a level's first iteration reads the
    # coarser level's estimate (the very first none); pyramids: the raw read and level-0
    # copy (2 + 2 B per px, both images), levels 1 and 2 written, level 1 read once.
    sys.path.insert(0, ROOT)
    import bench
    N = [1048576, 262144, 65536]
    pyr = 2 * (2 * N[0] + 2 * N[0] + 2 * (N[1] + N[2]) + 2 * N[1])
    it = sum(5 * N[l] * (4 + 8) + 4 * N[l] * 8 for l in range(3)) + 8 * N[1] + 8 * N[2]
    assert bench.algorithmic_bytes(1024, 1024, 3, 5, 2, 2) == (pyr + it, pyr, it) == (139984896, 10747904, 129236992)
    # the plain dataflow: level 0 re-read for the first reduction, every iteration reading a
    # full-level estimate
    plain = 2 * (2 * N[0] + 2 * sum(N) + 2 * (N[0] + N[1])) + 5 * sum(N) * 20
    assert bench.unfused_dataflow_bytes(1024, 1024, 3, 5, 2, 2) == plain == 152567808
