"""bench.py's output contract, checked on CPU through its reference arm (the
FP64 oracle timed on the host) and the arms that have none."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*args):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], capture_output=True, text=True,
                         timeout=600, cwd=ROOT, env={**os.environ, "WORLD_SIZE": "1", "RANK": "0"})
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, out.stdout
    return json.loads(lines[0])


def test_reference_arm_line():
    d = _run("--impl", "reference", "--steps", "1", "--warmup", "0")
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 1 and d["warmup"] == 0
    assert d["higher_is_better"] is True and d["scaling"] == "weak"
    assert d["config"]["workload"] == "pm2-256c-128x512mesh"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_arms_without_oracle_say_so():
    for wl in ("c4-ensemble-64x20", "c3-adjoint-128c-256mesh", "c5-force-1024c-512x2048mesh"):
        d = _run("--impl", "reference", "--workload", wl)
        assert d["impl"] == "reference" and "unavailable" in d


def test_numa_node_of_the_gpu_from_sysfs(tmp_path):
    # the e2e leg binds to the CPUs of the GPU's NUMA node before allocating its
    # pinned host buffers; the node and its CPU list come from sysfs
    sys.path.insert(0, ROOT)
    import bench
    dev = tmp_path / "bus" / "pci" / "devices" / "0009:01:00.0"
    dev.mkdir(parents=True)
    (dev / "numa_node").write_text("1\n")
    node = tmp_path / "devices" / "system" / "node" / "node1"
    node.mkdir(parents=True)
    (node / "cpulist").write_text("0-3,8,10-11\n")
    assert bench.numa_cpus("00000009:01:00.0", root=str(tmp_path)) == (1, {0, 1, 2, 3, 8, 10, 11})
    (dev / "numa_node").write_text("-1\n")                      # no affinity reported: nothing to bind
    assert bench.numa_cpus("00000009:01:00.0", root=str(tmp_path)) is None
    assert bench.numa_cpus("00000009:02:00.0", root=str(tmp_path)) is None   # no such device
    assert bench.numa_cpus(None, root=str(tmp_path)) is None
