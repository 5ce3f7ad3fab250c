"""Host logic of bench.py that needs no GPU: the reference arm's
unavailable line for a workload without a stored full oracle run, and the
silent exit of non-zero ranks in the reference arm."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(args, env=None):
    e = dict(os.environ)
    e.update(env or {})
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args,
                         capture_output=True, text=True, timeout=120, env=e, cwd=ROOT)
    return out


def test_reference_arm_unavailable_line():
    out = _run(["--impl", "reference", "--config", "5", "--steps", "1", "--warmup", "0"])
    assert out.returncode == 0, out.stderr
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and "unavailable" in line


def test_reference_arm_other_ranks_print_nothing():
    out = _run(["--impl", "reference", "--steps", "1", "--warmup", "0"],
               env={"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert out.returncode == 0, out.stderr
    assert out.stdout.strip() == ""


def _bench_module():
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_host_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_committed_traffic_matches_the_sources_and_scales_with_n():
    """The committed ncu traffic of the CG product kernel belongs to the
    sources as they are (SHA-256 recorded with the capture), and it is
    scaled to the workload's n by (n / n_capture)^2 (the operator's planes
    dominate the bytes)."""
    bench = _bench_module()
    rec = json.load(open(os.path.join(ROOT, "profiles", "dram_traffic.json")))["bf16x3_kernel"]
    t0, note0 = bench.committed_traffic("bf16x3_kernel", rec["n"])
    assert t0 == rec["dram_bytes_per_launch"], note0
    t1, _ = bench.committed_traffic("bf16x3_kernel", 2 * rec["n"])
    assert t1 == 4 * rec["dram_bytes_per_launch"]
    # traffic / algorithmic bytes (4 n^2 + 16 n c) stays near 1: no re-reads
    n, c = rec["n"], rec["c"]
    assert 1.0 <= t0 / (4.0 * n * n + 16.0 * n * c) < 1.05


def test_committed_traffic_is_withheld_when_a_source_changed(tmp_path, monkeypatch):
    bench = _bench_module()
    rec = json.load(open(os.path.join(ROOT, "profiles", "dram_traffic.json")))["bf16x3_kernel"]
    os.makedirs(tmp_path / "profiles")
    (tmp_path / "profiles" / "dram_traffic.json").write_text(
        json.dumps({"bf16x3_kernel": rec}))
    for src in rec["sources"]:
        dst = tmp_path / src
        os.makedirs(dst.parent, exist_ok=True)
        dst.write_bytes(open(os.path.join(ROOT, src), "rb").read())
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.committed_traffic("bf16x3_kernel", rec["n"])[0] == rec["dram_bytes_per_launch"]
    first = tmp_path / rec["sources"][0]
    first.write_bytes(first.read_bytes() + b"\n// edited\n")
    t, note = bench.committed_traffic("bf16x3_kernel", rec["n"])
    assert t is None and note.startswith("stale")
    assert bench.committed_traffic("no_such_kernel", 1024) == (None, None)
