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
