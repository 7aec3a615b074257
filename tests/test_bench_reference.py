"""The benchmark's reference arm (`bench.py --impl reference`: the FP64 oracle
timed on the host cores) without a GPU: its one JSON line carries the keys of
the benchmark's line, with the oracle described as the CPU baseline and an
end-to-end entry that moves no bytes, and under two ranks (gloo) rank 0
alone prints it while both ranks exit 0.  A small sample grid keeps it quick.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ARGS = ["--impl", "reference", "--steps", "1", "--warmup", "0", "--sample-grid", "8"]


def json_lines(text):
    return [json.loads(l) for l in text.splitlines() if l.startswith("{")]


def check_line(line, n_gpus):
    assert line["impl"] == "reference"
    assert isinstance(line["metric"], str) and line["unit"] == "unknowns/s"
    assert line["value"] > 0 and line["ms_per_step"] > 0
    assert line["n_gpus"] == n_gpus and line["steps"] == 1 and line["warmup"] == 0
    assert line["higher_is_better"] is True and line["data"] == "synthetic" and line["dtype"] == "f64"
    assert line["vs_baseline"] is None
    assert "8^3 sample" in line["config"]["workload"] and line["config"]["n"] > 0
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_line():
    p = subprocess.run([sys.executable, "bench.py", *ARGS], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr
    lines = json_lines(p.stdout)
    assert len(lines) == 1
    check_line(lines[0], 1)


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_reference_line_under_two_ranks():
    pytest.importorskip("torch.distributed")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(free_port()), "bench.py", *ARGS]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    p = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = json_lines(p.stdout)
    assert len(lines) == 1
    check_line(lines[0], 2)
