"""The N > 1 host path of bench.py (replicas only, no data-path collective), on CPU with two
ranks under torch.distributed.run:
* with a gloo process group each rank builds its own instance (seed + rank) and
  max_over_ranks returns the slowest rank's time on every rank;
* the reference arm under two ranks prints exactly one JSON line, from rank 0.
"""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _torchrun(script_args, timeout):
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(_port())] + script_args
    env = dict(os.environ, OMP_NUM_THREADS="1", CUDA_VISIBLE_DEVICES="")
    p = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=timeout)
    assert p.returncode == 0, p.stderr[-3000:]
    # the ranks share one stdout pipe, so two lines can arrive without a newline between them:
    # decode every JSON object in the text instead of splitting on lines
    out, dec, text, i = [], json.JSONDecoder(), p.stdout, 0
    while True:
        i = text.find("{", i)
        if i < 0:
            return out
        obj, i = dec.raw_decode(text, i)
        out.append(obj)


def test_gloo_replicas_max_and_seeds():
    lines = _torchrun([os.path.join(ROOT, "tests", "_replica_worker.py")], 600)
    assert sorted(l["rank"] for l in lines) == [0, 1]
    assert all(l["max"] == 2.5 for l in lines)            # max(1.5, 2.5) on both ranks
    assert lines[0]["n"] == lines[1]["n"]
    assert lines[0]["b0"] != lines[1]["b0"]                # seed + rank: different instances


def test_reference_arm_prints_once_under_two_ranks():
    lines = _torchrun([os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2", "--steps", "1",
                       "--warmup", "0", "--small"], 900)
    assert len(lines) == 1
    line = lines[0]
    assert line["impl"] == "reference" and line["n_gpus"] == 2
    assert line["cpu_baseline"]["kind"] == "oracle" and line["value"] > 0
    assert line["cpu_baseline"]["cores"] >= 1 and len(line["step_times_s"]) == 1
