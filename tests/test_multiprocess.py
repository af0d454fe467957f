"""The multi-process path of bench.py on the CPU: two ranks over gloo, launched the way
the benchmark is launched (torch.distributed.run, one process per rank, rendezvous on
127.0.0.1).  The solver path itself runs one independent replica per GPU (no
collective on the data path); what ranks share is the barrier around the timed region
and the max over ranks of the measured time, and the reference arm runs on rank 0
alone."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _torchrun(args, timeout=300):
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr=127.0.0.1", f"--master-port={_free_port()}", *args]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    return subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=timeout)


def _json_lines(text):
    """The JSON objects the ranks printed (two ranks may share a line of output)."""
    dec, out, i = json.JSONDecoder(), [], 0
    while True:
        i = text.find("{", i)
        if i < 0:
            return out
        try:
            obj, end = dec.raw_decode(text, i)
        except ValueError:
            i += 1
            continue
        out.append(obj)
        i = end


def test_two_gloo_ranks_barrier_and_max_over_ranks():
    r = _torchrun([os.path.join("tests", "gloo_ranks.py")])
    assert r.returncode == 0, r.stderr[-2000:]
    lines = sorted(_json_lines(r.stdout), key=lambda d: d["rank"])
    assert [d["rank"] for d in lines] == [0, 1]
    assert all(d["world"] == 2 for d in lines)
    assert all(d["max"] == 2.5 for d in lines)          # the slower rank's time, on both


def test_reference_arm_prints_one_line_from_rank_0():
    pytest.importorskip("torch")
    r = _torchrun(["bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1",
                   "--warmup", "0"])
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _json_lines(r.stdout)
    assert len(lines) == 1
    d = lines[0]
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"
