"""The multi-rank path of bench.py on CPU: world size 2 over gloo.

Chunks are independent, so ranks share nothing on the data path: each rank
times its own work, and the reported time is the maximum over ranks while the
value counts every rank's chunks (weak scaling).  These tests exercise the
rank set-up, the barrier and the max-over-ranks reduction with gloo, and the
reference arm's rule that only rank 0 runs and prints.
"""
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


WORKER = r"""
import os, sys, json
sys.path.insert(0, {root!r})
import bench
import torch.distributed as dist

class A: impl = "reference"
world, rank, local = bench.dist_setup(A())
assert world == 2 and dist.get_backend() == "gloo"
bench.barrier(world)
t = 10.0 + 5.0 * rank                       # rank 1 is the slow one
m = bench.max_over_ranks(t, world, device="cpu")
value = world * 4113 / m                    # every rank's chunks over the slowest rank's time
print(json.dumps({{"rank": rank, "max": m, "value": value}}))
dist.destroy_process_group()
"""


def _launch(code, nproc=2, extra_args=()):
    port = _free_port()
    procs = []
    for rank in range(nproc):
        env = dict(os.environ, RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(nproc),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable, "-c", code, *extra_args], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True, cwd=ROOT))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=120)
        assert p.returncode == 0, err
        outs.append(out)
    return outs


def test_max_over_ranks_and_weak_scaling_value():
    import json

    outs = _launch(WORKER.format(root=ROOT))
    res = [json.loads(o.strip().splitlines()[-1]) for o in outs]
    assert all(r["max"] == 15.0 for r in res)
    assert all(abs(r["value"] - 2 * 4113 / 15.0) < 1e-9 for r in res)


def test_reference_arm_prints_on_rank_zero_only():
    code = (f"import sys; sys.path.insert(0, {ROOT!r}); import bench; "
            "sys.exit(bench.main(['--impl', 'reference', '--gpus', '2', '--steps', '1', '--warmup', '3', "
            "'--ref-sample', '8']))")
    outs = _launch(code)
    import json

    lines0 = [l for l in outs[0].splitlines() if l.startswith("{")]
    lines1 = [l for l in outs[1].splitlines() if l.startswith("{")]
    assert len(lines0) == 1 and not lines1
    rec = json.loads(lines0[0])
    assert rec["impl"] == "reference" and rec["n_gpus"] == 2 and rec["value"] > 0
