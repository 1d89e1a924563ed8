"""Runs across ranks, on the host with the gloo backend (world size 2): the
helpers bench.py times N GPUs with, bench.py's reference arm under the same
launcher, and the sharding of an ensemble's instances over ranks. A single
mesh is not partitioned, so replicas exchange no data and only agree on the
slowest rank's time; a sharded ensemble's ranks meet only to gather the
per-instance results."""
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


def _torchrun(args, timeout=300, **extra_env):
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr=127.0.0.1", "--master-port=%d" % _port()] + args
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="", OMP_NUM_THREADS="1", **extra_env)
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=timeout, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    return [json.loads(l) for l in r.stdout.splitlines() if l.startswith("{")]


def test_two_ranks_agree_on_the_slowest_step_and_the_job_rate(tmp_path):
    _torchrun([os.path.join("tests", "replica_worker.py")], REPLICA_OUT=str(tmp_path))
    lines = [json.loads((tmp_path / ("rank%d.json" % r)).read_text()) for r in range(2)]
    assert [l["rank"] for l in lines] == [0, 1]
    for l in lines:
        assert l["ws"] == 2 and l["local"] == l["rank"]
        assert l["slowest"] == 5.0                        # rank 1's 5 ms, seen by both
        assert l["rate"] == 2 * 1000.0 / 5e-3             # both ranks' units over the slowest time


def test_reference_arm_prints_once_under_two_ranks():
    lines = _torchrun(["bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"])
    assert len(lines) == 1
    assert lines[0]["impl"] == "reference" and lines[0]["n_gpus"] == 2 and lines[0]["value"] > 0


def test_partition_balances_triangles_and_covers_every_instance():
    from paper_2306_04467_gb300 import inputs, replicas
    sizes = [2 * n * n for n in inputs.ensemble_sizes(256)]
    for ws in (1, 2, 3, 8):
        parts = replicas.partition_instances(sizes, ws)
        assert sorted(i for p in parts for i in p) == list(range(256))
        loads = [sum(sizes[i] for i in p) for p in parts]
        assert max(loads) - min(loads) <= max(sizes)        # greedy bound
        assert parts == replicas.partition_instances(sizes, ws)   # deterministic


def test_two_ranks_shard_an_ensemble_and_gather_its_instances(tmp_path):
    """Each rank advances only its own instances; both end with every
    instance's masses and time, equal to a single process running them all."""
    _torchrun([os.path.join("tests", "shard_worker.py")], REPLICA_OUT=str(tmp_path))
    out = [json.loads((tmp_path / ("shard%d.json" % r)).read_text()) for r in range(2)]
    assert sorted(out[0]["mine"] + out[1]["mine"]) == list(range(5)) and out[0]["mine"] and out[1]["mine"]
    assert out[0]["all"] == out[1]["all"]
    from oracle.oracle import Oracle
    from paper_2306_04467_gb300 import inputs
    for i, n in enumerate([4, 7, 5, 6, 3]):
        o = Oracle.from_problem(inputs.ensemble_member(n, seed=100 + i))
        o.advance(4)
        assert out[0]["all"][i] == [float(x) for x in o.mass()] + [o.t]
