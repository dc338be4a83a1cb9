"""Multi-rank logic of bench.py on the host: two gloo ranks (127.0.0.1) set
up the process group, pass the barrier, agree on the slowest rank's time,
and the reference arm runs on rank 0 only.  The whole-job value is the sum of
the replicas' atoms over the slowest rank's step time."""
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

RANK_SCRIPT = r"""
import os, sys, time
sys.path.insert(0, os.getcwd())
import bench
dist, rank, ws = bench.dist_setup()
assert ws == 2 and rank == int(os.environ["RANK"]) and dist.get_backend() == "gloo"
bench.barrier(dist)
t = bench.max_over_ranks(dist, 1.5 + rank)
class A: warmup = 0; steps = 1; gpus = 2
if rank == 1:
    t0 = time.perf_counter()
    assert bench.run_reference(A, dist, rank, ws) is None      # no work off rank 0
    assert time.perf_counter() - t0 < 1.0
bench.barrier(dist)
print("RESULT", rank, t, flush=True)
dist.destroy_process_group()
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_agree_on_the_slowest_time():
    port = str(_free_port())
    procs = []
    for r in range(2):
        env = dict(os.environ, RANK=str(r), LOCAL_RANK=str(r), WORLD_SIZE="2", MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=port, CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable, "-c", RANK_SCRIPT], cwd=ROOT, env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = [p.communicate(timeout=120) for p in procs]
    for p, (o, e) in zip(procs, outs):
        assert p.returncode == 0, e
    got = sorted(tuple(l.split()[1:]) for o, _ in outs for l in o.splitlines() if l.startswith("RESULT"))
    assert got == [("0", "2.5"), ("1", "2.5")]


def test_weak_scaling_value_sums_replicas():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.weak_value(1, 12288, 2.0) == 12288 / 0.002
    assert bench.weak_value(4, 12288, 2.0) == 4 * 12288 / 0.002
