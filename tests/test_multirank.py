"""The N > 1 path of bench.py on CPU: world-size-2 gloo ranks (no GPU).

Frozen states are independent, so ranks run replicas with no data-path collective; only
the job-wide figures cross ranks (the slowest rank's time, the units all ranks processed)."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    mx, sm = bench.over_ranks(dist, "cpu", [10.0 * (rank + 1), -rank], [rank + 1, 3])
    q.put((rank, mx, sm, _state_hashes(bench, rank)))
    dist.destroy_process_group()


def test_over_ranks_max_time_sum_units_and_distinct_states():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = dict((r, (mx, sm, h)) for r, mx, sm, h in (q.get(timeout=120) for _ in ps))
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in (0, 1):
        mx, sm, _ = out[r]
        assert mx == [20.0, 0.0] and sm == [3.0, 6.0]          # slowest rank's time; all ranks' units
    assert out[0][2] != out[1][2] and out[0][2][0] != out[0][2][1]   # each rank, each step its own state
    assert bench_states_single_process() == out[0][2]


def _state_hashes(bench, rank):
    """The rank's bench states applied to a fixed design (the design itself is made on the
    device; the per-rank, per-state part is the seeded forced-floor set)."""
    import synth
    base = np.linspace(0.05, 1.0, 4096)
    return [float((synth.force_to_floor(base, 0.3, s) * np.arange(base.size)).sum())
            for s in bench.state_seeds(rank, 2)]


def bench_states_single_process():
    sys.path.insert(0, ROOT)
    import bench
    return _state_hashes(bench, 0)


def test_reference_arm_under_two_ranks_prints_once():
    """bench.py --impl reference under torchrun with 2 ranks: rank 0 alone runs the oracle
    sample and prints one JSON line; rank 1 exits 0 without work."""
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "0"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
