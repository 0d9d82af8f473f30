"""The multi-process path of the benchmark on CPU ranks (gloo, world size 2).

The solver shards by independent problems (replicas: one solve per rank, no
collective on the data path), so what is tested here is the host-side
plumbing: the max-over-ranks timing reduction, the barrier, and the launch
under torch.distributed.run where rank 0 alone prints the JSON line — and
the row-sharded form of the gradient step that one problem split over ranks
would use: g = Σ_k A_kᵀ(b_k − A_k x) − λx, one all-reduce of a d-vector
(there are no inner products in the step, Section 3)."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    bench.barrier(ws)
    q.put((rank, bench.max_over_ranks(10.0 * rank + 0.5, ws)))
    dist.destroy_process_group()


def test_max_over_ranks_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got == {0: 10.5, 1: 10.5}


@pytest.mark.timeout(600)
def test_reference_arm_under_torchrun_prints_one_line():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes", "1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "0", "--rows", "4096", "--cols", "64"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    out = json.loads(lines[0])
    assert out["impl"] == "reference" and out["n_gpus"] == 2 and out["value"] > 0
    assert out["e2e"]["h2d_bytes_per_step"] == 0 and out["cpu_baseline"]["kind"] == "oracle"


@pytest.mark.timeout(600)
def test_reference_arm_single_process_rotates_pieces():
    """One process, several steps: the first step times every piece of the
    oracle's work and later steps re-time one piece each; the line carries
    the contract's keys."""
    cmd = [sys.executable, "bench.py", "--impl", "reference", "--steps", "6", "--warmup", "2",
           "--rows", "4096", "--cols", "64"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    out = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "higher_is_better", "scaling",
                "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in out, key
    assert out["impl"] == "reference" and out["n_gpus"] == 1 and out["steps"] == 6 and out["value"] > 0
    assert out["cpu_baseline"]["value"] == out["value"] and out["e2e"]["value"] == out["value"]
    assert "re-timed" in out["cpu_baseline"]["sample"]


def _shard_main(rank, ws, port, q, drop):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    sys.path.insert(0, ROOT)
    import numpy as np
    import torch
    import torch.distributed as dist
    from oracle import mihs_oracle as o
    from paper_1912_03514_gb300 import workloads as W
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    p = W.problem_scaled(3001, 96, seed=5)
    A, b = p.A.numpy().astype(np.float64), p.b.numpy().astype(np.float64)
    x = W.randn((96,), 6).double().numpy()
    lo, hi = rank * A.shape[0] // ws, (rank + 1) * A.shape[0] // ws
    # this rank's rows; λx is counted once (rank 0)
    part = o.gradient(A[lo:hi], b[lo:hi], x, p.lam if rank == 0 else 0.0)
    if drop and rank == 1:
        part = np.zeros_like(part)  # a shard whose contribution was lost
    t = torch.from_numpy(part)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    full = o.gradient(A, b, x, p.lam)
    q.put((rank, float(np.linalg.norm(t.numpy() - full) / np.linalg.norm(full))))
    dist.destroy_process_group()


@pytest.mark.parametrize("drop", [False, True])
def test_row_sharded_gradient_gloo(drop):
    """Two CPU ranks, each with half the rows: the all-reduced partial
    gradients equal the oracle's full gradient (fp64 summation order only);
    a lost shard is detected by the same comparison."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_main, args=(r, 2, port, q, drop)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, err in got.items():
        if drop:
            assert err > 1e-3, (r, err)
        else:
            assert err <= 1e-13, (r, err)
