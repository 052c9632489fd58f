"""The N > 1 path on the CPU with the gloo backend (world size 2).

The path shards by replicas: every rank advances its own lattice, and the only
collectives are the barrier and the max over ranks of the timing.  These tests
run that plumbing in two processes, and the reference arm of ``bench.py`` under
``torch.distributed.run`` (rank 0 prints one line, rank 1 exits 0 without work).
"""
import importlib.util
import json
import os
import socket
import subprocess
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    b = _bench()
    w, r, _ = b.dist_env()
    b.init_distributed(w, "gloo")
    local_ms = 10.0 + 5.0 * r                      # rank 1 is the slower one
    ms = b.max_over_ranks(local_ms, w, "cpu")
    value = b.whole_job_mlups(w, 1000, 20, ms)
    dist.barrier()
    with open(os.path.join(out, f"rank{r}.json"), "w") as fh:
        json.dump({"world": w, "rank": r, "ms": ms, "value": value}, fh)
    dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_value(tmp_path):
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, start_method="spawn")
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    for r in res:
        assert r["world"] == 2 and r["ms"] == 15.0      # every rank sees the slowest rank's time
        assert r["value"] == pytest.approx(2 * 1000 * 20 / 15e-3 / 1e6)


def test_single_process_needs_no_group():
    b = _bench()
    assert b.max_over_ranks(3.5, 1, "cpu") == 3.5
    assert b.whole_job_mlups(1, 10 ** 6, 100, 1000.0) == pytest.approx(100.0)


def test_reference_arm_under_torchrun():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0",
           "--workload", "periodic32"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    res = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [l for l in res.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, res.stdout
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle"


def _replica_worker(rank, world, port, out):
    """One replica per rank on the one GPU of the test: the same seeded lattice,
    stepped independently, with a gloo group for the exchange of the results."""
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import hashlib

    import numpy as np

    from paper_2608_15781_b300 import lbm, synth
    dist.init_process_group("gloo", rank=rank, world_size=world)
    solid = synth.grf_mask((24, 20, 16), 3, 0.5, 11, periodic_z=False)
    p = lbm.Params(sigma=0.01, theta_deg=60.0, k_rate=5e-3, u_in=0.01, c_in=1.0)
    with lbm.Lattice(solid, p, bc_z=1) as L:
        dist.barrier()                 # both ranks step at the same time
        L.step(50)
        h = hashlib.sha256(L.get_state().tobytes()).hexdigest()
    hashes = [None] * world
    dist.all_gather_object(hashes, h)
    with open(os.path.join(out, f"replica{rank}.json"), "w") as fh:
        json.dump(hashes, fh)
    dist.destroy_process_group()


@pytest.mark.gpu
def test_replicas_are_independent_of_each_other():
    """Two ranks advancing their own copy of one lattice at the same time (the
    replica form of the N > 1 path) end bit-identical to each other and to the same
    lattice stepped alone in this process."""
    import hashlib
    import tempfile

    from paper_2608_15781_b300 import build, lbm, synth
    build.build()
    solid = synth.grf_mask((24, 20, 16), 3, 0.5, 11, periodic_z=False)
    p = lbm.Params(sigma=0.01, theta_deg=60.0, k_rate=5e-3, u_in=0.01, c_in=1.0)
    with lbm.Lattice(solid, p, bc_z=1) as L:
        L.step(50)
        alone = hashlib.sha256(L.get_state().tobytes()).hexdigest()
    with tempfile.TemporaryDirectory() as out:
        mp.start_processes(_replica_worker, args=(2, _free_port(), out), nprocs=2, start_method="spawn")
        res = [json.load(open(os.path.join(out, f"replica{r}.json"))) for r in range(2)]
    assert res[0] == res[1] == [alone, alone]
