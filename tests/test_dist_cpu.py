"""The multi-rank path of bench.py on CPU: two gloo ranks. Each rank has its own
bundle (its own seed) and reconstructs it alone -- no collective touches the
data -- and the job's time is the slowest rank's, its throughput the units of
all ranks over that time. The reference arm prints on rank 0 only."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def rank_main(rank, ws, port, out_dir):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    import oracle
    import synth
    # each rank its own bundle, reconstructed with no collective
    wl = synth.make_workload(2, 12, seed=bench.rank_seed(rank))
    ref = oracle.reconstruct(wl, threads=1)
    step_s = 0.010 * (rank + 1)                     # a rank-dependent "step time"
    slowest = bench.max_over_ranks(step_s, ws)
    rate = bench.job_rate(wl.n_evt, ws, slowest)
    np.save(os.path.join(out_dir, f"hillas{rank}.npy"), ref["hillas"])
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump({"seed": bench.rank_seed(rank), "n_evt": wl.n_evt, "slowest": slowest, "rate": rate}, f)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.timeout(300)
def test_two_gloo_ranks_weak_scaling_bookkeeping(tmp_path):
    ws = 2
    mp.start_processes(rank_main, args=(ws, free_port(), str(tmp_path)), nprocs=ws, start_method="spawn")
    r = [json.load(open(tmp_path / f"rank{k}.json")) for k in range(ws)]
    assert r[0]["seed"] != r[1]["seed"]
    assert r[0]["slowest"] == r[1]["slowest"] == pytest.approx(0.020)
    assert r[0]["rate"] == r[1]["rate"] == pytest.approx(r[0]["n_evt"] * ws / 0.020)
    # the ranks reconstructed different bundles, each exactly as a single process does
    h = [np.load(tmp_path / f"hillas{k}.npy") for k in range(ws)]
    assert h[0].shape != h[1].shape or not np.array_equal(h[0], h[1])
    sys.path.insert(0, ROOT)
    import bench
    import oracle
    import synth
    for k in range(ws):
        alone = oracle.reconstruct(synth.make_workload(2, 12, seed=bench.rank_seed(k)), threads=1)["hillas"]
        np.testing.assert_array_equal(alone, h[k])


@pytest.mark.timeout(600)
def test_reference_arm_prints_on_rank_zero_only():
    port = free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2", "--master-addr",
           "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1",
           "--warmup", "1", "--events", "50", "--ref-events", "8"]
    p = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=550)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [json.loads(x) for x in p.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    assert lines[0]["impl"] == "reference" and lines[0]["n_gpus"] == 2 and lines[0]["value"] > 0
