"""The bench's multi-rank path on CPU (gloo, world size 2, 127.0.0.1): the
rank helpers (barrier, max over ranks for times, sum over ranks for the
whole-job count) and the reference arm under torch.distributed.run, where
rank 0 alone prints one JSON line.  The factorization of one matrix does not
shard: under torchrun every rank factors its own replica; the batching form
splits its independent systems over the ranks."""
import json
import os
import socket
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, ws, port, out_dir):
    os.environ.update({"RANK": str(rank), "LOCAL_RANK": str(rank), "WORLD_SIZE": str(ws),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    w, r, local = bench.dist_setup(None)
    bench.barrier(w)
    mx = bench.allmax(w, 10.0 * (r + 1))
    sm = bench.allsum(w, 3.0)
    with open(os.path.join(out_dir, f"rank{r}.json"), "w") as f:
        json.dump({"ws": w, "rank": r, "local": local, "max": mx, "sum": sm,
                   "backend": dist.get_backend()}, f)
    dist.destroy_process_group()


def test_rank_helpers_gloo_world_size_2():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("CPU test: with CUDA the helpers take NCCL")
    import torch.multiprocessing as mp
    out = tempfile.mkdtemp()
    mp.spawn(_worker, args=(2, _free_port(), out), nprocs=2, join=True)
    res = [json.load(open(os.path.join(out, f"rank{r}.json"))) for r in range(2)]
    for r, d in enumerate(res):
        assert d["ws"] == 2 and d["rank"] == r and d["local"] == r
        assert d["backend"] == "gloo"
        assert d["max"] == 20.0          # the slowest rank's time
        assert d["sum"] == 6.0           # whole-job total over ranks


def test_reference_arm_under_torchrun_prints_one_line():
    pytest.importorskip("torch")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py",
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0", "--cpu-seconds", "2"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    p = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["cpu_baseline"]["kind"] == "oracle"
    assert d["value"] > 0 and d["higher_is_better"] is False


def _split_worker(rank, ws, port, out_dir):
    os.environ.update({"RANK": str(rank), "LOCAL_RANK": str(rank), "WORLD_SIZE": str(ws),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    from paper_2509_07690_gb300 import synth
    w, r, _ = bench.dist_setup(None)
    sizes = [int(n) for n in synth.circuit_batch_sizes()]
    weights = [bench.batch_weight(n) for n in sizes]
    mine = bench.partition_systems(weights, w)[r]
    got = [None] * w
    dist.all_gather_object(got, mine)
    with open(os.path.join(out_dir, f"split{r}.json"), "w") as f:
        json.dump({"parts": got, "weights": weights}, f)
    dist.destroy_process_group()


def test_batch_split_across_ranks_gloo_world_size_2():
    """The batching form shards by system: each rank computes its share of
    the 512 systems on its own (no exchange on the data path).  Every system
    is on exactly one rank, both ranks derive the same split, and the
    heaviest rank's load is at most the mean plus the largest system."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("CPU test: with CUDA the helpers take NCCL")
    import torch.multiprocessing as mp
    out = tempfile.mkdtemp()
    mp.spawn(_split_worker, args=(2, _free_port(), out), nprocs=2, join=True)
    res = [json.load(open(os.path.join(out, f"split{r}.json"))) for r in range(2)]
    assert res[0]["parts"] == res[1]["parts"]
    parts, weights = res[0]["parts"], res[0]["weights"]
    flat = sorted(q for p in parts for q in p)
    assert flat == list(range(len(weights)))
    loads = [sum(weights[q] for q in p) for p in parts]
    assert max(loads) <= sum(weights) / 2 + max(weights)
    assert max(loads) / min(loads) < 1.01          # 512 systems balance closely
