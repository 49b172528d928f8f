"""Multi-process host logic of the replica benchmark on CPU (gloo, world size 2).

The step shards into independent replicas (one problem per rank, no data-path collective);
the only cross-rank work is the whole-job reduction of the timed region: the slowest rank's
time and the sum of the nodes all ranks updated.  The reference arm under torchrun prints
one line from rank 0 while the other ranks exit without work.
"""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r pretends to take (r + 1) seconds for (r + 1) * 1000 node updates
    sec, units = bench.reduce_over_ranks(dist, "cpu", rank + 1.0, (rank + 1) * 1000)
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump([sec, units], f)
    dist.barrier()
    dist.destroy_process_group()


def test_reduce_over_ranks_gloo_world_2(tmp_path):
    import torch.multiprocessing as mp
    mp.spawn(_rank_main, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    for r in range(2):
        sec, units = json.load(open(tmp_path / f"r{r}.json"))
        assert sec == 2.0 and units == 3000.0


def test_reduce_over_ranks_single_process():
    import bench
    assert bench.reduce_over_ranks(None, "cpu", 1.5, 42) == (1.5, 42.0)


def test_reference_arm_under_torchrun_two_ranks():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py",
           "--impl", "reference", "--gpus", "2", "--steps", "2", "--warmup", "1"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    rec = json.loads(lines[0])
    assert rec["impl"] == "reference" and rec["n_gpus"] == 2 and rec["steps"] == 2
    assert rec["value"] > 0 and rec["unit"] == "MLUPS" and rec["higher_is_better"] is True
    assert rec["cpu_baseline"]["kind"] == "oracle" and rec["cpu_baseline"]["value"] == rec["value"]
    assert rec["e2e"]["h2d_bytes_per_step"] == 0 and rec["e2e"]["d2h_bytes_per_step"] == 0

