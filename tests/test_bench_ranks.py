"""The N>1 replica path of bench.py, on CPU with the gloo backend (2 ranks).

Each rank runs its own solves (no exchange step on the data path); the only
collectives are the max of the timed region over ranks and the sum of the units
the ranks processed, which these tests check with rank-dependent values.  The
reference arm under torchrun prints one line, from rank 0 only.
"""
import json
import os
import socket
import subprocess
import sys


ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        ms = 100.0 + 50.0 * rank
        counts = {"edges": 1000 * (rank + 1), "solves": 3, "phases": 7 + rank}
        t, tot = bench.combine_ranks(dist, "cpu", ms, counts)
        solves = [(0, 10), (0, 20), (0, 30)]
        mine = [bench.rank_solve(solves, rank, k) for k in range(3)]
        q.put((rank, t, tot, mine))
    finally:
        dist.destroy_process_group()


def test_combine_ranks_gloo_world2():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, tot, mine in res:
        assert t == 150.0                       # slowest rank
        assert tot == {"edges": 3000, "solves": 6, "phases": 15}
    # ranks start at different sources and each covers every solve once per cycle
    assert res[0][3][0] != res[1][3][0]
    assert sorted(res[0][3]) == sorted(res[1][3])


def test_combine_ranks_single_process():
    sys.path.insert(0, ROOT)
    import bench
    t, tot = bench.combine_ranks(None, "cpu", 12.5, {"edges": 5})
    assert t == 12.5 and tot == {"edges": 5}


def test_reference_arm_torchrun_world2():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port),
           "bench.py", "--impl", "reference", "--gpus", "2", "--workload", "1", "--steps", "2", "--warmup", "1"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    rec = json.loads(lines[0])
    assert rec["impl"] == "reference" and rec["n_gpus"] == 2 and rec["value"] > 0
    assert rec["e2e"]["h2d_bytes_per_step"] == 0 and rec["cpu_baseline"]["kind"] == "oracle"
