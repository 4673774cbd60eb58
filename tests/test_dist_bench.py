"""Multi-process path of bench.py on CPU (gloo, world size 2): each rank times
its own replica; the job's time is the maximum over ranks."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench

    class A:
        impl = "reference"   # selects gloo

    w, r, local, pg = bench.dist_setup(A())
    t = bench.max_over_ranks(10.0 + 5.0 * rank, pg, device="cpu")
    pg.barrier()
    q.put((r, w, t))
    pg.destroy_process_group()


def test_max_over_ranks_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    res = sorted(q.get(timeout=10) for _ in range(2))
    assert [r for r, _, _ in res] == [0, 1]
    assert all(w == 2 for _, w, _ in res)
    assert all(t == 15.0 for _, _, t in res)


def test_single_process_needs_no_group():
    import bench
    os.environ.pop("WORLD_SIZE", None)

    class A:
        impl = "ours"

    w, r, local, pg = bench.dist_setup(A())
    assert (w, r, pg) == (1, 0, None)
    assert bench.max_over_ranks(3.5, None) == 3.5


def test_flop_and_byte_models():
    import bench
    # 2 * 2.5 N log2 N per pair, N = 1024^3
    assert bench.pair_flops(1024, 1024, 1024) == pytest.approx(5 * 2 ** 30 * 30)
    # three passes, each reading and writing the array: 25.81 GB per transform in FP32
    assert bench.pass_bytes(1024, 1024, 1024, 4) / 1e9 == pytest.approx(25.81, abs=0.01)


def test_reference_arm_under_torchrun():
    """bench.py --impl reference launched as the two-rank job of a scaling run:
    rank 0 alone runs the oracle, on the host's cores (torchrun's one OpenMP
    thread per rank is lifted for it), and prints one line; the other rank
    exits 0 without work."""
    import json
    import subprocess
    import sys
    import bench
    port = _free_port()
    r = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
                        "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl",
                        "reference", "--ref-n", "32", "--steps", "1", "--warmup", "3"],
                       capture_output=True, text=True, timeout=300, cwd=bench.ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.strip().splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2
    assert line["cpu_baseline"]["cores"] == len(os.sched_getaffinity(0))
