"""The N > 1 path of bench.py without a GPU: two gloo ranks on the CPU.
bench.py runs one independent solve per GPU (replicas, no collective on the
data path); the ranks meet only to take the slowest rank's time and the sum
of their cycles, and under --impl reference only rank 0 works and prints."""
import io
import json
import os
import socket
import sys
from contextlib import redirect_stdout

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as tdist
    import bench
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    ms, cycles = bench.combine_over_ranks(10.0 * (rank + 1), 37 + rank, "cpu", True)
    # the reference arm: rank 0 alone runs the oracle and prints one line
    args = type("A", (), dict(N=32, steps=1, warmup=0))()
    buf = io.StringIO()
    with redirect_stdout(buf):
        line = bench.run_reference(args)
    tdist.barrier()
    tdist.destroy_process_group()
    out.put((rank, ms, cycles, line is not None, buf.getvalue()))


def test_two_replicas_take_the_slowest_time_and_all_cycles():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, cycles, ran, printed in res:
        assert ms == 20.0 and cycles == 75.0
        assert ran == (rank == 0)
        if rank == 0:
            d = json.loads(printed.strip().splitlines()[-1])
            assert d["impl"] == "reference" and d["value"] > 0
        else:
            assert printed == ""
