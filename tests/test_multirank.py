"""Host-side multi-rank logic of bench.py on CPU with gloo, world size 2: the
job's time is the slowest rank's, the value counts every rank's transforms, and
only rank 0 reports.  (Replicas share nothing on the data path, so no GPU
collective exists to test.)"""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    d = bench.init_dist(world)
    assert d is not None and dist.get_backend() == "gloo"
    ms = bench.max_over_ranks(d, 100.0 * (rank + 1), "cpu")
    val = bench.job_value(10, 64, world, ms)

    # a bounded reference-arm run (bench's own argument defaults): only rank 0 times and prints
    A = bench.parse(["--n", "64", "--steps", "1", "--warmup", "0", "--batch", "64"])
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(A, rank, world)
    out[rank] = (ms, val, buf.getvalue())
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 200.0
    assert res[0][1] == res[1][1] == pytest.approx(10 * 64 * 2 / 0.2)
    assert '"impl": "reference"' in res[0][2] and res[1][2] == ""
