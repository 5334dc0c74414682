"""The N > 1 path of bench.py on CPU with two gloo ranks: every rank gets the
slowest rank's time, the whole-job rate counts the points of every replica,
replicas start from different seeded states, and the reference arm runs on
rank 0 only (the other ranks return without work or output). The GPU run of
the same path uses NCCL for the same two collectives (a barrier and one MAX
reduction); no collective touches the data path."""
import io
import contextlib
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    import synth
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    try:
        dist.barrier()
        local_ms = [12.5, 17.25][rank]
        ms = bench.max_over_ranks(local_ms, world, "cpu")
        rate = bench.whole_job_rate(1000, world, 4, ms)
        w = synth.workload("rb512", nx=16, ny=8, nz=6)
        st = bench.replica_state(w, rank)
        # the reference arm: only rank 0 prints a line
        os.environ["RANK"] = str(rank)
        buf = io.StringIO()
        args = bench.parse(["--impl", "reference", "--steps", "1", "--warmup", "0",
                                          "--grid", "16x16x8"])
        with contextlib.redirect_stdout(buf):
            bench.run_reference(args)
        out[rank] = (ms, rate, float(np.abs(st[3]).sum()), buf.getvalue())
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    (ms0, rate0, t0, line0), (ms1, rate1, t1, line1) = out[0], out[1]
    assert ms0 == ms1 == 17.25                      # max over ranks on every rank
    assert rate0 == rate1 == pytest.approx(1000 * 2 * 4 / 17.25e-3)
    assert t0 != t1                                 # different seeded replicas
    assert '"impl": "reference"' in line0 and line1 == ""
