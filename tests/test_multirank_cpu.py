"""The bench's multi-rank path on CPU (gloo, world size 2): every rank joins its own
rows (distinct query seeds), the timing is the max over ranks, and the job throughput
counts the rows of all ranks.  No GPU and no data-path collective are involved."""
import os
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_1011_2807_gb300 import synth
    ms = 100.0 + 50.0 * rank                      # a slower rank 1
    m = bench.max_over_ranks(ms, world, device="cpu")
    v = bench.job_rows_per_s(1000, world, 4, m)
    R = synth.spectrum_u8(5, bench.rank_seed(rank), role="R")
    digest = int(R.indices.sum())
    got = [None] * world
    dist.all_gather_object(got, digest)
    out[rank] = (m, v, got)
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_on_gloo():
    port = 29500 + (os.getpid() % 1000)
    with mp.get_context("spawn").Manager() as man:
        out = man.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for rank in (0, 1):
        m, v, digests = res[rank]
        assert m == 150.0                                   # max over ranks
        assert v == pytest.approx(2 * 1000 * 4 / 0.150)     # rows of both ranks
        assert digests[0] != digests[1]                     # different rows per rank
