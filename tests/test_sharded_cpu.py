"""The S-sharded join's exchange on CPU (gloo, world size 2): each rank joins the same
queries against its own range of S (the CPU oracle stands in for the GPU join), the
lists are all-gathered with their S offsets and merged (a plain sort stands in for the
GPU merge); the result must equal the oracle's join over the whole S."""
import os
import sys

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _plain_merge(parts, offsets, k):
    ids = np.concatenate([p[0].numpy() + np.where(p[0].numpy() >= 0, o, 0) for p, o in zip(parts, offsets)], axis=1)
    sc = np.concatenate([p[1].numpy() for p in parts], axis=1)
    out_i = np.full((ids.shape[0], k), -1, np.int32)
    out_s = np.zeros((ids.shape[0], k), sc.dtype)
    for r in range(ids.shape[0]):
        cand = [(-s, i) for i, s in zip(ids[r], sc[r]) if i >= 0]
        cand.sort()
        for q, (ns, i) in enumerate(cand[:k]):
            out_i[r, q], out_s[r, q] = i, -ns
    return torch.from_numpy(out_i), torch.from_numpy(out_s)


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    from paper_1011_2807_gb300 import sharded, synth
    S = synth.spectrum_u8(3001, 71, role="S")
    R = synth.spectrum_u8(40, 72, role="R")
    a, b = sharded.shard_range(S.n_rows, rank, world)
    shard = S.slice_rows(a, b)

    def cpu_join(index, Rq, k):
        ids, sc, _ = oracle.iib_join(Rq, index, k, threads=2)
        return torch.from_numpy(ids.astype(np.int32)), torch.from_numpy(sc.astype(np.int32))

    ids, sc = sharded.knn_join_sharded(shard, R, 6, a, join=cpu_join, merge=_plain_merge)
    out[rank] = (ids.numpy().tolist(), sc.numpy().tolist(), (a, b))
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_exchange_on_gloo(oracle_mod):
    from paper_1011_2807_gb300 import synth, sharded
    assert sharded.shard_range(10, 0, 3) == (0, 4) and sharded.shard_range(10, 2, 3) == (7, 10)
    port = 29700 + (os.getpid() % 1000)
    with mp.get_context("spawn").Manager() as man:
        out = man.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    S = synth.spectrum_u8(3001, 71, role="S")
    R = synth.spectrum_u8(40, 72, role="R")
    eids, esc, _ = oracle_mod.iib_join(R, S, 6, threads=2)
    assert res[0][2] == (0, 1501) and res[1][2] == (1501, 3001)
    for rank in (0, 1):
        np.testing.assert_array_equal(np.array(res[rank][0]), eids)
        np.testing.assert_array_equal(np.array(res[rank][1]), esc.astype(np.int64))
