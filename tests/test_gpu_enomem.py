"""Running out of device memory, simulated on the host through the allocator hook.

An allocator callback (knn_set_allocator) that returns NULL on its n-th call stands in
for an exhausted device.  For every n up to the number of allocations a call makes,
the index build, the join and the batched form must return KNN_ENOMEM, give back every
buffer they obtained before the failure, and leave the library usable: the next call
with a working allocator returns the exact result.  No GPU fault is involved: the
failing call never reaches a kernel that would use the missing buffer.
"""
import numpy as np
import pytest

from paper_1011_2807_gb300 import synth
import compare

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def knn():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1011_2807_gb300 as knn
    knn.lib()
    return knn


class FailingAllocator:
    """Delegates to torch's caching allocator, but returns NULL on call `fail_at`
    (1-based); records what is still outstanding."""

    def __init__(self, knn, fail_at):
        import torch
        self.knn, self.fail_at, self.calls = knn, fail_at, 0
        self.outstanding = {}
        B = knn.binding

        def alloc(nbytes, stream, ctx):
            self.calls += 1
            if self.calls == self.fail_at:
                return None
            p = torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))
            self.outstanding[int(p)] = int(nbytes)
            return p

        def free(ptr, nbytes, stream, ctx):   # buffers from before the install come back here too
            self.outstanding.pop(int(ptr), None)
            torch.cuda.caching_allocator_delete(int(ptr))

        self.cbs = (B._ALLOC_FN(alloc), B._FREE_FN(free))

    def __enter__(self):
        assert self.knn.lib().knn_set_allocator(self.cbs[0], self.cbs[1], None) == 0
        return self

    def __exit__(self, *exc):
        B = self.knn.binding
        assert self.knn.lib().knn_set_allocator(B._alloc_cbs[0], B._alloc_cbs[1], None) == 0


def fail_each_allocation(knn, call, limit=64):
    """Runs call() with the n-th allocation failing, n = 1, 2, ... until it succeeds;
    every failing run must report KNN_ENOMEM and leave nothing allocated.  Returns
    (the successful call's result, the number of failing runs)."""
    import torch
    from paper_1011_2807_gb300.binding import KNN_ENOMEM, KnnError
    for n in range(1, limit + 1):
        with FailingAllocator(knn, n) as fa:
            try:
                out = call()
                torch.cuda.synchronize()
            except KnnError as e:
                torch.cuda.synchronize()
                assert e.status == KNN_ENOMEM, (n, e)
                assert not fa.outstanding, (n, fa.outstanding)
                continue
        return out, n - 1
    raise AssertionError(f"still failing after {limit} allocations")


def test_build_index_enomem(knn, oracle_mod):
    S = synth.spectrum_u8(5000, 951, role="S")
    idx, fails = fail_each_allocation(knn, lambda: knn.knn_join_build_index(S, block_size=1024))
    assert fails >= 5                      # the build allocates several arrays
    R = synth.spectrum_u8(50, 952, role="R")
    ids, sc = knn.knn_join(idx, knn.DeviceCSR.from_host(R), 5)
    eids, esc, _ = oracle_mod.iib_join(R, S, 5, threads=8)
    compare.assert_exact(ids.cpu().numpy(), sc.cpu().numpy(), eids, esc, "index built after ENOMEM")
    idx.close()


@pytest.mark.parametrize("kw", [dict(), dict(s_groups=3), dict(outputs_on_host=True)])
def test_join_enomem(knn, oracle_mod, kw):
    import torch
    S = synth.spectrum_u8(6000, 961, role="S")
    R = synth.spectrum_u8(70, 962, role="R")        # host R: the call uploads it
    idx = knn.knn_join_build_index(S, block_size=1024)
    k = 5
    if kw.get("outputs_on_host"):
        ids = torch.empty((R.n_rows, k), dtype=torch.int32, pin_memory=True)
        sc = torch.empty((R.n_rows, k), dtype=torch.int32, pin_memory=True)
        call = lambda: knn.knn_join(idx, R, k, out_ids=ids, out_scores=sc, **kw)
    else:
        call = lambda: knn.knn_join(idx, R, k, **kw)
    (ids, sc), fails = fail_each_allocation(knn, call)
    assert fails >= 1
    eids, esc, _ = oracle_mod.iib_join(R, S, k, threads=8)
    compare.assert_exact(ids.cpu().numpy(), sc.cpu().numpy(), eids, esc, f"join after ENOMEM {kw}")
    # and a plain call with the working allocator afterwards
    ids, sc = knn.knn_join(idx, knn.DeviceCSR.from_host(R), k)
    compare.assert_exact(ids.cpu().numpy(), sc.cpu().numpy(), eids, esc, "join after ENOMEM runs")
    idx.close()


def test_batch_create_enomem(knn, oracle_mod):
    import torch
    S = synth.spectrum_u8(8000, 971, role="S")
    idx = knn.knn_join_build_index(S, block_size=2048)     # 4 S blocks, 2 per group
    Rs = [synth.spectrum_u8(n, 972 + i, role="R") for i, n in enumerate((40, 90))]
    jobs = [(idx, knn.DeviceCSR.from_host(R), k) for R, k in zip(Rs, (5, 9))]
    b, fails = fail_each_allocation(knn, lambda: knn.Batch(jobs, use_graph=False, blocks_per_group=2))
    assert fails >= 1
    b.launch()
    torch.cuda.synchronize()
    for (ids, sc), R, k in zip(b.outputs, Rs, (5, 9)):
        eids, esc, _ = oracle_mod.iib_join(R, S, k, threads=8)
        compare.assert_exact(ids.cpu().numpy(), sc.cpu().numpy(), eids, esc, "batch after ENOMEM")
    b.close()
    idx.close()
