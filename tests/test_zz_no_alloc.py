"""knn_join_noalloc, the entry point that allocates no device memory, against knn_join.

Some callers cannot let a library allocate device memory while a call runs (a process
that has divided the GPU into its own fixed pools, or a latency-critical loop that must
not pay for an allocation or for the synchronisation a free can trigger).  For them
knn_join_noalloc works in the library's one fixed scratch array.  These tests call it
through the C ABI and check that it returns exactly what knn_join returns, on two calls
in a row with different inputs (the array keeps the previous call's contents), and
that it refuses work that does not fit its scratch.

This file is collected last on purpose, and passes both alone and after the others.
"""
import ctypes

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


class CountingAllocator:
    """Installs allocator callbacks that count calls (and delegate to torch)."""

    def __init__(self, knn):
        import torch
        self.knn, self.n_alloc, self.n_free = knn, 0, 0
        B = knn.binding

        def alloc(nbytes, stream, ctx):
            self.n_alloc += 1
            return torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))

        def free(ptr, nbytes, stream, ctx):
            self.n_free += 1
            torch.cuda.caching_allocator_delete(int(ptr))

        self.cbs = (B._ALLOC_FN(alloc), B._FREE_FN(free))

    def __enter__(self):
        assert self.knn.lib().knn_set_allocator(self.cbs[0], self.cbs[1], None) == 0
        return self

    def __exit__(self, *exc):
        B = self.knn.binding
        assert self.knn.lib().knn_set_allocator(B._alloc_cbs[0], B._alloc_cbs[1], None) == 0


def test_noalloc_equals_knn_join_on_two_calls(knn):
    import torch
    S = synth.spectrum_u8(60000, 911, role="S")
    idx = knn.knn_join_build_index(S, block_size=4096)          # 15 S blocks: carried top-k
    calls = [(synth.spectrum_u8(700, 912, role="R"), 5), (synth.spectrum_u8(300, 913, role="R"), 12)]
    for R, k in calls:                      # two calls in a row, different inputs
        Rd = knn.DeviceCSR.from_host(R)
        want_ids, want_sc = knn.knn_join(idx, Rd, k, s_groups=1)
        ids = torch.full((R.n_rows, k), -7, dtype=torch.int32, device="cuda")
        sc = torch.full((R.n_rows, k), -7, dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()
        with CountingAllocator(knn) as ca:
            knn.knn_join_noalloc(idx, Rd, k, ids, sc)
            torch.cuda.synchronize()
        assert ca.n_alloc == 0 and ca.n_free == 0, "knn_join_noalloc used the allocator"
        assert torch.equal(ids, want_ids) and torch.equal(sc, want_sc)    # uint8: bit-exact
    idx.close()


def test_noalloc_float_within_tolerance(knn, oracle_mod):
    import torch
    S = synth.uniform_f32(20000, 3000, 5, 40, 921)
    R = synth.uniform_f32(400, 3000, 5, 40, 922)
    idx = knn.knn_join_build_index(S, block_size=2048)
    Rd = knn.DeviceCSR.from_host(R)
    want_ids, want_sc = knn.knn_join(idx, Rd, 10, s_groups=1)
    eids, esc, _ = oracle_mod.iib_join(R, S, 10, threads=8)
    for _ in range(2):
        ids = torch.empty((R.n_rows, 10), dtype=torch.int32, device="cuda")
        sc = torch.empty((R.n_rows, 10), dtype=torch.float32, device="cuda")
        knn.knn_join_noalloc(idx, Rd, 10, ids, sc)
        torch.cuda.synchronize()
        # against the fp64 oracle: scores within 1e-5, ids equal but for boundary ties
        compare.assert_close(R, S, list(range(R.n_rows)), ids.cpu().numpy(), sc.cpu().numpy(), eids, esc,
                             what="knn_join_noalloc float")
        # and against knn_join (the same method; summation order may differ)
        np.testing.assert_allclose(sc.cpu().numpy(), want_sc.cpu().numpy(), rtol=1e-5, atol=0)
    idx.close()


def test_noalloc_refuses_what_does_not_fit(knn):
    import torch
    from paper_1011_2807_gb300.binding import KNN_EINVAL, KNN_EUNSUPPORTED, KnnError
    S = synth.spectrum_u8(3000, 931, role="S")
    idx = knn.knn_join_build_index(S)
    R = synth.spectrum_u8(40000, 932, role="R", nnz=np.full(40000, 3))
    Rd = knn.DeviceCSR.from_host(R)
    ids = torch.empty((R.n_rows, 64), dtype=torch.int32, device="cuda")
    sc = torch.empty((R.n_rows, 64), dtype=torch.int32, device="cuda")
    with pytest.raises(KnnError) as e:      # 40,000 x 64 keys > 2,097,120
        knn.knn_join_noalloc(idx, Rd, 64, ids, sc)
    assert e.value.status == KNN_EUNSUPPORTED and "scratch" in str(e.value)
    # host-resident R would need an upload buffer: refused
    c = knn.binding._csr(R, [])
    opts = knn.binding._JoinOpts()
    st = knn.lib().knn_join_noalloc(idx.handle, ctypes.byref(c), 5, ctypes.byref(opts),
                                    ids.data_ptr(), sc.data_ptr(), None)
    assert st == KNN_EINVAL and "device memory" in knn.knn_last_error()
    # a negative row count is an invalid argument, as for knn_join
    c = knn.binding._csr(Rd, [])
    c.n_rows = -1
    st = knn.lib().knn_join_noalloc(idx.handle, ctypes.byref(c), 5, ctypes.byref(opts),
                                    ids.data_ptr(), sc.data_ptr(), None)
    assert st == KNN_EINVAL and "n_rows" in knn.knn_last_error()
    idx.close()
