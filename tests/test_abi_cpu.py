"""CPU-side checks of the C ABI: the library builds, loads, and exports every entry
point declared in include/*.h; the binding marshals CSR arguments; the product path
refuses to run without the CUDA library."""
import ctypes
import glob
import os
import re
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"\b(knn_[a-z0-9_]+)\s*\(", src):
            names.add(m.group(1))
    # typedef'd function-pointer types are not exports
    return sorted(n for n in names if not n.endswith("_fn"))


@pytest.fixture(scope="module")
def libpath():
    from paper_1011_2807_gb300 import build_lib
    return build_lib.build()


def test_every_declared_symbol_is_exported(libpath):
    L = ctypes.CDLL(libpath)
    names = declared_functions()
    assert "knn_join" in names and "knn_join_build_index" in names
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, f"declared but not exported: {missing}"


def test_exports_match_nm(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (knn_[a-z0-9_]+)", out))
    assert set(declared_functions()) <= exported


def test_version_and_allocator_hook_without_gpu(libpath):
    import paper_1011_2807_gb300 as knn
    assert "sm_103a" in knn.knn_version()
    L = knn.lib()
    # NULL/NULL restores the default; a half-set pair is rejected
    assert L.knn_set_allocator(ctypes.cast(None, knn.binding._ALLOC_FN),
                               ctypes.cast(None, knn.binding._FREE_FN), None) == 0
    assert L.knn_set_allocator(knn.binding._alloc_cbs[0], ctypes.cast(None, knn.binding._FREE_FN), None) == 1
    assert "both" in knn.knn_last_error()
    assert L.knn_set_allocator(knn.binding._alloc_cbs[0], knn.binding._alloc_cbs[1], None) == 0


def test_null_arguments_are_rejected_without_touching_the_gpu(libpath):
    import paper_1011_2807_gb300 as knn
    L = knn.lib()
    out = ctypes.c_void_p()
    assert L.knn_join_build_index(None, None, None, ctypes.byref(out)) == knn.binding.KNN_EINVAL
    assert L.knn_join(None, None, 5, None, None, None, None) == knn.binding.KNN_EINVAL
    assert "NULL" in knn.knn_last_error()


def test_csr_marshalling():
    from paper_1011_2807_gb300 import binding, synth
    S = synth.from_rows([[(1, 2), (3, 1)], [], [(0, 7)]], 6)
    keep = []
    c = binding._csr(S, keep)
    assert c.n_rows == 3 and c.dim == 6 and c.dtype == binding.KNN_U8 and c.on_device == 0
    assert ctypes.cast(c.indptr, ctypes.POINTER(ctypes.c_int64))[3] == 3
    F = synth.from_rows([[(1, 0.5)]], 4, np.float32)
    assert binding._csr(F, keep).dtype == binding.KNN_F32
    with pytest.raises(TypeError):
        binding._csr(synth.CSR(S.indptr, S.indices, S.values.astype(np.int16), 6), keep)


def test_missing_library_fails_loudly(tmp_path):
    code = ("import paper_1011_2807_gb300.binding as b; b.LIB_PATH = '/nonexistent/libknnjoin.so'\n"
            "try:\n    b.lib()\nexcept RuntimeError as e:\n    print('RAISED', 'missing' in str(e))\n")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True)
    assert "RAISED True" in r.stdout, r.stdout + r.stderr


def test_oracle_is_not_imported_by_the_product():
    pkg = os.path.join(ROOT, "paper_1011_2807_gb300")
    for f in glob.glob(os.path.join(pkg, "**", "*.py"), recursive=True) + \
            glob.glob(os.path.join(pkg, "csrc", "*")):
        src = open(f).read()
        assert "import oracle" not in src and "from oracle" not in src and "knn_oracle" not in src, f
