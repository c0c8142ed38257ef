"""Spectra files to KNN join: R as MGF, S as MS2 (seeded synthetic peak lists, with the
noise real files carry), read by the library with a shared dimension, indexed and joined
on the GPU; results against the oracle's brute force on the oracle's own reading of the
same files (uint8 bit-exact, float32 within the float tolerance)."""
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


@pytest.mark.parametrize("weights", ["u8", "f32"])
def test_spectra_files_join(knn, oracle_mod, tmp_path, weights):
    from oracle import spectra as osp
    r_text = synth.spectra_text(150, 1401, fmt="mgf")
    s_text = synth.spectra_text(6000, 1402, fmt="ms2", peaks_lo=20, peaks_hi=60)
    (tmp_path / "r.mgf").write_bytes(r_text.encode())
    (tmp_path / "s.ms2").write_bytes(s_text.encode())
    dim = 10000
    R, _ = knn.spectra_read(str(tmp_path / "r.mgf"), weights=weights, dim=dim)
    S, _ = knn.spectra_read(str(tmp_path / "s.ms2"), weights=weights, dim=dim)
    # the oracle reads the files its own way; the vectors must be the same
    for X, text in ((R, r_text), (S, s_text)):
        ip, ix, v, d = osp.spectra_to_csr(osp.read_peak_lists(text), weights=weights, dim=dim)
        assert np.array_equal(X.indptr, ip) and np.array_equal(X.indices, ix) and np.array_equal(X.values, v)
    k = 10
    eids, esc, _ = oracle_mod.bf_join(R, S, k, threads=8)
    idx = knn.knn_join_build_index(S, block_size=2048)
    for mode in ("iiib", "iib"):
        ids, sc = knn.knn_join(idx, R, k, mode=mode)
        ids, sc = ids.cpu().numpy(), sc.cpu().numpy()
        if weights == "u8":
            compare.assert_exact(ids, sc, eids, esc, f"spectra {mode}")
        else:
            compare.assert_close(R, S, list(range(R.n_rows)), ids, sc, eids, esc, what=f"spectra {mode}")
    idx.close()


def test_spectra_join_command(knn, tmp_path, capsys):
    """The command-line join of two spectra files writes what knn_join returns."""
    import json
    from paper_1011_2807_gb300 import spectra_join
    (tmp_path / "r.mgf").write_bytes(synth.spectra_text(60, 1411, fmt="mgf").encode())
    (tmp_path / "s.ms2").write_bytes(synth.spectra_text(3000, 1412, fmt="ms2", peaks_hi=80).encode())
    out = tmp_path / "knn.npz"
    assert spectra_join.main([str(tmp_path / "r.mgf"), str(tmp_path / "s.ms2"), "-k", "5", "--weights", "u8",
                              "--out", str(out)]) == 0
    summary = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    got = np.load(out)
    R, _ = knn.spectra_read(str(tmp_path / "r.mgf"), weights="u8")
    S, _ = knn.spectra_read(str(tmp_path / "s.ms2"), weights="u8")
    dim = max(R.dim, S.dim)
    assert summary["dim"] == dim and summary["r"]["n_spectra"] == 60
    R = synth.CSR(R.indptr, R.indices, R.values, dim)
    S = synth.CSR(S.indptr, S.indices, S.values, dim)
    idx = knn.knn_join_build_index(S)
    ids, sc = knn.knn_join(idx, knn.DeviceCSR.from_host(R), 5)
    assert np.array_equal(got["ids"], ids.cpu().numpy()) and np.array_equal(got["scores"], sc.cpu().numpy())
    idx.close()
