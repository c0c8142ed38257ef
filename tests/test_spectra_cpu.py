"""Section 5's preprocessing of MS/MS spectra (peak -> feature, m/z x 10 -> dimension,
intensity -> value): the oracle pinned to a hand-worked example and to invariants checked
in exact decimal arithmetic, then the library's MGF/MS2 reader against the oracle,
element by element, on seeded synthetic files.  Host code only: no GPU."""
import math
import os
from decimal import ROUND_FLOOR, Decimal

import numpy as np
import pytest

from paper_1011_2807_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def oracle():
    from oracle import spectra
    return spectra


def golden_expected():
    """{(merge, weights): (indptr, indices, values)} from spectra_small_expected.txt."""
    out, key = {}, None
    for ln in open(os.path.join(GOLDEN, "spectra_small_expected.txt")):
        ln = ln.strip()
        if not ln or ln.startswith("#"):
            continue
        if ln.startswith("["):
            key = tuple(ln[1:-1].split())
            out[key] = {}
            continue
        name, *vals = ln.split()
        out[key][name] = [float(v) for v in vals]
    return out


def oracle_csr(text, fmt="auto", **kw):
    o = oracle()
    return o.spectra_to_csr(o.read_peak_lists(text, fmt), **kw)


@pytest.mark.parametrize("fmt", ["mgf", "ms2"])
@pytest.mark.parametrize("merge", ["max", "sum"])
@pytest.mark.parametrize("weights", ["f32", "u8"])
def test_oracle_hand_worked_example(fmt, merge, weights):
    text = open(os.path.join(GOLDEN, f"spectra_small.{fmt}"), newline="").read()
    indptr, indices, values, dim = oracle_csr(text, merge=merge, weights=weights)
    e = golden_expected()[(merge, weights)]
    assert indptr.tolist() == e["indptr"] and indices.tolist() == e["indices"]
    assert values.astype(np.float64).tolist() == e["values"] and dim == 2506


@pytest.mark.parametrize("fmt", ["mgf", "ms2"])
@pytest.mark.parametrize("merge", ["max", "sum"])
@pytest.mark.parametrize("weights", ["f32", "u8"])
def test_library_hand_worked_example(fmt, merge, weights):
    import paper_1011_2807_gb300 as knn
    csr, info = knn.spectra_read(os.path.join(GOLDEN, f"spectra_small.{fmt}"), merge=merge, weights=weights)
    e = golden_expected()[(merge, weights)]
    assert csr.indptr.tolist() == e["indptr"] and csr.indices.tolist() == e["indices"]
    assert csr.values.astype(np.float64).tolist() == e["values"] and csr.dim == 2506
    assert (info["n_spectra"], info["n_peaks"], info["n_dropped"], info["n_merged"]) == (3, 9, 2, 2)
    assert csr.values.dtype == (np.uint8 if weights == "u8" else np.float32)


def decimal_peaks(text, fmt):
    """Each spectrum's (m/z, intensity) as the Decimals the file spells, read with a
    parser of its own (independent of the oracle's)."""
    spectra, cur = [], None
    for raw in text.replace("\r", "").split("\n"):
        ln = raw.strip()
        if not ln or ln[0] in "#;!":
            continue
        if fmt == "mgf":
            if ln == "BEGIN IONS":
                cur = []
            elif ln == "END IONS":
                spectra.append(cur)
                cur = None
            elif cur is not None and not ln[0].isalpha():
                f = ln.split()
                cur.append((Decimal(f[0]), Decimal(f[1])))
        else:
            if ln[0] == "S":
                if cur is not None:
                    spectra.append(cur)
                cur = []
            elif not ln[0].isalpha():
                f = ln.split()
                cur.append((Decimal(f[0]), Decimal(f[1])))
    if fmt == "ms2" and cur is not None:
        spectra.append(cur)
    return spectra


@pytest.mark.parametrize("fmt", ["mgf", "ms2"])
def test_oracle_invariants_in_exact_decimals(fmt):
    """On 40 synthetic spectra (4-decimal m/z, so the binary snap never decides): the
    dimensions are floor(10 m/z) in exact decimal arithmetic, max-merged values are the
    largest kept intensity of their bin, sums keep each spectrum's kept total, rows are
    ascending, uint8 rows peak at 100 and stay in 1..100."""
    text = synth.spectra_text(40, 71 if fmt == "mgf" else 72, fmt=fmt)
    peaks = decimal_peaks(text, fmt)
    mx = oracle_csr(text, merge="max")
    sm = oracle_csr(text, merge="sum")
    u8 = oracle_csr(text, merge="max", weights="u8")
    assert len(peaks) == len(mx[0]) - 1 == 40
    for i, pk in enumerate(peaks):
        bins = {}
        for mz, w in pk:
            if w > 0:
                d = int((mz * 10).to_integral_value(rounding=ROUND_FLOOR))
                bins.setdefault(d, []).append(w)
        a, b = mx[0][i], mx[0][i + 1]
        ds = mx[1][a:b].tolist()
        assert ds == sorted(bins) and all(x < y for x, y in zip(ds, ds[1:]))
        for d, v in zip(ds, mx[2][a:b]):
            assert v == np.float32(float(max(bins[d])))
        total = float(sum(sum(ws) for ws in bins.values()))
        assert math.isclose(float(sm[2][sm[0][i]:sm[0][i + 1]].astype(np.float64).sum()), total, rel_tol=1e-6)
        q = u8[2][u8[0][i]:u8[0][i + 1]]
        if q.size:
            assert q.max() == 100 and q.min() >= 1


@pytest.mark.parametrize("fmt", ["mgf", "ms2"])
@pytest.mark.parametrize("merge", ["max", "sum"])
@pytest.mark.parametrize("weights", ["f32", "u8"])
@pytest.mark.parametrize("seed", [1, 2])
def test_library_matches_oracle(fmt, merge, weights, seed):
    import paper_1011_2807_gb300 as knn
    text = synth.spectra_text(120, 900 + seed, fmt=fmt)
    csr, info = knn.spectra_parse(text, merge=merge, weights=weights)
    indptr, indices, values, dim = oracle_csr(text, merge=merge, weights=weights)
    assert np.array_equal(csr.indptr, indptr) and np.array_equal(csr.indices, indices)
    assert csr.values.dtype == values.dtype and np.array_equal(csr.values, values)
    assert csr.dim == dim and info["n_spectra"] == 120 and info["n_features"] == indices.size
    assert info["n_dropped"] > 0 and info["n_merged"] > 0   # the noise reached both rules


def test_library_fixed_dim_scale_and_threshold():
    import paper_1011_2807_gb300 as knn
    text = synth.spectra_text(30, 31, fmt="mgf")
    csr, _ = knn.spectra_parse(text, dim=10000)
    assert csr.dim == 10000
    kw = dict(mz_scale=100.0, min_intensity=500.0, dim=100000)
    csr, info = knn.spectra_parse(text, **kw)
    indptr, indices, values, dim = oracle_csr(text, **kw)
    assert np.array_equal(csr.indptr, indptr) and np.array_equal(csr.indices, indices)
    assert np.array_equal(csr.values, values) and csr.dim == dim == 100000
    assert values.min() > 500.0


def test_library_reads_files_as_it_parses_text(tmp_path):
    import paper_1011_2807_gb300 as knn
    for fmt in ("mgf", "ms2"):
        text = synth.spectra_text(25, 41, fmt=fmt)
        path = tmp_path / f"s.{fmt}"
        path.write_bytes(text.encode())
        a, ia = knn.spectra_read(str(path))
        b, ib = knn.spectra_parse(text)
        assert ia == ib
        assert all(np.array_equal(getattr(a, f), getattr(b, f)) for f in ("indptr", "indices", "values"))


def test_library_empty_and_comment_only_inputs():
    import paper_1011_2807_gb300 as knn
    for text in ("", "# nothing here\r\n; still nothing\n"):
        csr, info = knn.spectra_parse(text)
        assert csr.n_rows == 0 and csr.dim == 1 and info["n_spectra"] == 0
    csr, _ = knn.spectra_parse("BEGIN IONS\nTITLE=empty\nEND IONS\n")
    assert csr.indptr.tolist() == [0, 0]


@pytest.mark.parametrize("text, fmt", [
    ("BEGIN IONS\n100 5\n", "auto"),                       # no END IONS
    ("END IONS\n", "mgf"),                                 # END without BEGIN
    ("BEGIN IONS\nBEGIN IONS\nEND IONS\n", "auto"),        # nested BEGIN
    ("BEGIN IONS\nnot a peak\nEND IONS\n", "auto"),        # neither header nor peak
    ("BEGIN IONS\n100.5\nEND IONS\n", "auto"),             # a peak without intensity
    ("BEGIN IONS\n100.5 abc\nEND IONS\n", "auto"),         # not a number
    ("BEGIN IONS\n-1 5\nEND IONS\n", "auto"),              # negative m/z
    ("BEGIN IONS\n100 inf\nEND IONS\n", "auto"),           # non-finite intensity
    ("100 5\n", "auto"),                                   # no format
    ("100 5\n", "ms2"),                                    # a peak before the first S
    ("S 1 1 100\nX 1\n", "ms2"),                           # unknown record
    ("S 1 1 100\n10 1\nH late\n", "ms2"),                  # H after a spectrum
    ("Z 2 100\nS 1 1 1\n", "ms2"),                         # Z before the first S
])
def test_library_rejects_malformed_input(text, fmt):
    import paper_1011_2807_gb300 as knn
    from paper_1011_2807_gb300.binding import KNN_EINVAL, KnnError
    with pytest.raises(KnnError) as e:
        knn.spectra_parse(text, fmt=fmt)
    assert e.value.status == KNN_EINVAL
    with pytest.raises(ValueError):    # the oracle rejects the same inputs
        oracle_csr(text, fmt=fmt)


def test_library_rejects_bad_options_and_dimensions():
    import paper_1011_2807_gb300 as knn
    from paper_1011_2807_gb300.binding import KNN_EINVAL, KnnError
    text = "BEGIN IONS\n100.05 5\nEND IONS\n"
    for kw in (dict(mz_scale=-1.0), dict(min_intensity=-1.0), dict(dim=-3), dict(dim=1000)):
        with pytest.raises(KnnError) as e:
            knn.spectra_parse(text, **kw)
        assert e.value.status == KNN_EINVAL, kw
    with pytest.raises(KnnError) as e:
        knn.spectra_read("/nonexistent/spectra.mgf")
    assert e.value.status == KNN_EINVAL
    with pytest.raises(ValueError):
        knn.spectra_parse(text, merge="mean")


@pytest.mark.parametrize("fmt", ["mgf", "ms2"])
@pytest.mark.parametrize("chunk", [700, 5000, 60000])
def test_library_chunked_parse_equals_one_pass(fmt, chunk):
    """Cut into chunks of ~chunk bytes at spectrum starts and parsed by host threads, the
    input gives exactly the rows of one sequential pass (and of the oracle)."""
    import paper_1011_2807_gb300 as knn
    text = synth.spectra_text(150, 1500 + chunk, fmt=fmt)
    assert len(text) > 20 * chunk or chunk == 60000
    one, i1 = knn.spectra_parse(text, merge="sum", chunk_bytes=1 << 40)
    many, im = knn.spectra_parse(text, merge="sum", chunk_bytes=chunk)
    assert i1 == im
    for f in ("indptr", "indices", "values"):
        assert np.array_equal(getattr(one, f), getattr(many, f))
    indptr, indices, values, dim = oracle_csr(text, merge="sum")
    assert np.array_equal(many.indptr, indptr) and np.array_equal(many.values, values) and many.dim == dim


@pytest.mark.parametrize("fmt, bad", [
    ("mgf", "not a peak\n"),          # a line that is neither a header nor a peak
    ("mgf", "BEGIN IONS\n"),          # a spectrum left open: reported at the next BEGIN IONS
    ("ms2", "X 1\n"),                 # an unknown record
    ("ms2", "12.5\n"),                # a peak without intensity
])
def test_library_chunked_errors_match_one_pass(fmt, bad):
    """A malformed line deep in the input: parsed in many chunks, the error (status and
    message, line number included) is the one a sequential pass reports."""
    import paper_1011_2807_gb300 as knn
    from paper_1011_2807_gb300.binding import KnnError
    lines = synth.spectra_text(80, 1601, fmt=fmt, noise=False).split("\n")
    at = int(len(lines) * 0.7)
    if fmt == "mgf":   # put it inside a spectrum
        while lines[at] in ("BEGIN IONS", "END IONS") or "=" in lines[at]:
            at += 1
    text = "\n".join(lines[:at] + [bad.rstrip("\n")] + lines[at:])
    errs = []
    for chunk in (1 << 40, 900):
        with pytest.raises(KnnError) as e:
            knn.spectra_parse(text, chunk_bytes=chunk)
        errs.append((e.value.status, str(e.value)))
    assert errs[0] == errs[1], errs
    assert f"line {at + 1}" in errs[0][1] or (bad == "BEGIN IONS\n" and f"line " in errs[0][1])
