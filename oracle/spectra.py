"""CPU oracle of the spectra preprocessing -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU legs of ``bench.py`` may import
this module; it shares no code with the library's reader and never calls it.

Section 5 (experimental results) turns each MS/MS spectrum into one sparse vector:
every peak is a feature, the peak's m/z multiplied by 10 is the dimension index, and
its intensity is the value.  :func:`spectra_to_csr` restates that in plain Python, one
spectrum and one peak at a time, with the readings the paper leaves open:

* dimension = floor(m/z * mz_scale) (mz_scale 10), where a product within 2^-20 below
  an integer counts as that integer (decimal m/z such as 0.7 whose binary value falls
  just short of the bin its digits name);
* two peaks of one spectrum in the same dimension: the larger intensity ("max"), or
  their sum in file order ("sum");
* a peak whose intensity is <= min_intensity (default 0) is dropped: weights are > 0;
* float32 weights: the intensity rounded to float32 (a value that rounds to 0 is
  dropped); uint8 weights: ceil(100 * I / I_max), I_max the spectrum's largest merged
  intensity.

:func:`read_peak_lists` is a plain reader of the two text formats (MGF: BEGIN IONS /
KEY=VALUE / "m/z intensity [charge]" / END IONS; MS2: H, S, I, Z, D records and "m/z
intensity" lines), returning each spectrum's peaks in file order.

Parity status: pinned by ``tests/test_spectra_cpu.py`` -- a hand-worked MGF example
(``tests/golden/spectra_small.mgf`` with its expected vectors worked out by hand from
the rule above), and invariants that a slip in the binning, the merge or the weight
rule breaks (each kept peak lies in its bin's m/z interval; max-merged values are
peak intensities; sum merging keeps each spectrum's total; uint8 rows peak at 100).
"""
from __future__ import annotations

import math

import numpy as np

BIN_SNAP = 2.0 ** -20


def read_peak_lists(text: str, fmt: str = "auto"):
    """[[(mz, intensity), ...] per spectrum] in file order, from MGF or MS2 text."""
    lines = text.replace("\r\n", "\n").split("\n")
    body = [ln.strip() for ln in lines]
    body = [ln for ln in body if ln and ln[0] not in "#;!"]
    if fmt == "auto":
        if not body:
            return []
        first = body[0]
        if first.upper() == "BEGIN IONS" or "=" in first:
            fmt = "mgf"
        elif first[0] in "HS" and (len(first) == 1 or first[1] in " \t"):
            fmt = "ms2"
        else:
            raise ValueError("neither MGF nor MS2")
    spectra = []
    if fmt == "mgf":
        cur = None
        for ln in body:
            if cur is None:
                if ln.upper() == "BEGIN IONS":
                    cur = []
                elif ln.upper() == "END IONS":
                    raise ValueError("END IONS without BEGIN IONS")
                continue
            if ln.upper() == "END IONS":
                spectra.append(cur)
                cur = None
            elif ln.upper() == "BEGIN IONS":
                raise ValueError("BEGIN IONS inside a spectrum")
            elif ln[0].isalpha():
                if "=" not in ln:
                    raise ValueError(f"not a header: {ln!r}")
            else:
                fields = ln.split()
                if len(fields) < 2:
                    raise ValueError(f"not a peak: {ln!r}")
                spectra_peak(cur, fields)
        if cur is not None:
            raise ValueError("no END IONS")
    else:
        cur = None
        for ln in body:
            if ln[0].isalpha():
                if len(ln) > 1 and ln[1] not in " \t":
                    raise ValueError(f"bad record: {ln!r}")
                if ln[0] == "S":
                    if cur is not None:
                        spectra.append(cur)
                    cur = []
                elif ln[0] == "H":
                    if cur is not None or spectra:
                        raise ValueError("H after the first spectrum")
                elif ln[0] in "IZD":
                    if cur is None:
                        raise ValueError("record before the first S")
                else:
                    raise ValueError(f"unknown record {ln[0]!r}")
            else:
                if cur is None:
                    raise ValueError("peak before the first S")
                fields = ln.split()
                if len(fields) < 2:
                    raise ValueError(f"not a peak: {ln!r}")
                spectra_peak(cur, fields)
        if cur is not None:
            spectra.append(cur)
    return spectra


def spectra_peak(cur, fields):
    mz, inten = float(fields[0]), float(fields[1])
    if not math.isfinite(mz) or mz < 0.0 or not math.isfinite(inten):
        raise ValueError("bad peak")
    cur.append((mz, inten))


def dimension_of(mz: float, mz_scale: float = 10.0) -> int:
    """Section 5: the m/z times 10, as an integer index (the binary snap above)."""
    x = mz * mz_scale
    d = math.floor(x)
    if x - d >= 1.0 - BIN_SNAP:
        d += 1
    return int(d)


def spectra_to_csr(spectra, *, mz_scale: float = 10.0, merge: str = "max", weights: str = "f32",
                   dim: int = 0, min_intensity: float = 0.0):
    """(indptr int64, indices int32, values float32|uint8, dim) of the spectra."""
    indptr, indices, values = [0], [], []
    max_d = -1
    for peaks in spectra:
        bins = {}       # dimension -> merged intensity
        order = []
        for mz, inten in peaks:
            if not inten > min_intensity:
                continue
            d = dimension_of(mz, mz_scale)
            if dim > 0 and d >= dim:
                raise ValueError("dimension past dim")
            if d not in bins:
                bins[d] = inten
                order.append(d)
            elif merge == "sum":
                bins[d] = bins[d] + inten
            else:
                bins[d] = max(bins[d], inten)
        ds = sorted(order)
        if weights == "u8":
            imax = max((bins[d] for d in ds), default=0.0)
            for d in ds:
                c = math.ceil(100.0 * bins[d] / imax)
                indices.append(d)
                values.append(min(100, max(1, c)))
                max_d = max(max_d, d)
        else:
            for d in ds:
                f = np.float32(bins[d])
                if not f > 0:
                    continue
                indices.append(d)
                values.append(f)
                max_d = max(max_d, d)
        indptr.append(len(indices))
    out_dim = dim if dim > 0 else max(1, max_d + 1)
    vdt = np.uint8 if weights == "u8" else np.float32
    return (np.asarray(indptr, np.int64), np.asarray(indices, np.int32), np.asarray(values, vdt), out_dim)
