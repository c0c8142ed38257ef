"""Joins two MS/MS spectra files on the GPU (Section 5's setting: every spectrum of R
against all spectra of S, e.g. Yeast as R and Worm as S).

    python -m paper_1011_2807_gb300.spectra_join R.ms2 S.mgf -k 10 --out knn.npz

Both files are read by the library (knn_spectra_read: peak -> feature, m/z x 10 ->
dimension, intensity -> value) with one shared dimension, S is indexed on the device and
R joined against it; the result (ids and scores, [|R|, k], best first, -1 / 0 padding)
goes to an .npz file, and a one-line JSON summary to stdout.
"""
from __future__ import annotations

import argparse
import json
import time


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("r", help="query spectra (MGF or MS2)")
    ap.add_argument("s", help="database spectra (MGF or MS2)")
    ap.add_argument("-k", type=int, default=10)
    ap.add_argument("--weights", choices=("f32", "u8"), default="f32",
                    help="float32 intensities, or uint8 ceil(100 I / I_max) per spectrum")
    ap.add_argument("--merge", choices=("max", "sum"), default="max",
                    help="two peaks of a spectrum in one dimension: the larger intensity or the sum")
    ap.add_argument("--mz-scale", type=float, default=10.0, help="dimension = floor(m/z x this)")
    ap.add_argument("--min-intensity", type=float, default=0.0, help="drop peaks at or below this")
    ap.add_argument("--dim", type=int, default=0, help="shared dimension (0: from the files)")
    ap.add_argument("--mode", choices=("iiib", "iib", "bf"), default="iiib")
    ap.add_argument("--out", default="knn.npz")
    a = ap.parse_args(argv)

    import numpy as np
    import torch
    from . import binding as B
    from .synth import CSR

    kw = dict(weights=a.weights, merge=a.merge, mz_scale=a.mz_scale, min_intensity=a.min_intensity)
    t0 = time.perf_counter()
    R, ri = B.spectra_read(a.r, dim=a.dim, **kw)
    S, si = B.spectra_read(a.s, dim=a.dim, **kw)
    dim = a.dim or max(R.dim, S.dim)
    R = CSR(R.indptr, R.indices, R.values, dim)
    S = CSR(S.indptr, S.indices, S.values, dim)
    read_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    idx = B.knn_join_build_index(S)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    Rd = B.DeviceCSR.from_host(R)
    t0 = time.perf_counter()
    ids, scores = B.knn_join(idx, Rd, a.k, mode=a.mode)
    torch.cuda.synchronize()
    join_s = time.perf_counter() - t0
    np.savez(a.out, ids=ids.cpu().numpy(), scores=scores.cpu().numpy())
    idx.close()
    print(json.dumps({"r": ri, "s": si, "dim": dim, "k": a.k, "mode": a.mode, "read_s": read_s,
                      "index_build_s": build_s, "join_s": join_s,
                      "rows_per_s": R.n_rows / join_s if join_s > 0 else None, "out": a.out}))
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
