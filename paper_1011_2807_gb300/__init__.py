"""GB300 sparse-vector KNN join (inverted-index join with threshold refinement).

The compute path is the CUDA library ``libknnjoin.so`` (C ABI in include/knn_join.h);
:mod:`.binding` marshals arguments to it.  :mod:`.synth` draws seeded inputs.
"""
from .binding import (Batch, DeviceCSR, Index, KnnError, ThresholdModel, knn_join,  # noqa: F401
                      knn_join_batched, knn_join_build_index, knn_join_learned, knn_join_noalloc,
                      knn_kernel_launch_count, knn_last_error, knn_merge_topk, knn_version, lib,
                      spectra_parse, spectra_read)
