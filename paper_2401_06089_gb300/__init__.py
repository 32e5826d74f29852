"""GB300-native single-linkage dendrograms of weighted trees (PANDORA method).

The compute path is a C-ABI CUDA library (``libpandora.so``, sm_103a) whose
entry points are declared in ``include/pandora.h``; this package is a thin
ctypes binding over it.  Nothing is loaded at import time; the first call
loads the library and raises if it is missing or no GPU is present.  There is
no CPU fallback.
"""
from ._binding import (  # noqa: F401
    PandoraError,
    dendrogram,
    dendrogram_async,
    dendrogram_batched,
    dendrogram_batched_async,
    dendrogram_batched_planned,
    dendrogram_host,
    get_tuning,
    hdbscan_labels,
    library_path,
    load_tuning,
    profile_read,
    profile_start,
    load_library,
    membench,
    mr_emst,
    set_tuning,
    set_wait_report_limit,
    sort_pairs,
    status_string,
    workspace_size,
    workspace_status,
)
