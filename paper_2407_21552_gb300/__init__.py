"""GB300-native partitioned distance maps for fast transfer-function updates.

Rauter, Zimmermann & Zeilinger, "Accelerating Transfer Function Update for Distance Map
based Volume Rendering" (IEEE VIS 2024): K partitioned distance maps are built once per
volume (§3.1), and each TF change combines the active ones with an element-wise min
(§3.1 steps 1-2, Eq. 1) instead of recomputing the distance map.

Every step runs in hand-written sm_103a CUDA kernels behind the C ABI of libdm
(include/dm.h); this package is the ctypes binding (``_abi``, same names as the C ABI)
and a torch-buffer wrapper (``maps.PartitionedDistanceMaps``).  Importing the package
does not load the library; the first call does, and fails loudly if it is not built.
"""
from . import _abi  # noqa: F401
from ._abi import (DM_OK, DM_ERR_INVALID_ARG, DM_ERR_UNSUPPORTED, DM_ERR_CUDA,  # noqa: F401
                   DM_ERR_NOT_BOUND, DM_U8, DM_U16, DM_OCC_MINMAX, DM_OCC_EXACT, DM_INDEX_NONE,
                   DM_INDEX_RANGES, DmError,
                   dm_create, dm_query_sizes, dm_bind, dm_build_partitions,
                   dm_build_partitions_batch, dm_update_tf, dm_update_tf_host,
                   dm_full_recompute, dm_set_profile_events, dm_set_profile_counter,
                   dm_update_tf_batch,
                   dm_batch_workspace_bytes, dm_update_tf_batch_ws, dm_update_tf_noalloc,
                   dm_render,
                   dm_sync, dm_destroy,
                   dm_last_error_string, dm_status_string, dm_version, make_config)


def build(force: bool = False) -> str:
    from .build import build as _build
    return _build(force=force)


def load():
    return _abi.load()


def __getattr__(name):
    if name == "PartitionedDistanceMaps":
        from .maps import PartitionedDistanceMaps
        return PartitionedDistanceMaps
    raise AttributeError(name)
