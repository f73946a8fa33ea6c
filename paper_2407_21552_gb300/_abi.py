"""ctypes binding of libdm's C ABI (include/dm.h): same names, argument marshalling only.

Loading fails loudly when libdm.so has not been built: there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libdm.so")

DM_OK = 0
DM_ERR_INVALID_ARG = 1
DM_ERR_UNSUPPORTED = 2
DM_ERR_CUDA = 3
DM_ERR_NOT_BOUND = 4
DM_U8 = 1
DM_U16 = 2
DM_OCC_MINMAX = 0
DM_OCC_EXACT = 1
DM_INDEX_NONE = 0
DM_INDEX_RANGES = 1
DM_MAX_PARTITIONS = 256
DM_MAX_TF_SIZE = 65536
DM_MAX_BLOCK = 16
DM_NOALLOC_MAX_TF_SIZE = 16384
DM_NOALLOC_SCRATCH_BYTES = 4096
DM_BATCH_MAX_ITEMS = 64
DM_BATCH_MAX_EDITS_PER_GROUP = 8
DM_BUILD_BATCH_MAX_ITEMS = 64

#: every function declared in include/dm.h
EXPORTED = ("dm_create", "dm_query_sizes", "dm_bind", "dm_build_partitions",
            "dm_build_partitions_batch", "dm_update_tf",
            "dm_update_tf_host", "dm_full_recompute", "dm_set_profile_events",
            "dm_set_profile_counter",
            "dm_update_tf_noalloc", "dm_update_tf_batch", "dm_batch_workspace_bytes",
            "dm_update_tf_batch_ws", "dm_render", "dm_config_hash",
            "dm_mark_built", "dm_sync", "dm_destroy",
            "dm_last_error_string", "dm_status_string", "dm_version")


class dm_config(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int32 * 3), ("dtype", ctypes.c_int32),
                ("block", ctypes.c_int32), ("apron", ctypes.c_int32),
                ("num_partitions", ctypes.c_int32), ("borders", ctypes.POINTER(ctypes.c_int32)),
                ("tf_size", ctypes.c_int32), ("occ_mode", ctypes.c_int32),
                ("index_mode", ctypes.c_int32)]


class dm_sizes(ctypes.Structure):
    _fields_ = [("mask_bytes", ctypes.c_size_t), ("pdm_bytes", ctypes.c_size_t),
                ("plane_stride", ctypes.c_size_t), ("minmax_bytes", ctypes.c_size_t),
                ("scratch_bytes", ctypes.c_size_t), ("out_bytes", ctypes.c_size_t),
                ("grid", ctypes.c_int32 * 3), ("mask_words", ctypes.c_int32),
                ("pdm_planes", ctypes.c_int32)]


class dm_batch_item(ctypes.Structure):
    _fields_ = [("ctx", ctypes.c_void_p), ("d_tf_rgba", ctypes.c_void_p),
                ("d_out", ctypes.c_void_p)]


class dm_batch_tuning(ctypes.Structure):
    _fields_ = [("combine_ctas_per_sm", ctypes.c_int32), ("loads_per_stage", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 2)]


class dm_camera(ctypes.Structure):
    _fields_ = [("origin", ctypes.c_float * 3), ("pixel_dx", ctypes.c_float * 3),
                ("pixel_dy", ctypes.c_float * 3), ("direction", ctypes.c_float * 3),
                ("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("step", ctypes.c_float), ("ert", ctypes.c_float)]


class DmError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        super().__init__(f"{where}: {status_name(status)}" + (f" ({detail})" if detail else ""))


_lib = None


def load(path: str = LIB_PATH):
    """Load libdm.so (build it first with paper_2407_21552_gb300.build.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libdm.so not found at {path}: build the CUDA library first "
                          "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    S = ctypes.c_int32
    lib.dm_create.argtypes = [ctypes.POINTER(P), ctypes.POINTER(dm_config)]
    lib.dm_query_sizes.argtypes = [P, ctypes.POINTER(dm_sizes)]
    lib.dm_bind.argtypes = [P, P, P, P, P]
    lib.dm_build_partitions.argtypes = [P, P, P]
    lib.dm_build_partitions_batch.argtypes = [ctypes.POINTER(P), ctypes.POINTER(P), S, P]
    lib.dm_update_tf.argtypes = [P, P, P, P, P]
    lib.dm_update_tf_host.argtypes = [P, P, P, P]
    lib.dm_full_recompute.argtypes = [P, P, P, P, P]
    lib.dm_set_profile_events.argtypes = [P, P, P]
    lib.dm_set_profile_counter.argtypes = [P, P]
    lib.dm_update_tf_noalloc.argtypes = [P, ctypes.c_size_t, ctypes.c_int64, S, P, S, P, P, P]
    lib.dm_update_tf_batch.argtypes = [ctypes.POINTER(dm_batch_item), S,
                                       ctypes.POINTER(dm_batch_tuning), P]
    lib.dm_batch_workspace_bytes.argtypes = [S]
    lib.dm_batch_workspace_bytes.restype = ctypes.c_size_t
    lib.dm_update_tf_batch_ws.argtypes = [ctypes.POINTER(dm_batch_item), S,
                                          ctypes.POINTER(dm_batch_tuning), P, ctypes.c_size_t, P]
    lib.dm_render.argtypes = [P, S, P, S, P, P, S, ctypes.POINTER(dm_camera), P, P, P]
    lib.dm_config_hash.argtypes = [P, ctypes.POINTER(ctypes.c_uint64)]
    lib.dm_mark_built.argtypes = [P, ctypes.c_uint64, S, P]
    lib.dm_sync.argtypes = [P, P]
    lib.dm_destroy.argtypes = [P]
    lib.dm_destroy.restype = None
    lib.dm_last_error_string.argtypes = [P]
    lib.dm_last_error_string.restype = ctypes.c_char_p
    lib.dm_status_string.argtypes = [S]
    lib.dm_status_string.restype = ctypes.c_char_p
    lib.dm_version.argtypes = []
    for n in ("dm_create", "dm_query_sizes", "dm_bind", "dm_build_partitions",
              "dm_build_partitions_batch", "dm_update_tf",
              "dm_update_tf_host", "dm_full_recompute", "dm_set_profile_events",
              "dm_set_profile_counter",
              "dm_update_tf_noalloc", "dm_update_tf_batch", "dm_update_tf_batch_ws",
              "dm_render", "dm_config_hash", "dm_mark_built", "dm_sync", "dm_version"):
        getattr(lib, n).restype = S
    _lib = lib
    return lib


def status_name(s: int) -> str:
    try:
        return load().dm_status_string(int(s)).decode()
    except ImportError:
        return str(s)


def _check(ctx, status, where):
    if status != DM_OK:
        detail = load().dm_last_error_string(ctx).decode() if ctx else ""
        raise DmError(status, where, detail)


# ---------------------------------------------------------------- same-name wrappers
def make_config(dims, dtype, block=4, apron=1, num_partitions=16, tf_size=256, borders=None,
                occ_mode=DM_OCC_MINMAX, index_mode=DM_INDEX_NONE):
    cfg = dm_config()
    cfg.dims[:] = [int(d) for d in dims]
    cfg.dtype = int(dtype)
    cfg.block = int(block)
    cfg.apron = int(apron)
    cfg.num_partitions = int(num_partitions)
    cfg.tf_size = int(tf_size)
    cfg.occ_mode = int(occ_mode)
    cfg.index_mode = int(index_mode)
    keep = None
    if borders is not None:
        keep = (ctypes.c_int32 * len(borders))(*[int(v) for v in borders])
        cfg.borders = ctypes.cast(keep, ctypes.POINTER(ctypes.c_int32))
    return cfg, keep


def dm_create(cfg: dm_config):
    """Returns the opaque context handle (int); raises DmError on a non-OK status."""
    h = ctypes.c_void_p()
    _check(None, load().dm_create(ctypes.byref(h), ctypes.byref(cfg)), "dm_create")
    return h.value


def dm_create_status(cfg: dm_config) -> int:
    """dm_create returning the raw status (the context, if any, is destroyed)."""
    h = ctypes.c_void_p()
    s = load().dm_create(ctypes.byref(h), ctypes.byref(cfg))
    if s == DM_OK:
        load().dm_destroy(h)
    return s


def dm_query_sizes(ctx) -> dm_sizes:
    s = dm_sizes()
    _check(ctx, load().dm_query_sizes(ctx, ctypes.byref(s)), "dm_query_sizes")
    return s


def dm_bind(ctx, d_mask, d_pdm, d_minmax, d_scratch):
    _check(ctx, load().dm_bind(ctx, d_mask, d_pdm, d_minmax, d_scratch), "dm_bind")


def dm_build_partitions(ctx, d_volume, stream):
    _check(ctx, load().dm_build_partitions(ctx, d_volume, stream), "dm_build_partitions")


def dm_build_partitions_batch(ctxs, d_volumes, stream=None):
    """The precompute of several contexts in one call: ctxs[i] from the device volume
    pointer d_volumes[i]."""
    n = len(ctxs)
    if len(d_volumes) != n:
        raise ValueError(f"{n} contexts but {len(d_volumes)} volumes")
    carr = (ctypes.c_void_p * max(1, n))(*ctxs)
    varr = (ctypes.c_void_p * max(1, n))(*d_volumes)
    st = load().dm_build_partitions_batch(carr, varr, n, stream)
    if st != DM_OK:
        # the library reports in the context concerned: the first one with a message
        detail = ""
        for c in ctxs:
            if c:
                detail = load().dm_last_error_string(c).decode()
                if detail:
                    break
        raise DmError(st, "dm_build_partitions_batch", detail)


def dm_update_tf(ctx, d_tf_rgba, d_out, d_active_mask_out, stream):
    _check(ctx, load().dm_update_tf(ctx, d_tf_rgba, d_out, d_active_mask_out, stream),
           "dm_update_tf")


def dm_update_tf_host(ctx, h_tf_rgba, h_out, stream):
    _check(ctx, load().dm_update_tf_host(ctx, h_tf_rgba, h_out, stream), "dm_update_tf_host")


def dm_full_recompute(ctx, d_volume, d_tf_rgba, d_out, stream):
    _check(ctx, load().dm_full_recompute(ctx, d_volume, d_tf_rgba, d_out, stream),
           "dm_full_recompute")


def dm_set_profile_events(ctx, ev_begin, ev_end):
    _check(ctx, load().dm_set_profile_events(ctx, ev_begin, ev_end), "dm_set_profile_events")


def dm_set_profile_counter(ctx, d_bytes):
    """d_bytes: device address of a zeroed uint64 (or None to stop)."""
    _check(ctx, load().dm_set_profile_counter(ctx, d_bytes), "dm_set_profile_counter")


def dm_update_tf_noalloc(d_pdm, plane_stride, num_blocks, num_partitions, borders, tf_size,
                         d_tf_rgba, d_out, stream):
    """Context-free update whose working memory is the library's fixed device array.
    `borders` is None (uniform) or a sequence of K+1 ints."""
    keep = None
    if borders is not None:
        if len(borders) != int(num_partitions) + 1:
            raise ValueError(f"borders holds {len(borders)} entries; the library reads "
                             f"num_partitions + 1 = {int(num_partitions) + 1}")
        keep = (ctypes.c_int32 * len(borders))(*[int(v) for v in borders])
    st = load().dm_update_tf_noalloc(d_pdm, plane_stride, num_blocks, num_partitions, keep,
                                     tf_size, d_tf_rgba, d_out, stream)
    if st != DM_OK:
        raise DmError(st, "dm_update_tf_noalloc")


class PreparedBatch:
    """The C item array of a batch, marshalled once from (ctx, d_tf_rgba, d_out) triples and
    reusable by every dm_update_tf_batch call on the same pointers."""

    def __init__(self, items):
        self.n = len(items)
        self.arr = (dm_batch_item * max(1, self.n))()
        for i, (c, tf, out) in enumerate(items):
            self.arr[i].ctx, self.arr[i].d_tf_rgba, self.arr[i].d_out = c, tf, out
        self.first_ctx = items[0][0] if self.n else None


def _tuning(tuning):
    """dm_batch_tuning from None (library defaults), an int (combine CTAs per SM) or a
    (ctas_per_sm, loads_per_stage) pair."""
    if tuning is None:
        return None
    t = dm_batch_tuning()
    if isinstance(tuning, (tuple, list)):
        t.combine_ctas_per_sm = int(tuning[0])
        t.loads_per_stage = int(tuning[1])
    else:
        t.combine_ctas_per_sm = int(tuning)
    return ctypes.byref(t)


def dm_update_tf_batch(items, tuning=None, stream=None):
    """items: sequence of (ctx, d_tf_rgba, d_out) device pointers, or a PreparedBatch of
    them; tuning: see _tuning (None = library defaults)."""
    if not isinstance(items, PreparedBatch):
        items = PreparedBatch(items)
    n, arr = items.n, items.arr
    st = load().dm_update_tf_batch(arr, n, _tuning(tuning), stream)
    if st != DM_OK:
        detail = load().dm_last_error_string(items.first_ctx).decode() if n else ""
        raise DmError(st, "dm_update_tf_batch", detail)


def dm_batch_workspace_bytes(n: int) -> int:
    return int(load().dm_batch_workspace_bytes(int(n)))


def dm_update_tf_batch_ws(items, tuning, d_workspace, workspace_bytes, stream=None):
    """Batched update whose items may repeat a context (several TFs of one volume); the
    active sets live in the caller's device workspace of dm_batch_workspace_bytes(n)."""
    if not isinstance(items, PreparedBatch):
        items = PreparedBatch(items)
    n, arr = items.n, items.arr
    st = load().dm_update_tf_batch_ws(arr, n, _tuning(tuning), d_workspace,
                                      int(workspace_bytes), stream)
    if st != DM_OK:
        detail = load().dm_last_error_string(items.first_ctx).decode() if n else ""
        raise DmError(st, "dm_update_tf_batch_ws", detail)


def orbit_camera(dims, angle_rad, width, height, step=0.5, ert=0.98, elevation_rad=0.3):
    """Orthographic camera circling the volume's vertical (y) axis, its image plane
    covering the volume's bounding sphere."""
    import math
    X, Y, Z = (float(d) for d in dims)
    c = [(X - 1) / 2, (Y - 1) / 2, (Z - 1) / 2]
    r = 0.5 * math.sqrt(X * X + Y * Y + Z * Z)
    d = [math.cos(elevation_rad) * math.sin(angle_rad), -math.sin(elevation_rad),
         math.cos(elevation_rad) * math.cos(angle_rad)]
    up = [0.0, 1.0, 0.0]
    u = [d[1] * up[2] - d[2] * up[1], d[2] * up[0] - d[0] * up[2], d[0] * up[1] - d[1] * up[0]]
    nu = math.sqrt(sum(x * x for x in u))
    u = [x / nu for x in u]
    v = [u[1] * d[2] - u[2] * d[1], u[2] * d[0] - u[0] * d[2], u[0] * d[1] - u[1] * d[0]]
    cam = dm_camera()
    px = 2 * r / max(width, height)
    for a in range(3):
        cam.direction[a] = d[a]
        cam.pixel_dx[a] = u[a] * px
        cam.pixel_dy[a] = v[a] * px
        cam.origin[a] = c[a] - d[a] * 2 * r - u[a] * px * width / 2 - v[a] * px * height / 2
    cam.width, cam.height, cam.step, cam.ert = int(width), int(height), float(step), float(ert)
    return cam


def dm_render(d_volume, dtype, dims, block, d_dmap, d_tf_rgba, tf_size, cam, d_image, d_samples,
              stream):
    d = (ctypes.c_int32 * 3)(*[int(x) for x in dims])
    st = load().dm_render(d_volume, int(dtype), d, int(block), d_dmap, d_tf_rgba, int(tf_size),
                          ctypes.byref(cam), d_image, d_samples, stream)
    if st != DM_OK:
        raise DmError(st, "dm_render")


def dm_config_hash(ctx) -> int:
    h = ctypes.c_uint64()
    _check(ctx, load().dm_config_hash(ctx, ctypes.byref(h)), "dm_config_hash")
    return int(h.value)


def dm_mark_built(ctx, hash_, with_minmax, stream):
    _check(ctx, load().dm_mark_built(ctx, ctypes.c_uint64(hash_), int(bool(with_minmax)), stream),
           "dm_mark_built")


def dm_sync(ctx, stream):
    _check(ctx, load().dm_sync(ctx, stream), "dm_sync")


def dm_destroy(ctx):
    if ctx:
        load().dm_destroy(ctx)


def dm_last_error_string(ctx) -> str:
    return load().dm_last_error_string(ctx).decode()


def dm_status_string(s: int) -> str:
    return load().dm_status_string(int(s)).decode()


def dm_version() -> int:
    return int(load().dm_version())
