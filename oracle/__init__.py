"""CPU oracle for partitioned distance maps -- TEST INFRASTRUCTURE ONLY.

A ctypes wrapper around ``dm_oracle.c`` (plain single-threaded C, built with gcc).  Only
``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may import it;
the product library never does, and this package imports nothing from it.

Functions take and return numpy arrays.  Definitions (see the C file for the full list):
§3.1 partitions / POMs / PDMs, §3.1 step 1 (active set S), Eq. 1 (D' = min over S),
§3.2 (uint8 storage, clamped at 255), and the plain full recompute it replaces.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libdm_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library with gcc (no CUDA involved)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-Wall",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    """The oracle library: this package's build, or the one DM_ORACLE_LIB names (the
    planted-mistake tests load altered builds of the same source that way)."""
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(os.environ.get("DM_ORACLE_LIB") or build())
        P = ctypes.c_void_p
        i32, i64 = ctypes.c_int32, ctypes.c_int64
        sig = {
            "oracle_partition_lut": [i32, i32, P, P],
            "oracle_pom": [P, i32, P, i32, i32, i32, i32, P, P, P, P],
            "oracle_chamfer_dt": [P, P, P],
            "oracle_dt_at": [P, P, i32, i32, i32],
            "oracle_build_partitions": [P, i32, P, i32, i32, i32, i32, P, P, P, P, P],
            "oracle_active_set": [P, i32, i32, P, P],
            "oracle_combine": [P, i32, i64, P, P],
            "oracle_update_tf": [P, i32, i64, P, i32, P, P, P],
            "oracle_full_recompute_minmax": [P, P, P, P, i32, P],
            "oracle_occ_minmax": [P, P, i64, P, i32, P],
            "oracle_full_recompute_exact": [P, i32, P, i32, i32, P, i32, P],
        }
        for name, args in sig.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _i32(v):
    return np.ascontiguousarray(np.asarray(v, dtype=np.int32))


def _check(rc, what):
    if rc != 0:
        raise ValueError(f"oracle: {what} rejected its arguments")


def grid_of(dims, b):
    """Block grid (Gx, Gy, Gz) = ceil(dims / b)."""
    return tuple(-(-int(d) // int(b)) for d in dims)


def _vol(vol):
    v = np.ascontiguousarray(vol)
    if v.dtype == np.uint8:
        return v, 1
    if v.dtype == np.uint16:
        return v, 2
    raise TypeError("volume must be uint8 or uint16 [Z][Y][X]")


def partition_lut(N, K, borders=None):
    lut = np.empty(N, dtype=np.uint8)
    b = None if borders is None else _i32(borders)
    _check(_load().oracle_partition_lut(N, K, _p(b), _p(lut)), "partition_lut")
    return lut


def pom(vol, b, a, N, K, borders=None):
    """(mask [Gz,Gy,Gx,W] uint64, vmin, vmax [Gz,Gy,Gx] uint16) for volume [Z][Y][X]."""
    v, bpv = _vol(vol)
    dims = _i32([v.shape[2], v.shape[1], v.shape[0]])
    gx, gy, gz = grid_of(dims, b)
    W = (K + 63) // 64
    lut = partition_lut(N, K, borders)
    mask = np.empty((gz, gy, gx, W), dtype=np.uint64)
    vmin = np.empty((gz, gy, gx), dtype=np.uint16)
    vmax = np.empty((gz, gy, gx), dtype=np.uint16)
    _check(_load().oracle_pom(_p(v), bpv, _p(dims), b, a, N, K, _p(lut), _p(mask),
                              _p(vmin), _p(vmax)), "pom")
    return mask, vmin, vmax


def chamfer_dt(occ):
    """Chessboard DT (clamped to 255) of a [Gz][Gy][Gx] occupancy array."""
    o = np.ascontiguousarray(occ != 0, dtype=np.uint8)
    grid = _i32([o.shape[2], o.shape[1], o.shape[0]])
    out = np.empty_like(o)
    _check(_load().oracle_chamfer_dt(_p(o), _p(grid), _p(out)), "chamfer_dt")
    return out


def dt_at(occ, x, y, z):
    """Chessboard distance (clamped to 255) at block (x, y, z) by shell search."""
    o = np.ascontiguousarray(occ != 0, dtype=np.uint8)
    grid = _i32([o.shape[2], o.shape[1], o.shape[0]])
    r = _load().oracle_dt_at(_p(o), _p(grid), int(x), int(y), int(z))
    _check(0 if r >= 0 else -1, "dt_at")
    return r


def dt_at_many(occ_u8, points):
    """dt_at for many (x, y, z) points over an already-contiguous uint8 occupancy grid."""
    o = np.ascontiguousarray(occ_u8, dtype=np.uint8)
    grid = _i32([o.shape[2], o.shape[1], o.shape[0]])
    f = _load().oracle_dt_at
    return np.array([f(_p(o), _p(grid), int(x), int(y), int(z)) for x, y, z in points],
                    dtype=np.int32)


def build_partitions(vol, b, a, N, K, borders=None):
    """One-time precompute: (mask [Gz,Gy,Gx,W], pdm [K,Gz,Gy,Gx] uint8, vmin, vmax)."""
    v, bpv = _vol(vol)
    dims = _i32([v.shape[2], v.shape[1], v.shape[0]])
    gx, gy, gz = grid_of(dims, b)
    W = (K + 63) // 64
    mask = np.empty((gz, gy, gx, W), dtype=np.uint64)
    pdm = np.empty((K, gz, gy, gx), dtype=np.uint8)
    vmin = np.empty((gz, gy, gx), dtype=np.uint16)
    vmax = np.empty((gz, gy, gx), dtype=np.uint16)
    bb = None if borders is None else _i32(borders)
    _check(_load().oracle_build_partitions(_p(v), bpv, _p(dims), b, a, N, K, _p(bb),
                                           _p(mask), _p(pdm), _p(vmin), _p(vmax)),
           "build_partitions")
    return mask, pdm, vmin, vmax


def active_set(tf, K, borders=None):
    """S as a list of 0-based partition indices (ascending)."""
    t = np.ascontiguousarray(tf, dtype=np.float32)
    N = t.shape[0]
    s = np.zeros(4, dtype=np.uint64)
    bb = None if borders is None else _i32(borders)
    _check(_load().oracle_active_set(_p(t), N, K, _p(bb), _p(s)), "active_set")
    return [p for p in range(K) if (int(s[p // 64]) >> (p % 64)) & 1]


def active_mask(tf, K, borders=None):
    t = np.ascontiguousarray(tf, dtype=np.float32)
    s = np.zeros(4, dtype=np.uint64)
    bb = None if borders is None else _i32(borders)
    _check(_load().oracle_active_set(_p(t), t.shape[0], K, _p(bb), _p(s)), "active_set")
    return s[: (K + 63) // 64].copy()


def combine(pdm, smask):
    """Eq. 1 over an explicit active bit set."""
    pd = np.ascontiguousarray(pdm, dtype=np.uint8)
    K = pd.shape[0]
    G = int(np.prod(pd.shape[1:]))
    s = np.zeros(4, dtype=np.uint64)
    s[: len(smask)] = smask
    out = np.empty(pd.shape[1:], dtype=np.uint8)
    _check(_load().oracle_combine(_p(pd), K, G, _p(s), _p(out)), "combine")
    return out


def update_tf(pdm, tf, borders=None):
    """Per-TF update: (D' [Gz,Gy,Gx] uint8, S bit mask words)."""
    pd = np.ascontiguousarray(pdm, dtype=np.uint8)
    t = np.ascontiguousarray(tf, dtype=np.float32)
    K = pd.shape[0]
    G = int(np.prod(pd.shape[1:]))
    out = np.empty(pd.shape[1:], dtype=np.uint8)
    s = np.zeros(4, dtype=np.uint64)
    bb = None if borders is None else _i32(borders)
    _check(_load().oracle_update_tf(_p(pd), K, G, _p(t), t.shape[0], _p(bb), _p(out), _p(s)),
           "update_tf")
    return out, s[: (K + 63) // 64].copy()


def full_recompute_minmax(vmin, vmax, tf):
    mn = np.ascontiguousarray(vmin, dtype=np.uint16)
    mx = np.ascontiguousarray(vmax, dtype=np.uint16)
    t = np.ascontiguousarray(tf, dtype=np.float32)
    grid = _i32([mn.shape[2], mn.shape[1], mn.shape[0]])
    out = np.empty(mn.shape, dtype=np.uint8)
    _check(_load().oracle_full_recompute_minmax(_p(mn), _p(mx), _p(grid), _p(t), t.shape[0],
                                                _p(out)), "full_recompute_minmax")
    return out


def occ_minmax(vmin, vmax, tf):
    """0/1 occupancy of the min/max recompute: one visible intensity in [min, max]."""
    mn = np.ascontiguousarray(vmin, dtype=np.uint16)
    mx = np.ascontiguousarray(vmax, dtype=np.uint16)
    t = np.ascontiguousarray(tf, dtype=np.float32)
    occ = np.empty(mn.shape, dtype=np.uint8)
    _check(_load().oracle_occ_minmax(_p(mn), _p(mx), int(mn.size), _p(t), t.shape[0], _p(occ)),
           "occ_minmax")
    return occ


def full_recompute_exact(vol, b, a, tf):
    v, bpv = _vol(vol)
    t = np.ascontiguousarray(tf, dtype=np.float32)
    dims = _i32([v.shape[2], v.shape[1], v.shape[0]])
    gx, gy, gz = grid_of(dims, b)
    out = np.empty((gz, gy, gx), dtype=np.uint8)
    _check(_load().oracle_full_recompute_exact(_p(v), bpv, _p(dims), b, a, _p(t), t.shape[0],
                                               _p(out)), "full_recompute_exact")
    return out


def mask_plane(mask, p):
    """Occupancy plane (uint8 0/1) of partition p from a [...,W] mask array."""
    return ((mask[..., p // 64] >> np.uint64(p % 64)) & np.uint64(1)).astype(np.uint8)


def union_plane(mask, parts):
    """Occupancy (uint8 0/1) of the union of the POMs of `parts`."""
    out = np.zeros(mask.shape[:-1], dtype=np.uint8)
    for p in parts:
        out |= mask_plane(mask, p)
    return out
