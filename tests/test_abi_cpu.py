"""Host-side checks of libdm without a GPU: the library loads, exports every function that
include/dm.h declares, validates configurations, reports sizes (the memory formula of §5)
and refuses calls on unbound or misaligned buffers before touching the device."""
import ctypes
import os
import re

import pytest

import paper_2407_21552_gb300 as pkg
from paper_2407_21552_gb300 import _abi as A

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def lib():
    pkg.build()
    return A.load()


def header_functions():
    text = open(os.path.join(ROOT, "include", "dm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(dm_[a-z_]+)\s*\(", text)))


def test_exports_every_declared_function(lib):
    declared = header_functions()
    assert set(declared) == set(A.EXPORTED)
    for name in declared:
        assert hasattr(lib, name), name
    out = os.popen(f"nm -D --defined-only {A.LIB_PATH}").read()
    for name in declared:
        assert re.search(rf"\bT {name}\b", out), f"{name} not exported"


def test_version_and_status_names():
    assert A.dm_version() == 10000
    assert A.dm_status_string(A.DM_OK) == "DM_OK"
    assert A.dm_status_string(A.DM_ERR_UNSUPPORTED) == "DM_ERR_UNSUPPORTED"
    assert A.dm_status_string(99) == "DM_ERR_UNKNOWN"


def cfg(**kw):
    base = dict(dims=(128, 128, 128), dtype=A.DM_U8, block=4, apron=1, num_partitions=16,
                tf_size=256, borders=None, occ_mode=A.DM_OCC_MINMAX)
    base.update(kw)
    return A.make_config(**base)


@pytest.mark.parametrize("kw,status", [
    (dict(), A.DM_OK),
    (dict(dims=(0, 4, 4)), A.DM_ERR_INVALID_ARG),
    (dict(dtype=3), A.DM_ERR_INVALID_ARG),
    (dict(block=0), A.DM_ERR_INVALID_ARG),
    (dict(block=17), A.DM_ERR_UNSUPPORTED),
    (dict(apron=-1), A.DM_ERR_INVALID_ARG),
    (dict(apron=5), A.DM_ERR_UNSUPPORTED),
    (dict(num_partitions=0), A.DM_ERR_INVALID_ARG),
    (dict(num_partitions=257, tf_size=4096), A.DM_ERR_UNSUPPORTED),
    (dict(num_partitions=300, tf_size=256), A.DM_ERR_UNSUPPORTED),
    (dict(num_partitions=20, tf_size=16), A.DM_ERR_INVALID_ARG),
    (dict(tf_size=1), A.DM_ERR_INVALID_ARG),
    (dict(tf_size=70000), A.DM_ERR_UNSUPPORTED),
    (dict(occ_mode=2), A.DM_ERR_INVALID_ARG),
    (dict(num_partitions=4, borders=[0, 1, 5, 200, 256]), A.DM_OK),
    (dict(num_partitions=4, borders=[0, 5, 5, 200, 256]), A.DM_ERR_INVALID_ARG),
    (dict(num_partitions=4, borders=[1, 5, 9, 200, 256]), A.DM_ERR_INVALID_ARG),
    (dict(num_partitions=4, borders=[0, 5, 9, 200, 255]), A.DM_ERR_INVALID_ARG),
    (dict(dims=(4, 4, 4 * 2000)), A.DM_OK),                  # 2000-block z lines
    (dict(dims=(4, 4, 4 * 5886)), A.DM_OK),                  # the longest line a tile holds
    (dict(dims=(4, 4, 4 * 5887)), A.DM_ERR_UNSUPPORTED),     # z lines beyond the tiling
    (dict(dims=(1, 1, 1), block=1, apron=0, num_partitions=1, tf_size=2), A.DM_OK),
])
def test_create_validation(kw, status):
    c, keep = cfg(**kw)
    assert A.dm_create_status(c) == status


@pytest.mark.parametrize("dims,b,K,bpv", [
    ((512, 512, 460), 4, 16, 1),         # manix-sized grid 128x128x115
    ((1024, 1024, 1795), 4, 64, 2),      # 256x256x449
    ((37, 29, 23), 4, 7, 1),             # ragged edges: ceil
    ((5, 7, 9), 1, 256, 2),
])
def test_query_sizes_memory_formula(dims, b, K, bpv):
    c, keep = cfg(dims=dims, block=b, num_partitions=K, dtype=bpv,
                  tf_size=4096 if bpv == 2 else 256, apron=min(1, b))
    ctx = A.dm_create(c)
    try:
        s = A.dm_query_sizes(ctx)
        g = [-(-d // b) for d in dims]
        G = g[0] * g[1] * g[2]
        assert list(s.grid) == g
        assert s.out_bytes == G
        assert s.plane_stride == -(-G // 64) * 64
        assert s.pdm_bytes == K * s.plane_stride
        if G % 64 == 0:
            assert s.pdm_bytes == K * G          # §5: n * volumesize / b^3 bytes
        assert s.mask_words == -(-K // 64)
        assert s.mask_bytes == G * s.mask_words * 8
        assert s.minmax_bytes == 2 * bpv * G
        assert s.scratch_bytes >= G + 16 * c.tf_size
    finally:
        A.dm_destroy(ctx)


def test_unbound_and_misaligned_calls_are_refused_on_the_host():
    c, keep = cfg()
    ctx = A.dm_create(c)
    lib = A.load()
    try:
        fake = ctypes.c_void_p(1 << 20)       # never dereferenced: refused before any launch
        assert lib.dm_build_partitions(ctx, fake, None) == A.DM_ERR_NOT_BOUND
        assert lib.dm_update_tf(ctx, fake, fake, None, None) == A.DM_ERR_NOT_BOUND
        assert lib.dm_full_recompute(ctx, fake, fake, fake, None) == A.DM_ERR_NOT_BOUND
        assert "bound" in A.dm_last_error_string(ctx)
        assert lib.dm_bind(ctx, ctypes.c_void_p((1 << 20) + 3), None, None, None) == \
            A.DM_ERR_INVALID_ARG
        assert "misaligned" in A.dm_last_error_string(ctx)
        assert lib.dm_bind(ctx, None, None, None, ctypes.c_void_p((1 << 20) + 16)) == \
            A.DM_ERR_INVALID_ARG
        # pdm bound but never built: the update refuses
        assert lib.dm_bind(ctx, fake, fake, fake, fake) == A.DM_OK
        assert lib.dm_update_tf(ctx, fake, fake, None, None) == A.DM_ERR_NOT_BOUND
        assert "build" in A.dm_last_error_string(ctx)
        assert lib.dm_update_tf(ctx, None, fake, None, None) == A.DM_ERR_INVALID_ARG
        assert lib.dm_update_tf_host(ctx, None, None, None) == A.DM_ERR_INVALID_ARG
        assert lib.dm_build_partitions(ctx, None, None) == A.DM_ERR_INVALID_ARG
        assert lib.dm_query_sizes(None, None) == A.DM_ERR_INVALID_ARG
        assert lib.dm_create(None, None) == A.DM_ERR_INVALID_ARG
    finally:
        A.dm_destroy(ctx)
    A.dm_destroy(None)


def test_package_fails_loudly_without_the_library(tmp_path):
    with pytest.raises(ImportError):
        A._lib_backup = A._lib
        try:
            A._lib = None
            A.load(str(tmp_path / "missing.so"))
        finally:
            A._lib = A._lib_backup


@pytest.mark.parametrize("K,planes", [(1, 1), (2, 3), (5, 5 + 4 + 2), (32, 135), (64, 328),
                                      (256, 256 + 255 + 253 + 249 + 241 + 225 + 193 + 129 + 1)])
def test_range_index_plane_count(K, planes):
    """Planes of the optional range index: level k holds K - 2^k + 1 planes, k <= log2 K."""
    c, keep = cfg(num_partitions=K, tf_size=4096, dtype=A.DM_U16, index_mode=A.DM_INDEX_RANGES)
    ctx = A.dm_create(c)
    try:
        s = A.dm_query_sizes(ctx)
        assert s.pdm_planes == planes
        assert s.pdm_bytes == planes * s.plane_stride
    finally:
        A.dm_destroy(ctx)
    c2, keep2 = cfg(index_mode=7)
    assert A.dm_create_status(c2) == A.DM_ERR_INVALID_ARG


def test_config_hash_tracks_everything_that_shapes_the_maps():
    base = dict()
    variants = [dict(dims=(128, 128, 127)), dict(block=2), dict(apron=0), dict(num_partitions=8),
                dict(tf_size=512), dict(num_partitions=4, borders=[0, 1, 5, 200, 256]),
                dict(index_mode=A.DM_INDEX_RANGES), dict(dtype=A.DM_U16)]
    hashes = []
    for kw in [base] + variants:
        c, keep = cfg(**kw)
        ctx = A.dm_create(c)
        hashes.append(A.dm_config_hash(ctx))
        A.dm_destroy(ctx)
    assert len(set(hashes)) == len(hashes)
    c, keep = cfg()
    ctx = A.dm_create(c)
    try:
        assert A.dm_config_hash(ctx) == hashes[0]            # stable
        # occ_mode does not change the maps: same hash
        c2, keep2 = cfg(occ_mode=A.DM_OCC_EXACT)
        ctx2 = A.dm_create(c2)
        assert A.dm_config_hash(ctx2) == hashes[0]
        A.dm_destroy(ctx2)
        lib = A.load()
        assert lib.dm_mark_built(ctx, hashes[0] ^ 1, 0, None) == A.DM_ERR_INVALID_ARG
        assert lib.dm_mark_built(ctx, hashes[0], 0, None) == A.DM_ERR_NOT_BOUND
    finally:
        A.dm_destroy(ctx)


def test_batched_update_is_refused_on_the_host_for_bad_items():
    """dm_update_tf_batch checks every item before it launches: a null context or buffer,
    an unbuilt context and a context given twice are refused, whether the items come as
    a list or as a PreparedBatch (marshalled once)."""
    c, keep = cfg()
    ctxs = [A.dm_create(c) for _ in range(2)]
    lib = A.load()
    fake = (1 << 20)
    try:
        for ctx in ctxs:
            assert lib.dm_bind(ctx, ctypes.c_void_p(fake), ctypes.c_void_p(fake),
                               ctypes.c_void_p(fake), ctypes.c_void_p(fake)) == A.DM_OK
        items = [(ctxs[0], fake, fake + 4096), (ctxs[1], fake + 64, fake + 8192)]
        pb = A.PreparedBatch(items)
        assert pb.n == 2 and pb.first_ctx == ctxs[0]
        assert [(pb.arr[i].d_tf_rgba, pb.arr[i].d_out) for i in range(2)] == \
            [(fake, fake + 4096), (fake + 64, fake + 8192)]
        for form in (items, pb):                          # bound, never built
            with pytest.raises(A.DmError) as e:
                A.dm_update_tf_batch(form, None, None)
            assert e.value.status == A.DM_ERR_NOT_BOUND
            assert "not built" in str(e.value)
        with pytest.raises(A.DmError) as e:               # misaligned TF
            A.dm_update_tf_batch([(ctxs[0], fake + 2, fake)], None, None)
        assert e.value.status == A.DM_ERR_INVALID_ARG
        with pytest.raises(A.DmError) as e:               # null output
            A.dm_update_tf_batch(A.PreparedBatch([(ctxs[1], fake, None)]), 12, None)
        assert e.value.status == A.DM_ERR_INVALID_ARG
        A.dm_update_tf_batch([], None, None)              # nothing to do
    finally:
        for ctx in ctxs:
            A.dm_destroy(ctx)


def test_noalloc_wrapper_checks_the_border_count():
    """The C side reads num_partitions + 1 borders: a shorter or longer list is refused by
    the binding before the call (no GPU needed: nothing reaches the library)."""
    fake = 1 << 20
    for borders in ([0, 128, 256], [0, 64, 128, 192, 256, 256]):
        with pytest.raises(ValueError):
            A.dm_update_tf_noalloc(fake, 64, 64, 4, borders, 256, fake, fake, None)


def test_workspace_batch_is_refused_on_the_host():
    """dm_update_tf_batch_ws checks its workspace (present, 256-byte aligned, at least
    dm_batch_workspace_bytes(n)) and then every item, before it launches; unlike
    dm_update_tf_batch it accepts a context given twice (it fails here only because the
    contexts were never built)."""
    c, keep = cfg()
    ctxs = [A.dm_create(c) for _ in range(2)]
    lib = A.load()
    fake = 1 << 20
    per = A.dm_batch_workspace_bytes(1)
    assert per > 0 and per % 256 == 0
    assert A.dm_batch_workspace_bytes(5) == 5 * per and A.dm_batch_workspace_bytes(0) == 0
    try:
        for ctx in ctxs:
            assert lib.dm_bind(ctx, ctypes.c_void_p(fake), ctypes.c_void_p(fake),
                               ctypes.c_void_p(fake), ctypes.c_void_p(fake)) == A.DM_OK
        items = [(ctxs[0], fake, fake + 4096), (ctxs[0], fake + 64, fake + 8192),
                 (ctxs[1], fake + 128, fake + 12288)]
        need = A.dm_batch_workspace_bytes(len(items))
        for ws, size in ((None, need), (fake + 128, need), (fake, need - 1)):
            with pytest.raises(A.DmError) as e:
                A.dm_update_tf_batch_ws(items, None, ws, size, None)
            assert e.value.status == A.DM_ERR_INVALID_ARG
            assert "workspace" in str(e.value)
        with pytest.raises(A.DmError) as e:               # repeated context: allowed
            A.dm_update_tf_batch_ws(items, (12, 8), fake, need, None)
        assert e.value.status == A.DM_ERR_NOT_BOUND
        A.dm_update_tf_batch_ws([], None, None, 0, None)  # nothing to do
    finally:
        for ctx in ctxs:
            A.dm_destroy(ctx)


def test_batched_precompute_is_refused_on_the_host():
    """dm_build_partitions_batch checks every item before it launches: a null context, a
    null or misaligned volume, an unbound context, a context listed twice and two contexts
    sharing a buffer are refused, each reported in the context concerned."""
    c8, keep8 = cfg()
    c16, keep16 = cfg(dtype=A.DM_U16, tf_size=4096)
    ctxs = [A.dm_create(c8), A.dm_create(c16), A.dm_create(c8)]
    lib = A.load()
    base = 1 << 20

    def bind(ctx, k, shared_pdm=None):
        b = base + k * (1 << 16)
        pdm = shared_pdm if shared_pdm is not None else b + 4096
        assert lib.dm_bind(ctx, ctypes.c_void_p(b), ctypes.c_void_p(pdm),
                           ctypes.c_void_p(b + 8192), ctypes.c_void_p(b + 12288)) == A.DM_OK

    def refused(cs, vols, status, text):
        with pytest.raises(A.DmError) as e:
            A.dm_build_partitions_batch(cs, vols, None)
        assert e.value.status == status, str(e.value)
        assert text in str(e.value), str(e.value)

    try:
        A.dm_build_partitions_batch([], [], None)            # nothing to do
        with pytest.raises(ValueError):
            A.dm_build_partitions_batch(ctxs, [base], None)
        vols = [base, base + 64, base + 128]
        bind(ctxs[0], 0)
        refused(ctxs, vols, A.DM_ERR_NOT_BOUND, "item 1")     # ctxs[1] unbound
        bind(ctxs[1], 1)
        bind(ctxs[2], 2)
        refused(ctxs, [base, None, base], A.DM_ERR_INVALID_ARG, "item 1: null")
        refused(ctxs, [base, base + 65, base], A.DM_ERR_INVALID_ARG, "misaligned")  # u16
        assert lib.dm_build_partitions_batch(None, None, 1, None) == A.DM_ERR_INVALID_ARG
        assert lib.dm_build_partitions_batch(
            (ctypes.c_void_p * 1)(ctxs[0]), (ctypes.c_void_p * 1)(base), -1, None) == \
            A.DM_ERR_INVALID_ARG
        refused([ctxs[0], None], [base, base], A.DM_ERR_INVALID_ARG, "null context")
        refused([ctxs[0], ctxs[1], ctxs[0]], vols, A.DM_ERR_INVALID_ARG, "items 0 and 2")
        bind(ctxs[2], 2, shared_pdm=base + (1 << 16) + 4096)  # ctxs[1]'s pdm
        refused(ctxs, vols, A.DM_ERR_INVALID_ARG, "items 1 and 2 share")
    finally:
        for ctx in ctxs:
            A.dm_destroy(ctx)


def test_profile_counter_is_checked_on_the_host():
    """dm_set_profile_counter takes an 8-byte aligned device address or NULL; a misaligned
    counter is refused with DM_ERR_INVALID_ARG before any launch could use it."""
    c, keep = cfg()
    ctx = A.dm_create(c)
    try:
        A.dm_set_profile_counter(ctx, 1 << 20)              # aligned: accepted (not used)
        A.dm_set_profile_counter(ctx, None)                 # stop
        with pytest.raises(A.DmError) as e:
            A.dm_set_profile_counter(ctx, (1 << 20) + 4)
        assert e.value.status == A.DM_ERR_INVALID_ARG
        assert "misaligned" in str(e.value)
        assert A.load().dm_set_profile_counter(None, None) == A.DM_ERR_INVALID_ARG
    finally:
        A.dm_destroy(ctx)
