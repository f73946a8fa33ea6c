"""PyTorch-facing wrapper: torch owns the device buffers, libdm does every step.

PartitionedDistanceMaps allocates the buffers that dm_query_sizes() asks for as torch
uint8 tensors on the device, binds them, and forwards each call to the C ABI on the
current torch stream.  It performs no computation of its own.
"""
from __future__ import annotations

import ctypes

import torch

from . import _abi as A


_raw_current_stream = getattr(torch._C, "_cuda_getCurrentRawStream", None)


def _stream_handle(stream):
    """cudaStream_t of `stream`, or of torch's current stream on the current device.  The
    raw query skips building a torch Stream object (about 3 us per call)."""
    if stream is None:
        if _raw_current_stream is not None:
            return ctypes.c_void_p(_raw_current_stream(torch.cuda.current_device()))
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dtype_code(t: torch.Tensor) -> int:
    if t.dtype == torch.uint8:
        return A.DM_U8
    if t.dtype in (torch.int16, getattr(torch, "uint16", torch.int16)):
        return A.DM_U16
    raise TypeError("volume must be uint8, or int16/uint16 holding unsigned 16-bit intensities")


class PartitionedDistanceMaps:
    """One volume's partitioned distance maps (§3.1) resident on a CUDA device."""

    def __init__(self, dims, dtype: int, block: int = 4, apron: int = 1,
                 num_partitions: int = 16, tf_size: int = 256, borders=None,
                 occ_mode: int = A.DM_OCC_MINMAX, device="cuda", with_minmax: bool = True,
                 index_mode: int = A.DM_INDEX_NONE):
        self.cfg, self._keep = A.make_config(dims, dtype, block, apron, num_partitions, tf_size,
                                             borders, occ_mode, index_mode)
        self.ctx = A.dm_create(self.cfg)
        self.sizes = A.dm_query_sizes(self.ctx)
        self.device = torch.device(device)
        s = self.sizes
        self.K = int(num_partitions)
        self.N = int(tf_size)
        self.grid = tuple(int(v) for v in s.grid)          # (Gx, Gy, Gz)
        self.G = self.grid[0] * self.grid[1] * self.grid[2]
        self.plane_stride = int(s.plane_stride)
        alloc = dict(dtype=torch.uint8, device=self.device)
        self._mask = torch.empty(max(16, s.mask_bytes), **alloc)
        self._pdm = torch.empty(max(16, s.pdm_bytes), **alloc)
        self._with_minmax = bool(with_minmax)
        self._minmax = torch.empty(max(16, s.minmax_bytes), **alloc) if with_minmax else None
        self._scratch = torch.empty(max(256, s.scratch_bytes), **alloc)
        self._host = None                                   # set while offloaded
        self._host_bufs = None                              # pinned copies, reused
        self._host_valid = False                            # they hold the current maps
        self.ready_event = None                             # end of an async reload
        self._bind()

    def _bind(self):
        A.dm_bind(self.ctx,
                  self._mask.data_ptr() if self._mask is not None else None,
                  self._pdm.data_ptr() if self._pdm is not None else None,
                  self._minmax.data_ptr() if self._minmax is not None else None,
                  self._scratch.data_ptr() if self._scratch is not None else None)

    # ------------------------------------------------------------------ the three calls
    def build_partitions(self, volume: torch.Tensor, stream=None):
        self._prepare_build(volume)
        A.dm_build_partitions(self.ctx, volume.data_ptr(), _stream_handle(stream))
        self._host_valid = False

    def _prepare_build(self, volume: torch.Tensor):
        assert volume.is_cuda and volume.is_contiguous()
        assert _dtype_code(volume) == self.cfg.dtype
        if self._mask is None or self._pdm is None:    # released or offloaded before
            alloc = dict(dtype=torch.uint8, device=self.device)
            s = self.sizes
            if self._mask is None:
                self._mask = torch.empty(max(16, s.mask_bytes), **alloc)
            if self._pdm is None:
                self._pdm = torch.empty(max(16, s.pdm_bytes), **alloc)
                self._scratch = torch.empty(max(256, s.scratch_bytes), **alloc)
                if self._with_minmax:
                    self._minmax = torch.empty(max(16, s.minmax_bytes), **alloc)
                self._host = None
            self._bind()

    def update_tf(self, tf: torch.Tensor, out: torch.Tensor | None = None,
                  active_mask: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        assert tf.is_cuda and tf.dtype == torch.float32 and tf.is_contiguous()
        assert tf.numel() == 4 * self.N
        if out is None:
            out = torch.empty(self.G, dtype=torch.uint8, device=self.device)
        am = active_mask.data_ptr() if active_mask is not None else None
        A.dm_update_tf(self.ctx, tf.data_ptr(), out.data_ptr(), am, _stream_handle(stream))
        return out

    def update_tf_host(self, tf_host: torch.Tensor, out_host: torch.Tensor, stream=None):
        """Host in, host out (the call waits); pinned host tensors give async copies."""
        assert not tf_host.is_cuda and not out_host.is_cuda
        assert tf_host.dtype == torch.float32 and tf_host.numel() == 4 * self.N
        assert out_host.dtype == torch.uint8 and out_host.numel() >= self.G
        A.dm_update_tf_host(self.ctx, tf_host.data_ptr(), out_host.data_ptr(),
                            _stream_handle(stream))
        return out_host

    def full_recompute(self, tf: torch.Tensor, out: torch.Tensor | None = None,
                       volume: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        assert tf.is_cuda and tf.dtype == torch.float32 and tf.is_contiguous()
        if out is None:
            out = torch.empty(self.G, dtype=torch.uint8, device=self.device)
        vp = volume.data_ptr() if volume is not None else None
        A.dm_full_recompute(self.ctx, vp, tf.data_ptr(), out.data_ptr(), _stream_handle(stream))
        return out

    def set_profile_counter(self, counter: torch.Tensor | None):
        """Count the bytes of PDM planes that later updates load into `counter` (a zeroed
        device int64 tensor of one element, kept alive by the caller), or stop (None)."""
        if counter is not None and (counter.device.type != "cuda" or counter.numel() != 1
                                    or counter.element_size() != 8):
            raise ValueError("the counter is one 8-byte element in device memory")
        A.dm_set_profile_counter(self.ctx, counter.data_ptr() if counter is not None else None)

    def sync(self, stream=None):
        A.dm_sync(self.ctx, _stream_handle(stream))

    # ------------------------------------------------------------------ views for tests
    def pdm_planes(self) -> torch.Tensor:
        """[K, Gz, Gy, Gx] view of the PDM planes."""
        gx, gy, gz = self.grid
        v = self._pdm[: self.K * self.plane_stride].view(self.K, self.plane_stride)
        return v[:, : self.G].reshape(self.K, gz, gy, gx)

    def mask_words(self) -> torch.Tensor:
        gx, gy, gz = self.grid
        W = int(self.sizes.mask_words)
        return self._mask[: self.G * W * 8].view(torch.int64).view(gz, gy, gx, W)

    def minmax_pairs(self) -> torch.Tensor:
        """[Gz, Gy, Gx, 2] (min, max); int16 storage for 16-bit volumes."""
        gx, gy, gz = self.grid
        if self.cfg.dtype == A.DM_U8:
            return self._minmax[: 2 * self.G].view(gz, gy, gx, 2)
        return self._minmax[: 4 * self.G].view(torch.int16).view(gz, gy, gx, 2)

    # ------------------------------------------------------------------ checkpoint / resume
    def save(self, path: str):
        """Write the built maps (and min/max) with the configuration hash to `path`."""
        import numpy as np
        self.sync()
        h = A.dm_config_hash(self.ctx)
        arrays = {"hash": np.array([h], dtype=np.uint64),
                  "pdm": self._pdm[: self.sizes.pdm_bytes].cpu().numpy()}
        if self._minmax is not None:
            arrays["minmax"] = self._minmax[: self.sizes.minmax_bytes].cpu().numpy()
        np.savez(path, **arrays)

    def load(self, path: str, stream=None):
        """Restore maps saved by save() from a context with the same configuration."""
        import numpy as np
        z = np.load(path)
        h = int(z["hash"][0])
        if h != A.dm_config_hash(self.ctx):
            raise A.DmError(A.DM_ERR_INVALID_ARG, "load", "maps of another configuration")
        self._pdm[: self.sizes.pdm_bytes].copy_(torch.from_numpy(z["pdm"]))
        mm = "minmax" in z.files and self._minmax is not None
        if mm:
            self._minmax[: self.sizes.minmax_bytes].copy_(torch.from_numpy(z["minmax"]))
        torch.cuda.current_stream().synchronize()
        A.dm_mark_built(self.ctx, h, mm, _stream_handle(stream))
        self._host_valid = False

    # ------------------------------------------------------------------ eviction
    def offload(self, stream=None, wait: bool = True):
        """Move the built maps (PDM planes, and min/max if kept) to pinned host memory and
        free their device buffers and the scratch; reload() brings them back without a
        recompute.  The context stays valid but unbuilt in between (updates refuse to run).
        The host buffers are kept: the maps depend on the volume only (§3.1), so a later
        offload copies nothing unless the maps were rebuilt or loaded since.  With
        wait=False the copy stays queued on `stream`; the device memory is handed back to
        torch's allocator only once that copy has run."""
        if self._host is not None:
            return
        st = stream if stream is not None else torch.cuda.current_stream(self.device)
        st.wait_stream(torch.cuda.current_stream(self.device))   # the maps' last writer
        s = self.sizes
        if self._host_bufs is None:
            self._host_bufs = {
                "pdm": torch.empty(s.pdm_bytes, dtype=torch.uint8, pin_memory=True),
                "minmax": (torch.empty(s.minmax_bytes, dtype=torch.uint8, pin_memory=True)
                           if self._minmax is not None else None)}
        hb = self._host_bufs
        copy = not self._host_valid or (self._minmax is not None and hb["minmax"] is None)
        with torch.cuda.stream(st):
            if copy:
                if self._minmax is not None and hb["minmax"] is None:
                    hb["minmax"] = torch.empty(s.minmax_bytes, dtype=torch.uint8,
                                               pin_memory=True)
                hb["pdm"].copy_(self._pdm[: s.pdm_bytes], non_blocking=True)
                if self._minmax is not None:
                    hb["minmax"].copy_(self._minmax[: s.minmax_bytes], non_blocking=True)
            moved = torch.cuda.Event()
            moved.record(st)
        self._host_valid = True
        for t in (self._pdm, self._minmax, self._scratch, self._mask):
            if t is not None:
                t.record_stream(st)
        self._host = {"hash": A.dm_config_hash(self.ctx), "minmax": self._minmax is not None,
                      "moved": moved}
        self._pdm = None
        self._minmax = None
        self._scratch = None
        self._mask = None
        self.ready_event = None
        A.dm_bind(self.ctx, None, None, None, None)
        if wait:
            moved.synchronize()

    def reload(self, stream=None, wait: bool = True):
        """Inverse of offload(): device buffers again, the maps copied back, the context
        marked built (dm_mark_built rewrites the scratch's partition table and plane
        order).  With wait=False the work stays queued on `stream` and `ready_event` marks
        its end: work on another stream that reads the maps must wait for that event
        first."""
        h = self._host
        if h is None:
            return
        st = stream if stream is not None else torch.cuda.current_stream(self.device)
        st.wait_event(h["moved"])                               # the offload's copy landed
        s = self.sizes
        hb = self._host_bufs
        alloc = dict(dtype=torch.uint8, device=self.device)
        with torch.cuda.stream(st):
            self._pdm = torch.empty(max(16, s.pdm_bytes), **alloc)
            self._pdm[: s.pdm_bytes].copy_(hb["pdm"], non_blocking=True)
            if h["minmax"]:
                self._minmax = torch.empty(max(16, s.minmax_bytes), **alloc)
                self._minmax[: s.minmax_bytes].copy_(hb["minmax"], non_blocking=True)
            self._scratch = torch.empty(max(256, s.scratch_bytes), **alloc)
        self._bind()
        A.dm_mark_built(self.ctx, h["hash"], h["minmax"], _stream_handle(st))
        ready = torch.cuda.Event()
        ready.record(st)
        self._host = None
        if wait:
            ready.synchronize()
            self.ready_event = None
        else:
            self.ready_event = ready

    @property
    def offloaded(self) -> bool:
        return self._host is not None

    def release_mask(self):
        """The POMs are an intermediate (§5): drop their buffer after the precompute."""
        self._mask = None
        self._bind()

    def close(self):
        if self.ctx:
            A.dm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def build_partitions_batch(maps, volumes, stream=None):
    """The precompute of several volumes in one libdm call (dm_build_partitions_batch):
    maps[i] is built from volumes[i] exactly as maps[i].build_partitions(volumes[i])."""
    maps, volumes = list(maps), list(volumes)
    if len(maps) != len(volumes):
        raise ValueError(f"{len(maps)} maps but {len(volumes)} volumes")
    for m, v in zip(maps, volumes):
        m._prepare_build(v)
    A.dm_build_partitions_batch([m.ctx for m in maps], [v.data_ptr() for v in volumes],
                                _stream_handle(stream))
    for m in maps:
        m._host_valid = False
