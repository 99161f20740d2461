"""Object wrappers over the C ABI for Python callers (tests, benchmark, applications).

`HashMap` and `Volume` own a libvbh handle plus the torch CUDA tensors that receive outputs
(per-op results, the Marching Cubes stream).  They only allocate buffers and marshal arguments;
every step of the method runs in libvbh's kernels.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import torch

from . import vbh as V


def _stream() -> int:
    return torch.cuda.current_stream().cuda_stream


def _check_keys3(keys3: torch.Tensor):
    """Block keys handed to the library by pointer: a dense [n, 3] int32 CUDA tensor."""
    if keys3.dtype != torch.int32 or keys3.dim() != 2 or keys3.shape[1] != 3:
        raise ValueError(f"keys3 must be int32 [n, 3], got {keys3.dtype} {tuple(keys3.shape)}")
    if not (keys3.is_cuda and keys3.is_contiguous()):
        raise ValueError("keys3 must be a contiguous CUDA tensor")


class HashMap:
    """GPU map of int3 keys (Sec. 5).  With max_blocks > 0 the values are voxel-block pool
    indices (a voxel-block map); otherwise they are the caller's uint32 values."""

    def __init__(self, n_buckets: int, hash_fn: int = V.VBH_HASH_MIX, max_batch: int = 1 << 22,
                 max_blocks: int = 0):
        cfg = V.vbh_config(n_buckets=n_buckets, slots_per_bucket=4, hash_fn=hash_fn,
                           max_batch=max_batch, max_blocks=max_blocks)
        if max_blocks:
            cfg.voxel_size, cfg.trunc, cfg.max_weight, cfg.depth_scale = 0.01, 0.04, 64.0, 0.001
            cfg.width, cfg.height, cfg.fx, cfg.fy, cfg.cx, cfg.cy = 1, 1, 1.0, 1.0, 0.0, 0.0
        self.cfg = cfg
        self.h = V.vbh_create(cfg, _stream())

    def close(self):
        if getattr(self, "h", None):
            V.vbh_destroy(self.h)
            self.h = None

    __del__ = close

    def batch(self, ops: torch.Tensor, keys3: torch.Tensor, vals: torch.Tensor | None = None,
              results: torch.Tensor | None = None, status: torch.Tensor | None = None):
        n = int(ops.shape[0])
        if keys3.shape != (n, 3) or (vals is not None and vals.shape[0] < n):
            raise ValueError(f"batch of {n} ops needs keys3 [{n}, 3] (got {tuple(keys3.shape)})"
                             " and at least as many values")
        # the kernels read and write these as dense device arrays of exactly these types
        arrays = [(name, t, types) for name, t, types in (
            ("ops", ops, (torch.uint8,)), ("keys3", keys3, (torch.int32,)),
            ("vals", vals, (torch.int32, torch.uint32)),
            ("results", results, (torch.int32, torch.uint32)),
            ("status", status, (torch.uint8,))) if t is not None]
        for name, t, types in arrays:
            if t.dtype not in types:
                raise ValueError(f"{name} must be {' or '.join(map(str, types))}, got {t.dtype}")
        for name, t, _ in arrays:
            if not (t.is_cuda and t.is_contiguous()):
                raise ValueError(f"{name} must be a contiguous CUDA tensor")
            if name in ("results", "status") and t.shape[0] < n:
                raise ValueError(f"{name} holds {t.shape[0]} entries, the batch has {n} ops")
        if results is None:
            results = torch.empty(n, dtype=torch.int32, device=ops.device)
        if status is None:
            status = torch.empty(n, dtype=torch.uint8, device=ops.device)
        V.vbh_hash_batch(self.h, ops, keys3, vals, results, status, n)
        return results, status

    def rebuild(self):
        V.vbh_hash_rebuild(self.h)

    def counters(self) -> V.vbh_counters:
        return V.vbh_get_counters(self.h)

    def dump(self):
        n = self.counters().live
        k = np.zeros((max(n, 1), 3), np.int32)
        v = np.zeros(max(n, 1), np.uint32)
        m = V.vbh_dump(self.h, k, None, None, v, n)
        return k[:m], v[:m]


@dataclasses.dataclass
class McStream:
    """Device buffers of one extraction (see vbh_mc_stream)."""
    keys3: torch.Tensor
    info: torch.Tensor
    offsets: torch.Tensor
    counts: torch.Tensor
    local: torch.Tensor
    index: torch.Tensor
    n: torch.Tensor        # [n_blocks, n_entries] (uint32 on the device)

    @classmethod
    def allocate(cls, cap_blocks: int, cap_entries: int, device="cuda"):
        z = lambda n, dt: torch.zeros(max(n, 1), dtype=dt, device=device)
        return cls(z(3 * cap_blocks, torch.int32).view(-1, 3), z(cap_blocks, torch.int32),
                   z(cap_blocks, torch.int32), z(cap_blocks, torch.int32),
                   z(cap_entries, torch.int16), z(cap_entries, torch.uint8), z(2, torch.int32))

    def c_struct(self) -> V.vbh_mc_stream:
        cs = self.__dict__.get("_cs")
        if cs is None:
            cs = self.__dict__["_cs"] = self._make_struct()
        return cs

    def _make_struct(self) -> V.vbh_mc_stream:
        return V.vbh_mc_stream(self.keys3.data_ptr(), self.info.data_ptr(), self.offsets.data_ptr(),
                               self.counts.data_ptr(), self.local.data_ptr(), self.index.data_ptr(),
                               self.info.shape[0], self.local.shape[0], self.n.data_ptr(),
                               self.n.data_ptr() + 4)

    def to_host(self):
        """{(x, y, z): (info, local idx array, cube idx array)} of the produced records."""
        nb, ne = (int(x) & 0xFFFFFFFF for x in self.n.cpu().tolist())
        if nb > self.info.shape[0] or ne > self.local.shape[0]:
            raise RuntimeError(f"stream overflow: {nb} blocks / {ne} entries")
        keys = self.keys3[:nb].cpu().numpy()
        info = self.info[:nb].cpu().numpy().view(np.uint32)
        off = self.offsets[:nb].cpu().numpy().view(np.uint32)
        cnt = self.counts[:nb].cpu().numpy().view(np.uint32)
        loc = self.local[:ne].cpu().numpy().view(np.uint16)
        idx = self.index[:ne].cpu().numpy()
        out = {}
        for i in range(nb):
            k = tuple(int(x) for x in keys[i])
            if k in out:
                raise RuntimeError(f"block {k} emitted twice")
            o, c = int(off[i]), int(cnt[i])
            out[k] = (int(info[i]), loc[o:o + c].copy(), idx[o:o + c].copy())
        return out


@dataclasses.dataclass
class HostStream:
    """Pinned host buffers of one frame's MC stream (see vbh_mc_stream_host)."""
    keys3: torch.Tensor
    info: torch.Tensor
    offsets: torch.Tensor
    counts: torch.Tensor
    local: torch.Tensor
    index: torch.Tensor

    @classmethod
    def allocate(cls, cap_blocks: int, cap_entries: int):
        z = lambda n, dt: torch.zeros(max(n, 1), dtype=dt).pin_memory()
        return cls(z(3 * cap_blocks, torch.int32).view(-1, 3), z(cap_blocks, torch.int32),
                   z(cap_blocks, torch.int32), z(cap_blocks, torch.int32),
                   z(cap_entries, torch.int16), z(cap_entries, torch.uint8))

    def c_struct(self) -> V.vbh_mc_stream_host:
        cs = self.__dict__.get("_cs")
        if cs is None:
            cs = self.__dict__["_cs"] = V.vbh_mc_stream_host(
                self.keys3.data_ptr(), self.info.data_ptr(), self.offsets.data_ptr(),
                self.counts.data_ptr(), self.local.data_ptr(), self.index.data_ptr(),
                self.info.shape[0], self.local.shape[0], 0, 0, 0, 0)
        return cs

    @property
    def done(self) -> bool:
        return bool(self.c_struct().done)

    @property
    def n(self) -> tuple[int, int]:
        """(records, entries) the frame produced (valid once done)."""
        cs = self.c_struct()
        return cs.n_blocks, cs.n_entries

    def to_host(self):
        """{(x, y, z): (info, local idx array, cube idx array)} of the frame's records."""
        cs = self.c_struct()
        if not cs.done:
            raise RuntimeError("frame not complete")
        nb, ne = cs.n_blocks, cs.n_entries
        if nb > self.info.shape[0] or ne > self.local.shape[0]:
            raise RuntimeError(f"stream overflow: {nb} blocks / {ne} entries")
        keys = self.keys3[:nb].numpy()
        info = self.info[:nb].numpy().view(np.uint32)
        off = self.offsets[:nb].numpy().view(np.uint32)
        cnt = self.counts[:nb].numpy().view(np.uint32)
        loc = self.local[:ne].numpy().view(np.uint16)
        idx = self.index[:ne].numpy()
        out = {}
        for i in range(nb):
            k = tuple(int(x) for x in keys[i])
            if k in out:
                raise RuntimeError(f"block {k} emitted twice")
            o, c = int(off[i]), int(cnt[i])
            out[k] = (int(info[i]), loc[o:o + c].copy(), idx[o:o + c].copy())
        return out


class Volume:
    """Voxel-block TSDF volume on one GPU (Sec. 4.1 fusion, Sec. 4.2 MC indices)."""

    def __init__(self, voxel_size, trunc, width, height, fx, fy, cx, cy, n_buckets, max_blocks,
                 max_weight=64.0, depth_scale=0.001, zmax=0.0, hash_fn=V.VBH_HASH_MIX,
                 mc_cap_blocks=None, mc_cap_entries=None):
        cfg = V.vbh_config(voxel_size=voxel_size, trunc=trunc, max_weight=max_weight,
                           depth_scale=depth_scale, zmax=zmax, width=width, height=height,
                           fx=fx, fy=fy, cx=cx, cy=cy, n_buckets=n_buckets, slots_per_bucket=4,
                           max_blocks=max_blocks, hash_fn=hash_fn, max_batch=max(max_blocks, 1))
        self.cfg = cfg
        self.h = V.vbh_create(cfg, _stream())
        cb = mc_cap_blocks if mc_cap_blocks is not None else max_blocks
        ce = mc_cap_entries if mc_cap_entries is not None else max_blocks * 512
        self.stream = McStream.allocate(cb, ce)
        self.erased_keys = torch.zeros((max_blocks, 3), dtype=torch.int32, device="cuda")
        self.n_erased = torch.zeros(1, dtype=torch.int32, device="cuda")

    def close(self):
        srv = getattr(self, "_server", None)
        if srv is not None:
            srv.close()
            self._server = None
        if getattr(self, "h", None):
            V.vbh_destroy(self.h)
            self.h = None

    __del__ = close

    def integrate(self, depth: torch.Tensor, T_wc, frame_id: int, stats: bool = False):
        assert depth.dtype == torch.uint16 and depth.is_cuda and depth.is_contiguous()
        return V.vbh_integrate_frame(self.h, depth, T_wc, frame_id, stats)

    def process_frame(self, depth: torch.Tensor, T_wc, frame_id: int, erase_radius: float,
                      stream: McStream | None = None):
        """Erase beyond `erase_radius` of the camera, fuse the frame, extract the touched MC
        blocks into `stream` -- one CUDA-graph launch."""
        assert depth.dtype == torch.uint16 and depth.is_cuda and depth.is_contiguous()
        s = stream or self.stream
        V.vbh_process_frame(self.h, depth, T_wc, frame_id, erase_radius, s.c_struct())
        return s

    def process_frame_host(self, depth_host, T_wc, frame_id: int, erase_radius: float,
                           out: HostStream) -> int:
        """The frame from host depth (pinned uint16 for overlap) with its MC stream copied into
        `out` (pinned host buffers) while the next frames run: enqueues this frame and returns
        once the `out` of two calls earlier is complete (status VBH_OK or
        VBH_ERR_BUFFER_TOO_SMALL); process_frame_host_flush completes every pending frame."""
        if isinstance(depth_host, torch.Tensor):
            assert depth_host.dtype == torch.uint16 and not depth_host.is_cuda
            assert depth_host.is_contiguous()
        else:
            assert depth_host.dtype == np.uint16 and depth_host.flags["C_CONTIGUOUS"]
        assert tuple(depth_host.shape) == (self.cfg.height, self.cfg.width)
        return V.vbh_process_frame_host(self.h, depth_host, T_wc, frame_id, erase_radius,
                                        out.c_struct())

    def process_frame_host_flush(self) -> int:
        return V.vbh_process_frame_host_flush(self.h)

    def erase_radius(self, centre, radius, keys_out: bool = True):
        sel = V.vbh_erase_selector(mode=V.VBH_ERASE_RADIUS, radius=float(radius))
        sel.centre[:] = [float(c) for c in centre]
        V.vbh_erase_blocks(self.h, sel, self.erased_keys if keys_out else None,
                           self.n_erased if keys_out else None)

    def erase_frustum(self, T_wc, zfar: float = 0.0, keys_out: bool = True):
        """Scene reset: erase every block in view of pose T_wc (3x4) up to depth zfar."""
        sel = V.vbh_erase_selector(mode=V.VBH_ERASE_FRUSTUM, zfar=float(zfar))
        sel.T_wc[:] = [float(x) for x in np.asarray(T_wc, np.float32).reshape(12)]
        V.vbh_erase_blocks(self.h, sel, self.erased_keys if keys_out else None,
                           self.n_erased if keys_out else None)

    def set_integration_mode(self, visible: bool):
        """Fuse the touched blocks only (default) or also every live block in view."""
        V.vbh_set_integration_mode(self.h, V.VBH_INTEGRATE_VISIBLE if visible
                                   else V.VBH_INTEGRATE_TOUCHED)

    def erase_keys(self, keys3: torch.Tensor, keys_out: bool = True):
        _check_keys3(keys3)
        sel = V.vbh_erase_selector(mode=V.VBH_ERASE_KEYS, keys3_dev=keys3.data_ptr(),
                                   n_keys=int(keys3.shape[0]))
        V.vbh_erase_blocks(self.h, sel, self.erased_keys if keys_out else None,
                           self.n_erased if keys_out else None)

    def erased(self) -> np.ndarray:
        n = int(self.n_erased.item())
        return self.erased_keys[:n].cpu().numpy()

    def extract(self, mode=V.VBH_MC_TOUCHED, keys3: torch.Tensor | None = None, since=0,
                stream: McStream | None = None, sync=False):
        s = stream or self.stream
        if keys3 is not None:
            _check_keys3(keys3)
        sel = V.vbh_mc_selector(mode=mode, keys3_dev=keys3.data_ptr() if keys3 is not None else None,
                                n_keys=int(keys3.shape[0]) if keys3 is not None else 0,
                                since_version=since)
        need = V.vbh_extract_mc_indices(self.h, sel, s.c_struct(), want_needed=sync)
        return s if not sync else (s, need)

    def counters(self) -> V.vbh_counters:
        return V.vbh_get_counters(self.h)

    def clear_errors(self):
        V.vbh_clear_errors(self.h)

    def set_wait_limit(self, polls: int):
        V.vbh_set_wait_limit(self.h, polls)

    def dump(self):
        n = self.counters().live
        k = np.zeros((max(n, 1), 3), np.int32)
        F = np.zeros((max(n, 1), 512), np.float32)
        W = np.zeros((max(n, 1), 512), np.float32)
        m = V.vbh_dump(self.h, k, F, W, None, n)
        order = np.lexsort((k[:m, 2], k[:m, 1], k[:m, 0]))
        return k[:m][order], F[:m][order], W[:m][order]

    def load(self, keys3, tsdf, weight):
        V.vbh_load(self.h, np.ascontiguousarray(keys3, np.int32),
                   np.ascontiguousarray(tsdf, np.float32), np.ascontiguousarray(weight, np.float32))

    def triangulate(self, stream: McStream | None = None, cap: int | None = None):
        """Triangles (n, 3, 3) float32 in metres of an MC stream (default: the volume's last
        extraction), vertices at edge midpoints."""
        s = stream or self.stream
        cap = cap if cap is not None else int(s.local.shape[0])
        tris = torch.empty((max(cap, 1), 9), dtype=torch.float32, device="cuda")
        n = torch.zeros(1, dtype=torch.int32, device="cuda")
        V.vbh_mc_triangulate(s.c_struct(), float(self.cfg.voxel_size), tris, cap, n,
                             torch.cuda.current_stream().cuda_stream)
        m = int(n.item())
        if m > cap:
            raise RuntimeError(f"{m} triangles, capacity {cap}")
        return tris[:m].view(-1, 3, 3)

    # ---- stream-out of erased blocks to the host map, explicit stream-in
    def stream_out_enable(self, ring_blocks: int = 0):
        V.vbh_stream_out_enable(self.h, ring_blocks)

    def stream_out_poll(self) -> int:
        return V.vbh_stream_out_poll(self.h)

    def stream_out_flush(self):
        V.vbh_stream_out_flush(self.h)

    def stream_out_stats(self):
        """(blocks streamed out so far, blocks lost for want of ring room, host map size)."""
        return V.vbh_stream_out_stats(self.h)

    def host_map(self):
        """The host map of streamed-out blocks: keys sorted, TSDF, weights."""
        n = V.vbh_stream_out_stats(self.h)[2]
        k = np.zeros((max(n, 1), 3), np.int32)
        F = np.zeros((max(n, 1), 512), np.float32)
        W = np.zeros((max(n, 1), 512), np.float32)
        m = V.vbh_host_map_dump(self.h, k, F, W, n)
        order = np.lexsort((k[:m, 2], k[:m, 1], k[:m, 0]))
        return k[:m][order], F[:m][order], W[:m][order]

    def stream_in(self, keys3) -> int:
        return V.vbh_stream_in(self.h, keys3)

    def timing(self, stages=("erase", "alloc", "integrate", "mcset", "mc", "hash")):
        """Record CUDA events around the named stages (empty / None: off)."""
        mask = 0
        for s in stages or ():
            mask |= 1 << V.VBH_STAGES.index(s)
        V.vbh_timing_enable(self.h, mask)

    def timing_read(self, reset=False):
        return V.vbh_timing_read(self.h, reset)
