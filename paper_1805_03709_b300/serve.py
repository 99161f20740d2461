"""Multi-client delta streaming (vbh_serve_* in include/vbh.h): argument marshalling only.

A `Server` attaches to a `Volume`; each client holds a change sequence number on the device and
asks for the MC blocks refreshed (or removed) since it.  Requests are served by continuous
batching in libvbh's native scheduler; results are views of the server's stream buffer until
released.  Nothing here computes any part of the method.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import vbh as V
from .volume import Volume


class _DevView:
    """A raw device buffer exposed to torch through __cuda_array_interface__ (no copy)."""

    def __init__(self, ptr: int, shape, typestr: str):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr,
                                         "data": (int(ptr), False), "version": 3}


def done_dict(d: V.vbh_serve_done) -> dict:
    return {k: getattr(d, k) for k, _ in V.vbh_serve_done._fields_}


class Server:
    def __init__(self, vol: Volume, n_clients: int, max_batch: int = 64, chunk_records: int = 0,
                 iter_records: int = 0, max_inflight: int = 2, bypass_iters: int = 8,
                 budget_bytes: int = 4 << 30, log_bits: int = 0, rem_bits: int = 0):
        self.vol = vol
        self.n_clients = n_clients
        self.cfg = V.vbh_serve_config(n_clients=n_clients, max_batch=max_batch,
                                      chunk_records=chunk_records, iter_records=iter_records,
                                      max_inflight=max_inflight, bypass_iters=bypass_iters,
                                      log_bits=log_bits, rem_bits=rem_bits,
                                      budget_bytes=budget_bytes)
        self.s = V.vbh_serve_create(vol.h, self.cfg)
        vol._server = self

    def close(self):
        loop = getattr(self, "_loop", None)
        if loop is not None and getattr(loop, "L", None):
            loop.stop()
        if getattr(self, "s", None):
            if getattr(self.vol, "h", None):
                V.vbh_serve_destroy(self.s)
            self.s = None

    __del__ = close

    def set_policy(self, max_batch: int, chunk_records: int = 0, iter_records: int = 0,
                   max_inflight: int = 2, bypass_iters: int = 8):
        c = V.vbh_serve_config(n_clients=self.n_clients, max_batch=max_batch,
                               chunk_records=chunk_records, iter_records=iter_records,
                               max_inflight=max_inflight, bypass_iters=bypass_iters)
        V.vbh_serve_set_policy(self.s, c)

    def set_versions(self, clients, versions):
        V.vbh_serve_set_versions(self.s, clients, versions)

    def versions(self) -> np.ndarray:
        return V.vbh_serve_get_versions(self.s, self.n_clients)

    def versions_for_backlog(self, backlogs) -> np.ndarray:
        return V.vbh_serve_versions_for_backlog(self.s, backlogs)

    def submit(self, client: int, t_arrival_ns: int = 0) -> int:
        return V.vbh_serve_submit(self.s, client, t_arrival_ns)

    def step(self) -> int:
        return V.vbh_serve_step(self.s)

    def poll(self) -> list[dict]:
        out = []
        while True:
            got = V.vbh_serve_poll(self.s, 256)
            out += [done_dict(d) for d in got]
            if len(got) < 256:
                return out

    def drain(self) -> list[dict]:
        V.vbh_serve_drain(self.s)
        return self.poll()

    def result(self, rid: int, copy: bool = True):
        """(records int32 [n, 4] = x, y, z, info bits; indices uint8 [n, 512], flags)."""
        v = V.vbh_serve_result(self.s, rid)
        n = v.n_records
        if n == 0:
            return (torch.zeros((0, 4), dtype=torch.int32, device="cuda"),
                    torch.zeros((0, 512), dtype=torch.uint8, device="cuda"), v.flags)
        recs = torch.as_tensor(_DevView(v.recs_dev, (n, 4), "<i4"), device="cuda")
        idx = torch.as_tensor(_DevView(v.indices_dev, (n, 512), "|u1"), device="cuda")
        if copy:
            recs, idx = recs.clone(), idx.clone()
        return recs, idx, v.flags

    def release(self, rid: int):
        V.vbh_serve_release(self.s, rid)

    def stats(self) -> dict:
        st = V.vbh_serve_stats_read(self.s)
        return {k: getattr(st, k) for k, _ in V.vbh_serve_stats._fields_}

    def run(self, t_ns, client, depth_frames=None, poses=None, frame_ids=None,
            erase_radius: float = 0.0, cap: int | None = None) -> list[dict]:
        """Real-time script: request arrivals (client >= 0) and frames (client -1) at t_ns."""
        sc, keep, n_req = _script(self.vol, t_ns, client, depth_frames, poses, frame_ids,
                                  erase_radius)
        got = V.vbh_serve_run(self.s, sc, cap if cap is not None else n_req)
        return [done_dict(d) for d in got]


def _script(vol, t_ns, client, depth_frames, poses, frame_ids, erase_radius):
    """A vbh_serve_script and the host arrays it points to (kept alive by the caller)."""
    t = np.ascontiguousarray(t_ns, np.uint64)
    c = np.ascontiguousarray(client, np.int32)
    nf = int((c < 0).sum())
    sc = V.vbh_serve_script(n_events=len(t), t_ns=t.ctypes.data, client=c.ctypes.data,
                            erase_radius=float(erase_radius))
    keep = [t, c]
    if nf:
        ptrs = (ctypes.c_void_p * nf)(*[d.data_ptr() for d in depth_frames[:nf]])
        P = np.ascontiguousarray(np.asarray(poses[:nf], np.float32).reshape(nf, 12))
        ids = np.ascontiguousarray(np.asarray(frame_ids[:nf]), np.uint32)
        sc.depth_dev = ctypes.cast(ptrs, ctypes.c_void_p)
        sc.T_wc = P.ctypes.data
        sc.frame_id = ids.ctypes.data
        ms = vol.stream.c_struct()
        sc.frame_out = ctypes.pointer(ms)
        keep += [ptrs, P, ids, ms]
    return sc, keep, int((c >= 0).sum())


class ServeLoop:
    """The device-resident request loop of a Server (vbh_serve_loop_*): one persistent kernel
    admits, batches and serves the requests while frames run on the volume's stream.  While it
    runs, synchronise streams rather than the whole device (a device-wide synchronisation waits
    for the loop to stop)."""

    def __init__(self, server: Server, ctas: int = 0, max_slots: int = 0, chunk_records: int = 0,
                 bypass_rounds: int = 8, ring: int = 0, idle_timeout_us: int = 0):
        self.server = server
        self.cfg = V.vbh_serve_loop_config(ctas=ctas, max_slots=max_slots,
                                           chunk_records=chunk_records,
                                           bypass_rounds=bypass_rounds, ring=ring,
                                           idle_timeout_us=idle_timeout_us)
        self.L = V.vbh_serve_loop_start(server.s, self.cfg)
        server._loop = self

    def stop(self):
        """Stop the loop; raises VbhError with the status it stopped with by itself."""
        if getattr(self, "L", None):
            L, self.L = self.L, None
            V.vbh_serve_loop_stop(L)

    close = stop

    def __del__(self):
        if getattr(self, "L", None):
            try:
                self.stop()
            except V.VbhError:
                pass

    def submit(self, client: int, t_arrival_ns: int = 0) -> int:
        return V.vbh_serve_loop_submit(self.L, client, t_arrival_ns)

    def poll(self) -> list[dict]:
        out = []
        while True:
            got = V.vbh_serve_loop_poll(self.L, 256)
            out += [done_dict(d) for d in got]
            if len(got) < 256:
                return out

    def drain(self, timeout_s: float = 60.0) -> list[dict]:
        V.vbh_serve_loop_drain(self.L, int(timeout_s * 1e9))
        return self.poll()

    def result(self, rid: int, copy: bool = True):
        """(records int32 [n, 4] = x, y, z, info bits; indices uint8 [n, 512], flags)."""
        v = V.vbh_serve_loop_result(self.L, rid)
        n = v.n_records
        if n == 0:
            return (torch.zeros((0, 4), dtype=torch.int32, device="cuda"),
                    torch.zeros((0, 512), dtype=torch.uint8, device="cuda"), v.flags)
        recs = torch.as_tensor(_DevView(v.recs_dev, (n, 4), "<i4"), device="cuda")
        idx = torch.as_tensor(_DevView(v.indices_dev, (n, 512), "|u1"), device="cuda")
        if copy:
            recs, idx = recs.clone(), idx.clone()
        return recs, idx, v.flags

    def release(self, rid: int):
        V.vbh_serve_loop_release(self.L, rid)

    def stats(self) -> dict:
        st = V.vbh_serve_loop_stats_read(self.L)
        return {k: getattr(st, k) for k, _ in V.vbh_serve_loop_stats._fields_}

    def run(self, t_ns, client, depth_frames=None, poses=None, frame_ids=None,
            erase_radius: float = 0.0, cap: int | None = None) -> list[dict]:
        """Real-time script as Server.run, served by the device-resident loop."""
        sc, keep, n_req = _script(self.server.vol, t_ns, client, depth_frames, poses,
                                  frame_ids, erase_radius)
        got = V.vbh_serve_loop_run(self.L, sc, cap if cap is not None else n_req)
        return [done_dict(d) for d in got]


class StreamSets:
    """The paper's per-client stream sets (vbh_sets_*), beside a Server whose store they read."""

    def __init__(self, server: Server, n_clients: int, cap_log2: int = 18):
        self.server = server
        self.n_clients = n_clients
        self.q = V.vbh_sets_create(server.s, n_clients, cap_log2)

    def close(self):
        if getattr(self, "q", None):
            if getattr(self.server, "s", None):
                V.vbh_sets_destroy(self.q)
            self.q = None

    __del__ = close

    def insert_last(self):
        V.vbh_sets_insert_last(self.q)

    def fill(self, client: int):
        V.vbh_sets_fill(self.q, client)

    def fetch(self, clients, limits):
        """[(records int32 [n, 4], indices uint8 [n, 512])] per request (device tensors)."""
        total = int(np.sum(limits))
        recs = torch.empty((total, 4), dtype=torch.int32, device="cuda")
        idx = torch.empty((total, 512), dtype=torch.uint8, device="cuda")
        n_out = torch.empty(len(clients), dtype=torch.int32, device="cuda")
        V.vbh_sets_fetch(self.q, clients, limits, recs, idx, n_out)
        n = n_out.cpu().numpy()
        out, off = [], 0
        for i, lim in enumerate(limits):
            out.append((recs[off:off + n[i]], idx[off:off + n[i]]))
            off += int(lim)
        return out

    def counts(self):
        return V.vbh_sets_counts(self.q, self.n_clients)

    def rebuild(self, client: int):
        V.vbh_sets_rebuild(self.q, client)
