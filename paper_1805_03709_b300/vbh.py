"""Python binding of libvbh (include/vbh.h): ctypes argument marshalling only.

Every function below forwards to the C entry point of the same name; device buffers are torch
CUDA tensors (their data_ptr() is passed), host buffers are numpy arrays.  Nothing here computes
any part of the method, and there is no fallback: if libvbh.so is missing or cannot be loaded,
`lib()` raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libvbh.so")

VBH_OK, VBH_ERR_INVALID_ARG, VBH_ERR_CAPACITY, VBH_ERR_CUDA, VBH_ERR_TIMEOUT, \
    VBH_ERR_BUFFER_TOO_SMALL, VBH_ERR_UNSUPPORTED = range(7)
VBH_OP_FIND, VBH_OP_INSERT, VBH_OP_ERASE = 0, 1, 2
VBH_ST_FOUND, VBH_ST_NOT_FOUND, VBH_ST_INSERTED, VBH_ST_EXISTS, VBH_ST_ERASED, \
    VBH_ST_CAPACITY, VBH_ST_INVALID = range(1, 8)
VBH_NONE = 0xFFFFFFFF
VBH_HASH_PRIMES, VBH_HASH_MIX = 0, 1
VBH_ERASE_RADIUS, VBH_ERASE_KEYS, VBH_ERASE_FRUSTUM = 0, 1, 2
VBH_INTEGRATE_TOUCHED, VBH_INTEGRATE_VISIBLE = 0, 1
VBH_MC_TOUCHED, VBH_MC_ALL, VBH_MC_KEYS, VBH_MC_SINCE = 0, 1, 2, 3
VBH_REC_REMOVED = 0x80000000
VBH_STAGES = ("erase", "alloc", "integrate", "mcset", "mc", "hash")

_u32, _i32, _f32, _u64, _p = ctypes.c_uint32, ctypes.c_int32, ctypes.c_float, ctypes.c_uint64, ctypes.c_void_p


class vbh_config(ctypes.Structure):
    _fields_ = [("voxel_size", _f32), ("trunc", _f32), ("max_weight", _f32),
                ("depth_scale", _f32), ("zmax", _f32), ("width", _i32), ("height", _i32),
                ("fx", _f32), ("fy", _f32), ("cx", _f32), ("cy", _f32), ("n_buckets", _u32),
                ("slots_per_bucket", _u32), ("max_blocks", _u32), ("hash_fn", _u32),
                ("max_batch", _u32)]


class vbh_counters(ctypes.Structure):
    _fields_ = [("live", _u32), ("tombstones", _u32), ("empty", _u32), ("free_blocks", _u32),
                ("last_touched", _u32), ("last_new", _u32), ("last_candidates", _u32),
                ("error_flags", _u32), ("kernel_launches", _u64), ("rebuilds", _u32),
                ("last_mc_blocks", _u32), ("last_mc_entries", _u32), ("last_erased", _u32),
                ("voxels_written", _u64), ("total_frames", _u64), ("total_touched", _u64),
                ("total_new", _u64), ("total_written", _u64)]


class vbh_frame_stats(ctypes.Structure):
    _fields_ = [("touched", _u32), ("new_blocks", _u32), ("candidates", _u32),
                ("error_flags", _u32)]


class vbh_erase_selector(ctypes.Structure):
    _fields_ = [("mode", _u32), ("centre", _f32 * 3), ("radius", _f32), ("keys3_dev", _p),
                ("n_keys", _u32), ("T_wc", _f32 * 12), ("zfar", _f32)]


class vbh_mc_selector(ctypes.Structure):
    _fields_ = [("mode", _u32), ("keys3_dev", _p), ("n_keys", _u32), ("since_version", _u32)]


class vbh_mc_stream(ctypes.Structure):
    _fields_ = [("keys3", _p), ("info", _p), ("offsets", _p), ("counts", _p), ("local", _p),
                ("index", _p), ("cap_blocks", _u32), ("cap_entries", _u32),
                ("n_blocks_dev", _p), ("n_entries_dev", _p)]


class vbh_mc_stream_host(ctypes.Structure):
    _fields_ = [("keys3", _p), ("info", _p), ("offsets", _p), ("counts", _p), ("local", _p),
                ("index", _p), ("cap_blocks", _u32), ("cap_entries", _u32), ("n_blocks", _u32),
                ("n_entries", _u32), ("frame_id", _u32), ("done", _u32)]


class vbh_diff_config(ctypes.Structure):
    _fields_ = [("voxel_size", _f32), ("trunc", _f32), ("width", _i32), ("height", _i32),
                ("fx", _f32), ("fy", _f32), ("cx", _f32), ("cy", _f32), ("n_frames", _u32)]


# every symbol include/vbh.h declares: (name, restype, argtypes)
SYMBOLS = [
    ("vbh_abi_version", ctypes.c_int, []),
    ("vbh_last_error", ctypes.c_char_p, []),
    ("vbh_bucket_of", _u32, [_i32, _i32, _i32, _u32, _u32]),
    ("vbh_create", ctypes.c_int, [ctypes.POINTER(vbh_config), _p, ctypes.POINTER(_p)]),
    ("vbh_destroy", ctypes.c_int, [_p]),
    ("vbh_set_stream", ctypes.c_int, [_p, _p]),
    ("vbh_hash_batch", ctypes.c_int, [_p, _p, _p, _p, _p, _p, _u32]),
    ("vbh_hash_rebuild", ctypes.c_int, [_p]),
    ("vbh_integrate_frame", ctypes.c_int, [_p, _p, _p, _u32, ctypes.POINTER(vbh_frame_stats)]),
    ("vbh_erase_blocks", ctypes.c_int, [_p, ctypes.POINTER(vbh_erase_selector), _p, _p]),
    ("vbh_extract_mc_indices", ctypes.c_int,
     [_p, ctypes.POINTER(vbh_mc_selector), ctypes.POINTER(vbh_mc_stream), ctypes.POINTER(_u64)]),
    ("vbh_process_frame", ctypes.c_int,
     [_p, _p, _p, _u32, _f32, ctypes.POINTER(vbh_mc_stream)]),
    ("vbh_process_frame_host", ctypes.c_int,
     [_p, _p, _p, _u32, _f32, ctypes.POINTER(vbh_mc_stream_host)]),
    ("vbh_process_frame_host_flush", ctypes.c_int, [_p]),
    ("vbh_dump", ctypes.c_int, [_p, _p, _p, _p, _p, _u32, ctypes.POINTER(_u32)]),
    ("vbh_load", ctypes.c_int, [_p, _p, _p, _p, _u32]),
    ("vbh_get_counters", ctypes.c_int, [_p, ctypes.POINTER(vbh_counters)]),
    ("vbh_clear_errors", ctypes.c_int, [_p]),
    ("vbh_set_wait_limit", ctypes.c_int, [_p, _u32]),
    ("vbh_timing_enable", ctypes.c_int, [_p, ctypes.c_int]),
    ("vbh_timing_read", ctypes.c_int, [_p, _p, _p, ctypes.c_int]),
    ("vbh_diff_create", ctypes.c_int,
     [ctypes.POINTER(vbh_diff_config), _p, ctypes.POINTER(_p)]),
    ("vbh_diff_destroy", ctypes.c_int, [_p]),
    ("vbh_diff_poses", ctypes.c_int, [_p, _p, _p]),
    ("vbh_diff_masks", ctypes.c_int, [_p, _p, _u32, _p, _p, _p]),
    ("vbh_diff_forward", ctypes.c_int, [_p, _p, _u32, _p, _p, _p, _p, _p, _p]),
    ("vbh_diff_backward", ctypes.c_int, [_p, _p, _u32, _p, _p, _p, _p, _p, _p, _p]),
    ("vbh_mc_from_tsdf_static", ctypes.c_int,
     [_p, _p, _p, _u32, ctypes.POINTER(vbh_mc_stream), _p, _p]),
]


_lib = None


VBH_SERVE_RESET, VBH_SERVE_PARTIAL, VBH_SERVE_ERR_OVERRUN, VBH_SERVE_ERR_CAPACITY, \
    VBH_SERVE_ERR_VERSION = 1, 2, 4, 8, 16


class vbh_serve_config(ctypes.Structure):
    _fields_ = [("n_clients", _u32), ("max_batch", _u32), ("chunk_records", _u32),
                ("iter_records", _u32), ("max_inflight", _u32), ("bypass_iters", _u32),
                ("log_bits", _u32), ("rem_bits", _u32), ("budget_bytes", _u64)]


class vbh_serve_done(ctypes.Structure):
    _fields_ = [("id", _u32), ("client", _u32), ("v_before", _u32), ("v_after", _u32),
                ("n_records", _u32), ("flags", _u32), ("t_arrival_ns", _u64),
                ("t_admit_ns", _u64), ("t_done_ns", _u64), ("bytes_reserved", _u64)]


class vbh_serve_view(ctypes.Structure):
    _fields_ = [("recs_dev", _p), ("indices_dev", _p), ("n_records", _u32), ("flags", _u32)]


class vbh_serve_stats(ctypes.Structure):
    _fields_ = [("iterations", _u64), ("requests_done", _u64), ("records_served", _u64),
                ("changes_scanned", _u64), ("bytes_in_use", _u64), ("bytes_peak", _u64),
                ("deferred_memory", _u64), ("err_flags", _u32), ("sigma", _u32)]


class vbh_serve_loop_config(ctypes.Structure):
    _fields_ = [("ctas", _u32), ("max_slots", _u32), ("chunk_records", _u32),
                ("bypass_rounds", _u32), ("ring", _u32), ("idle_timeout_us", _u32)]


class vbh_serve_loop_stats(ctypes.Structure):
    _fields_ = [("requests_done", _u64), ("records_served", _u64),
                ("change_records_scanned", _u64), ("chunks", _u64), ("rounds", _u64),
                ("deferred_memory", _u64), ("bytes_in_use", _u64), ("bytes_peak", _u64),
                ("max_active", _u32), ("status", _u32), ("launches", _u32)]


class vbh_serve_script(ctypes.Structure):
    _fields_ = [("n_events", _u32), ("t_ns", _p), ("client", _p), ("depth_dev", _p),
                ("T_wc", _p), ("frame_id", _p), ("erase_radius", _f32),
                ("frame_out", ctypes.POINTER(vbh_mc_stream))]


SYMBOLS += [
    ("vbh_mc_tri_table", ctypes.c_int, [_p, _p]),
    ("vbh_mc_triangulate", ctypes.c_int, [ctypes.POINTER(vbh_mc_stream), _f32, _p, _u32, _p,
                                          _p]),
    ("vbh_sets_create", ctypes.c_int, [_p, _u32, _u32, ctypes.POINTER(_p)]),
    ("vbh_sets_destroy", ctypes.c_int, [_p]),
    ("vbh_sets_insert_last", ctypes.c_int, [_p]),
    ("vbh_sets_fill", ctypes.c_int, [_p, _u32]),
    ("vbh_sets_fetch", ctypes.c_int, [_p, _p, _p, _u32, _p, _p, _p]),
    ("vbh_sets_counts", ctypes.c_int, [_p, _p, _p, _p]),
    ("vbh_sets_rebuild", ctypes.c_int, [_p, _u32]),
    ("vbh_set_integration_mode", ctypes.c_int, [_p, _u32]),
    ("vbh_stream_out_enable", ctypes.c_int, [_p, _u32]),
    ("vbh_stream_out_poll", ctypes.c_int, [_p, ctypes.POINTER(_u64)]),
    ("vbh_stream_out_flush", ctypes.c_int, [_p]),
    ("vbh_stream_out_stats", ctypes.c_int, [_p, ctypes.POINTER(_u64), ctypes.POINTER(_u64),
                                            ctypes.POINTER(_u32)]),
    ("vbh_host_map_dump", ctypes.c_int, [_p, _p, _p, _p, _u32, ctypes.POINTER(_u32)]),
    ("vbh_stream_in", ctypes.c_int, [_p, _p, _u32, ctypes.POINTER(_u32)]),
    ("vbh_serve_create", ctypes.c_int, [_p, ctypes.POINTER(vbh_serve_config), ctypes.POINTER(_p)]),
    ("vbh_serve_destroy", ctypes.c_int, [_p]),
    ("vbh_serve_set_policy", ctypes.c_int, [_p, ctypes.POINTER(vbh_serve_config)]),
    ("vbh_serve_set_versions", ctypes.c_int, [_p, _p, _p, _u32]),
    ("vbh_serve_get_versions", ctypes.c_int, [_p, _p]),
    ("vbh_serve_versions_for_backlog", ctypes.c_int, [_p, _p, _u32, _p]),
    ("vbh_serve_submit", ctypes.c_int, [_p, _u32, _u64, ctypes.POINTER(_u32)]),
    ("vbh_serve_step", ctypes.c_int, [_p, ctypes.POINTER(_u32)]),
    ("vbh_serve_poll", ctypes.c_int, [_p, _p, _u32, ctypes.POINTER(_u32)]),
    ("vbh_serve_result", ctypes.c_int, [_p, _u32, ctypes.POINTER(vbh_serve_view)]),
    ("vbh_serve_release", ctypes.c_int, [_p, _u32]),
    ("vbh_serve_drain", ctypes.c_int, [_p]),
    ("vbh_serve_stats_read", ctypes.c_int, [_p, ctypes.POINTER(vbh_serve_stats)]),
    ("vbh_serve_run", ctypes.c_int, [_p, ctypes.POINTER(vbh_serve_script), _p, _u32, ctypes.POINTER(_u32)]),
    ("vbh_serve_now_ns", _u64, []),
    ("vbh_serve_loop_start", ctypes.c_int, [_p, ctypes.POINTER(vbh_serve_loop_config),
                                            ctypes.POINTER(_p)]),
    ("vbh_serve_loop_submit", ctypes.c_int, [_p, _u32, _u64, ctypes.POINTER(_u32)]),
    ("vbh_serve_loop_poll", ctypes.c_int, [_p, _p, _u32, ctypes.POINTER(_u32)]),
    ("vbh_serve_loop_result", ctypes.c_int, [_p, _u32, ctypes.POINTER(vbh_serve_view)]),
    ("vbh_serve_loop_release", ctypes.c_int, [_p, _u32]),
    ("vbh_serve_loop_drain", ctypes.c_int, [_p, _u64]),
    ("vbh_serve_loop_run", ctypes.c_int, [_p, ctypes.POINTER(vbh_serve_script), _p, _u32,
                                          ctypes.POINTER(_u32)]),
    ("vbh_serve_loop_stats_read", ctypes.c_int, [_p, ctypes.POINTER(vbh_serve_loop_stats)]),
    ("vbh_serve_loop_stop", ctypes.c_int, [_p]),
]


class VbhError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where} -> status {status}: {msg}")
        self.status = status


def lib() -> ctypes.CDLL:
    """Load libvbh.so from the package directory (build it with `python -m
    paper_1805_03709_b300.build`); raises if it is absent -- there is no CPU fallback."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libvbh.so not built at {LIB_PATH}; run paper_1805_03709_b300/build.py")
        L = ctypes.CDLL(LIB_PATH)
        for name, res, args in SYMBOLS:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(st: int, where: str):
    if st != VBH_OK:
        raise VbhError(st, where, lib().vbh_last_error().decode())


def _ptr(t) -> int | None:
    """data_ptr of a torch tensor (device) or numpy array (host); None stays None."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        assert t.flags["C_CONTIGUOUS"]
        return t.ctypes.data
    assert t.is_contiguous()
    return t.data_ptr()


# ---------------------------------------------------------------------------- same-name calls
def vbh_abi_version() -> int:
    return lib().vbh_abi_version()


def vbh_bucket_of(x: int, y: int, z: int, n_buckets: int, hash_fn: int) -> int:
    return lib().vbh_bucket_of(x, y, z, n_buckets, hash_fn)


def vbh_create(cfg: vbh_config, stream: int | None = None) -> int:
    h = _p()
    _check(lib().vbh_create(ctypes.byref(cfg), stream, ctypes.byref(h)), "vbh_create")
    return h.value


def vbh_destroy(h: int):
    _check(lib().vbh_destroy(h), "vbh_destroy")


def vbh_set_stream(h: int, stream: int | None):
    _check(lib().vbh_set_stream(h, stream), "vbh_set_stream")


def vbh_hash_batch(h, ops, keys3, vals, results, status, n=None):
    n = int(ops.shape[0]) if n is None else int(n)
    _check(lib().vbh_hash_batch(h, _ptr(ops), _ptr(keys3), _ptr(vals), _ptr(results),
                                _ptr(status), n), "vbh_hash_batch")


def vbh_hash_rebuild(h):
    _check(lib().vbh_hash_rebuild(h), "vbh_hash_rebuild")


def vbh_integrate_frame(h, depth, T_wc, frame_id: int, want_stats: bool = False):
    T = np.ascontiguousarray(np.asarray(T_wc, np.float32).reshape(12))
    st = vbh_frame_stats() if want_stats else None
    _check(lib().vbh_integrate_frame(h, _ptr(depth), T.ctypes.data, int(frame_id),
                                     ctypes.byref(st) if st is not None else None),
           "vbh_integrate_frame")
    return st


def vbh_erase_blocks(h, sel: vbh_erase_selector, erased_keys3=None, n_erased=None):
    _check(lib().vbh_erase_blocks(h, ctypes.byref(sel), _ptr(erased_keys3), _ptr(n_erased)),
           "vbh_erase_blocks")


def vbh_extract_mc_indices(h, sel: vbh_mc_selector, out: vbh_mc_stream, want_needed=False):
    need = _u64(0) if want_needed else None
    _check(lib().vbh_extract_mc_indices(h, ctypes.byref(sel), ctypes.byref(out),
                                        ctypes.byref(need) if need is not None else None),
           "vbh_extract_mc_indices")
    return None if need is None else need.value


def vbh_process_frame(h, depth, T_wc, frame_id: int, erase_radius: float, out: vbh_mc_stream):
    T = np.ascontiguousarray(np.asarray(T_wc, np.float32).reshape(12))
    _check(lib().vbh_process_frame(h, _ptr(depth), T.ctypes.data, int(frame_id),
                                   float(erase_radius), ctypes.byref(out)), "vbh_process_frame")


def vbh_process_frame_host(h, depth_host, T_wc, frame_id: int, erase_radius: float,
                           out: vbh_mc_stream_host) -> int:
    """Enqueue a frame from host depth; completes the `out` of two calls earlier (returns its
    status: VBH_OK or VBH_ERR_BUFFER_TOO_SMALL).  `out` is kept by the library until its frame is
    done."""
    T = np.ascontiguousarray(np.asarray(T_wc, np.float32).reshape(12))
    st = lib().vbh_process_frame_host(h, _ptr(depth_host), T.ctypes.data, int(frame_id),
                                      float(erase_radius), ctypes.byref(out))
    if st not in (VBH_OK, VBH_ERR_BUFFER_TOO_SMALL):
        _check(st, "vbh_process_frame_host")
    return st


def vbh_process_frame_host_flush(h) -> int:
    st = lib().vbh_process_frame_host_flush(h)
    if st not in (VBH_OK, VBH_ERR_BUFFER_TOO_SMALL):
        _check(st, "vbh_process_frame_host_flush")
    return st


def vbh_dump(h, keys3, tsdf, weight, vals, cap: int) -> int:
    n = _u32(0)
    _check(lib().vbh_dump(h, _ptr(keys3), _ptr(tsdf), _ptr(weight), _ptr(vals), cap,
                          ctypes.byref(n)), "vbh_dump")
    return n.value


def vbh_load(h, keys3, tsdf, weight):
    _check(lib().vbh_load(h, _ptr(keys3), _ptr(tsdf), _ptr(weight), int(keys3.shape[0])),
           "vbh_load")


def vbh_get_counters(h) -> vbh_counters:
    c = vbh_counters()
    _check(lib().vbh_get_counters(h, ctypes.byref(c)), "vbh_get_counters")
    return c


def vbh_clear_errors(h):
    _check(lib().vbh_clear_errors(h), "vbh_clear_errors")


def vbh_set_wait_limit(h, polls: int):
    """Polls of the fusion kernel's bounded copy wait (default 2^24; 0 = give up at once)."""
    _check(lib().vbh_set_wait_limit(h, int(polls)), "vbh_set_wait_limit")


def vbh_timing_enable(h, stage_mask: int):
    """stage_mask: bit (1 << i) times stage VBH_STAGES[i]; 0 turns timing off."""
    _check(lib().vbh_timing_enable(h, int(stage_mask)), "vbh_timing_enable")


def vbh_timing_read(h, reset: bool = False):
    ms = np.zeros(len(VBH_STAGES), np.float64)
    n = np.zeros(len(VBH_STAGES), np.uint64)
    _check(lib().vbh_timing_read(h, ms.ctypes.data, n.ctypes.data, int(reset)), "vbh_timing_read")
    return dict(zip(VBH_STAGES, ms.tolist())), dict(zip(VBH_STAGES, n.tolist()))


def _check_static_mc_args(keys3, tsdf, weight, error_flags):
    """The kernels read 3 n int32 keys and 512 n floats from each of tsdf and weight, and write
    one uint32 error word: refuse anything else before the library call (dtypes and shapes
    first, then placement)."""
    import torch
    if keys3.dtype != torch.int32 or keys3.dim() != 2 or keys3.shape[1] != 3:
        raise ValueError(f"keys3 must be int32 [n, 3], got {keys3.dtype} {tuple(keys3.shape)}")
    n = int(keys3.shape[0])
    for name, t in (("tsdf", tsdf), ("weight", weight)):
        if t.dtype != torch.float32 or t.numel() != n * 512:
            raise ValueError(f"{name} must be float32 with n * 512 = {n * 512} elements, got "
                             f"{t.dtype} {tuple(t.shape)}")
    if error_flags is not None and (error_flags.dtype not in (torch.int32, torch.uint32)
                                    or error_flags.numel() < 1):
        raise ValueError("error_flags must be int32 or uint32 with at least one element")
    arrays = [keys3, tsdf, weight] + ([error_flags] if error_flags is not None else [])
    for t in arrays:
        if not (t.is_cuda and t.is_contiguous()):
            raise ValueError("keys3, tsdf, weight and error_flags must be contiguous CUDA tensors")
    if len({t.device for t in arrays}) != 1:
        raise ValueError("keys3, tsdf, weight and error_flags must be on one device")


def vbh_mc_from_tsdf_static(keys3, tsdf, weight, out: vbh_mc_stream, stream=None,
                            error_flags=None):
    """MC stream of caller-owned TSDF blocks using only the library's fixed scratch array (no
    device allocation inside the call; at most 32768 blocks)."""
    _check_static_mc_args(keys3, tsdf, weight, error_flags)
    _check(lib().vbh_mc_from_tsdf_static(_ptr(keys3), _ptr(tsdf), _ptr(weight),
                                         int(keys3.shape[0]), ctypes.byref(out), stream,
                                         _ptr(error_flags)), "vbh_mc_from_tsdf_static")


def vbh_diff_create(cfg: vbh_diff_config, stream=None) -> int:
    h = _p()
    _check(lib().vbh_diff_create(ctypes.byref(cfg), stream, ctypes.byref(h)), "vbh_diff_create")
    return h.value


def vbh_diff_destroy(h):
    _check(lib().vbh_diff_destroy(h), "vbh_diff_destroy")


def vbh_diff_poses(h, xi, T=None):
    _check(lib().vbh_diff_poses(h, _ptr(xi), _ptr(T)), "vbh_diff_poses")


def vbh_diff_masks(h, samples, depth, T0, masks):
    _check(lib().vbh_diff_masks(h, _ptr(samples), int(samples.shape[0]), _ptr(depth), _ptr(T0),
                                _ptr(masks)), "vbh_diff_masks")


def vbh_diff_forward(h, samples, depth, T0, xi, masks, F, loss=None):
    _check(lib().vbh_diff_forward(h, _ptr(samples), int(samples.shape[0]), _ptr(depth), _ptr(T0),
                                  _ptr(xi), _ptr(masks), _ptr(F), _ptr(loss)), "vbh_diff_forward")


def vbh_diff_backward(h, samples, depth, T0, xi, masks, F, gdepth, gxi):
    _check(lib().vbh_diff_backward(h, _ptr(samples), int(samples.shape[0]), _ptr(depth),
                                   _ptr(T0), _ptr(xi), _ptr(masks), _ptr(F), _ptr(gdepth),
                                   _ptr(gxi)), "vbh_diff_backward")


# ------------------------------------------------------------------------------- serving
def vbh_serve_create(h, cfg: vbh_serve_config) -> int:
    out = _p()
    _check(lib().vbh_serve_create(h, ctypes.byref(cfg), ctypes.byref(out)), "vbh_serve_create")
    return out.value


def vbh_serve_destroy(s):
    _check(lib().vbh_serve_destroy(s), "vbh_serve_destroy")


def vbh_serve_set_policy(s, cfg: vbh_serve_config):
    _check(lib().vbh_serve_set_policy(s, ctypes.byref(cfg)), "vbh_serve_set_policy")


def vbh_serve_set_versions(s, clients, versions):
    c = np.ascontiguousarray(clients, dtype=np.uint32)
    v = np.ascontiguousarray(versions, dtype=np.uint32)
    _check(lib().vbh_serve_set_versions(s, _ptr(c), _ptr(v), len(c)), "vbh_serve_set_versions")


def vbh_serve_get_versions(s, n_clients: int) -> np.ndarray:
    v = np.zeros(n_clients, np.uint32)
    _check(lib().vbh_serve_get_versions(s, _ptr(v)), "vbh_serve_get_versions")
    return v


def vbh_serve_versions_for_backlog(s, backlog) -> np.ndarray:
    b = np.ascontiguousarray(backlog, dtype=np.uint32)
    v = np.zeros(len(b), np.uint32)
    _check(lib().vbh_serve_versions_for_backlog(s, _ptr(b), len(b), _ptr(v)),
           "vbh_serve_versions_for_backlog")
    return v


def vbh_serve_submit(s, client: int, t_arrival_ns: int = 0) -> int:
    rid = _u32()
    _check(lib().vbh_serve_submit(s, client, t_arrival_ns, ctypes.byref(rid)), "vbh_serve_submit")
    return rid.value


def vbh_serve_step(s) -> int:
    n = _u32()
    _check(lib().vbh_serve_step(s, ctypes.byref(n)), "vbh_serve_step")
    return n.value


def vbh_serve_poll(s, cap: int = 256) -> list:
    buf = (vbh_serve_done * cap)()
    n = _u32()
    _check(lib().vbh_serve_poll(s, buf, cap, ctypes.byref(n)), "vbh_serve_poll")
    return [buf[i] for i in range(n.value)]


def vbh_serve_result(s, rid: int) -> vbh_serve_view:
    v = vbh_serve_view()
    _check(lib().vbh_serve_result(s, rid, ctypes.byref(v)), "vbh_serve_result")
    return v


def vbh_serve_release(s, rid: int):
    _check(lib().vbh_serve_release(s, rid), "vbh_serve_release")


def vbh_serve_drain(s):
    _check(lib().vbh_serve_drain(s), "vbh_serve_drain")


def vbh_serve_stats_read(s) -> vbh_serve_stats:
    st = vbh_serve_stats()
    _check(lib().vbh_serve_stats_read(s, ctypes.byref(st)), "vbh_serve_stats_read")
    return st


def vbh_serve_run(s, script: vbh_serve_script, cap: int) -> list:
    buf = (vbh_serve_done * max(cap, 1))()
    n = _u32()
    _check(lib().vbh_serve_run(s, ctypes.byref(script), buf, cap, ctypes.byref(n)),
           "vbh_serve_run")
    return [buf[i] for i in range(n.value)]


def vbh_serve_now_ns() -> int:
    return int(lib().vbh_serve_now_ns())


def vbh_serve_loop_start(s, cfg: vbh_serve_loop_config) -> int:
    out = _p()
    _check(lib().vbh_serve_loop_start(s, ctypes.byref(cfg), ctypes.byref(out)),
           "vbh_serve_loop_start")
    return out.value


def vbh_serve_loop_submit(L, client: int, t_arrival_ns: int = 0) -> int:
    rid = _u32()
    _check(lib().vbh_serve_loop_submit(L, client, t_arrival_ns, ctypes.byref(rid)),
           "vbh_serve_loop_submit")
    return rid.value


def vbh_serve_loop_poll(L, cap: int = 256) -> list:
    buf = (vbh_serve_done * cap)()
    n = _u32()
    _check(lib().vbh_serve_loop_poll(L, buf, cap, ctypes.byref(n)), "vbh_serve_loop_poll")
    return [buf[i] for i in range(n.value)]


def vbh_serve_loop_result(L, rid: int) -> vbh_serve_view:
    v = vbh_serve_view()
    _check(lib().vbh_serve_loop_result(L, rid, ctypes.byref(v)), "vbh_serve_loop_result")
    return v


def vbh_serve_loop_release(L, rid: int):
    _check(lib().vbh_serve_loop_release(L, rid), "vbh_serve_loop_release")


def vbh_serve_loop_drain(L, timeout_ns: int):
    _check(lib().vbh_serve_loop_drain(L, int(timeout_ns)), "vbh_serve_loop_drain")


def vbh_serve_loop_run(L, script: vbh_serve_script, cap: int) -> list:
    buf = (vbh_serve_done * max(cap, 1))()
    n = _u32()
    _check(lib().vbh_serve_loop_run(L, ctypes.byref(script), buf, cap, ctypes.byref(n)),
           "vbh_serve_loop_run")
    return [buf[i] for i in range(n.value)]


def vbh_serve_loop_stats_read(L) -> vbh_serve_loop_stats:
    st = vbh_serve_loop_stats()
    _check(lib().vbh_serve_loop_stats_read(L, ctypes.byref(st)), "vbh_serve_loop_stats_read")
    return st


def vbh_serve_loop_stop(L):
    _check(lib().vbh_serve_loop_stop(L), "vbh_serve_loop_stop")


# ---------------------------------------------------------------------------- stream-out / in
def vbh_stream_out_enable(h, ring_blocks: int = 0):
    _check(lib().vbh_stream_out_enable(h, ring_blocks), "vbh_stream_out_enable")


def vbh_stream_out_poll(h) -> int:
    n = _u64()
    _check(lib().vbh_stream_out_poll(h, ctypes.byref(n)), "vbh_stream_out_poll")
    return n.value


def vbh_stream_out_flush(h):
    _check(lib().vbh_stream_out_flush(h), "vbh_stream_out_flush")


def vbh_stream_out_stats(h):
    s, l, m = _u64(), _u64(), _u32()
    _check(lib().vbh_stream_out_stats(h, ctypes.byref(s), ctypes.byref(l), ctypes.byref(m)),
           "vbh_stream_out_stats")
    return s.value, l.value, m.value


def vbh_host_map_dump(h, keys3, tsdf, weight, cap: int) -> int:
    n = _u32()
    _check(lib().vbh_host_map_dump(h, _ptr(keys3), _ptr(tsdf), _ptr(weight), cap,
                                   ctypes.byref(n)), "vbh_host_map_dump")
    return n.value


def vbh_stream_in(h, keys3) -> int:
    k = np.ascontiguousarray(keys3, dtype=np.int32).reshape(-1, 3)
    n = _u32()
    _check(lib().vbh_stream_in(h, _ptr(k), k.shape[0], ctypes.byref(n)), "vbh_stream_in")
    return n.value


def vbh_set_integration_mode(h, mode: int):
    _check(lib().vbh_set_integration_mode(h, mode), "vbh_set_integration_mode")


# ------------------------------------------------------------------ per-client stream sets
def vbh_sets_create(server, n_clients: int, cap_log2: int) -> int:
    out = _p()
    _check(lib().vbh_sets_create(server, n_clients, cap_log2, ctypes.byref(out)),
           "vbh_sets_create")
    return out.value


def vbh_sets_destroy(q):
    _check(lib().vbh_sets_destroy(q), "vbh_sets_destroy")


def vbh_sets_insert_last(q):
    _check(lib().vbh_sets_insert_last(q), "vbh_sets_insert_last")


def vbh_sets_fill(q, client: int):
    _check(lib().vbh_sets_fill(q, client), "vbh_sets_fill")


def vbh_sets_fetch(q, clients, limits, recs, indices, n_out):
    c = np.ascontiguousarray(clients, np.uint32)
    l = np.ascontiguousarray(limits, np.uint32)
    _check(lib().vbh_sets_fetch(q, _ptr(c), _ptr(l), len(c), _ptr(recs), _ptr(indices),
                                _ptr(n_out)), "vbh_sets_fetch")


def vbh_sets_counts(q, n_clients: int):
    a = np.zeros(n_clients, np.uint32)
    b = np.zeros(n_clients, np.uint32)
    e = np.zeros(1, np.uint32)
    _check(lib().vbh_sets_counts(q, _ptr(a), _ptr(b), _ptr(e)), "vbh_sets_counts")
    return a, b, int(e[0])


def vbh_sets_rebuild(q, client: int):
    _check(lib().vbh_sets_rebuild(q, client), "vbh_sets_rebuild")


# ------------------------------------------------------------------------- triangulation
def vbh_mc_tri_table():
    n = np.zeros(256, np.uint8)
    e = np.zeros((256, 15), np.uint8)
    _check(lib().vbh_mc_tri_table(_ptr(n), _ptr(e)), "vbh_mc_tri_table")
    return n, e


def vbh_mc_triangulate(stream: "vbh_mc_stream", voxel_size: float, tris, cap: int, n_tris,
                       cuda_stream=None):
    _check(lib().vbh_mc_triangulate(ctypes.byref(stream), voxel_size, _ptr(tris), cap,
                                    _ptr(n_tris), cuda_stream), "vbh_mc_triangulate")
