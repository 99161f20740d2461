"""CPU oracle of the voxel-block-hashing hot path -- TEST INFRASTRUCTURE ONLY.

Only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline leg of `bench.py` may import this
package.  The product library never routes through it.  It wraps `vbh_oracle.cpp` (plain C++,
FP64 values, std::unordered_map store) through ctypes and shares no code with the CUDA path.

Parity status of each function (what pins it; see the tests named in brackets):
  map_batch          pinned: brute-force set/dict model on random sequences [test_oracle_hash]
  alloc_keys         pinned: exact FP64 ray/band traversal bounds on tiny frames [test_oracle_alloc]
  vol_integrate      pinned: closed-form plane and sphere SDFs, running-average closed forms
                     [test_oracle_tsdf]
  vol_erase_radius   pinned: FP64 distance away from the boundary [test_oracle_erase]
  mc_dense / mc_set  pinned: analytic sphere classification, complement symmetry, S^c, and
                     incremental == full re-extraction [test_oracle_mc]
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vbh_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")

OP_FIND, OP_INSERT, OP_ERASE = 0, 1, 2
ST_FOUND, ST_NOT_FOUND, ST_INSERTED, ST_EXISTS, ST_ERASED, ST_CAPACITY, ST_INVALID = 1, 2, 3, 4, 5, 6, 7
NONE = 0xFFFFFFFF


def build(force: bool = False) -> str:
    """Compile the oracle with the flags its canonical binary32 arithmetic needs."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call([
            "g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
            "-fno-fast-math", "-fexcess-precision=standard", _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        P, U32, I32, F = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_int, ctypes.c_float
        L.orc_map_create.restype = P
        L.orc_map_destroy.argtypes = [P]
        L.orc_map_size.argtypes = [P]
        L.orc_map_size.restype = U32
        L.orc_map_batch.argtypes = [P, U32, P, P, P, P, P]
        L.orc_map_dump.argtypes = [P, P, P, U32]
        L.orc_map_dump.restype = U32
        L.orc_vol_create.argtypes = [P, I32, I32]
        L.orc_vol_create.restype = P
        L.orc_vol_destroy.argtypes = [P]
        L.orc_vol_size.argtypes = [P]
        L.orc_vol_size.restype = U32
        L.orc_alloc_keys.argtypes = [P, P, P, P, U32]
        L.orc_alloc_keys.restype = U32
        L.orc_vol_integrate.argtypes = [P, P, P]
        L.orc_vol_integrate.restype = U32
        L.orc_vol_integrate_mode.argtypes = [P, P, P, ctypes.c_int]
        L.orc_vol_integrate_mode.restype = U32
        L.orc_in_view.argtypes = [P, P, U32, P, ctypes.c_float, P]
        L.orc_vol_erase_frustum.argtypes = [P, P, ctypes.c_float, P, U32]
        L.orc_vol_erase_frustum.restype = U32
        L.orc_vol_touched.argtypes = [P, P, U32]
        L.orc_vol_touched.restype = U32
        L.orc_vol_erase_radius.argtypes = [P, P, F, P, U32]
        L.orc_vol_erase_radius.restype = U32
        L.orc_vol_erase_keys.argtypes = [P, P, U32]
        L.orc_vol_erase_keys.restype = U32
        L.orc_vol_dump.argtypes = [P, P, P, P, U32]
        L.orc_vol_dump.restype = U32
        L.orc_vol_load.argtypes = [P, P, P, P, U32]
        L.orc_tri_case.argtypes = [ctypes.c_int, P, U32]
        L.orc_tri_case.restype = U32
        L.orc_vol_triangles.argtypes = [P, P, U32, P, U32]
        L.orc_vol_triangles.restype = U32
        L.orc_vol_host_dump.argtypes = [P, P, P, P, U32]
        L.orc_vol_host_dump.restype = U32
        L.orc_vol_stream_in.argtypes = [P, P, U32]
        L.orc_vol_stream_in.restype = U32
        L.orc_vol_mc_set.argtypes = [P, I32, P, U32, P, U32, P]
        L.orc_vol_mc_set.restype = U32
        L.orc_vol_mc_dense.argtypes = [P, P, U32, P, P]
        L.orc_set_threads.argtypes = [I32]
        L.orc_get_threads.restype = I32
        _lib = L
    return _lib


def set_threads(n: int) -> None:
    """Timing mode of every oracle call: 1 = the single-threaded reference (default); n > 1 runs
    the allocation's image rows and the fusion's and MC classification's blocks on n OpenMP
    threads.  Results are identical in every mode (blocks are independent; the allocation is a
    set union); hash operations always run serially."""
    lib().orc_set_threads(int(n))


def get_threads() -> int:
    return lib().orc_get_threads()


def _p(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


class OracleMap:
    """Sec. 5 map of unique int3 keys to uint32 values, with the phased batch reading."""

    def __init__(self):
        self._h = lib().orc_map_create()

    def __del__(self):
        if getattr(self, "_h", None):
            lib().orc_map_destroy(self._h)
            self._h = None

    def __len__(self):
        return lib().orc_map_size(self._h)

    def batch(self, ops, keys3, vals=None):
        ops = np.ascontiguousarray(ops, np.uint8)
        keys3 = np.ascontiguousarray(keys3, np.int32).reshape(-1, 3)
        n = ops.shape[0]
        vals = None if vals is None else np.ascontiguousarray(vals, np.uint32)
        res = np.zeros(n, np.uint32)
        st = np.zeros(n, np.uint8)
        lib().orc_map_batch(self._h, n, _p(ops), _p(keys3), _p(vals), _p(res), _p(st))
        return res, st

    def dump(self):
        n = len(self)
        k = np.zeros((n, 3), np.int32)
        v = np.zeros(n, np.uint32)
        lib().orc_map_dump(self._h, _p(k), _p(v), n)
        return k, v


class OracleVolume:
    """Voxel-block volume with FP64 TSDF values (allocation, fusion, erase, MC indices)."""

    def __init__(self, voxel_size, trunc, max_weight, depth_scale, zmax, width, height,
                 fx, fy, cx, cy):
        self.params = np.array([voxel_size, trunc, max_weight, depth_scale, zmax, fx, fy, cx, cy],
                               np.float32)
        self.width, self.height = int(width), int(height)
        self._h = lib().orc_vol_create(_p(self.params), self.width, self.height)

    def __del__(self):
        if getattr(self, "_h", None):
            lib().orc_vol_destroy(self._h)
            self._h = None

    def __len__(self):
        return lib().orc_vol_size(self._h)

    def _frame(self, depth, T):
        depth = np.ascontiguousarray(depth, np.uint16)
        assert depth.shape == (self.height, self.width)
        T = np.ascontiguousarray(T, np.float32).reshape(12)
        return depth, T

    def alloc_keys(self, depth, T):
        depth, T = self._frame(depth, T)
        n = lib().orc_alloc_keys(self._h, _p(depth), _p(T), None, 0)
        out = np.zeros((n, 3), np.int32)
        lib().orc_alloc_keys(self._h, _p(depth), _p(T), _p(out), n)
        return out

    def integrate(self, depth, T, visible: bool = False) -> int:
        """R4/R5 fusion of the touched set; with `visible`, R8 (touched + every block in view)."""
        depth, T = self._frame(depth, T)
        return lib().orc_vol_integrate_mode(self._h, _p(depth), _p(T), 1 if visible else 0)

    def in_view(self, keys3, T, zfar: float = 0.0):
        """R7 flags of the given block keys for pose T (3x4)."""
        k = np.ascontiguousarray(keys3, np.int32).reshape(-1, 3)
        T = np.ascontiguousarray(T, np.float32).reshape(12)
        out = np.zeros(k.shape[0], np.uint8)
        lib().orc_in_view(self._h, _p(k), k.shape[0], _p(T), float(zfar), _p(out))
        return out.astype(bool)

    def erase_frustum(self, T, zfar: float = 0.0):
        """R9: erase every live block in view of T; returns the erased keys (sorted)."""
        T = np.ascontiguousarray(T, np.float32).reshape(12)
        cap = len(self)
        out = np.zeros((max(cap, 1), 3), np.int32)
        n = lib().orc_vol_erase_frustum(self._h, _p(T), float(zfar), _p(out), cap)
        return out[:n]

    def touched(self):
        n = lib().orc_vol_touched(self._h, None, 0)
        out = np.zeros((n, 3), np.int32)
        lib().orc_vol_touched(self._h, _p(out), n)
        return out

    def erase_radius(self, centre, R):
        c = np.ascontiguousarray(centre, np.float32).reshape(3)
        cap = len(self)
        out = np.zeros((cap, 3), np.int32)
        n = lib().orc_vol_erase_radius(self._h, _p(c), float(R), _p(out), cap)
        return out[:n]

    def erase_keys(self, keys3) -> int:
        k = np.ascontiguousarray(keys3, np.int32).reshape(-1, 3)
        return lib().orc_vol_erase_keys(self._h, _p(k), k.shape[0])

    def dump(self):
        n = len(self)
        k = np.zeros((n, 3), np.int32)
        F = np.zeros((n, 512), np.float64)
        W = np.zeros((n, 512), np.float64)
        lib().orc_vol_dump(self._h, _p(k), _p(F), _p(W), n)
        return k, F, W

    def triangles(self, keys3):
        """R10: triangles (m, 3, 3) in metres of the cubes at the voxels of the given blocks."""
        k = np.ascontiguousarray(keys3, np.int32).reshape(-1, 3)
        m = lib().orc_vol_triangles(self._h, _p(k), k.shape[0], None, 0)
        out = np.zeros((max(m, 1), 9), np.float64)
        lib().orc_vol_triangles(self._h, _p(k), k.shape[0], _p(out), m)
        return out[:m].reshape(-1, 3, 3)

    def host_dump(self):
        """The passive host map of streamed-out (erased) blocks: keys sorted, F, W."""
        n = lib().orc_vol_host_dump(self._h, None, None, None, 0)
        k = np.zeros((n, 3), np.int32)
        F = np.zeros((n, 512), np.float64)
        W = np.zeros((n, 512), np.float64)
        lib().orc_vol_host_dump(self._h, _p(k), _p(F), _p(W), n)
        return k, F, W

    def stream_in(self, keys3) -> int:
        k = np.ascontiguousarray(keys3, np.int32).reshape(-1, 3)
        return lib().orc_vol_stream_in(self._h, _p(k), k.shape[0])

    def load(self, keys3, F, W):
        k = np.ascontiguousarray(keys3, np.int32).reshape(-1, 3)
        F = np.ascontiguousarray(F, np.float64).reshape(-1, 512)
        W = np.ascontiguousarray(W, np.float64).reshape(-1, 512)
        lib().orc_vol_load(self._h, _p(k), _p(F), _p(W), k.shape[0])

    def mc_set(self, mode: int):
        """mode 0: touched blocks + seven negative neighbours (+ removals); 1: all blocks."""
        cap = len(self) + 1
        k = np.zeros((cap, 3), np.int32)
        rcap = 1 << 20
        rem = np.zeros((rcap, 3), np.int32)
        nr = np.zeros(1, np.uint32)
        n = lib().orc_vol_mc_set(self._h, mode, _p(k), cap, _p(rem), rcap, _p(nr))
        return k[:n], rem[:int(nr[0])]

    def mc_dense(self, keys3):
        k = np.ascontiguousarray(keys3, np.int32).reshape(-1, 3)
        n = k.shape[0]
        idx = np.zeros((n, 512), np.uint8)
        margin = np.zeros((n, 512), np.float32)
        lib().orc_vol_mc_dense(self._h, _p(k), n, _p(idx), _p(margin))
        return idx, margin


# ------------------------------------------------------------------ differentiable window fusion
def _diff_lib():
    L = lib()
    if not getattr(L, "_diff_bound", False):
        P, U32, I32 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_int
        L.orc_se3_exp.argtypes = [P, P, P, P, P]
        L.orc_diff_masks.argtypes = [P, I32, I32, I32, P, U32, P, P, P]
        L.orc_diff_forward.argtypes = [P, I32, I32, I32, P, U32, P, P, P, P, P]
        L.orc_diff_forward.restype = ctypes.c_double
        L.orc_diff_backward.argtypes = [P, I32, I32, I32, P, U32, P, P, P, P, P, P]
        L._diff_bound = True
    return L


def se3_exp(xi):
    """Exponential map of an se(3) vector (rho, omega): R (3x3), t (3,), dR (6,3,3), dt (6,3)."""
    xi = np.ascontiguousarray(xi, np.float64).reshape(6)
    R = np.zeros(9)
    t = np.zeros(3)
    dR = np.zeros(54)
    dt = np.zeros(18)
    _diff_lib().orc_se3_exp(_p(xi), _p(R), _p(t), _p(dR), _p(dt))
    return R.reshape(3, 3), t, dR.reshape(6, 3, 3), dt.reshape(6, 3)


def nominal_pose_f32(xi):
    """float32 3x4 [R | t] of exp(xi), the nominal pose at which cells and masks are fixed."""
    R, t, _, _ = se3_exp(xi)
    T = np.zeros((3, 4))
    T[:, :3] = R
    T[:, 3] = t
    return T.astype(np.float32)


class OracleDiffFusion:
    """FP64 window fusion of float32 depth at fixed sample voxels, with its analytic gradient."""

    def __init__(self, voxel_size, trunc, width, height, fx, fy, cx, cy, samples, depth, T0):
        self.params = np.array([voxel_size, trunc, fx, fy, cx, cy], np.float32)
        self.W, self.H = int(width), int(height)
        self.samples = np.ascontiguousarray(samples, np.int32).reshape(-1, 3)
        self.depth = np.ascontiguousarray(depth, np.float32)
        self.nf = self.depth.shape[0]
        assert self.depth.shape == (self.nf, self.H, self.W)
        self.T0 = np.ascontiguousarray(T0, np.float32).reshape(self.nf, 12)
        self.words = (self.nf + 31) // 32
        self.masks = np.zeros((len(self.samples), self.words), np.uint32)
        _diff_lib().orc_diff_masks(_p(self.params), self.W, self.H, self.nf, _p(self.samples),
                                   len(self.samples), _p(self.depth), _p(self.T0), _p(self.masks))

    def forward(self, xi, depth=None):
        xi = np.ascontiguousarray(xi, np.float64).reshape(self.nf, 6)
        d = self.depth if depth is None else np.ascontiguousarray(depth, np.float32)
        F = np.zeros(len(self.samples))
        L = _diff_lib().orc_diff_forward(_p(self.params), self.W, self.H, self.nf,
                                         _p(self.samples), len(self.samples), _p(d), _p(self.T0),
                                         _p(xi), _p(self.masks), _p(F))
        return L, F

    def backward(self, xi):
        xi = np.ascontiguousarray(xi, np.float64).reshape(self.nf, 6)
        gd = np.zeros((self.nf, self.H, self.W))
        gx = np.zeros((self.nf, 6))
        _diff_lib().orc_diff_backward(_p(self.params), self.W, self.H, self.nf, _p(self.samples),
                                      len(self.samples), _p(self.depth), _p(self.T0), _p(xi),
                                      _p(self.masks), _p(gd), _p(gx))
        return gd, gx


def tri_case(c: int) -> np.ndarray:
    """R10: the triangles of cube index c as (t, 3) edge indices."""
    out = np.zeros((16, 3), np.int32)
    n = lib().orc_tri_case(int(c), _p(out), 16)
    assert n <= 16
    return out[:n]
