"""Pins of the oracle's block allocation (voxel block hashing, Sec. 4.1) on tiny frames by brute
force in FP64: every allocated block must meet the exact band segment [d - mu, d + mu] of some
valid pixel ray, and every block that contains an exact band sample point with a clear margin
from the block faces must be allocated."""
import numpy as np
import pytest

from oracle import OracleVolume

from test_oracle_tsdf import pose

W_IMG, H_IMG, FX, FY, CX, CY = 4, 4, 3.0, 3.0, 2.0, 2.0


def segment_hits_box(o, d, t0, t1, lo, hi):
    """Does the segment o + t d, t in [t0, t1], meet the closed box [lo, hi]? (slab test, FP64)"""
    tmin, tmax = t0, t1
    for a in range(3):
        if abs(d[a]) < 1e-300:
            if o[a] < lo[a] or o[a] > hi[a]:
                return False
            continue
        ta, tb = (lo[a] - o[a]) / d[a], (hi[a] - o[a]) / d[a]
        tmin, tmax = max(tmin, min(ta, tb)), min(tmax, max(ta, tb))
    return tmin <= tmax


@pytest.mark.parametrize("seed,voxel,mu", [(1, 0.01, 0.04), (2, 0.005, 0.02), (3, 0.02, 0.05),
                                           (4, 0.01, 0.015)])
def test_alloc_tiny_frames_brute_force(seed, voxel, mu):
    rng = np.random.default_rng(seed)
    T = pose(seed, t=tuple(rng.uniform(-0.5, 0.5, 3)))
    depth = rng.integers(300, 3000, size=(H_IMG, W_IMG)).astype(np.uint16)
    depth[rng.uniform(size=depth.shape) < 0.2] = 0
    o = OracleVolume(voxel, mu, 64.0, 0.001, 0.0, W_IMG, H_IMG, FX, FY, CX, CY)
    keys = {tuple(k) for k in o.alloc_keys(depth, T).tolist()}
    assert keys
    R = T[:, :3].astype(np.float64)
    t = T[:, 3].astype(np.float64)
    s = float(np.float32(voxel))
    m = float(np.float32(mu))
    bs = 8 * s
    eps = 1e-5
    J = int(np.ceil(2 * m / s - 1e-6))
    must = set()
    rays = []
    for v in range(H_IMG):
        for u in range(W_IMG):
            if depth[v, u] == 0:
                continue
            d = float(np.float32(depth[v, u]) * np.float32(0.001))
            dirc = R @ np.array([(u - CX) / FX, (v - CY) / FY, 1.0])
            rays.append((dirc, d))
            for j in range(J + 1):
                z = d - m + j * s
                X = R @ np.array([(u - CX) / FX * z, (v - CY) / FY * z, z]) + t
                q = X / bs
                if np.all(np.abs(q - np.round(q)) > eps / bs):
                    must.add(tuple(np.floor(q).astype(int).tolist()))
    missing = must - keys
    assert not missing, f"blocks holding a band sample are missing: {sorted(missing)[:5]}"
    for k in keys:
        lo = np.array(k, np.float64) * bs - eps
        hi = lo + bs + 2 * eps
        assert any(segment_hits_box(t, dirc, d - m - eps, d + m + eps, lo, hi) for dirc, d in rays), k


def test_alloc_sample_count():
    """J + 1 samples spaced s apart span exactly [d - mu, d + mu] when 2 mu / s is an integer:
    a ray along a world axis through a block grid then touches exactly the blocks that the
    interval [d - mu, d + mu] overlaps (one pixel, camera looking down +x)."""
    T = np.array([[0, 0, 1, 0.0001], [1, 0, 0, 0.0001], [0, 1, 0, 0.0001]], np.float32)
    o = OracleVolume(0.01, 0.04, 64.0, 0.001, 0.0, 1, 1, 1.0, 1.0, 0.0, 0.0)
    for raw in (1000, 1037, 1100, 1150):
        d = float(np.float32(raw) * np.float32(0.001))
        keys = o.alloc_keys(np.array([[raw]], np.uint16), T)
        lo, hi = d - 0.04, d + 0.04
        expect = set(range(int(np.floor((lo + 0.0001) / 0.08)), int(np.floor((hi + 0.0001) / 0.08)) + 1))
        assert {k[0] for k in keys.tolist()} == expect
        assert {(k[1], k[2]) for k in keys.tolist()} == {(0, 0)}
