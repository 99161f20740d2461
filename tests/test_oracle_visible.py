"""Pins of the oracle's visibility test (R7), visible-set integration (R8, free-space carving)
and frustum erase (R9, the scene reset of Sec. 4.1).

R7 is conservative by construction: every block that has a voxel projecting into the image
(brute force over its 512 voxels in FP64) must be in view, and a block whose bounding sphere is
far outside the frustum must not.  R8 is pinned by the closed form of a wall that moves back:
voxels of the old surface now see free space, f = 1, and their running average becomes
(n f_old + m) / (n + m); with the touched-set integration they keep f_old."""
import numpy as np
import pytest

import oracle


def vol(W=40, H=30, f=30.0, s=0.01, mu=0.04, zmax=0.0):
    return oracle.OracleVolume(s, mu, 64.0, 0.001, zmax, W, H, f, f, W / 2.0, H / 2.0)


def rand_pose(rng):
    a = rng.normal(size=3)
    a *= rng.uniform(0, np.pi) / np.linalg.norm(a)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    th = np.linalg.norm(a)
    R = np.eye(3) + np.sin(th) / th * K + (1 - np.cos(th)) / th ** 2 * K @ K
    t = rng.uniform(-0.3, 0.3, 3)
    return np.concatenate([R, t[:, None]], 1).astype(np.float32)


def voxel_in_image(k, T, W, H, f, s):
    R = T[:, :3].astype(np.float64)
    t = T[:, 3].astype(np.float64)
    g = np.stack(np.meshgrid(*[np.arange(8)] * 3, indexing="ij"), -1).reshape(-1, 3) + 8 * np.asarray(k)
    p = (g * np.float64(np.float32(s)) - t) @ R
    ok = p[:, 2] > 1e-9
    u = f * p[ok, 0] / p[ok, 2] + W / 2.0 + 0.5
    v = f * p[ok, 1] / p[ok, 2] + H / 2.0 + 0.5
    return bool(np.any((u >= 0) & (u < W) & (v >= 0) & (v < H)))


def test_in_view_keeps_every_block_with_a_voxel_in_the_image():
    rng = np.random.default_rng(0)
    o = vol()
    n_in = n_cases = 0
    for _ in range(20):
        T = rand_pose(rng)
        keys = rng.integers(-12, 12, (300, 3)).astype(np.int32)
        flags = o.in_view(keys, T)
        for k, fl in zip(keys, flags):
            if voxel_in_image(k, T, 40, 30, 30.0, 0.01):
                n_in += 1
                assert fl, (k, T)
            n_cases += 1
    assert n_in > 200


def test_in_view_rejects_blocks_far_outside_and_behind():
    o = vol()
    T = np.concatenate([np.eye(3), np.zeros((3, 1))], 1).astype(np.float32)   # looks along +z
    # one metre ahead, on the axis: in view; the same block 2 m to the side: out
    assert o.in_view([[0, 0, 12]], T).all()
    assert not o.in_view([[25, 0, 12]], T).any()       # x = 2 m at z = 1 m, fov 67 deg
    assert not o.in_view([[0, 0, -12]], T).any()       # behind the camera
    assert not o.in_view([[0, 0, 30]], T, zfar=1.0).any()   # beyond the far limit
    assert o.in_view([[0, 0, 30]], T).all()


def wall(Z, W=16, H=16):
    return np.full((H, W), int(round(Z * 1000)), np.uint16)


@pytest.mark.parametrize("visible", [False, True])
def test_moving_wall_carving_closed_form(visible):
    W = H = 16
    f, s, mu = 16.0, 0.01, 0.04
    o = vol(W, H, f, s, mu)
    T = np.concatenate([np.eye(3), np.zeros((3, 1))], 1).astype(np.float32)
    n, m = 3, 2
    for _ in range(n):
        o.integrate(wall(1.0), T, visible=visible)
    for _ in range(m):
        o.integrate(wall(1.3), T, visible=visible)
    k, F, Wt = o.dump()
    keys = {tuple(x): i for i, x in enumerate(k.tolist())}
    # voxel (0, 0, 99): z = 0.99 m, projects to the image centre
    b = keys[(0, 0, 12)]
    li = 0 + 8 * 0 + 64 * (99 - 96)
    ds = np.float32(0.001)
    d1 = np.float64(np.float32(np.float32(1000) * ds))
    z = 99 * np.float64(np.float32(s))
    f1 = np.clip((d1 - z) / np.float64(np.float32(mu)), -1, 1)
    if visible:
        assert Wt[b, li] == n + m
        assert F[b, li] == pytest.approx((n * f1 + m * 1.0) / (n + m), abs=1e-12)
    else:
        assert Wt[b, li] == n
        assert F[b, li] == pytest.approx(f1, abs=1e-12)


def test_frustum_erase_removes_exactly_the_blocks_in_view():
    rng = np.random.default_rng(3)
    o = vol()
    keys = rng.integers(-10, 10, (400, 3)).astype(np.int32)
    keys = np.unique(keys, axis=0)
    o.load(keys, np.zeros((len(keys), 512)), np.ones((len(keys), 512)))
    T = rand_pose(rng)
    before = o.in_view(keys, T, zfar=1.5)
    gone = o.erase_frustum(T, zfar=1.5)
    assert len(gone) == int(before.sum()) > 0
    live = o.dump()[0]
    assert not o.in_view(live, T, zfar=1.5).any()
    assert len(live) + len(gone) == len(keys)
    assert {tuple(x) for x in o.host_dump()[0].tolist()} == {tuple(x) for x in gone.tolist()}
