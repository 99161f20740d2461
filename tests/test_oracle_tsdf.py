"""Pins of the oracle's projective TSDF fusion against closed forms that do not go through its
code: a plane perpendicular to the optical axis (constant depth, so the value is independent of
which pixel a voxel lands on), the projective SDF read at the FP64-projected pixel of an
arbitrary depth image (sphere), and the closed forms of the capped running average."""
import numpy as np
import pytest

from oracle import OracleVolume

S, MU, WMAX, DS = 0.01, 0.04, 64.0, np.float32(0.001)
W_IMG, H_IMG, FX, FY, CX, CY = 32, 24, 30.0, 30.0, 16.0, 12.0


def rot(seed):
    q = np.random.default_rng(seed).standard_normal(4)
    q /= np.linalg.norm(q)
    a, b, c, d = q
    return np.array([[a*a+b*b-c*c-d*d, 2*(b*c-a*d), 2*(b*d+a*c)],
                     [2*(b*c+a*d), a*a-b*b+c*c-d*d, 2*(c*d-a*b)],
                     [2*(b*d-a*c), 2*(c*d+a*b), a*a-b*b-c*c+d*d]])


def pose(seed, t=(0.3, -0.2, 0.5)):
    T = np.zeros((3, 4))
    T[:, :3] = rot(seed)
    T[:, 3] = t
    return T.astype(np.float32)


def vol(zmax=0.0, w=W_IMG, h=H_IMG):
    return OracleVolume(S, MU, WMAX, float(DS), zmax, w, h, FX, FY, CX, CY)


def voxel_geometry(keys, T):
    """FP64 camera coordinates and pixel coordinates of every voxel of the given blocks."""
    l = np.arange(512)
    loc = np.stack([l % 8, (l // 8) % 8, l // 64], -1)
    g = keys[:, None, :].astype(np.float64) * 8 + loc[None]
    X = g * np.float64(np.float32(S))
    R = T[:, :3].astype(np.float64)
    t = T[:, 3].astype(np.float64)
    p = (X - t) @ R                    # R^T (X - t), row-vector form
    u = FX * p[..., 0] / p[..., 2] + CX
    v = FY * p[..., 1] / p[..., 2] + CY
    return p, u, v


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_plane_closed_form(seed):
    T = pose(seed)
    Z0 = 1200 + 37 * seed                      # mm, the plane z_cam = Z0
    depth = np.full((H_IMG, W_IMG), Z0, np.uint16)
    o = vol()
    n_frames = 3
    for _ in range(n_frames):
        o.integrate(depth, T)
    keys, F, W = o.dump()
    assert keys.shape[0] > 0
    p, u, v = voxel_geometry(keys, T)
    d32 = float(np.float32(Z0) * DS)
    sdf = d32 - p[..., 2]
    inside = (u > 0.01) & (u < W_IMG - 1 - 0.01) & (v > 0.01) & (v < H_IMG - 1 - 0.01) & (p[..., 2] > 0)
    band = sdf >= -MU + 1e-6
    behind = sdf < -MU - 1e-6
    upd = inside & band
    assert upd.sum() > 1000
    np.testing.assert_array_equal(W[upd], n_frames)
    np.testing.assert_allclose(F[upd], np.clip(sdf[upd] / np.float64(np.float32(MU)), -1, 1), atol=1e-9)
    assert np.all(W[inside & behind] == 0)
    # voxels projecting outside the image are never updated
    outside = (u < -0.6) | (u > W_IMG - 0.4) | (v < -0.6) | (v > H_IMG - 0.4) | (p[..., 2] <= 0)
    assert np.all(W[outside] == 0)


def test_projective_sdf_reads_projected_pixel():
    """Arbitrary (sphere) depth image: F = clamp((depth[v, u] * ds - p_z) / mu) with (u, v) the
    FP64-rounded projection, at voxels whose projection is well inside a pixel."""
    from paper_1805_03709_b300 import synth
    cam = synth.Camera(W_IMG, H_IMG, FX, FY, CX, CY)
    T = synth.look_at((0.0, -1.2, 0.3), (0.05, 0.0, 0.0))
    scene = synth.Scene(spheres=np.array([[0.0, 0.0, 0.0, 0.35]]), boxes=np.zeros((0, 6)))
    depth = synth.quantize_mm(synth.render_depth_m(scene, cam, T))
    assert (depth > 0).sum() > 50
    o = vol()
    o.integrate(depth, T)
    keys, F, W = o.dump()
    p, u, v = voxel_geometry(keys, T)
    ur, vr = np.rint(u), np.rint(v)
    crisp = (np.abs(u - ur) < 0.49) & (np.abs(v - vr) < 0.49) & (p[..., 2] > 0)
    crisp &= (ur >= 0) & (ur < W_IMG) & (vr >= 0) & (vr < H_IMG)
    ui, vi = ur.astype(np.int64).clip(0, W_IMG - 1), vr.astype(np.int64).clip(0, H_IMG - 1)
    raw = depth[vi, ui]
    d32 = raw.astype(np.float32) * DS
    sdf = d32.astype(np.float64) - p[..., 2]
    upd = crisp & (raw > 0) & (sdf >= -MU + 1e-6)
    assert upd.sum() > 500
    np.testing.assert_array_equal(W[upd], 1)
    np.testing.assert_allclose(F[upd], np.clip(sdf[upd] / np.float64(np.float32(MU)), -1, 1), atol=1e-9)
    skip = crisp & ((raw == 0) | (sdf < -MU - 1e-6))
    assert skip.sum() > 100 and np.all(W[skip] == 0)


def test_running_average_mean_below_cap():
    T = pose(7)
    Zs = [1100, 1112, 1090, 1125, 1101, 1118, 1095]
    o = vol()
    every = None
    for Z in Zs:
        o.integrate(np.full((H_IMG, W_IMG), Z, np.uint16), T)
        tk = {tuple(k) for k in o.touched().tolist()}
        every = tk if every is None else every & tk
    keys, F, W = o.dump()
    p, u, v = voxel_geometry(keys, T)
    # R4: a frame updates only the blocks its own allocation touched
    in_every = np.array([tuple(k) in every for k in keys.tolist()])[:, None]
    inside = (u > 0.01) & (u < W_IMG - 1.01) & (v > 0.01) & (v < H_IMG - 1.01) & in_every
    d32 = [float(np.float32(Z) * DS) for Z in Zs]
    sdfs = np.stack([d - p[..., 2] for d in d32])
    in_all = inside & np.all(sdfs >= -MU + 1e-6, axis=0)
    assert in_all.sum() > 500
    mu64 = np.float64(np.float32(MU))
    expect = np.mean(np.clip(sdfs / mu64, -1, 1), axis=0)
    np.testing.assert_array_equal(W[in_all], len(Zs))
    np.testing.assert_allclose(F[in_all], expect[in_all], atol=1e-9)


def test_running_average_cap_closed_form():
    """64 frames at Z1 saturate W; m more frames at Z2 give F = c^m f1 + (1 - c^m) f2, c = 64/65."""
    T = pose(11)
    Z1, Z2, m = 1000, 1010, 9
    o = vol()
    o.integrate(np.full((H_IMG, W_IMG), Z1, np.uint16), T)
    every = {tuple(k) for k in o.touched().tolist()}
    for _ in range(63):
        o.integrate(np.full((H_IMG, W_IMG), Z1, np.uint16), T)
    o.integrate(np.full((H_IMG, W_IMG), Z2, np.uint16), T)
    every &= {tuple(k) for k in o.touched().tolist()}
    for _ in range(m - 1):
        o.integrate(np.full((H_IMG, W_IMG), Z2, np.uint16), T)
    keys, F, W = o.dump()
    p, u, v = voxel_geometry(keys, T)
    in_every = np.array([tuple(k) in every for k in keys.tolist()])[:, None]
    inside = (u > 0.01) & (u < W_IMG - 1.01) & (v > 0.01) & (v < H_IMG - 1.01) & in_every
    mu64 = np.float64(np.float32(MU))
    s1 = float(np.float32(Z1) * DS) - p[..., 2]
    s2 = float(np.float32(Z2) * DS) - p[..., 2]
    both = inside & (s1 >= -MU + 1e-6) & (s2 >= -MU + 1e-6)
    assert both.sum() > 500
    c = (64.0 / 65.0) ** m
    expect = c * np.clip(s1 / mu64, -1, 1) + (1 - c) * np.clip(s2 / mu64, -1, 1)
    np.testing.assert_array_equal(W[both], 64.0)
    np.testing.assert_allclose(F[both], expect[both], atol=1e-12)


def test_zmax_and_empty_frame():
    T = pose(5)
    o = vol(zmax=1.0)
    assert o.integrate(np.zeros((H_IMG, W_IMG), np.uint16), T) == 0
    assert o.integrate(np.full((H_IMG, W_IMG), 1001, np.uint16), T) == 0   # beyond zmax
    assert o.integrate(np.full((H_IMG, W_IMG), 1000, np.uint16), T) > 0
