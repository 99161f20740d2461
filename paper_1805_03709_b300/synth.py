"""Seeded synthetic RGB-D-like depth streams (depth only) for the voxel-block-hashing path.

This module is the one input source shared by the CUDA path, the CPU oracle, the tests and the
benchmark.  It holds no arithmetic of the reconstruction method itself: it only simulates a
pinhole depth sensor moving through an analytic scene (ray casting in FP64, Kinect-like axial
noise, random dropout, quantisation to uint16 millimetres).

The paper evaluates on recorded Kinect v1/v2 sequences (heating_room, pool, TUM fr1/desk2 and
fr1/room; Sec. 6, Tables 2-3) that are not available here; the scenes below stand in for them
with the same sensor geometry (640x480, f=525 for the Kinect v1 shaped room sequence) and the
voxel / truncation settings of the workloads this library is measured on.

Conventions
-----------
* World frame: z up.  Camera frame: x right, y down, z forward (optical axis).
* A pose T_wc is a float32 3x4 row-major matrix [R | t] mapping camera to world: X = R p + t.
* Pixel (u, v) has its centre at image coordinates (u, v); the principal point is (cx, cy).
* Raw depth is the camera-frame z of the first surface hit, in millimetres, rounded to the
  nearest integer; 0 marks an invalid pixel (no hit, dropout, or out of the uint16 range).
"""
from __future__ import annotations

import dataclasses
import numpy as np

__all__ = [
    "Camera", "Scene", "make_tiny_scene", "make_room_scene", "render_depth_m",
    "quantize_mm", "tiny_sequence", "room_sequence", "room_frames", "room_camera", "look_at",
    "room_static_frames",
    "random_hash_keys", "distinct_keys", "zipf_cluster_keys", "diff_window", "surface_samples",
]


@dataclasses.dataclass(frozen=True)
class Camera:
    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float


@dataclasses.dataclass
class Scene:
    """Analytic scene: axis-aligned boxes (solid), spheres (solid), optional room (hollow box)
    and optional finite floor rectangle at z = 0."""
    spheres: np.ndarray            # (n, 4): cx, cy, cz, r
    boxes: np.ndarray              # (m, 6): xmin, ymin, zmin, xmax, ymax, zmax
    room: np.ndarray | None = None  # (6,): interior extent, rays hit its inside faces
    floor: np.ndarray | None = None  # (4,): xmin, ymin, xmax, ymax of a floor patch at z = 0


def look_at(eye, target, up=(0.0, 0.0, 1.0)) -> np.ndarray:
    """Camera-to-world pose (float32 3x4) for a camera at `eye` looking at `target`."""
    eye = np.asarray(eye, np.float64)
    fwd = np.asarray(target, np.float64) - eye
    fwd /= np.linalg.norm(fwd)
    right = np.cross(fwd, np.asarray(up, np.float64))
    right /= np.linalg.norm(right)
    down = np.cross(fwd, right)
    R = np.stack([right, down, fwd], axis=1)  # columns: camera x, y, z axes in world
    T = np.zeros((3, 4), np.float64)
    T[:, :3] = R
    T[:, 3] = eye
    return T.astype(np.float32)


def _rays(cam: Camera, T: np.ndarray):
    u = np.arange(cam.width, dtype=np.float64)
    v = np.arange(cam.height, dtype=np.float64)
    uu, vv = np.meshgrid(u, v)
    dc = np.stack([(uu - cam.cx) / cam.fx, (vv - cam.cy) / cam.fy, np.ones_like(uu)], axis=-1)
    R = T[:, :3].astype(np.float64)
    o = T[:, 3].astype(np.float64)
    d = dc @ R.T  # world direction with unit camera-z component: hit parameter t == camera z
    return o, d


def _screen_rect(cam: Camera, T: np.ndarray, centre, radius):
    """Conservative pixel rectangle [v0, v1) x [u0, u1) containing the projection of a sphere
    (the bounding sphere of an object); None if it lies entirely behind the camera."""
    R = T[:, :3].astype(np.float64)
    p = R.T @ (np.asarray(centre, np.float64) - T[:, 3].astype(np.float64))
    if p[2] + radius <= 1e-6:
        return None
    if p[2] - radius <= 1e-3:
        return 0, cam.height, 0, cam.width
    zs = (p[2] - radius, p[2] + radius)
    us = [cam.cx + cam.fx * (p[0] + sx * radius) / z for sx in (-1, 1) for z in zs]
    vs = [cam.cy + cam.fy * (p[1] + sy * radius) / z for sy in (-1, 1) for z in zs]
    u0, u1 = max(0, int(np.floor(min(us))) - 1), min(cam.width, int(np.ceil(max(us))) + 2)
    v0, v1 = max(0, int(np.floor(min(vs))) - 1), min(cam.height, int(np.ceil(max(vs))) + 2)
    if u0 >= u1 or v0 >= v1:
        return None
    return v0, v1, u0, u1


def render_depth_m(scene: Scene, cam: Camera, T: np.ndarray) -> np.ndarray:
    """Exact (FP64) camera-frame depth of the first hit for every pixel; +inf where nothing is hit."""
    o, d = _rays(cam, T)
    best = np.full(d.shape[:2], np.inf)
    eps = 1e-9
    with np.errstate(divide="ignore", invalid="ignore"):
        inv = 1.0 / d
        if scene.room is not None:
            lo, hi = scene.room[:3], scene.room[3:]
            # from inside the room: exit distance of the slab intersection
            t1 = (lo - o) * inv
            t2 = (hi - o) * inv
            tfar = np.nanmin(np.maximum(t1, t2), axis=-1)
            best = np.where((tfar > eps) & (tfar < best), tfar, best)
        if scene.floor is not None:
            x0, y0, x1, y1 = scene.floor
            t = -o[2] / d[..., 2]
            px = o[0] + t * d[..., 0]
            py = o[1] + t * d[..., 1]
            hit = (t > eps) & (px >= x0) & (px <= x1) & (py >= y0) & (py <= y1)
            best = np.where(hit & (t < best), t, best)
        for b in scene.boxes:
            lo, hi = b[:3], b[3:]
            rect = _screen_rect(cam, T, (lo + hi) / 2, 0.5 * np.linalg.norm(hi - lo))
            if rect is None:
                continue
            v0, v1, u0, u1 = rect
            sub_inv = inv[v0:v1, u0:u1]
            t1 = (lo - o) * sub_inv
            t2 = (hi - o) * sub_inv
            mn = np.minimum(t1, t2)
            mx = np.maximum(t1, t2)
            tnear = np.maximum(np.maximum(mn[..., 0], mn[..., 1]), mn[..., 2])
            tfar = np.minimum(np.minimum(mx[..., 0], mx[..., 1]), mx[..., 2])
            hit = (tnear <= tfar) & (tnear > eps)
            sb = best[v0:v1, u0:u1]
            best[v0:v1, u0:u1] = np.where(hit & (tnear < sb), tnear, sb)
        for s in scene.spheres:
            c, r = s[:3], s[3]
            rect = _screen_rect(cam, T, c, r)
            if rect is None:
                continue
            v0, v1, u0, u1 = rect
            sd = d[v0:v1, u0:u1]
            a = np.einsum("hwc,hwc->hw", sd, sd)
            oc = o - c
            b = np.einsum("hwc,c->hw", sd, oc)
            cc = float(oc @ oc - r * r)
            disc = b * b - a * cc
            sq = np.sqrt(np.maximum(disc, 0.0))
            t = (-b - sq) / a
            hit = (disc >= 0) & (t > eps)
            sb = best[v0:v1, u0:u1]
            best[v0:v1, u0:u1] = np.where(hit & (t < sb), t, sb)
    return best


def quantize_mm(depth_m: np.ndarray) -> np.ndarray:
    """Round metres to integer millimetres; non-finite, non-positive or >65535 mm -> 0."""
    mm = np.rint(np.where(np.isfinite(depth_m), depth_m, 0.0) * 1000.0)
    mm = np.where((mm > 0) & (mm <= 65535), mm, 0)
    return mm.astype(np.uint16)


def make_tiny_scene(seed: int = 1805) -> Scene:
    """Floor patch (2 x 2 m at z = 0) and 3 spheres of radius 0.2-0.5 m inside a 2 x 2 x 2 m box."""
    rng = np.random.default_rng(seed)
    sph = []
    for _ in range(3):
        r = rng.uniform(0.2, 0.5)
        c = [rng.uniform(-1 + r, 1 - r), rng.uniform(-1 + r, 1 - r), rng.uniform(r, 2 - r)]
        sph.append(c + [r])
    return Scene(spheres=np.array(sph), boxes=np.zeros((0, 6)), floor=np.array([-1.0, -1.0, 1.0, 1.0]))


def tiny_sequence(n_frames: int = 10, seed: int = 1805, width: int = 160, height: int = 120,
                  f: float = 140.0):
    """Small workload: camera on a seeded circular path of radius 1.5 m around the 2 m box,
    looking at its centre.  Returns (camera, poses (n,3,4) f32, depth (n,H,W) u16 mm)."""
    rng = np.random.default_rng(seed + 1)
    scene = make_tiny_scene(seed)
    cam = Camera(width, height, f, f, width / 2.0, height / 2.0)
    phase = rng.uniform(0, 2 * np.pi)
    h = rng.uniform(0.9, 1.3)
    poses, depths = [], []
    for i in range(n_frames):
        a = phase + 0.12 * i
        eye = (1.5 * np.cos(a), 1.5 * np.sin(a), h)
        T = look_at(eye, (0.0, 0.0, 0.4))
        poses.append(T)
        depths.append(quantize_mm(render_depth_m(scene, cam, T)))
    return cam, np.stack(poses), np.stack(depths)


def make_room_scene(seed: int = 1805, n_objects: int = 40) -> Scene:
    """8 x 8 x 3 m room with `n_objects` random boxes and spheres (sizes 0.15-0.9 m)."""
    rng = np.random.default_rng(seed)
    boxes, sph = [], []
    for i in range(n_objects):
        x, y = rng.uniform(0.5, 7.5, size=2)
        if i % 2 == 0:
            sx, sy, sz = rng.uniform(0.15, 0.9, size=3)
            z0 = 0.0 if rng.uniform() < 0.7 else rng.uniform(0.3, 1.8)
            boxes.append([x - sx / 2, y - sy / 2, z0, x + sx / 2, y + sy / 2, min(z0 + sz, 2.9)])
        else:
            r = rng.uniform(0.1, 0.45)
            z = r if rng.uniform() < 0.5 else rng.uniform(r, 2.9 - r)
            sph.append([x, y, z, r])
    return Scene(spheres=np.array(sph).reshape(-1, 4), boxes=np.array(boxes).reshape(-1, 6),
                 room=np.array([0.0, 0.0, 0.0, 8.0, 8.0, 3.0]))


def room_trajectory(n_frames: int, seed: int = 1805, fps: float = 30.0):
    """Seeded smooth walking trajectory at ~1.5 m eye height inside the 8 x 8 m room."""
    rng = np.random.default_rng(seed + 7)
    ph = rng.uniform(0, 2 * np.pi, size=6)
    w1, w2 = rng.uniform(0.10, 0.16), rng.uniform(0.07, 0.12)
    poses = []
    for i in range(n_frames):
        t = i / fps
        x = 4.0 + 2.2 * np.cos(w1 * 2 * np.pi * t + ph[0])
        y = 4.0 + 2.2 * np.sin(w2 * 2 * np.pi * t + ph[1])
        z = 1.5 + 0.05 * np.sin(0.5 * 2 * np.pi * t + ph[2])
        yaw = ph[3] + 0.6 * t + 0.5 * np.sin(0.2 * 2 * np.pi * t + ph[4])
        pitch = -0.25 + 0.12 * np.sin(0.15 * 2 * np.pi * t + ph[5])
        fwd = np.array([np.cos(yaw) * np.cos(pitch), np.sin(yaw) * np.cos(pitch), np.sin(pitch)])
        poses.append(look_at((x, y, z), (x + fwd[0], y + fwd[1], z + fwd[2])))
    return np.stack(poses)


def room_camera(width: int = 640, height: int = 480, f: float = 525.0) -> Camera:
    """Kinect-v1-like pinhole camera (f scaled with the image width)."""
    return Camera(width, height, f * width / 640.0, f * width / 640.0, width / 2.0, height / 2.0)


def room_frames(indices, n_frames: int, seed: int = 1805, width: int = 640, height: int = 480,
                f: float = 525.0, noise: bool = True, dropout: float = 0.02,
                metric_depth: bool = False):
    """Depth frames `indices` of the room walk of `n_frames` frames (each frame has its own
    seeded noise stream, so any subset can be rendered independently)."""
    scene = make_room_scene(seed)
    cam = room_camera(width, height, f)
    poses = room_trajectory(n_frames, seed)
    out = []
    for i in indices:
        rng = np.random.default_rng([seed + 11, int(i)])
        z = render_depth_m(scene, cam, poses[i])
        if noise:
            z = z + rng.standard_normal(z.shape) * (0.0015 * np.where(np.isfinite(z), z, 0.0) ** 2)
        if dropout > 0:
            z = np.where(rng.uniform(size=z.shape) < dropout, np.inf, z)
        if metric_depth:
            out.append(np.where(np.isfinite(z) & (z > 0), z, 0.0).astype(np.float32))
        else:
            out.append(quantize_mm(z))
    return np.stack(out) if out else np.zeros((0, height, width),
                                               np.float32 if metric_depth else np.uint16)


def room_sequence(n_frames: int = 300, seed: int = 1805, width: int = 640, height: int = 480,
                  f: float = 525.0, noise: bool = True, dropout: float = 0.02,
                  metric_depth: bool = False, workers: int = 1):
    """Room-scale workload: depth along a smooth walk through the 8 x 8 x 3 m room, axial noise
    sigma = 1.5 mm * z^2 (z in m) and `dropout` random invalid pixels.  Returns (camera, poses,
    depth) with depth as uint16 mm, or float32 metres (0 = invalid) when `metric_depth` is set.
    `workers` > 1 renders in that many spawned processes (call it before any CUDA work)."""
    cam = room_camera(width, height, f)
    poses = room_trajectory(n_frames, seed)
    kw = dict(n_frames=n_frames, seed=seed, width=width, height=height, f=f, noise=noise,
              dropout=dropout, metric_depth=metric_depth)
    if workers <= 1 or n_frames < 8:
        return cam, poses, room_frames(range(n_frames), **kw)
    import concurrent.futures as cf
    import functools
    import multiprocessing as mp
    chunks = [list(c) for c in np.array_split(np.arange(n_frames), workers) if len(c)]
    with cf.ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as ex:
        parts = list(ex.map(functools.partial(room_frames, **kw), chunks))
    return cam, poses, np.concatenate(parts)


def room_static_frames(n_frames: int, pose_index: int = 0, seed: int = 1805, width: int = 160,
                       height: int = 120, f: float = 525.0, dropout: float = 0.02):
    """`n_frames` depth frames seen from ONE pose of the room walk (frame `pose_index` of a
    300-frame walk), each with its own seeded axial noise (sigma = 1.5 mm * z^2) and dropout:
    a camera held still, so every voxel in view is observed once per frame and its weight runs
    up to and past any cap.  Returns (camera, pose (3,4) f32, depth (n,H,W) u16 mm)."""
    scene = make_room_scene(seed)
    cam = room_camera(width, height, f)
    T = room_trajectory(300, seed)[pose_index]
    z0 = render_depth_m(scene, cam, T)
    out = []
    for i in range(n_frames):
        rng = np.random.default_rng([seed + 13, int(i)])
        z = z0 + rng.standard_normal(z0.shape) * (0.0015 * np.where(np.isfinite(z0), z0, 0.0) ** 2)
        if dropout > 0:
            z = np.where(rng.uniform(size=z.shape) < dropout, np.inf, z)
        out.append(quantize_mm(z))
    return cam, T, np.stack(out)


def distinct_keys(n: int, seed: int) -> np.ndarray:
    """`n` distinct int3 keys spread over [-2^20, 2^20)^3: a seeded bijection of the 63-bit
    packed key space (odd multiplier and xor-shifts are invertible mod 2^63) applied to
    0..n-1, unpacked into three 21-bit coordinates.  Vectorised; no de-duplication needed."""
    m = np.uint64((1 << 63) - 1)
    x = (np.arange(n, dtype=np.uint64) + np.uint64(seed * 0x9E3779B9 & ((1 << 62) - 1))) & m
    for c in (0x5DEECE66D2B79F5, 0x2545F4914F6CDD1D):
        x = (x * np.uint64(c | 1)) & m
        x ^= x >> np.uint64(29)
    f = np.uint64((1 << 21) - 1)
    out = np.stack([(x & f), (x >> np.uint64(21)) & f, (x >> np.uint64(42)) & f], 1).astype(np.int64)
    return (out - (1 << 20)).astype(np.int32)


def random_hash_keys(n: int, seed: int, lo: int = -(1 << 20), hi: int = (1 << 20)) -> np.ndarray:
    """`n` distinct int3 keys uniform in [lo, hi)^3 (int32, shape (n, 3))."""
    rng = np.random.default_rng(seed)
    out = np.zeros((0, 3), np.int32)
    while out.shape[0] < n:
        k = rng.integers(lo, hi, size=(int((n - out.shape[0]) * 1.1) + 16, 3), dtype=np.int64)
        out = np.unique(np.concatenate([out.astype(np.int64), k]), axis=0).astype(np.int32)
    perm = rng.permutation(out.shape[0])[:n]
    return np.ascontiguousarray(out[perm])


def zipf_cluster_keys(n_draws: int, seed: int, hot_side: int = 64, s: float = 1.1) -> np.ndarray:
    """Clustered keys: a seeded cube of hot_side^3 contiguous block coordinates, drawn with
    Zipf(s) popularity over a seeded ranking (int32, shape (n_draws, 3); duplicates expected)."""
    rng = np.random.default_rng(seed)
    n_hot = hot_side ** 3
    origin = rng.integers(-(1 << 20), (1 << 20) - hot_side, size=3)
    ranks = np.arange(1, n_hot + 1, dtype=np.float64)
    p = ranks ** (-s)
    p /= p.sum()
    order = rng.permutation(n_hot)
    idx = order[rng.choice(n_hot, size=n_draws, p=p)]
    g = np.stack([idx % hot_side, (idx // hot_side) % hot_side, idx // (hot_side * hot_side)], -1)
    return (g + origin).astype(np.int32)


def diff_window(n_frames: int = 64, width: int = 320, height: int = 240, f: float = 262.5,
                seed: int = 1805, noise: bool = True, dropout: float = 0.02):
    """Window of the room walk for differentiable fusion: float32 metric depth (0 = invalid),
    the camera, the look-at poses (float32 3x4) and the same poses as se(3) vectors
    xi = (rho, omega), read off the matrix logarithm of the 4x4 pose (scipy.linalg.logm)."""
    import scipy.linalg
    cam, poses, depth = room_sequence(n_frames, seed=seed, width=width, height=height,
                                      f=f * 640.0 / width, noise=noise, dropout=dropout,
                                      metric_depth=True)
    xi = np.zeros((n_frames, 6))
    for i, T in enumerate(poses):
        M = np.eye(4)
        M[:3, :] = T.astype(np.float64)
        L = np.real(scipy.linalg.logm(M))
        xi[i, :3] = L[:3, 3]
        xi[i, 3:] = [L[2, 1], L[0, 2], L[1, 0]]
    return cam, poses, xi, depth


def surface_samples(cam: Camera, poses, depth_m, n: int, seed: int, voxel: float, band: float):
    """`n` distinct voxel coordinates (int32, shape (n, 3)) near observed surfaces: random valid
    pixels of random frames are lifted to world points, shifted by a uniform offset in
    [-band, band]^3 and snapped to the voxel grid."""
    rng = np.random.default_rng(seed)
    out = np.zeros((0, 3), np.int64)
    nf = len(poses)
    while len(out) < n:
        m = int((n - len(out)) * 1.3) + 64
        f = rng.integers(0, nf, m)
        u = rng.integers(0, cam.width, m)
        v = rng.integers(0, cam.height, m)
        d = depth_m[f, v, u].astype(np.float64)
        ok = d > 0
        f, u, v, d = f[ok], u[ok], v[ok], d[ok]
        pc = np.stack([(u - cam.cx) / cam.fx * d, (v - cam.cy) / cam.fy * d, d], -1)
        T = np.asarray(poses, np.float64)[f]
        P = np.einsum("nij,nj->ni", T[:, :, :3], pc) + T[:, :, 3]
        P += rng.uniform(-band, band, size=P.shape)
        g = np.round(P / voxel).astype(np.int64)
        out = np.unique(np.concatenate([out, g]), axis=0)
    keep = rng.permutation(len(out))[:n]
    return np.ascontiguousarray(out[keep].astype(np.int32))
