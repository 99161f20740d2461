"""Pins of the oracle's differentiable window fusion: the se(3) exponential map against
scipy.linalg.expm of the twist matrix, its derivatives against central differences, the fused
value of a fronto-parallel plane against its closed form, and the analytic FP64 gradient
(depth and pose) against FP64 central finite differences with h = 1e-6."""
import numpy as np
import pytest
import scipy.linalg

import oracle
from paper_1805_03709_b300 import synth


def twist(xi):
    rho, w = xi[:3], xi[3:]
    M = np.zeros((4, 4))
    M[:3, :3] = [[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]]
    M[:3, 3] = rho
    return M


@pytest.mark.parametrize("theta", [0.0, 1e-7, 1e-4, 2e-3, 0.3, 1.5, 3.0])
def test_exp_matches_matrix_exponential(theta):
    rng = np.random.default_rng(int(theta * 1e6) + 1)
    axis = rng.standard_normal(3)
    axis /= np.linalg.norm(axis)
    xi = np.concatenate([rng.uniform(-2, 2, 3), axis * theta])
    R, t, _, _ = oracle.se3_exp(xi)
    E = scipy.linalg.expm(twist(xi))
    np.testing.assert_allclose(R, E[:3, :3], atol=1e-12)
    np.testing.assert_allclose(t, E[:3, 3], atol=1e-12)
    np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-12)


@pytest.mark.parametrize("theta", [1e-6, 5e-4, 0.7, 2.5])
def test_exp_derivatives_central_differences(theta):
    rng = np.random.default_rng(7)
    axis = rng.standard_normal(3)
    axis /= np.linalg.norm(axis)
    xi = np.concatenate([rng.uniform(-1, 1, 3), axis * theta])
    _, _, dR, dt = oracle.se3_exp(xi)
    h = 1e-6
    for k in range(6):
        e = np.zeros(6)
        e[k] = h
        Rp, tp, _, _ = oracle.se3_exp(xi + e)
        Rm, tm, _, _ = oracle.se3_exp(xi - e)
        np.testing.assert_allclose(dR[k], (Rp - Rm) / (2 * h), atol=1e-8)
        np.testing.assert_allclose(dt[k], (tp - tm) / (2 * h), atol=1e-8)


def plane_setup(nf=3, W=40, H=30, Z0=1.3):
    """Camera looking along world +x from the origin; a wall at camera depth Z0 fills the view."""
    T = np.array([[0, 0, 1, 0.0], [-1, 0, 0, 0.0], [0, -1, 0, 0.0]], np.float64)
    M = np.eye(4)
    M[:3] = T
    L = np.real(scipy.linalg.logm(M))
    xi = np.array([L[0, 3], L[1, 3], L[2, 3], L[2, 1], L[0, 2], L[1, 0]])
    xis = np.tile(xi, (nf, 1))
    T0 = np.stack([oracle.nominal_pose_f32(x) for x in xis])
    depth = np.full((nf, H, W), np.float32(Z0), np.float32)
    return xis, T0, depth


def test_plane_value_closed_form():
    s, mu = 0.01, 0.04
    xis, T0, depth = plane_setup()
    nf, H, W = depth.shape
    f = 20.0
    g = np.array([(x, y, z) for x in range(110, 140) for y in range(-12, 13, 3) for z in range(-9, 10, 3)],
                 np.int32)
    o = oracle.OracleDiffFusion(s, mu, W, H, f, f, W / 2, H / 2, g, depth, T0)
    L, F = o.forward(xis)
    R, t, _, _ = oracle.se3_exp(xis[0])
    p = (g * np.float64(np.float32(s)) - t) @ R          # camera coordinates (rows)
    sdf = np.float64(np.float32(1.3)) - p[:, 2]
    valid = o.masks[:, 0] != 0
    assert valid.sum() > 100 and (~valid).sum() > 20
    q = sdf / np.float64(np.float32(mu))
    expect = np.clip(q, -1, 1)
    clear = valid & (np.abs(np.abs(q) - 1) > 1e-5)   # the side of the clamp is decided in float32
    np.testing.assert_allclose(F[clear], expect[clear], atol=1e-12)
    # invalid samples are the ones clearly behind the wall (or outside the view)
    u = f * p[:, 0] / p[:, 2] + W / 2
    v = f * p[:, 1] / p[:, 2] + H / 2
    inside = (u > 0.01) & (u < W - 1.01) & (v > 0.01) & (v < H - 1.01)
    assert np.all(valid[inside & (sdf > -mu + 1e-6)])
    assert not np.any(valid[sdf < -mu - 1e-6])
    assert L == pytest.approx(np.sum(F ** 2), rel=1e-14)


def small_window():
    cam, poses, xi, depth = synth.diff_window(4, 48, 36, seed=11)
    T0 = np.stack([oracle.nominal_pose_f32(x) for x in xi])
    S = synth.surface_samples(cam, poses, depth, 600, seed=5, voxel=0.005, band=0.01)
    o = oracle.OracleDiffFusion(0.005, 0.02, cam.width, cam.height, cam.fx, cam.fy, cam.cx, cam.cy,
                                S, depth, T0)
    return o, xi, depth


def rel_l2(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def test_gradient_vs_central_differences():
    o, xi, depth = small_window()
    gd, gx = o.backward(xi)
    h = 1e-6
    fd = np.zeros_like(gx)
    for f in range(xi.shape[0]):
        for k in range(6):
            e = np.zeros_like(xi)
            e[f, k] = h
            fd[f, k] = (o.forward(xi + e)[0] - o.forward(xi - e)[0]) / (2 * h)
    for f in range(xi.shape[0]):
        assert rel_l2(gx[f], fd[f]) < 1e-5, (f, gx[f], fd[f])
    rng = np.random.default_rng(2)
    nz = np.argwhere(np.abs(gd) > 1e-6 * np.abs(gd).max())
    pick = nz[rng.choice(len(nz), size=min(64, len(nz)), replace=False)]
    ga, gf = [], []
    for f, v, u in pick:
        dp = depth.copy()
        dm = depth.copy()
        # perturb in float64 around the float32 value: the oracle reads depth as float32, so use
        # a step that float32 represents exactly
        step = np.float32(2.0 ** -14)
        dp[f, v, u] += step
        dm[f, v, u] -= step
        ga.append(gd[f, v, u])
        gf.append((o.forward(xi, dp)[0] - o.forward(xi, dm)[0]) / (2 * float(step)))
    assert rel_l2(np.array(ga), np.array(gf)) < 1e-5
