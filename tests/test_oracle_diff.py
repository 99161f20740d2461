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


def wall_camera_xyz(g, xi, s):
    """FP64 camera coordinates (rows) of voxels g at pose exp(xi)."""
    R, t, _, _ = oracle.se3_exp(xi)
    return (g * np.float64(np.float32(s)) - t) @ R


def clear_of_pixel_edges(p, f, W, H, eps=1e-4):
    """Projections (FP64) that are not within eps of a pixel edge, and their cells."""
    u = f * p[:, 0] / p[:, 2] + W / 2
    v = f * p[:, 1] / p[:, 2] + H / 2
    clear = (np.abs(u - np.rint(u)) > eps) & (np.abs(v - np.rint(v)) > eps)
    return clear, np.floor(u).astype(int), np.floor(v).astype(int)


@pytest.mark.parametrize("delta_over_mu, valid_across", [
    (0.5, True), (1.0, True), (1.0 + 2.0 ** -15, False), (1.5, False), (2.5, False)])
def test_depth_span_rule_isolated_spikes(delta_over_mu, valid_across):
    """R-diff-3's discontinuity rule: a cell is valid only when its FOUR depths span at most mu.
    The wall at Z0 carries isolated pixels raised by delta on a 4 x 4 grid, so a raised pixel
    sits in each corner position (00, 10, 01, 11) of some cells.  Expected validity is computed
    here from the FP64 projection: inside the image, and no raised corner unless delta <= mu.
    mu = 2^-5 and Z0 = 1.25 make Z0 + delta and the float32 span exact, so delta = mu must be
    valid (the bound is inclusive) and delta = mu (1 + 2^-15) must not be.  A span over two
    corners, a strict bound, or a bound of 2 mu each fail one of the cases."""
    s, mu, Z0, f, W, H = 0.01, 2.0 ** -5, 1.25, 20.0, 40, 30
    xis, T0, depth = plane_setup(nf=1, W=W, H=H, Z0=Z0)
    delta = np.float32(mu * delta_over_mu)
    spike = np.zeros((H, W), bool)
    spike[2::4, 1::4] = True
    depth[0][spike] = np.float32(Z0) + delta
    assert np.float32(depth[0][spike][0] - np.float32(Z0)) == delta
    # samples in front of the wall (sdf > 0 >= -mu whatever the cell interpolates)
    g = np.array([(x, y, z) for x in range(100, 124, 2) for y in range(-30, 31)
                  for z in range(-22, 23)], np.int32)
    o = oracle.OracleDiffFusion(s, mu, W, H, f, f, W / 2, H / 2, g, depth, T0)
    valid = o.masks[:, 0] != 0
    p = wall_camera_xyz(g, xis[0], s)
    clear, iu, iv = clear_of_pixel_edges(p, f, W, H)
    inside = (iu >= 0) & (iu <= W - 2) & (iv >= 0) & (iv <= H - 2)
    iu_c, iv_c = np.clip(iu, 0, W - 2), np.clip(iv, 0, H - 2)
    corners = [spike[iv_c + b, iu_c + a] for b in (0, 1) for a in (0, 1)]
    raised = np.any(corners, axis=0)
    expect = inside & (~raised | valid_across)
    np.testing.assert_array_equal(valid[clear], expect[clear])
    # every corner position of a raised pixel is exercised by clear samples
    for c in corners:
        assert np.sum(clear & inside & c) > 10
    assert np.sum(clear & inside & ~raised) > 100


@pytest.mark.parametrize("eps_over_mu", [0.3, -0.3])
def test_clamp_side_fixed_at_nominal_pose(eps_over_mu):
    """R-diff-3's fixed clamp side: at the nominal pose a valid term is live (f = sdf / mu)
    when sdf0 < mu and saturated (f = 1) otherwise, and keeps that side at every other pose --
    a live term is extended linearly past +-1, a saturated one stays 1.  The camera moves by eps
    along its optical axis in front of a uniform wall, so every sdf grows by exactly eps; F of
    a single frame is compared with that closed form."""
    s, mu, Z0, f, W, H = 0.004, 0.04, 1.3, 20.0, 40, 30
    xis, T0, depth = plane_setup(nf=1, W=W, H=H, Z0=Z0)
    g = np.array([(x, y, z) for x in range(303, 348) for y in range(-200, 201, 50)
                  for z in range(-150, 151, 50)], np.int32)
    o = oracle.OracleDiffFusion(s, mu, W, H, f, f, W / 2, H / 2, g, depth, T0)
    valid = o.masks[:, 0] != 0
    eps = eps_over_mu * mu
    # the moved pose: camera centre at world (eps, 0, 0), same rotation
    M = np.eye(4)
    M[:3, :3] = oracle.se3_exp(xis[0])[0]
    M[:3, 3] = [eps, 0.0, 0.0]
    Lg = np.real(scipy.linalg.logm(M))
    xi1 = np.array([[Lg[0, 3], Lg[1, 3], Lg[2, 3], Lg[2, 1], Lg[0, 2], Lg[1, 0]]])
    _, F = o.forward(xi1)
    p0 = wall_camera_xyz(g, xis[0], s)
    p1 = wall_camera_xyz(g, xi1[0], s)
    np.testing.assert_allclose(p1[:, 2], p0[:, 2] - eps, atol=1e-12)
    q0 = (np.float64(np.float32(Z0)) - p0[:, 2]) / np.float64(np.float32(mu))
    q1 = (np.float64(np.float32(Z0)) - p1[:, 2]) / np.float64(np.float32(mu))
    decided = valid & (np.abs(q0 - 1) > 1e-5)          # float32 side decision unambiguous
    live0 = q0 < 1
    expect = np.where(live0, q1, 1.0)
    np.testing.assert_allclose(F[decided], expect[decided], atol=1e-9)
    if eps > 0:   # live terms pushed past the clamp are extended linearly, not clamped
        assert np.sum(decided & live0 & (q1 > 1.05)) > 5
    else:         # saturated terms pulled inside stay saturated; valid terms pass below -1
        assert np.sum(decided & ~live0 & (q1 < 0.95)) > 5
        assert np.sum(decided & (q1 < -1.05)) > 5


def small_window(n_samples=600):
    cam, poses, xi, depth = synth.diff_window(4, 48, 36, seed=11)
    T0 = np.stack([oracle.nominal_pose_f32(x) for x in xi])
    S = synth.surface_samples(cam, poses, depth, n_samples, seed=5, voxel=0.005, band=0.01)
    o = oracle.OracleDiffFusion(0.005, 0.02, cam.width, cam.height, cam.fx, cam.fy, cam.cx, cam.cy,
                                S, depth, T0)
    return o, xi, depth


def rel_l2(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def test_gradient_vs_central_differences():
    o, xi, depth = small_window(3000)
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
    assert len(nz) >= 256
    pick = nz[rng.choice(len(nz), size=256, replace=False)]
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
