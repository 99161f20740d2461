"""Pins of the oracle's Marching Cubes index extraction (Sec. 4.2): the analytic classification of
a sphere, the single-corner cases that fix the corner numbering, the S^c rule (0 and 255 are
written as 0), complement symmetry, invalid cubes, and the rule that refreshing each updated
block together with its seven negative neighbours keeps an incrementally maintained MC model
equal to a full re-extraction."""
import numpy as np
import pytest

from oracle import OracleVolume

# Classic Lorensen-Cline corner numbering (reading of the paper, which names no order).
CORNERS = [(0, 0, 0), (1, 0, 0), (1, 1, 0), (0, 1, 0), (0, 0, 1), (1, 0, 1), (1, 1, 1), (0, 1, 1)]


def make_vol(s=0.01, mu=0.04):
    return OracleVolume(s, mu, 64.0, 0.001, 0.0, 16, 16, 8.0, 8.0, 8.0, 8.0)


def local_grid(keys):
    l = np.arange(512)
    loc = np.stack([l % 8, (l // 8) % 8, l // 64], -1)
    return keys[:, None, :].astype(np.int64) * 8 + loc[None]


def test_analytic_sphere():
    s, mu = 0.01, 0.04
    c = np.array([0.013, -0.021, 0.007])
    r = 0.17
    rng = range(-4, 4)
    keys = np.array([(x, y, z) for x in rng for y in rng for z in rng], np.int32)
    g = local_grid(keys)
    dist = np.linalg.norm(g * s - c, axis=-1)
    F = np.clip((dist - r) / mu, -1, 1)
    o = make_vol(s, mu)
    o.load(keys, F, np.ones_like(F))
    idx, margin = o.mc_dense(keys)
    expect = np.zeros(g.shape[:2], np.int64)
    robust = np.ones(g.shape[:2], bool)
    valid = np.ones(g.shape[:2], bool)
    for i, off in enumerate(CORNERS):
        gc = g + np.array(off)
        dc = np.linalg.norm(gc * s - c, axis=-1)
        expect |= (dc < r).astype(np.int64) << i
        robust &= np.abs(dc - r) > 1e-4 * mu
        valid &= np.all((gc >= -32) & (gc < 32), axis=-1)   # corner inside the loaded blocks
    expect[expect == 255] = 0
    expect[~valid] = 0
    sel = robust | ~valid
    assert (expect[sel] != 0).sum() > 1000
    np.testing.assert_array_equal(idx[sel], expect[sel])
    assert not np.any(idx == 255)
    # margins agree with the analytic corner distances
    assert np.all(margin[~valid] == np.inf)


@pytest.mark.parametrize("corner", range(8))
def test_single_corner(corner):
    """One negative voxel: the cube whose corner `corner` is that voxel gets index 1 << corner."""
    keys = np.array([(x, y, z) for x in (-1, 0) for y in (-1, 0) for z in (-1, 0)], np.int32)
    F = np.ones((8, 512))
    W = np.ones((8, 512))
    # voxel g* = (0,0,0) lives in block (0,0,0) at local index 0
    b0 = [tuple(k) for k in keys.tolist()].index((0, 0, 0))
    F[b0, 0] = -0.5
    o = make_vol()
    o.load(keys, F, W)
    gc = -np.array(CORNERS[corner])   # cube origin g with g + c_corner = g*
    kb = tuple((gc // 8).tolist())
    li = int((gc % 8)[0] + 8 * (gc % 8)[1] + 64 * (gc % 8)[2])
    idx, _ = o.mc_dense(np.array([kb], np.int32))
    assert idx[0, li] == (1 << corner)
    assert np.count_nonzero(idx) == 1   # each of the 8 blocks holds exactly one cube using g*


def test_complement_and_invalid():
    rng = np.random.default_rng(3)
    keys = np.array([(x, y, z) for x in (0, 1) for y in (0, 1) for z in (0, 1)], np.int32)
    F = rng.uniform(-1, 1, size=(8, 512))
    F[np.abs(F) < 1e-3] = 0.5
    W = np.ones((8, 512))
    a = make_vol()
    a.load(keys, F, W)
    b = make_vol()
    b.load(keys, -F, W)
    ia, _ = a.mc_dense(keys[:1])
    ib, _ = b.mc_dense(keys[:1])
    both = (ia != 0) & (ib != 0)
    np.testing.assert_array_equal(ia[both].astype(int), 255 - ib[both].astype(int))
    # a zero weight anywhere invalidates every cube that uses the voxel
    W2 = W.copy()
    W2[0, 9] = 0.0           # voxel (1,1,0) of block (0,0,0)
    c = make_vol()
    c.load(keys, F, W2)
    ic, _ = c.mc_dense(keys[:1])
    for off in CORNERS:
        g = np.array([1, 1, 0]) - np.array(off)
        if np.all(g >= 0):
            assert ic[0, g[0] + 8 * g[1] + 64 * g[2]] == 0


def test_incremental_equals_full_reextraction():
    """Maintain an MC model by refreshing only the blocks in the per-frame set (touched blocks and
    their seven negative neighbours, plus removals) and compare with a full extraction."""
    from paper_1805_03709_b300 import synth
    cam, poses, depth = synth.tiny_sequence(n_frames=6, width=64, height=48, f=56.0)
    o = OracleVolume(0.02, 0.06, 64.0, 0.001, 0.0, cam.width, cam.height, cam.fx, cam.fy, cam.cx, cam.cy)
    model = {}
    for i in range(len(poses)):
        if i == 4:   # remove a few blocks mid-sequence
            o.erase_radius(poses[i][:, 3], 1.6)
        o.integrate(depth[i], poses[i])
        M, rem = o.mc_set(0)
        for k in rem.tolist():
            model.pop(tuple(k), None)
        idx, _ = o.mc_dense(M)
        for k, row in zip(M.tolist(), idx):
            model[tuple(k)] = row.copy()
        full, _ = o.mc_set(1)
        fidx, _ = o.mc_dense(full)
        assert set(model) == {tuple(k) for k in full.tolist()}
        for k, row in zip(full.tolist(), fidx):
            np.testing.assert_array_equal(model[tuple(k)], row)
