"""Pins of the oracle's stream-out / stream-in (blocks leaving the active model move to a
passive host map, Sec. 4.1): an erased block arrives in the host map with exactly the values it
had, a later erase of the same key replaces them, and stream-in restores only keys that are not
live (a live block is newer)."""
import numpy as np

import oracle
from paper_1805_03709_b300 import synth


def vol_with_blocks(keys, seed=0):
    o = oracle.OracleVolume(0.01, 0.04, 64.0, 0.001, 0.0, 8, 8, 4.0, 4.0, 4.0, 4.0)
    rng = np.random.default_rng(seed)
    F = rng.uniform(-1, 1, (len(keys), 512))
    W = rng.integers(0, 65, (len(keys), 512)).astype(np.float64)
    o.load(np.asarray(keys, np.int32), F, W)
    return o, F, W


def test_erase_moves_exact_values_to_the_host_map():
    keys = [(x, y, 0) for x in range(-3, 3) for y in range(-2, 2)]
    o, F, W = vol_with_blocks(keys)
    gone = [(0, 0, 0), (-3, -2, 0), (2, 1, 0)]
    assert o.erase_keys(np.array(gone + [(9, 9, 9)], np.int32)) == 3
    hk, hF, hW = o.host_dump()
    assert [tuple(k) for k in hk.tolist()] == sorted(gone)
    for j, k in enumerate(map(tuple, hk.tolist())):
        i = keys.index(k)
        np.testing.assert_array_equal(hF[j], F[i])
        np.testing.assert_array_equal(hW[j], W[i])
    lk = {tuple(k) for k in o.dump()[0].tolist()}
    assert lk == set(keys) - set(gone)


def test_radius_erase_streams_out_what_leaves_the_sphere():
    keys = [(x, 0, 0) for x in range(-6, 7)]
    o, F, W = vol_with_blocks(keys, seed=1)
    # block centre (8k + 3.5) s with s = 1 cm: beyond 0.3 m from the origin -> |8x + 3.5| > 30
    o.erase_radius(np.zeros(3, np.float32), 0.3)
    hk = {tuple(k) for k in o.host_dump()[0].tolist()}
    expect = {k for k in keys if abs(8 * k[0] + 3.5) * 0.01 > 0.3}
    assert hk == expect and len(expect) > 0


def test_last_erase_wins_and_stream_in_restores_only_absent_keys():
    keys = [(0, 0, 0), (1, 0, 0), (2, 0, 0)]
    o, F, W = vol_with_blocks(keys, seed=2)
    o.erase_keys(np.array(keys, np.int32))
    # key (0,0,0) comes back with new values and is erased again: the host keeps the newest
    F2 = np.full((1, 512), 0.25)
    W2 = np.full((1, 512), 3.0)
    o.load(np.array([(0, 0, 0)], np.int32), F2, W2)
    o.erase_keys(np.array([(0, 0, 0)], np.int32))
    hk, hF, hW = o.host_dump()
    j = [tuple(k) for k in hk.tolist()].index((0, 0, 0))
    np.testing.assert_array_equal(hF[j], F2[0])
    # (1,0,0) is live again (new values): stream-in must not replace it
    o.load(np.array([(1, 0, 0)], np.int32), F2, W2)
    assert o.stream_in(np.array(keys + [(5, 5, 5)], np.int32)) == 2   # (0,0,0) and (2,0,0)
    lk, lF, lW = o.dump()
    live = {tuple(k): i for i, k in enumerate(lk.tolist())}
    np.testing.assert_array_equal(lF[live[(1, 0, 0)]], F2[0])
    np.testing.assert_array_equal(lF[live[(2, 0, 0)]], F[2])
    np.testing.assert_array_equal(lF[live[(0, 0, 0)]], F2[0])
    assert [tuple(k) for k in o.host_dump()[0].tolist()] == [(1, 0, 0)]


def test_frame_erase_streams_out_the_fused_values():
    """A fused block that leaves the radius is in the host map with the values it was fused to."""
    cam, poses, depth = synth.tiny_sequence(n_frames=2)
    o = oracle.OracleVolume(0.01, 0.04, 64.0, 0.001, 0.0, cam.width, cam.height, cam.fx, cam.fy,
                            cam.cx, cam.cy)
    o.integrate(depth[0], poses[0])
    k0, F0, W0 = o.dump()
    gone = o.erase_radius(poses[1][:, 3], 1.5)
    hk, hF, hW = o.host_dump()
    assert len(gone) == len(hk) > 0
    idx = {tuple(k): i for i, k in enumerate(k0.tolist())}
    for j, k in enumerate(map(tuple, hk.tolist())):
        np.testing.assert_array_equal(hF[j], F0[idx[k]])
        np.testing.assert_array_equal(hW[j], W0[idx[k]])
