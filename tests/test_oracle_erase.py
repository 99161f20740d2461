"""Pin of the oracle's out-of-region erase (Sec. 4.1: blocks leaving the active region are
removed from the GPU model): FP64 distance of each block centre (8k + 3.5) s from the camera,
checked wherever it is not within 1e-5 m of the radius."""
import numpy as np

from oracle import OracleVolume


def test_erase_radius_fp64():
    rng = np.random.default_rng(5)
    s = 0.05
    keys = np.unique(rng.integers(-30, 30, size=(3000, 3)), axis=0).astype(np.int32)
    o = OracleVolume(s, 0.2, 64.0, 0.001, 0.0, 8, 8, 4.0, 4.0, 4.0, 4.0)
    o.load(keys, np.zeros((len(keys), 512)), np.ones((len(keys), 512)))
    centre = np.array([0.31, -0.42, 0.17], np.float32)
    R = 4.0
    gone = {tuple(k) for k in o.erase_radius(centre, R).tolist()}
    left = {tuple(k) for k in o.dump()[0].tolist()}
    assert gone and left and not (gone & left) and len(gone) + len(left) == len(keys)
    c = (keys.astype(np.float64) * 8 + 3.5) * float(np.float32(s))
    dist = np.linalg.norm(c - centre.astype(np.float64), axis=1)
    for k, dd in zip(map(tuple, keys.tolist()), dist):
        if abs(dd - R) > 1e-5:
            assert (k in gone) == (dd > R), (k, dd)


def test_erase_keys_and_removal_list():
    o = OracleVolume(0.01, 0.04, 64.0, 0.001, 0.0, 8, 8, 4.0, 4.0, 4.0, 4.0)
    keys = np.array([[0, 0, 0], [1, 0, 0], [5, 5, 5]], np.int32)
    o.load(keys, np.zeros((3, 512)), np.ones((3, 512)))
    assert o.erase_keys(np.array([[1, 0, 0], [9, 9, 9]], np.int32)) == 1
    M, rem = o.mc_set(0)
    assert rem.tolist() == [[1, 0, 0]]
    # nothing was touched; the removed block's live negative neighbour (0,0,0) must be refreshed
    assert M.tolist() == [[0, 0, 0]]
    M2, rem2 = o.mc_set(0)
    assert M2.shape[0] == 0 and rem2.shape[0] == 0
