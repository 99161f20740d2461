"""The oracle's OpenMP timing mode gives exactly the single-threaded reference's results: the
allocation is a union of per-row block sets and fusion / MC classification work on independent
blocks, so neither the block sets nor a single FP64 value may depend on the thread count."""
import os

import numpy as np

import oracle
from paper_1805_03709_b300 import synth


def _run(threads, cam, poses, depth):
    oracle.set_threads(threads)
    try:
        o = oracle.OracleVolume(0.005, 0.02, 64.0, 0.001, 4.0, cam.width, cam.height, cam.fx,
                                cam.fy, cam.cx, cam.cy)
        sets = []
        for i in range(len(poses)):
            gone = o.erase_radius(poses[i][:, 3], 2.5)
            n = o.integrate(depth[i], poses[i])
            M, rem = o.mc_set(0)
            sets.append((gone.copy(), n, M.copy(), rem.copy()))
        k, F, W = o.dump()
        idx, margin = o.mc_dense(k)
        return sets, k, F, W, idx, margin
    finally:
        oracle.set_threads(1)


def test_threads_reproduce_the_reference_bit_for_bit():
    cam, poses, depth = synth.room_sequence(n_frames=4, width=160, height=120)
    ref = _run(1, cam, poses, depth)
    par = _run(max(2, min(8, os.cpu_count() or 2)), cam, poses, depth)
    for (g0, n0, M0, r0), (g1, n1, M1, r1) in zip(ref[0], par[0]):
        np.testing.assert_array_equal(g0, g1)
        assert n0 == n1
        np.testing.assert_array_equal(M0, M1)
        np.testing.assert_array_equal(r0, r1)
    for a, b in zip(ref[1:], par[1:]):
        np.testing.assert_array_equal(a, b)   # exact, FP64 values included
    assert len(ref[1]) > 1000
