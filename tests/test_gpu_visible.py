"""GPU parity of the visible-set integration (touched blocks + every live block in view, with
free-space carving) and of the frustum erase (the scene reset) against the oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_1805_03709_b300 import synth, vbh as V

pytestmark = pytest.mark.gpu

TSDF_TOL = 1e-5
MC_MARGIN = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1805_03709_b300 import build
    build.build()
    assert torch.cuda.is_available()


def make_pair(cam, s, mu, n_buckets, max_blocks, zmax):
    from paper_1805_03709_b300.volume import Volume
    vol = Volume(voxel_size=s, trunc=mu, width=cam.width, height=cam.height, fx=cam.fx,
                 fy=cam.fy, cx=cam.cx, cy=cam.cy, n_buckets=n_buckets, max_blocks=max_blocks,
                 zmax=zmax)
    orc = oracle.OracleVolume(s, mu, 64.0, 0.001, zmax, cam.width, cam.height, cam.fx, cam.fy,
                              cam.cx, cam.cy)
    return vol, orc


def compare_volume(vol, orc):
    kg, Fg, Wg = vol.dump()
    ko, Fo, Wo = orc.dump()
    np.testing.assert_array_equal(kg, ko)
    np.testing.assert_array_equal(Wg, Wo.astype(np.float32))
    if len(ko):
        assert np.abs(Fg.astype(np.float64) - Fo).max() <= TSDF_TOL


def compare_mc(recs, orc, keys, removed):
    live = {k: r for k, r in recs.items() if not (r[0] & V.VBH_REC_REMOVED)}
    tomb = {k for k, r in recs.items() if r[0] & V.VBH_REC_REMOVED}
    assert set(live) == set(map(tuple, np.asarray(keys).reshape(-1, 3).tolist()))
    assert tomb == set(map(tuple, np.asarray(removed).reshape(-1, 3).tolist()))
    if not len(keys):
        return
    idx, margin = orc.mc_dense(keys)
    for b, k in enumerate(map(tuple, np.asarray(keys).tolist())):
        d = np.zeros(512, np.uint8)
        _, loc, ix = live[k]
        d[loc.astype(np.int64)] = ix
        sel = margin[b] > MC_MARGIN
        assert np.array_equal(d[sel], idx[b][sel]), k


@pytest.fixture(scope="module")
def room():
    return synth.room_sequence(n_frames=8, width=160, height=120)


@pytest.mark.parametrize("graph", [True, False])
def test_visible_integration_matches_oracle(room, graph):
    cam, poses, depth = room
    vol, orc = make_pair(cam, 0.005, 0.02, 1 << 16, 1 << 17, 4.0)
    vol.set_integration_mode(True)
    grew = 0
    for i in range(len(poses)):
        T = poses[i]
        d = torch.from_numpy(depth[i]).cuda()
        if graph:
            s = vol.process_frame(d, T, i + 1, 2.5)
        else:
            vol.erase_radius(T[:, 3], 2.5, keys_out=False)
            vol.integrate(d, T, i + 1)
            s = vol.extract(V.VBH_MC_TOUCHED)
        orc.erase_radius(T[:, 3], 2.5)
        n_o = orc.integrate(depth[i], T, visible=True)
        n_touched_only = len(orc.touched())   # same as n_o (the fused set)
        assert vol.counters().last_touched == n_o == n_touched_only
        M, rem = orc.mc_set(0)
        compare_mc(s.to_host(), orc, M, rem)
        compare_volume(vol, orc)
        grew += n_o
    assert vol.counters().error_flags == 0


def test_visible_set_is_larger_and_carves(room):
    """The visible set adds blocks the band does not reach; the volumes of the two modes differ
    only in blocks that were fused in the visible mode."""
    cam, poses, depth = room
    a, oa = make_pair(cam, 0.005, 0.02, 1 << 16, 1 << 17, 4.0)
    b, ob = make_pair(cam, 0.005, 0.02, 1 << 16, 1 << 17, 4.0)
    b.set_integration_mode(True)
    extra = 0
    for i in range(4):
        d = torch.from_numpy(depth[i]).cuda()
        a.process_frame(d, poses[i], i + 1, 0.0)
        b.process_frame(d, poses[i], i + 1, 0.0)
        torch.cuda.synchronize()
        extra += b.counters().last_touched - a.counters().last_touched
    assert extra > 0
    ka, Fa, Wa = a.dump()
    kb, Fb, Wb = b.dump()
    np.testing.assert_array_equal(ka, kb)   # the same blocks are allocated
    assert (Wb >= Wa).all() and (Wb > Wa).any()   # extra observations only


def test_frustum_erase_matches_oracle(room):
    cam, poses, depth = room
    vol, orc = make_pair(cam, 0.005, 0.02, 1 << 16, 1 << 17, 4.0)
    vol.stream_out_enable()
    for i in range(4):
        vol.process_frame(torch.from_numpy(depth[i]).cuda(), poses[i], i + 1, 0.0)
        orc.integrate(depth[i], poses[i])
        orc.mc_set(0)
    T = poses[2]
    vol.erase_frustum(T, zfar=1.5)
    gone_o = orc.erase_frustum(T, zfar=1.5)
    gone_g = vol.erased()
    assert len(gone_o) > 100
    assert {tuple(k) for k in gone_g.tolist()} == {tuple(k) for k in gone_o.tolist()}
    compare_volume(vol, orc)
    # the erased blocks reach the host map and are reported as removal records
    vol.stream_out_flush()
    hk = vol.host_map()[0]
    assert {tuple(k) for k in hk.tolist()} == {tuple(k) for k in gone_o.tolist()}
    s = vol.extract(V.VBH_MC_TOUCHED)
    M, rem = orc.mc_set(0)
    compare_mc(s.to_host(), orc, M, rem)
