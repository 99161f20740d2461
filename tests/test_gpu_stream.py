"""GPU parity of stream-out (blocks leaving the active model move to a host map, Sec. 4.1) and
stream-in against the oracle: the host map after a room sequence with a moving erase radius
(through the frame graph and through separate calls), stream-in of every host key, and a ring
too small for one erase (the blocks that do not fit are counted and flagged, never silently
dropped)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1805_03709_b300 import synth, vbh as V

pytestmark = pytest.mark.gpu

TSDF_TOL = 1e-5


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


def compare_maps(a, b):
    ka, Fa, Wa = a
    kb, Fb, Wb = b
    np.testing.assert_array_equal(ka, kb)
    np.testing.assert_array_equal(Wa, Wb.astype(np.float32))
    if len(kb):
        assert np.abs(Fa.astype(np.float64) - Fb).max() <= TSDF_TOL


@pytest.fixture(scope="module")
def room():
    return synth.room_sequence(n_frames=10, width=160, height=120)


@pytest.mark.parametrize("graph", [True, False])
def test_stream_out_host_map_matches_oracle(room, graph):
    cam, poses, depth = room
    vol, orc = make_pair(cam, 0.005, 0.02, 1 << 16, 1 << 17, 4.0)
    vol.stream_out_enable()
    for i in range(len(poses)):
        T = poses[i]
        d = torch.from_numpy(depth[i]).cuda()
        if graph:
            vol.process_frame(d, T, i + 1, 2.5)
        else:
            vol.erase_radius(T[:, 3], 2.5, keys_out=False)
            vol.integrate(d, T, i + 1)
            vol.extract(V.VBH_MC_TOUCHED)
        orc.erase_radius(T[:, 3], 2.5)
        orc.integrate(depth[i], T)
        orc.mc_set(0)
    vol.stream_out_flush()
    streamed, lost, held = vol.stream_out_stats()
    assert lost == 0 and held > 500 and streamed >= held
    compare_maps(vol.host_map(), orc.host_dump())
    compare_maps(vol.dump(), orc.dump())
    assert vol.counters().error_flags == 0


def test_stream_in_moves_host_blocks_back(room):
    cam, poses, depth = room
    vol, orc = make_pair(cam, 0.005, 0.02, 1 << 16, 1 << 17, 4.0)
    vol.stream_out_enable()
    for i in range(6):
        vol.process_frame(torch.from_numpy(depth[i]).cuda(), poses[i], i + 1, 2.5)
        orc.erase_radius(poses[i][:, 3], 2.5)
        orc.integrate(depth[i], poses[i])
        orc.mc_set(0)
    hk = orc.host_dump()[0]
    assert len(hk) > 100
    extra = np.array([[1000, 1000, 1000]], np.int32)   # not in the map: ignored
    n_o = orc.stream_in(np.concatenate([hk, extra]))
    n_g = vol.stream_in(np.concatenate([hk, extra]))
    assert n_g == n_o > 0
    compare_maps(vol.dump(), orc.dump())
    compare_maps(vol.host_map(), orc.host_dump())
    # fusion continues on the streamed-in blocks exactly as in the oracle
    vol.process_frame(torch.from_numpy(depth[6]).cuda(), poses[6], 7, 2.5)
    orc.erase_radius(poses[6][:, 3], 2.5)
    orc.integrate(depth[6], poses[6])
    orc.mc_set(0)
    vol.stream_out_flush()
    compare_maps(vol.dump(), orc.dump())
    compare_maps(vol.host_map(), orc.host_dump())


def test_back_to_back_frames_do_not_outrun_the_ring(room):
    """Frames submitted with no synchronisation, through a ring of 32 frames' worth of removals:
    the host keeps only a few frames queued while it drains the ring, so nothing is lost and
    the host map equals that of a run with a ring larger than all removals."""
    cam, poses, depth = room
    order = [i % len(poses) for i in range(60)]
    D = [torch.from_numpy(depth[i]).cuda() for i in range(len(poses))]
    maps, per_frame = [], []
    for ring in (0, None):
        vol, _ = make_pair(cam, 0.005, 0.02, 1 << 16, 1 << 17, 4.0)
        if ring is None:
            ring = 32 * max(per_frame)
        vol.stream_out_enable(ring_blocks=ring)
        for k, i in enumerate(order):
            vol.process_frame(D[i], poses[i], k + 1, 1.0)
            if not maps:
                torch.cuda.synchronize()
                per_frame.append(vol.counters().last_erased)
        vol.stream_out_flush()
        streamed, lost, held = vol.stream_out_stats()
        assert lost == 0 and vol.counters().error_flags == 0
        maps.append(vol.host_map())
        vol.close()
    assert sum(per_frame) > 32 * max(per_frame) > 0   # the small ring wraps several times
    compare_maps(maps[1], maps[0])


def test_small_ring_counts_and_flags_lost_blocks():
    cam = synth.Camera(8, 8, 4.0, 4.0, 4.0, 4.0)
    vol, orc = make_pair(cam, 0.01, 0.04, 1 << 12, 1 << 10, 0.0)
    vol.stream_out_enable(ring_blocks=64)
    keys = np.array([(x, y, 0) for x in range(20) for y in range(10)], np.int32)
    rng = np.random.default_rng(4)
    F = rng.uniform(-1, 1, (len(keys), 512)).astype(np.float32)
    W = np.full((len(keys), 512), 2.0, np.float32)
    vol.load(keys, F, W)
    vol.erase_keys(torch.from_numpy(keys).cuda(), keys_out=False)
    vol.stream_out_flush()
    streamed, lost, held = vol.stream_out_stats()
    assert (streamed, lost, held) == (64, len(keys) - 64, 64)
    assert vol.counters().error_flags & 16
    hk, hF, hW = vol.host_map()
    pos = {tuple(k): i for i, k in enumerate(keys.tolist())}
    for j, k in enumerate(map(tuple, hk.tolist())):
        np.testing.assert_array_equal(hF[j], F[pos[k]])
        np.testing.assert_array_equal(hW[j], W[pos[k]])
