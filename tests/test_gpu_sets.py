"""GPU tests of the paper's per-client stream sets (vbh_sets_*): what a client's set holds is set
algebra over the oracle's per-frame refreshed blocks and removal records (plus every live block
for a filled client); fetches drain it as random subsets of at most the request size, each key
exactly once, with every live block's MC indices equal to the model's (and the oracle's at
every cube clear of the margin) and removal records for keys that are not live."""
import numpy as np
import pytest
import torch

import oracle
from paper_1805_03709_b300 import synth, vbh as V

pytestmark = pytest.mark.gpu

MC_MARGIN = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1805_03709_b300 import build
    build.build()
    assert torch.cuda.is_available()


def all_blocks_dense(vol):
    out = {}
    for k, (info, loc, idx) in vol.extract(V.VBH_MC_ALL).to_host().items():
        d = np.zeros(512, np.uint8)
        d[loc.astype(np.int64)] = idx
        out[k] = (info, d)
    return out


def drain(sets, client, limit):
    got, sizes = {}, []
    for _ in range(10000):
        recs, idx = sets.fetch([client], [limit])[0]
        r = recs.cpu().numpy()
        ix = idx.cpu().numpy()
        sizes.append(len(r))
        if not len(r):
            break
        for i in range(len(r)):
            k = tuple(int(x) for x in r[i, :3])
            assert k not in got, f"{k} fetched twice"
            info = int(r[i, 3]) & 0xFFFFFFFF
            got[k] = (info, None if info & V.VBH_REC_REMOVED else ix[i].copy())
    return got, sizes


def test_sets_hold_the_oracle_frame_sets_and_drain_exactly_once():
    from paper_1805_03709_b300.serve import Server, StreamSets
    from paper_1805_03709_b300.volume import Volume
    cam, poses, depth = synth.room_sequence(n_frames=8, width=160, height=120)
    vol = Volume(voxel_size=0.005, trunc=0.02, width=cam.width, height=cam.height, fx=cam.fx,
                 fy=cam.fy, cx=cam.cx, cy=cam.cy, n_buckets=1 << 16, max_blocks=1 << 17,
                 zmax=4.0)
    orc = oracle.OracleVolume(0.005, 0.02, 64.0, 0.001, 4.0, cam.width, cam.height, cam.fx,
                              cam.fy, cam.cx, cam.cy)
    vol.process_frame(torch.from_numpy(depth[0]).cuda(), poses[0], 1, 2.5)
    orc.erase_radius(poses[0][:, 3], 2.5)
    orc.integrate(depth[0], poses[0])
    orc.mc_set(0)
    srv = Server(vol, n_clients=2, budget_bytes=1 << 28, log_bits=20)
    sets = StreamSets(srv, n_clients=3, cap_log2=17)
    sets.fill(0)   # client 0 (re)connects: every live block is queued
    expect0 = {tuple(k) for k in orc.dump()[0].tolist()}
    expect1 = set()
    for i in range(1, len(poses)):
        vol.process_frame(torch.from_numpy(depth[i]).cuda(), poses[i], i + 1, 2.5)
        sets.insert_last()
        orc.erase_radius(poses[i][:, 3], 2.5)
        orc.integrate(depth[i], poses[i])
        M, R = orc.mc_set(0)
        upd = set(map(tuple, M.tolist())) | set(map(tuple, R.tolist()))
        expect0 |= upd
        expect1 |= upd
    queued, tombs, err = sets.counts()
    assert err == 0
    # every client's set receives the updates; only client 0 was filled
    assert (queued[0], queued[1], queued[2]) == (len(expect0), len(expect1), len(expect1))
    model = all_blocks_dense(vol)
    live = set(map(tuple, orc.dump()[0].tolist()))
    for client, expect, limit in ((0, expect0, 512), (1, expect1, 1000)):
        got, sizes = drain(sets, client, limit)
        assert set(got) == expect
        assert all(s == limit for s in sizes[:-2]) and sizes[-1] == 0
        for k, (info, d) in got.items():
            if k in live:
                assert d is not None and model[k][0] == info
                np.testing.assert_array_equal(d, model[k][1])
            else:
                assert d is None
        keys = np.array(sorted(k for k in got if k in live), np.int32)
        idx, margin = orc.mc_dense(keys)
        for j, k in enumerate(map(tuple, keys.tolist())):
            sel = margin[j] > MC_MARGIN
            assert np.array_equal(got[k][1][sel], idx[j][sel]), k
    queued, tombs, err = sets.counts()
    assert queued.tolist() == [0, 0, len(expect1)] and tombs[0] == len(expect0)
    # a rebuild drops the tombstones; a refill queues the live model again
    sets.rebuild(0)
    sets.fill(0)
    queued, tombs, _ = sets.counts()
    assert tombs[0] == 0 and queued[0] == len(live)
    sets.close()
    srv.close()
    vol.close()


def test_fetch_of_many_clients_in_one_launch():
    from paper_1805_03709_b300.serve import Server, StreamSets
    from paper_1805_03709_b300.volume import Volume
    cam, poses, depth = synth.tiny_sequence(n_frames=3)
    vol = Volume(voxel_size=0.01, trunc=0.04, width=cam.width, height=cam.height, fx=cam.fx,
                 fy=cam.fy, cx=cam.cx, cy=cam.cy, n_buckets=1 << 14, max_blocks=1 << 14)
    for i in range(3):
        vol.process_frame(torch.from_numpy(depth[i]).cuda(), poses[i], i + 1, 0.0)
    srv = Server(vol, n_clients=1, budget_bytes=1 << 26, log_bits=16)
    sets = StreamSets(srv, n_clients=16, cap_log2=14)
    for c in range(16):
        sets.fill(c)
    live = vol.counters().live
    limits = [128 * (1 + c % 8) for c in range(16)]
    seen = [set() for _ in range(16)]
    for _ in range(100):
        out = sets.fetch(list(range(16)), limits)
        if not any(len(r) for r, _ in out):
            break
        for c, (r, _) in enumerate(out):
            ks = {tuple(x) for x in r[:, :3].cpu().numpy().tolist()}
            assert not (ks & seen[c]) and len(ks) == len(r) <= limits[c]
            seen[c] |= ks
    assert all(len(s) == live for s in seen)
    sets.close()
    srv.close()
    vol.close()
