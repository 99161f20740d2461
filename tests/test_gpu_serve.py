"""GPU tests of multi-client delta streaming (vbh_serve_*): served MC blocks against the oracle,
client replicas that converge to the server's model through deltas and removals, every request
identical alone and in a continuously batched mix (chunked, under memory pressure), partial
ranges under a tight budget, and the real-time loop."""
import numpy as np
import pytest
import torch

import oracle
from paper_1805_03709_b300 import synth, vbh as V

pytestmark = pytest.mark.gpu

MC_MARGIN = 1e-4   # oracle |TSDF| margin of the MC parity bar (normalised TSDF units)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1805_03709_b300 import build
    build.build()
    assert torch.cuda.is_available()


def make_volume(cam, s, mu, n_buckets, max_blocks, zmax):
    from paper_1805_03709_b300.volume import Volume
    vol = Volume(voxel_size=s, trunc=mu, width=cam.width, height=cam.height, fx=cam.fx,
                 fy=cam.fy, cx=cam.cx, cy=cam.cy, n_buckets=n_buckets, max_blocks=max_blocks,
                 zmax=zmax)
    orc = oracle.OracleVolume(s, mu, 64.0, 0.001, zmax, cam.width, cam.height, cam.fx, cam.fy,
                              cam.cx, cam.cy)
    return vol, orc


def frame(vol, orc, depth, T, fid, R):
    """One fused frame on the GPU (erase, fuse, touched MC extraction) and the same in the
    oracle; returns the oracle's refreshed block set M and removal records of the frame."""
    vol.process_frame(torch.from_numpy(depth).cuda(), T, fid, R)
    if orc is not None:
        if R > 0:   # process_frame takes radius 0 as "no erase"
            orc.erase_radius(T[:, 3], R)
        orc.integrate(depth, T)
        return orc.mc_set(0)
    return None


def result_map(srv, rid):
    """{key: (info, dense 512 cube indices or None for a removal record)} of one result."""
    recs, idx, flags = srv.result(rid)
    recs = recs.cpu().numpy()
    idx = idx.cpu().numpy()
    out = {}
    for i in range(recs.shape[0]):
        k = tuple(int(x) for x in recs[i, :3])
        assert k not in out, f"block {k} served twice"
        info = int(recs[i, 3]) & 0xFFFFFFFF
        out[k] = (info, None if info & V.VBH_REC_REMOVED else idx[i].copy())
    return out, flags


def apply(replica, m, flags):
    if flags & V.VBH_SERVE_RESET:
        replica.clear()
    for k, (info, d) in m.items():
        if d is None:
            replica.pop(k, None)
        else:
            replica[k] = (info, d)


def all_blocks_dense(vol):
    s = vol.extract(V.VBH_MC_ALL)
    out = {}
    for k, (info, loc, idx) in s.to_host().items():
        d = np.zeros(512, np.uint8)
        d[loc.astype(np.int64)] = idx
        out[k] = (info, d)
    return out


def assert_matches_model(replica, vol, orc):
    model = all_blocks_dense(vol)
    assert set(replica) == set(model)
    for k, (info, d) in model.items():
        assert replica[k][0] == info, k
        np.testing.assert_array_equal(replica[k][1], d, err_msg=str(k))
    if orc is not None and model:
        keys = np.array(sorted(model), np.int32)
        idx, margin = orc.mc_dense(keys)
        for b, k in enumerate(map(tuple, keys.tolist())):
            sel = margin[b] > MC_MARGIN
            assert np.array_equal(replica[k][1][sel], idx[b][sel]), k


def consume(srv, n, timeout_s=120.0):
    """Step the loop, reading and releasing each result as it completes (as a server that
    sends results on frees their buffer), until n requests are done."""
    import time
    out = {}
    t0 = time.time()
    while len(out) < n:
        srv.step()
        for d in srv.poll():
            m, flags = result_map(srv, d["id"])
            srv.release(d["id"])
            out[d["id"]] = (d, m, flags)
        assert time.time() - t0 < timeout_s, "serving loop made no progress"
    return out


def serve_one(srv, client):
    rid = srv.submit(client)
    done = srv.drain()
    assert [d["id"] for d in done] == [rid]
    m, flags = result_map(srv, rid)
    srv.release(rid)
    return done[0], m, flags


@pytest.fixture(scope="module")
def room():
    cam, poses, depth = synth.room_sequence(n_frames=12, width=160, height=120)
    return cam, poses, depth


def test_reset_request_serves_the_full_model(room):
    """A new client (version 0) receives every live block -- the oracle's MC indices at every
    cube with all corners clear of the margin, and exactly the MC_ALL extraction."""
    from paper_1805_03709_b300.serve import Server
    cam, poses, depth = room
    vol, orc = make_volume(cam, 0.005, 0.02, 1 << 16, 1 << 17, 4.0)
    for i in range(3):
        frame(vol, orc, depth[i], poses[i], i + 1, 2.5)
    srv = Server(vol, n_clients=4, budget_bytes=1 << 28, log_bits=20)
    d, m, flags = serve_one(srv, 0)
    assert flags & V.VBH_SERVE_RESET and d["flags"] == V.VBH_SERVE_RESET
    assert d["v_after"] == srv.stats()["sigma"] and d["n_records"] == len(m) > 1000
    replica = {}
    apply(replica, m, flags)
    assert_matches_model(replica, vol, orc)
    assert srv.versions()[0] == d["v_after"]
    srv.close()
    vol.close()


def test_deltas_match_the_oracle_frame_sets(room):
    """From a version taken after frame a, a request after frame b holds exactly the oracle's
    blocks refreshed in frames a+1..b that are live at b (info = the last frame that refreshed
    them, MC indices as the oracle's at every cube clear of the margin) and removal records
    for the keys removed in those frames that are not live at b."""
    from paper_1805_03709_b300.serve import Server
    cam, poses, depth = room
    vol, orc = make_volume(cam, 0.005, 0.02, 1 << 16, 1 << 17, 4.0)
    frame(vol, orc, depth[0], poses[0], 1, 2.5)
    srv = Server(vol, n_clients=4, budget_bytes=1 << 28, log_bits=20)
    sigma = {0: srv.stats()["sigma"]}
    Ms, Rs = {}, {}
    for i in range(1, len(poses)):
        M, R = frame(vol, orc, depth[i], poses[i], i + 1, 2.5)
        Ms[i] = set(map(tuple, M.tolist()))
        Rs[i] = set(map(tuple, R.tolist()))
        sigma[i] = srv.stats()["sigma"]
    b = len(poses) - 1
    live = set(map(tuple, orc.dump()[0].tolist()))
    removed_seen = 0
    for c, a in enumerate((0, 4, 8, b - 1)):
        srv.set_versions([c], [sigma[a]])
        d, m, flags = serve_one(srv, c)
        assert flags == 0 and d["v_after"] == sigma[b]
        exp_live = {k for f in range(a + 1, b + 1) for k in Ms[f]} & live
        exp_rem = {k for f in range(a + 1, b + 1) for k in Rs[f]} - live
        got_live = {k for k, v in m.items() if v[1] is not None}
        got_rem = {k for k, v in m.items() if v[1] is None}
        assert got_live == exp_live
        assert got_rem == exp_rem
        removed_seen += len(got_rem)
        for k in got_live:
            last = max(f for f in range(a + 1, b + 1) if k in Ms[f])
            assert m[k][0] == last + 1, k
        keys = np.array(sorted(got_live), np.int32)
        idx, margin = orc.mc_dense(keys)
        for j, k in enumerate(map(tuple, keys.tolist())):
            sel = margin[j] > MC_MARGIN
            assert np.array_equal(m[k][1][sel], idx[j][sel]), k
    assert removed_seen > 0
    srv.close()
    vol.close()


def test_replicas_converge_through_deltas_and_removals(room):
    """Clients that ask at different rates (every frame, every third frame, one that reconnects
    with version 0) hold, after a final request, exactly the server's model; removal records
    are served for erased blocks."""
    from paper_1805_03709_b300.serve import Server
    cam, poses, depth = room
    vol, orc = make_volume(cam, 0.005, 0.02, 1 << 16, 1 << 17, 4.0)
    frame(vol, orc, depth[0], poses[0], 1, 2.5)
    srv = Server(vol, n_clients=3, budget_bytes=1 << 28, log_bits=20)
    replicas = [dict(), dict(), dict()]
    removals = 0
    for i in range(1, len(poses)):
        frame(vol, orc, depth[i], poses[i], i + 1, 2.5)
        asking = [0] + ([1] if i % 3 == 0 else [])
        if i == 7:
            srv.set_versions([2], [0])   # client 2 reconnects
            replicas[2] = {}
        if i % 4 == 0:
            asking.append(2)
        for c in asking:
            d, m, flags = serve_one(srv, c)
            assert not (flags & ~V.VBH_SERVE_RESET)
            removals += sum(1 for v in m.values() if v[1] is None)
            apply(replicas[c], m, flags)
    for c in range(3):
        d, m, flags = serve_one(srv, c)
        apply(replicas[c], m, flags)
        assert_matches_model(replicas[c], vol, orc if c == 0 else None)
    assert removals > 0
    st = srv.stats()
    assert st["err_flags"] == 0
    srv.close()
    vol.close()


def test_every_request_is_the_same_alone_and_in_the_mix(room):
    """32 clients with log-uniform backlogs (plus two resets) served by continuous batching --
    chunks of 256 change records, at most 2048 per iteration, a budget that defers admissions --
    then each request served again alone (unbatched, unchunked) from the same version at the
    same snapshot: identical as maps, and each log request holds exactly its backlog."""
    from paper_1805_03709_b300.serve import Server
    cam, poses, depth = room
    vol, orc = make_volume(cam, 0.005, 0.02, 1 << 16, 1 << 17, 4.0)
    frame(vol, None, depth[0], poses[0], 1, 2.5)
    srv = Server(vol, n_clients=34, max_batch=16, chunk_records=256, iter_records=2048,
                 budget_bytes=(1 << 17) * 528 + (1 << 20), bypass_iters=4, log_bits=20)
    for i in range(1, 10):
        frame(vol, None, depth[i], poses[i], i + 1, 2.5)
    torch.cuda.synchronize()
    live = vol.counters().live
    rng = np.random.default_rng(5)
    backlog = np.exp(rng.uniform(0, np.log(min(50000, live)), 32)).astype(np.int64)
    v0 = srv.versions_for_backlog(backlog)
    clients = np.arange(34)
    versions = np.concatenate([v0, [0, 0]]).astype(np.uint32)
    srv.set_versions(clients, versions)
    ids = {srv.submit(int(c)): int(c) for c in clients}
    got = consume(srv, len(ids))
    assert set(got) == set(ids)
    st = srv.stats()
    assert st["deferred_memory"] > 0 and st["bytes_peak"] <= (1 << 17) * 528 + (1 << 20)
    assert st["iterations"] > len(ids)
    mix = {ids[rid]: v for rid, v in got.items()}
    srv.set_policy(max_batch=1, chunk_records=0, iter_records=0)
    for c in clients.tolist():
        d0, m0, f0 = mix[c]
        assert d0["v_before"] == versions[c]
        if c < 32:
            assert not (f0 & V.VBH_SERVE_RESET)
            assert sum(1 for v in m0.values() if v[1] is not None) == min(int(backlog[c]), live)
        else:
            assert f0 & V.VBH_SERVE_RESET and len(m0) == live
        srv.set_versions([c], [versions[c]])
        d1, m1, f1 = serve_one(srv, c)
        assert (f1, d1["v_after"], d1["n_records"]) == (f0, d0["v_after"], d0["n_records"])
        assert m1.keys() == m0.keys()
        for k in m0:
            assert m1[k][0] == m0[k][0]
            assert (m1[k][1] is None) == (m0[k][1] is None)
            if m0[k][1] is not None:
                np.testing.assert_array_equal(m1[k][1], m0[k][1])
    srv.close()
    vol.close()


def test_budget_cuts_a_range_into_partial_requests():
    """A budget of one full model (528 B x max_blocks) cannot hold a range of more change
    records than that: the request is cut (VBH_SERVE_PARTIAL) and the client's next requests
    continue from where it stopped, ending with the server's model."""
    from paper_1805_03709_b300.serve import Server
    cam, poses, depth = synth.tiny_sequence(n_frames=10)
    vol, orc = make_volume(cam, 0.01, 0.04, 1 << 14, 1 << 13, 0.0)
    frame(vol, orc, depth[0], poses[0], 1, 0.0)
    srv = Server(vol, n_clients=2, budget_bytes=(1 << 13) * 528, log_bits=17)
    d, m, flags = serve_one(srv, 0)
    replica = {}
    apply(replica, m, flags)
    for i in range(1, 10):
        frame(vol, orc, depth[i], poses[i], i + 1, 0.0)
    sigma = srv.stats()["sigma"]
    assert sigma - d["v_after"] > (1 << 13)
    partial = 0
    while True:
        d, m, flags = serve_one(srv, 0)
        apply(replica, m, flags)
        partial += bool(flags & V.VBH_SERVE_PARTIAL)
        assert d["v_after"] - d["v_before"] <= (1 << 13)
        if d["v_after"] == sigma:
            break
    assert partial >= 1
    assert_matches_model(replica, vol, orc)
    srv.close()
    vol.close()


def test_realtime_loop_serves_every_request(room):
    """vbh_serve_run: frames every 33 ms and Poisson arrivals of 8 clients; every request
    completes without error, after it arrived, and the clients end at the last snapshot."""
    from paper_1805_03709_b300.serve import Server
    cam, poses, depth = room
    vol, _ = make_volume(cam, 0.005, 0.02, 1 << 16, 1 << 17, 4.0)
    frame(vol, None, depth[0], poses[0], 1, 2.5)
    srv = Server(vol, n_clients=8, max_batch=8, chunk_records=4096, budget_bytes=1 << 28,
                 log_bits=20)
    rng = np.random.default_rng(9)
    ev = [(int(33e6 * k), -1) for k in range(1, 10)]
    for c in range(8):
        t = np.cumsum(rng.exponential(1 / 40.0, 16)) * 1e9
        ev += [(int(x), c) for x in t if x < 3.2e8]
    ev += [(int(3.4e8 + c), c) for c in range(8)]   # a final request each, after the last frame
    ev.sort()
    t_ns = [e[0] for e in ev]
    cl = [e[1] for e in ev]
    D = [torch.from_numpy(depth[i]).cuda() for i in range(1, 10)]
    done = srv.run(t_ns, cl, D, poses[1:10], list(range(2, 11)), erase_radius=2.5)
    assert len(done) == sum(1 for c in cl if c >= 0)
    for d in done:
        assert d["flags"] & ~V.VBH_SERVE_RESET == 0
        assert d["t_done_ns"] >= d["t_admit_ns"] >= d["t_arrival_ns"]
    sigma = srv.stats()["sigma"]
    assert (srv.versions() == sigma).all()
    srv.close()
    vol.close()
