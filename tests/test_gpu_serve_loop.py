"""GPU tests of the device-resident serving loop (vbh_serve_loop_*): one persistent kernel that
admits, batches and serves client requests while frames keep running.  Its results are checked
against the oracle's per-frame sets and against the host scheduler's results for the same
requests alone; clients that ask while frames are fused concurrently converge to the model; a
host that falls silent makes the loop's bounded waits run out (VBH_ERR_TIMEOUT, no hang) and
the server is usable again afterwards.

While a loop runs these tests synchronise streams only: a device-wide synchronisation would
wait for the persistent kernel."""
import time

import numpy as np
import pytest
import torch

from paper_1805_03709_b300 import synth, vbh as V
from test_gpu_serve import (MC_MARGIN, all_blocks_dense, apply, assert_matches_model, frame,
                            make_volume, result_map, serve_one)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1805_03709_b300 import build
    build.build()
    assert torch.cuda.is_available()


@pytest.fixture(scope="module")
def room():
    cam, poses, depth = synth.room_sequence(n_frames=12, width=160, height=120)
    return cam, poses, depth


def collect(loop, ids, timeout_s=60.0):
    """Poll the loop until every request id in `ids` has completed; read and release each
    result as it arrives.  Returns {id: (done dict, result map, flags)}."""
    out = {}
    t0 = time.time()
    while len(out) < len(ids):
        for d in loop.poll():
            m, flags = result_map(loop, d["id"])
            loop.release(d["id"])
            out[d["id"]] = (d, m, flags)
        assert time.time() - t0 < timeout_s, "device loop made no progress"
    assert set(out) == set(ids)
    return out


def test_loop_deltas_and_reset_match_the_oracle(room):
    """Four clients at versions taken after frames a (deltas) and one new client (reset), all in
    flight in the loop at once: each delta holds exactly the oracle's blocks refreshed in
    frames a+1..b that are live (info = last refreshing frame, MC indices as the oracle's) and
    removal records for the keys removed and not live; the reset is the whole model."""
    from paper_1805_03709_b300.serve import Server, ServeLoop
    cam, poses, depth = room
    vol, orc = make_volume(cam, 0.005, 0.02, 1 << 16, 1 << 17, 4.0)
    frame(vol, orc, depth[0], poses[0], 1, 2.5)
    srv = Server(vol, n_clients=5, budget_bytes=1 << 28, log_bits=20)
    sigma = {0: srv.stats()["sigma"]}
    Ms, Rs = {}, {}
    for i in range(1, len(poses)):
        M, R = frame(vol, orc, depth[i], poses[i], i + 1, 2.5)
        Ms[i] = set(map(tuple, M.tolist()))
        Rs[i] = set(map(tuple, R.tolist()))
        sigma[i] = srv.stats()["sigma"]
    b = len(poses) - 1
    starts = (0, 4, 8, b - 1)
    srv.set_versions(list(range(5)), [sigma[a] for a in starts] + [0])
    loop = ServeLoop(srv, idle_timeout_us=5_000_000)
    with pytest.raises(V.VbhError) as e:   # the host scheduler is not used meanwhile
        srv.submit(0)
    assert e.value.status == V.VBH_ERR_UNSUPPORTED
    ids = {loop.submit(c): c for c in range(5)}
    got = {ids[r]: v for r, v in collect(loop, ids).items()}
    st = loop.stats()
    loop.stop()
    assert st["requests_done"] == 5 and st["launches"] == 1 and st["max_active"] >= 2
    live = set(map(tuple, orc.dump()[0].tolist()))
    removed_seen = 0
    for c, a in enumerate(starts):
        d, m, flags = got[c]
        assert flags == 0 and d["v_before"] == sigma[a] and d["v_after"] == sigma[b]
        exp_live = {k for f in range(a + 1, b + 1) for k in Ms[f]} & live
        exp_rem = {k for f in range(a + 1, b + 1) for k in Rs[f]} - live
        assert {k for k, v in m.items() if v[1] is not None} == exp_live
        assert {k for k, v in m.items() if v[1] is None} == exp_rem
        removed_seen += len(exp_rem)
        for k in exp_live:
            assert m[k][0] == max(f for f in range(a + 1, b + 1) if k in Ms[f]) + 1, k
        keys = np.array(sorted(exp_live), np.int32)
        idx, margin = orc.mc_dense(keys)
        for j, k in enumerate(map(tuple, keys.tolist())):
            sel = margin[j] > MC_MARGIN
            assert np.array_equal(m[k][1][sel], idx[j][sel]), k
    assert removed_seen > 0
    d, m, flags = got[4]
    assert flags == V.VBH_SERVE_RESET and d["v_after"] == sigma[b]
    replica = {}
    apply(replica, m, flags)
    assert_matches_model(replica, vol, orc)
    assert (srv.versions() == sigma[b]).all()
    srv.close()
    vol.close()


def test_loop_every_request_is_the_same_alone_and_in_the_mix(room):
    """32 clients with log-uniform backlogs and two resets in flight together in the device
    loop -- chunks of 256 change records, at most 16 requests at once, a stream buffer that
    defers admissions -- and each request served again alone by the host scheduler (one
    request per launch, unchunked) from the same version at the same snapshot: identical as
    maps, and each log request holds exactly its backlog."""
    from paper_1805_03709_b300.serve import Server, ServeLoop
    cam, poses, depth = room
    vol, _ = make_volume(cam, 0.005, 0.02, 1 << 16, 1 << 17, 4.0)
    frame(vol, None, depth[0], poses[0], 1, 2.5)
    budget = (1 << 17) * 528 + (1 << 20)
    srv = Server(vol, n_clients=34, max_batch=1, budget_bytes=budget, log_bits=20)
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
    loop = ServeLoop(srv, max_slots=16, chunk_records=256, bypass_rounds=4,
                     idle_timeout_us=5_000_000)
    ids = {loop.submit(int(c)): int(c) for c in clients}
    mix = {ids[r]: v for r, v in collect(loop, ids).items()}
    st = loop.stats()
    loop.stop()
    assert st["deferred_memory"] > 0 and st["bytes_peak"] <= budget
    assert st["chunks"] > len(ids) and st["max_active"] > 1 and st["status"] == 0
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


def test_loop_clients_converge_while_frames_run(room):
    """Frames are fused on the volume's stream while three clients' requests run in the loop
    (each request submitted right behind a frame launch, so extraction and serving overlap on
    the GPU); after a last request each, every client's replica is exactly the model, and the
    first one's MC indices are the oracle's."""
    from paper_1805_03709_b300.serve import Server, ServeLoop
    cam, poses, depth = room
    vol, orc = make_volume(cam, 0.005, 0.02, 1 << 16, 1 << 17, 4.0)
    frame(vol, orc, depth[0], poses[0], 1, 2.5)
    srv = Server(vol, n_clients=3, budget_bytes=1 << 28, log_bits=20)
    D = [torch.from_numpy(depth[i]).cuda() for i in range(len(poses))]
    torch.cuda.current_stream().synchronize()
    loop = ServeLoop(srv, idle_timeout_us=5_000_000)
    replicas = [dict(), dict(), dict()]
    removals = 0
    for i in range(1, len(poses)):
        vol.process_frame(D[i], poses[i], i + 1, 2.5)   # asynchronous on the volume's stream
        orc.erase_radius(poses[i][:, 3], 2.5)
        orc.integrate(depth[i], poses[i])
        orc.mc_set(0)
        asking = [0, 1] if i % 2 else [0, 2]
        ids = [loop.submit(c) for c in asking]
        for rid, (d, m, flags) in collect(loop, ids).items():
            assert not (flags & ~V.VBH_SERVE_RESET)
            removals += sum(1 for v in m.values() if v[1] is None)
            apply(replicas[d["client"]], m, flags)
    torch.cuda.current_stream().synchronize()
    ids = [loop.submit(c) for c in range(3)]
    for rid, (d, m, flags) in collect(loop, ids).items():
        apply(replicas[d["client"]], m, flags)
    st = loop.stats()
    loop.stop()
    assert st["status"] == 0 and st["launches"] == 1
    for c in range(3):
        assert_matches_model(replicas[c], vol, orc if c == 0 else None)
    assert removals > 0
    srv.close()
    vol.close()


def test_loop_realtime_script_serves_every_request(room):
    """vbh_serve_loop_run: frames every 33 ms and Poisson arrivals of 8 clients into the device
    loop; every request completes after it arrived (and is admitted in between), and the
    clients end at the last snapshot."""
    from paper_1805_03709_b300.serve import Server, ServeLoop
    cam, poses, depth = room
    vol, _ = make_volume(cam, 0.005, 0.02, 1 << 16, 1 << 17, 4.0)
    frame(vol, None, depth[0], poses[0], 1, 2.5)
    srv = Server(vol, n_clients=8, budget_bytes=1 << 28, log_bits=20)
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
    torch.cuda.current_stream().synchronize()
    loop = ServeLoop(srv, idle_timeout_us=5_000_000)
    done = loop.run(t_ns, cl, D, poses[1:10], list(range(2, 11)), erase_radius=2.5)
    loop.stop()
    assert len(done) == sum(1 for c in cl if c >= 0)
    served = 0
    for d in done:
        assert d["flags"] & ~V.VBH_SERVE_RESET == 0
        # admission time in the host clock from the GPU's admission-to-publication interval
        assert d["t_done_ns"] >= d["t_admit_ns"] >= d["t_arrival_ns"]
        served += d["n_records"] > 0 and d["t_done_ns"] > d["t_admit_ns"]
    assert served > 0   # served requests spent measurable time on the device
    sigma = srv.stats()["sigma"]
    assert (srv.versions() == sigma).all()
    srv.close()
    vol.close()


def test_loop_times_out_when_the_host_falls_silent_and_the_server_recovers(room):
    """A loop whose host makes no call for longer than its idle limit (20 ms here) stops by
    itself: its bounded waits run out, stop() reports VBH_ERR_TIMEOUT, nothing hangs, and a new
    loop on the same server serves requests again."""
    from paper_1805_03709_b300.serve import Server, ServeLoop
    cam, poses, depth = room
    vol, _ = make_volume(cam, 0.005, 0.02, 1 << 16, 1 << 17, 4.0)
    frame(vol, None, depth[0], poses[0], 1, 2.5)
    srv = Server(vol, n_clients=2, budget_bytes=1 << 28, log_bits=20)
    loop = ServeLoop(srv, ctas=4, idle_timeout_us=20_000)
    time.sleep(0.3)                                   # the host falls silent
    with pytest.raises(V.VbhError) as e:
        loop.submit(0)
    assert e.value.status == V.VBH_ERR_TIMEOUT
    with pytest.raises(V.VbhError) as e:
        loop.stop()
    assert e.value.status == V.VBH_ERR_TIMEOUT
    assert float(torch.ones(8, device="cuda").sum()) == 8.0   # the context is fine
    loop2 = ServeLoop(srv, idle_timeout_us=5_000_000)
    rid = loop2.submit(1)
    (d, m, flags), = collect(loop2, [rid]).values()
    loop2.stop()
    assert flags == V.VBH_SERVE_RESET and len(m) == vol.counters().live
    srv.close()
    vol.close()
