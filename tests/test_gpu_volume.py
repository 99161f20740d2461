"""GPU parity of the per-frame path (allocation, fusion, erase, MC extraction; Sec. 4.1, 4.2)
against the CPU oracle on seeded synthetic depth streams, through the C ABI.

Bar: allocated block sets, MC block sets and removal records bit-exact; weights exact; TSDF
values within TSDF_TOL (normalised units, i.e. 1e-5 x truncation in metres); MC indices exact
at every cube whose eight corners have |oracle TSDF| > MC_MARGIN (elsewhere the FP32 sign may
legitimately differ from the FP64 one)."""
import os

import numpy as np
import pytest
import torch

import oracle
from paper_1805_03709_b300 import synth
from paper_1805_03709_b300 import vbh as V

pytestmark = pytest.mark.gpu

TSDF_TOL = 1e-5
MC_MARGIN = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1805_03709_b300 import build
    build.build()
    assert torch.cuda.is_available()


def make_pair(cam, s, mu, n_buckets, max_blocks, zmax=0.0, hash_fn=V.VBH_HASH_MIX, **kw):
    from paper_1805_03709_b300.volume import Volume
    vol = Volume(voxel_size=s, trunc=mu, width=cam.width, height=cam.height, fx=cam.fx,
                 fy=cam.fy, cx=cam.cx, cy=cam.cy, n_buckets=n_buckets, max_blocks=max_blocks,
                 zmax=zmax, hash_fn=hash_fn, **kw)
    orc = oracle.OracleVolume(s, mu, 64.0, 0.001, zmax, cam.width, cam.height, cam.fx, cam.fy,
                              cam.cx, cam.cy)
    return vol, orc


def compare_volume(vol, orc):
    kg, Fg, Wg = vol.dump()
    ko, Fo, Wo = orc.dump()
    np.testing.assert_array_equal(kg, ko)
    np.testing.assert_array_equal(Wg, Wo.astype(np.float32))
    if len(ko):
        err = np.abs(Fg.astype(np.float64) - Fo)
        assert err.max() <= TSDF_TOL, f"max TSDF error {err.max():.3e}"
    return ko


def dense_from_records(recs, key):
    dense = np.zeros(512, np.uint8)
    _, loc, idx = recs[key]
    dense[loc.astype(np.int64)] = idx
    assert np.all(idx != 0) and np.all(idx != 255)
    return dense


def compare_mc(recs, orc, keys, removed=()):
    keys = np.asarray(keys, np.int32).reshape(-1, 3)
    live = {k: r for k, r in recs.items() if not (r[0] & V.VBH_REC_REMOVED)}
    tomb = {k for k, r in recs.items() if r[0] & V.VBH_REC_REMOVED}
    assert set(live) == set(map(tuple, keys.tolist()))
    assert tomb == set(map(tuple, np.asarray(removed).reshape(-1, 3).tolist()))
    if not len(keys):
        return 0
    idx, margin = orc.mc_dense(keys)
    checked = 0
    for b, k in enumerate(map(tuple, keys.tolist())):
        d = dense_from_records(live, k)
        sel = margin[b] > MC_MARGIN
        mism = np.nonzero(d[sel] != idx[b][sel])[0]
        assert mism.size == 0, f"block {k}: {mism.size} MC indices differ"
        checked += int(sel.sum())
    return checked


def run_sequence(vol, orc, depth, poses, erase_radius=None, check_every=1):
    for i in range(len(poses)):
        T = poses[i]
        if erase_radius is not None:
            vol.erase_radius(T[:, 3], erase_radius)
            gone_o = orc.erase_radius(T[:, 3], erase_radius)
            gone_g = vol.erased()
            assert {tuple(k) for k in gone_g.tolist()} == {tuple(k) for k in gone_o.tolist()}
        d = torch.from_numpy(depth[i]).cuda()
        st = vol.integrate(d, T, i + 1, stats=True)
        n_o = orc.integrate(depth[i], T)
        assert st.touched == n_o
        assert st.error_flags == 0
        s = vol.extract(V.VBH_MC_TOUCHED)
        M, rem = orc.mc_set(0)
        recs = s.to_host()
        assert all((r[0] & 0x7FFFFFFF) == i + 1 for r in recs.values())
        if i % check_every == 0 or i == len(poses) - 1:
            compare_volume(vol, orc)
            compare_mc(recs, orc, M, rem)
        else:
            live = {k for k, r in recs.items() if not (r[0] & V.VBH_REC_REMOVED)}
            assert live == set(map(tuple, M.tolist()))


def test_tiny_sequence_full_parity():
    """10 frames of 160 x 120 (f = 140), voxel 1 cm, truncation 4 cm, 2^16 x 4 table."""
    cam, poses, depth = synth.tiny_sequence()
    vol, orc = make_pair(cam, 0.01, 0.04, 1 << 16, 1 << 15)
    run_sequence(vol, orc, depth, poses)
    # whole-model extraction at the end
    s = vol.extract(V.VBH_MC_ALL)
    full, _ = orc.mc_set(1)
    n = compare_mc(s.to_host(), orc, full)
    assert n > 100000


@pytest.mark.parametrize("width,height", [(157, 113), (33, 17), (16, 1)])
def test_ragged_image_sizes(width, height):
    """Image sides that are no multiple of the band allocation's 16 x 16 pixel tiles (partial
    tiles in both directions, odd sides) and a one-row image: the separate calls and the frame
    graph both give the oracle's volume and MC blocks."""
    cam, poses, depth = synth.tiny_sequence(n_frames=4, width=width, height=height,
                                            f=140.0 * width / 160.0)
    vol, orc = make_pair(cam, 0.01, 0.04, 1 << 14, 1 << 13)
    run_sequence(vol, orc, depth, poses)
    vg, og = make_pair(cam, 0.01, 0.04, 1 << 14, 1 << 13)
    for i in range(len(poses)):
        vg.process_frame(torch.from_numpy(depth[i]).cuda(), poses[i], i + 1, 0.0)
        og.integrate(depth[i], poses[i])
    torch.cuda.synchronize()
    compare_volume(vg, og)
    assert vg.counters().error_flags == 0


@pytest.mark.parametrize("hash_fn", [V.VBH_HASH_MIX, V.VBH_HASH_PRIMES])
def test_room_reduced_with_erase(hash_fn):
    """Room scene at 160 x 120 (f scaled to 131.25), voxel 5 mm, truncation 2 cm, zmax 4 m,
    erase radius 2.5 m so blocks are removed and re-allocated every frame."""
    cam, poses, depth = synth.room_sequence(n_frames=8, width=160, height=120)
    vol, orc = make_pair(cam, 0.005, 0.02, 1 << 16, 1 << 17, zmax=4.0, hash_fn=hash_fn)
    run_sequence(vol, orc, depth, poses, erase_radius=2.5)


def test_room_full_size_frames():
    """640 x 480 (f = 525) room frames with the full configuration: 2^22 x 4 table, 2^19-block
    pool, voxel 5 mm, truncation 2 cm, blocks beyond 4 m erased each frame."""
    cam, poses, depth = synth.room_sequence(n_frames=40)
    sel = [0, 1, 39]
    vol, orc = make_pair(cam, 0.005, 0.02, 1 << 22, 1 << 19, zmax=4.0)
    run_sequence(vol, orc, depth[sel], poses[sel], erase_radius=4.0)


def test_room_full_size_long_sequence():
    """130 consecutive 640 x 480 frames of the room walk with the full configuration (2^22 x 4
    table, 2^19-block pool, voxel 5 mm, truncation 2 cm, 4 m erase from frame 46 on): touched
    counts, erased sets and MC block sets every frame; the whole volume (TSDF within 1e-5,
    weights exact) and every MC index at frames 0, 20, ..., 120 and 129.  Long sequences are
    where FP32 running-average error would compound."""
    ncpu = os.cpu_count() or 1
    cam, poses, depth = synth.room_sequence(n_frames=130, workers=min(8, ncpu))
    oracle.set_threads(ncpu)
    try:
        vol, orc = make_pair(cam, 0.005, 0.02, 1 << 22, 1 << 19, zmax=4.0)
        run_sequence(vol, orc, depth, poses, erase_radius=4.0, check_every=20)
        assert vol.counters().total_frames == 130
        _, _, W = orc.dump()
        assert W.max() >= 20       # voxels seen by many frames of the walk carry long histories
    finally:
        oracle.set_threads(1)


def test_weight_cap_static_pose_80_frames():
    """A camera held still for 80 noisy frames (the noise differs per frame): every voxel in view
    is fused once per frame, so its weight reaches the cap Wmax = 64 at frame 64 and the capped
    running average F <- (64 F + f) / 65 runs over the last 16 frames.  Volume and MC indices
    against the oracle at frames 1, 20, 40, 63, 64, 65, 72 and 80."""
    cam, T, depth = synth.room_static_frames(80)
    vol, orc = make_pair(cam, 0.005, 0.02, 1 << 16, 1 << 16, zmax=4.0)
    check = {1, 20, 40, 63, 64, 65, 72, 80}
    at64 = None
    for i in range(80):
        st = vol.integrate(torch.from_numpy(depth[i]).cuda(), T, i + 1, stats=True)
        assert st.touched == orc.integrate(depth[i], T) and st.error_flags == 0
        s = vol.extract(V.VBH_MC_TOUCHED)
        M, rem = orc.mc_set(0)
        if i + 1 in check:
            compare_volume(vol, orc)
            compare_mc(s.to_host(), orc, M, rem)
        if i + 1 == 64:
            at64 = orc.dump()
    k, F, W = orc.dump()
    pos = {tuple(b): i for i, b in enumerate(k.tolist())}
    sel = np.array([pos[tuple(b)] for b in at64[0].tolist()])   # blocks live at frame 64
    capped = (at64[2] == 64) & (W[sel] == 64)
    assert capped.sum() > 50000                   # voxels that ran 16 capped updates
    assert (np.abs(F[sel] - at64[1])[capped] > 1e-3).mean() > 0.5   # ... which moved their values


@pytest.mark.parametrize("wset", [(63.0,), (64.0,), (0.0, 1.0, 62.0, 63.0, 64.0)])
def test_loaded_weights_at_the_cap_then_frames(wset):
    """Blocks uploaded with weights at (64) and just below (63) the cap, then fused by three
    frames: the first update of a W = 63 voxel reaches the cap, a W = 64 voxel takes the capped
    average (64 F + f) / 65 at once.  Volume and MC indices against the oracle after each frame."""
    cam, poses, depth = synth.room_sequence(n_frames=3, width=160, height=120)
    vol, orc = make_pair(cam, 0.005, 0.02, 1 << 16, 1 << 16, zmax=4.0)
    keys = orc.alloc_keys(depth[0], poses[0])
    rng = np.random.default_rng(64)
    F = rng.uniform(-1.0, 1.0, (len(keys), 512)).astype(np.float32)
    W = rng.choice(np.array(wset, np.float32), (len(keys), 512))
    F[W == 0] = 0.0
    vol.load(keys, F, W)
    orc.load(keys, F.astype(np.float64), W.astype(np.float64))
    compare_volume(vol, orc)
    for i in range(3):
        st = vol.integrate(torch.from_numpy(depth[i]).cuda(), poses[i], i + 1, stats=True)
        assert st.touched == orc.integrate(depth[i], poses[i]) and st.error_flags == 0
        s = vol.extract(V.VBH_MC_TOUCHED)
        M, rem = orc.mc_set(0)
        compare_volume(vol, orc)
        compare_mc(s.to_host(), orc, M, rem)
    _, Fo, Wo = orc.dump()
    assert Wo.max() == 64.0
    if 64.0 in wset:
        assert Wo.min() >= 0.0 and (Wo == 64.0).mean() > 0.3


def test_empty_and_out_of_range_frames():
    cam, poses, depth = synth.tiny_sequence(n_frames=1)
    vol, orc = make_pair(cam, 0.01, 0.04, 1 << 12, 1 << 12, zmax=1.0)
    z = torch.zeros((cam.height, cam.width), dtype=torch.uint16, device="cuda")
    st = vol.integrate(z, poses[0], 1, stats=True)
    assert st.touched == 0 and st.new_blocks == 0
    far = torch.full((cam.height, cam.width), 1500, dtype=torch.uint16, device="cuda")
    st = vol.integrate(far, poses[0], 2, stats=True)     # every pixel beyond zmax
    assert st.touched == 0
    recs = vol.extract(V.VBH_MC_TOUCHED).to_host()
    assert recs == {}
    assert vol.counters().live == 0


def test_pool_exhaustion_fuses_what_fits():
    cam, poses, depth = synth.tiny_sequence(n_frames=1)
    vol, orc = make_pair(cam, 0.01, 0.04, 1 << 12, 300)
    with pytest.raises(V.VbhError) as e:
        vol.integrate(torch.from_numpy(depth[0]).cuda(), poses[0], 1, stats=True)
    assert e.value.status == V.VBH_ERR_CAPACITY
    orc.integrate(depth[0], poses[0])
    assert len(orc) > 300
    kg, Fg, Wg = vol.dump()
    ko, Fo, Wo = orc.dump()
    assert len(kg) == 300 and vol.counters().free_blocks == 0
    pos = {tuple(k): i for i, k in enumerate(ko.tolist())}
    idx = np.array([pos[tuple(k)] for k in kg.tolist()])     # every GPU block is an oracle block
    np.testing.assert_array_equal(Wg, Wo[idx].astype(np.float32))
    assert np.abs(Fg - Fo[idx]).max() <= TSDF_TOL


def sphere_blocks(s=0.01, mu=0.04, r=0.23, c=(0.011, -0.017, 0.006), span=range(-5, 5)):
    keys = np.array([(x, y, z) for x in span for y in span for z in span], np.int32)
    l = np.arange(512)
    loc = np.stack([l % 8, (l // 8) % 8, l // 64], -1)
    g = keys[:, None, :].astype(np.float64) * 8 + loc[None]
    F = np.clip((np.linalg.norm(g * np.float32(s) - np.array(c), axis=-1) - r) / mu, -1, 1)
    F = F.astype(np.float32)
    W = np.ones_like(F)
    W[:, ::97] = 0.0          # sprinkle invalid voxels
    return keys, F, W


def test_loaded_sphere_all_keys_since_modes():
    keys, F, W = sphere_blocks()
    cam = synth.Camera(8, 8, 4.0, 4.0, 4.0, 4.0)
    vol, orc = make_pair(cam, 0.01, 0.04, 1 << 12, 4096)
    vol.load(keys, F, W)
    orc.load(keys, F.astype(np.float64), W.astype(np.float64))
    compare_volume(vol, orc)
    s = vol.extract(V.VBH_MC_ALL)
    assert compare_mc(s.to_host(), orc, keys) > 50000
    # KEYS: the given blocks and their seven negative neighbours (live ones)
    pick = keys[::37][:20]
    live = {tuple(k) for k in keys.tolist()}
    expect = {(k[0] - ox, k[1] - oy, k[2] - oz) for k in pick.tolist()
              for ox in (0, 1) for oy in (0, 1) for oz in (0, 1)} & live
    s = vol.extract(V.VBH_MC_KEYS, keys3=torch.from_numpy(pick).cuda())
    compare_mc(s.to_host(), orc, sorted(expect))
    # SINCE: loaded blocks carry version 0, so nothing is newer than 0
    assert vol.extract(V.VBH_MC_SINCE, since=0).to_host() == {}


def test_erase_keys_and_removal_records():
    keys, F, W = sphere_blocks(span=range(-2, 2))
    cam = synth.Camera(8, 8, 4.0, 4.0, 4.0, 4.0)
    vol, orc = make_pair(cam, 0.01, 0.04, 1 << 10, 256)
    vol.load(keys, F, W)
    orc.load(keys, F.astype(np.float64), W.astype(np.float64))
    gone = np.array([[0, 0, 0], [1, 1, 1], [7, 7, 7]], np.int32)   # (7,7,7) is absent
    vol.erase_keys(torch.from_numpy(gone).cuda())
    assert orc.erase_keys(gone) == 2
    assert {tuple(k) for k in vol.erased().tolist()} == {(0, 0, 0), (1, 1, 1)}
    s = vol.extract(V.VBH_MC_TOUCHED)
    M, rem = orc.mc_set(0)
    compare_mc(s.to_host(), orc, M, rem)
    compare_volume(vol, orc)
    assert vol.counters().free_blocks == 256 - len(keys) + 2


def test_stream_too_small_reports_needed_bytes():
    keys, F, W = sphere_blocks(span=range(-2, 2))
    cam = synth.Camera(8, 8, 4.0, 4.0, 4.0, 4.0)
    from paper_1805_03709_b300.volume import McStream
    vol, _ = make_pair(cam, 0.01, 0.04, 1 << 10, 256)
    vol.load(keys, F, W)
    small = McStream.allocate(4, 100)
    with pytest.raises(V.VbhError) as e:
        vol.extract(V.VBH_MC_ALL, stream=small, sync=True)
    assert e.value.status == V.VBH_ERR_BUFFER_TOO_SMALL
    s, need = vol.extract(V.VBH_MC_ALL, sync=True)
    nb, ne = s.n.cpu().tolist()
    assert nb == len(keys) and need == nb * 24 + ne * 3


def test_version_stamps_since_mode():
    cam, poses, depth = synth.tiny_sequence(n_frames=3)
    vol, orc = make_pair(cam, 0.01, 0.04, 1 << 14, 1 << 14)
    last = None
    for i in range(3):
        vol.integrate(torch.from_numpy(depth[i]).cuda(), poses[i], 10 + i)
        last = {k for k, r in vol.extract(V.VBH_MC_TOUCHED).to_host().items()}
    since = vol.extract(V.VBH_MC_SINCE, since=11).to_host()
    assert set(since) == last
    assert all(r[0] == 12 for r in since.values())


@pytest.mark.parametrize("timed", [False, True])
def test_process_frame_graph_matches_oracle_and_separate_calls(timed):
    """vbh_process_frame (one CUDA graph per frame) against the oracle, and bit-identical to the
    three separate calls on a second volume."""
    cam, poses, depth = synth.room_sequence(n_frames=8, width=160, height=120)
    g, orc = make_pair(cam, 0.005, 0.02, 1 << 16, 1 << 17, zmax=4.0)
    sep, _ = make_pair(cam, 0.005, 0.02, 1 << 16, 1 << 17, zmax=4.0)
    if timed:
        g.timing(("integrate",))
    from paper_1805_03709_b300.volume import McStream
    s2 = McStream.allocate(1 << 17, 1 << 22)
    for i in range(len(poses)):
        d = torch.from_numpy(depth[i]).cuda()
        rg = g.process_frame(d, poses[i], i + 1, 2.5).to_host()
        sep.erase_radius(poses[i][:, 3], 2.5)
        sep.integrate(d, poses[i], i + 1)
        rs = sep.extract(V.VBH_MC_TOUCHED, stream=s2).to_host()
        orc.erase_radius(poses[i][:, 3], 2.5)
        orc.integrate(depth[i], poses[i])
        M, rem = orc.mc_set(0)
        compare_mc(rg, orc, M, rem)
        assert set(rg) == set(rs)
        for k in rg:
            assert rg[k][0] == rs[k][0]
            np.testing.assert_array_equal(dense_from_records(rg, k), dense_from_records(rs, k))
        kg, Fg, Wg = g.dump()
        ks, Fs, Ws = sep.dump()
        np.testing.assert_array_equal(kg, ks)
        np.testing.assert_array_equal(Fg, Fs)
        np.testing.assert_array_equal(Wg, Ws)
    compare_volume(g, orc)
    if timed:
        ms, n = g.timing_read()
        assert n["integrate"] == len(poses) and ms["integrate"] > 0
    c0 = g.counters().kernel_launches
    g.process_frame(torch.from_numpy(depth[0]).cuda(), poses[0], 99, 2.5)
    assert g.counters().kernel_launches - c0 == 8      # one graph: 8 kernels
