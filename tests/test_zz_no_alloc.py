"""The allocation-free entry point vbh_mc_from_tsdf_static against the handle-based path.

vbh_mc_from_tsdf_static exists for callers that cannot call cudaMalloc (code living inside
another framework's memory pool, real-time threads that must not risk an allocation's
device-wide synchronisation, hosts that reserve all GPU memory up front): they cannot create a
vbh_handle, so the function takes their own device buffers and keeps its scratch in a fixed
array inside the library.  This file checks, through the C ABI, that two calls in a row produce
exactly the stream the existing path produces (vbh_load + vbh_extract_mc_indices with
VBH_MC_ALL) for the same blocks -- MC indices are integers, so the comparison is exact -- and
that sizes above the fixed limit are refused.  It is collected last on purpose.
"""
import numpy as np
import pytest
import torch

from paper_1805_03709_b300 import vbh as V

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1805_03709_b300 import build
    build.build()
    assert torch.cuda.is_available()


def sphere_blocks(span, centre, r, s=0.01, mu=0.04, hole_stride=97):
    keys = np.array([(x, y, z) for x in span for y in span for z in span], np.int32)
    l = np.arange(512)
    loc = np.stack([l % 8, (l // 8) % 8, l // 64], -1)
    g = keys[:, None, :].astype(np.float64) * 8 + loc[None]
    F = np.clip((np.linalg.norm(g * s - np.array(centre), axis=-1) - r) / mu, -1, 1)
    W = np.ones_like(F)
    W[:, ::hole_stride] = 0.0
    return keys, F.astype(np.float32), W.astype(np.float32)


def dense(recs):
    out = {}
    for k, (info, loc, idx) in recs.items():
        d = np.zeros(512, np.uint8)
        d[loc.astype(np.int64)] = idx
        assert np.all(idx != 0) and np.all(idx != 255)
        out[k] = (info, d)
    return out


def reference_stream(keys, F, W):
    """The existing path: a handle holding exactly these blocks, whole-volume extraction."""
    from paper_1805_03709_b300.volume import Volume
    vol = Volume(voxel_size=0.01, trunc=0.04, width=8, height=8, fx=4.0, fy=4.0, cx=4.0, cy=4.0,
                 n_buckets=1 << 12, max_blocks=4096)
    vol.load(keys, F, W)
    recs = vol.extract(V.VBH_MC_ALL).to_host()
    vol.close()
    return dense(recs)


def static_stream(keys, F, W, stream):
    from paper_1805_03709_b300.volume import McStream
    out = McStream.allocate(len(keys), len(keys) * 512)
    err = torch.full((1,), 77, dtype=torch.int32, device="cuda")
    K = torch.from_numpy(keys).cuda()
    Ft = torch.from_numpy(F).cuda()
    Wt = torch.from_numpy(W).cuda()
    V.vbh_mc_from_tsdf_static(K, Ft, Wt, out.c_struct(), stream, err)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    return dense(out.to_host())


def test_static_matches_handle_path_twice_in_a_row():
    stream = torch.cuda.current_stream().cuda_stream
    cases = [sphere_blocks(range(-5, 5), (0.013, -0.021, 0.007), 0.23),
             sphere_blocks(range(-3, 4), (0.05, 0.02, -0.03), 0.11, hole_stride=61)]
    for keys, F, W in cases:               # second call reuses the scratch of the first
        got = static_stream(keys, F, W, stream)
        want = reference_stream(keys, F, W)
        assert set(got) == set(want) == {tuple(k) for k in keys.tolist()}
        for k in want:
            assert got[k][0] == want[k][0]
            np.testing.assert_array_equal(got[k][1], want[k][1])
        assert sum(int(np.count_nonzero(d)) for _, d in got.values()) > 1000


def test_static_rejects_sizes_above_its_scratch():
    from paper_1805_03709_b300.volume import McStream
    n = (1 << 15) + 1
    keys = torch.zeros((n, 3), dtype=torch.int32, device="cuda")
    F = torch.zeros((n, 512), dtype=torch.float32, device="cuda")
    out = McStream.allocate(4, 4)
    with pytest.raises(V.VbhError) as e:
        V.vbh_mc_from_tsdf_static(keys, F, F, out.c_struct(), None)
    assert e.value.status == V.VBH_ERR_INVALID_ARG


def _raw(out, keys):
    """Records as written (no overflow check): totals and per-record (key, offset, count)."""
    nb, ne = (int(x) & 0xFFFFFFFF for x in out.n.cpu().tolist())
    nrec = min(nb, out.info.shape[0])
    k = out.keys3[:nrec].cpu().numpy()
    off = out.offsets[:nrec].cpu().numpy().view(np.uint32)
    cnt = out.counts[:nrec].cpu().numpy().view(np.uint32)
    loc = out.local.cpu().numpy().view(np.uint16)
    idx = out.index.cpu().numpy()
    return nb, ne, k, off, cnt, loc, idx


def _call(keys, F, W, out, flags_init=77):
    err = torch.full((1,), flags_init, dtype=torch.int32, device="cuda")
    V.vbh_mc_from_tsdf_static(torch.from_numpy(keys).cuda(), torch.from_numpy(F).cuda(),
                              torch.from_numpy(W).cuda(), out.c_struct(),
                              torch.cuda.current_stream().cuda_stream, err)
    torch.cuda.synchronize()
    return int(err.item())


def test_static_error_flags_and_empty_input():
    """bit0 for a key outside [-2^20, 2^20), bit1 for a repeated key; an empty input writes
    zero totals and a clear flag word (what earlier calls left in the scratch does not leak)."""
    from paper_1805_03709_b300.volume import McStream
    keys, F, W = sphere_blocks(range(-2, 2), (0.01, 0.0, -0.01), 0.15)
    out = McStream.allocate(len(keys) + 1, (len(keys) + 1) * 512)
    bad = keys.copy()
    bad[5] = (1 << 20, 0, 0)
    assert _call(bad, F, W, out) & 3 == 1
    dup = keys.copy()
    dup[7] = dup[3]
    assert _call(dup, F, W, out) & 3 == 2
    out.n.fill_(99)
    e = np.zeros((0, 3), np.int32)
    assert _call(e, np.zeros((0, 512), np.float32), np.zeros((0, 512), np.float32), out) == 0
    assert out.n.cpu().tolist() == [0, 0]
    assert _call(keys, F, W, out) == 0     # clean input after the faulty ones: no stale bits


def _guarded_stream(cap_blocks, cap_entries, pad=64):
    """A stream whose arrays are the first cap_* elements of larger buffers filled with a
    sentinel, so that a write past a capacity shows up in the padding."""
    from paper_1805_03709_b300.volume import McStream
    big = McStream.allocate(cap_blocks + pad, cap_entries + pad)
    for t in (big.keys3, big.info, big.offsets, big.counts, big.local, big.index):
        t.fill_(0x5A)
    small = McStream(big.keys3[:cap_blocks], big.info[:cap_blocks], big.offsets[:cap_blocks],
                     big.counts[:cap_blocks], big.local[:cap_entries], big.index[:cap_entries],
                     big.n)
    return small, big


def _padding_untouched(big, cap_blocks, cap_entries):
    for t, cap in ((big.keys3, cap_blocks), (big.info, cap_blocks), (big.offsets, cap_blocks),
                   (big.counts, cap_blocks), (big.local, cap_entries), (big.index, cap_entries)):
        assert bool((t[cap:] == 0x5A).all())


def test_static_capacity_overflow_sets_bit2_and_writes_only_in_bounds():
    """Undersized stream capacities: bit2 is raised, the totals are the full counts, nothing is
    written beyond cap_blocks / cap_entries, and every record whose entries fit is exact (the
    handle path's records for the same blocks)."""
    keys, F, W = sphere_blocks(range(-3, 3), (0.013, -0.021, 0.007), 0.2)
    want = reference_stream(keys, F, W)
    full_entries = sum(int(np.count_nonzero(d)) for _, d in want.values())
    # (a) fewer record slots than blocks
    cap_b = len(keys) - 5
    out, big = _guarded_stream(cap_b, full_entries)
    assert _call(keys, F, W, out) & 4
    nb, ne, k, off, cnt, loc, idx = _raw(out, keys)
    assert nb == len(keys) and ne == full_entries and len(k) == cap_b
    for i in range(cap_b):
        kk = tuple(int(x) for x in k[i])
        d = np.zeros(512, np.uint8)
        d[loc[off[i]:off[i] + cnt[i]].astype(np.int64)] = idx[off[i]:off[i] + cnt[i]]
        np.testing.assert_array_equal(d, want[kk][1])
    _padding_untouched(big, cap_b, full_entries)
    # (b) fewer entry slots than entries
    cap_e = full_entries // 3
    out, big = _guarded_stream(len(keys), cap_e)
    assert _call(keys, F, W, out) & 4
    nb, ne, k, off, cnt, loc, idx = _raw(out, keys)
    assert nb == len(keys) and ne == full_entries and len(loc) == cap_e
    fitted = 0
    for i in range(nb):
        kk = tuple(int(x) for x in k[i])
        assert cnt[i] == np.count_nonzero(want[kk][1])
        if off[i] + cnt[i] <= cap_e:
            d = np.zeros(512, np.uint8)
            d[loc[off[i]:off[i] + cnt[i]].astype(np.int64)] = idx[off[i]:off[i] + cnt[i]]
            np.testing.assert_array_equal(d, want[kk][1])
            fitted += 1
    assert 0 < fitted < nb
    _padding_untouched(big, len(keys), cap_e)
    # (c) enough room again: no flag
    out, big = _guarded_stream(len(keys), full_entries)
    assert _call(keys, F, W, out) == 0
    _padding_untouched(big, len(keys), full_entries)
