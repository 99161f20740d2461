"""GPU parity of the Marching Cubes triangulation (vbh_mc_triangulate) against the oracle: on
volumes loaded with the same float32 values on both sides (so the MC indices agree exactly),
the GPU's triangles of a whole-model extraction equal the oracle's as a multiset, and the mesh
of a random sign field with an outside shell is closed and consistently oriented."""
import numpy as np
import pytest
import torch

import oracle
from paper_1805_03709_b300 import vbh as V

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1805_03709_b300 import build
    build.build()
    assert torch.cuda.is_available()


def blocks_from(F):
    n = F.shape[0]
    nb = (n + 7) // 8
    keys, vals = [], []
    for bx in range(nb):
        for by in range(nb):
            for bz in range(nb):
                blk = np.ones((8, 8, 8), np.float32)
                sub = F[8 * bx:8 * bx + 8, 8 * by:8 * by + 8, 8 * bz:8 * bz + 8]
                blk[:sub.shape[0], :sub.shape[1], :sub.shape[2]] = sub
                keys.append((bx - nb // 2, by, bz - 1))
                vals.append(blk.transpose(2, 1, 0).reshape(512))
    return np.array(keys, np.int32), np.array(vals, np.float32)


def pair(keys, F):
    from paper_1805_03709_b300.volume import Volume
    s = 0.01
    vol = Volume(voxel_size=s, trunc=0.04, width=8, height=8, fx=4, fy=4, cx=4, cy=4,
                 n_buckets=1 << 12, max_blocks=1 << 12)
    W = np.ones_like(F)
    vol.load(keys, F, W)
    o = oracle.OracleVolume(s, 0.04, 64.0, 0.001, 0.0, 8, 8, 4.0, 4.0, 4.0, 4.0)
    o.load(keys, F.astype(np.float64), W.astype(np.float64))
    return vol, o


def canon(tris):
    q = np.round(np.asarray(tris, np.float64) / 0.005).astype(np.int64).reshape(-1, 9)
    # a triangle up to rotation of its vertex list (orientation kept)
    out = []
    for t in q:
        v = [tuple(t[0:3]), tuple(t[3:6]), tuple(t[6:9])]
        i = v.index(min(v))
        out.append(tuple(v[i:] + v[:i]))
    return sorted(out)


@pytest.mark.parametrize("field", ["sphere", "random"])
def test_triangles_equal_the_oracle(field):
    rng = np.random.default_rng(7)
    n = 24
    if field == "sphere":
        g = np.arange(n) - 11.6
        X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
        F = (np.sqrt(X ** 2 + Y ** 2 + Z ** 2) - 9.3).astype(np.float32) * 0.1
    else:
        F = np.where(rng.random((n, n, n)) < 0.45, -0.5, 0.5).astype(np.float32)
        F[0, :, :] = F[-1, :, :] = F[:, 0, :] = F[:, -1, :] = F[:, :, 0] = F[:, :, -1] = 0.5
    keys, vals = blocks_from(F)
    vol, o = pair(keys, vals)
    s = vol.extract(V.VBH_MC_ALL)
    tris = vol.triangulate(s).cpu().numpy()
    ref = o.triangles(keys)
    assert len(tris) == len(ref) > 500
    assert canon(tris) == canon(ref)
    # closed and consistently oriented
    q = np.round(tris / 0.005).astype(np.int64)
    e = {}
    for t in q:
        for a, b in ((0, 1), (1, 2), (2, 0)):
            k = (tuple(t[a]), tuple(t[b]))
            e[k] = e.get(k, 0) + 1
    assert all(m == 1 and e.get((b, a), 0) == 1 for (a, b), m in e.items())
    vol.close()


def test_capacity_reports_the_needed_count():
    g = np.arange(16) - 7.6
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    F = (np.sqrt(X ** 2 + Y ** 2 + Z ** 2) - 5.2).astype(np.float32) * 0.1
    keys, vals = blocks_from(F)
    vol, o = pair(keys, vals)
    s = vol.extract(V.VBH_MC_ALL)
    full = vol.triangulate(s)
    tris = torch.empty((10, 9), dtype=torch.float32, device="cuda")
    n = torch.zeros(1, dtype=torch.int32, device="cuda")
    V.vbh_mc_triangulate(s.c_struct(), 0.01, tris, 10, n, torch.cuda.current_stream().cuda_stream)
    assert int(n.item()) == len(full) > 10
    vol.close()


def test_records_beyond_one_counting_group():
    """The kernel (8 CTAs of 8 warps per SM, one record per warp and round) counts the triangles
    of a few rounds of records before it writes them: a stream of many such groups of records
    (every record pointing at the entries of one extracted block, each with its own key) is
    written whole, each record's triangles being the oracle's triangles of that block moved by
    the record's key."""
    F = np.full((8, 8, 8), 0.5, np.float32)
    F[3, 4, 2] = -0.5   # eight cubes with one inside corner each
    keys, vals = blocks_from(F)
    vol, o = pair(keys, vals)
    s = vol.extract(V.VBH_MC_ALL)
    nb, ne = (int(x) for x in s.n.cpu().tolist())
    assert nb == 1 and ne == 8
    base = o.triangles(keys).reshape(-1, 9)
    m0 = len(base)
    assert m0 == 8
    from paper_1805_03709_b300.volume import McStream
    N = 2 * torch.cuda.get_device_properties(0).multi_processor_count * 64 * 16 + 5
    r = torch.arange(N, dtype=torch.int32, device="cuda")
    shift = torch.stack([r % 512, r // 512, torch.zeros_like(r)], 1)
    big = McStream(
        (torch.from_numpy(keys).cuda() + shift).contiguous(),
        torch.zeros(N, dtype=torch.int32, device="cuda"),
        torch.full((N,), int(s.offsets[0]), dtype=torch.int32, device="cuda"),
        torch.full((N,), int(s.counts[0]), dtype=torch.int32, device="cuda"),
        s.local, s.index, torch.tensor([N, ne], dtype=torch.int32, device="cuda"))
    tris = vol.triangulate(big, cap=N * m0).cpu().numpy().reshape(-1, 9)
    assert len(tris) == N * m0
    sh = (8 * 0.01) * np.repeat(shift.cpu().numpy().astype(np.float64), 3, axis=0).reshape(N, 9)
    ref = (base[None, :, :] + sh[:, None, :]).reshape(-1, 9)

    def canon_rows(t):
        q = np.round(np.asarray(t, np.float64) / 0.005).astype(np.int64).reshape(-1, 3, 3)
        code = ((q[..., 0] + (1 << 20)) << 42) | ((q[..., 1] + (1 << 20)) << 21) | (q[..., 2] + (1 << 20))
        first = np.argmin(code, axis=1)
        idx = (first[:, None] + np.arange(3)[None, :]) % 3
        rolled = np.take_along_axis(code, idx, axis=1)
        v = np.ascontiguousarray(rolled).view(np.dtype((np.void, 24))).ravel()
        return np.sort(v)

    assert np.array_equal(canon_rows(tris), canon_rows(ref))
    vol.close()


def test_empty_stream_and_blocks_without_surface():
    """A stream of no records, and one whose block holds no surface (every cube index 0, so the
    record has no entries): no triangles and no error."""
    from paper_1805_03709_b300.volume import Volume
    v0 = Volume(voxel_size=0.01, trunc=0.04, width=8, height=8, fx=4, fy=4, cx=4, cy=4,
                n_buckets=1 << 10, max_blocks=1 << 10)
    s0 = v0.extract(V.VBH_MC_ALL)
    assert int(s0.n[0]) == 0 and len(v0.triangulate(s0)) == 0
    F = np.full((8, 8, 8), 0.5, np.float32)
    keys, vals = blocks_from(F)
    vol, o = pair(keys, vals)
    s = vol.extract(V.VBH_MC_ALL)
    nb, ne = (int(x) for x in s.n.cpu().tolist())
    assert nb == 1 and ne == 0
    assert len(vol.triangulate(s)) == 0 and len(o.triangles(keys).reshape(-1, 9)) == 0
    assert vol.counters().error_flags == 0
    v0.close()
    vol.close()
