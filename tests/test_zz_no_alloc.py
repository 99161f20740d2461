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
