"""GPU tests of the pipelined host-buffer frame call (vbh_process_frame_host): every frame's MC
stream copied into host memory equals the stream vbh_process_frame writes for the same frame on a
second volume fed the same inputs (as a map keyed by block), each call completes exactly the
frame of two calls earlier, capacities that are too small cut the copy and are reported with the
true totals, and pageable depth works like pinned depth."""
import numpy as np
import pytest
import torch

from paper_1805_03709_b300 import synth, vbh as V

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1805_03709_b300 import build
    build.build()
    assert torch.cuda.is_available()


@pytest.fixture(scope="module")
def room():
    return synth.room_sequence(n_frames=10, width=160, height=120)


def volume(cam):
    from paper_1805_03709_b300.volume import Volume
    return Volume(voxel_size=0.005, trunc=0.02, width=cam.width, height=cam.height, fx=cam.fx,
                  fy=cam.fy, cx=cam.cx, cy=cam.cy, n_buckets=1 << 16, max_blocks=1 << 17,
                  zmax=4.0, mc_cap_blocks=1 << 14, mc_cap_entries=1 << 20)


def same_stream(a, b):
    assert a.keys() == b.keys()
    for k in a:
        assert a[k][0] == b[k][0]
        oa, ob = np.argsort(a[k][1]), np.argsort(b[k][1])
        np.testing.assert_array_equal(a[k][1][oa], b[k][1][ob])
        np.testing.assert_array_equal(a[k][2][oa], b[k][2][ob])


@pytest.mark.parametrize("pinned", [True, False])
def test_host_frames_equal_device_frames(room, pinned):
    from paper_1805_03709_b300.volume import HostStream
    cam, poses, depth = room
    va, vb = volume(cam), volume(cam)
    outs = [HostStream.allocate(1 << 14, 1 << 20) for _ in range(3)]
    ref = []
    host_depth = torch.from_numpy(depth).pin_memory() if pinned else depth
    for i in range(len(poses)):
        d = host_depth[i]
        if not pinned:
            d = np.ascontiguousarray(d)
        out = outs[i % 3]
        st = va.process_frame_host(d, poses[i], i + 1, 1.5, out)
        assert st == V.VBH_OK
        assert not out.done
        if i >= 2:   # the frame of two calls earlier is complete when the call returns
            prev = outs[(i - 2) % 3]
            assert prev.done and prev.c_struct().frame_id == i - 1
            same_stream(prev.to_host(), ref[i - 2])
        vb.process_frame(torch.from_numpy(depth[i]).cuda(), poses[i], i + 1, 1.5)
        ref.append(vb.stream.to_host())
    assert va.process_frame_host_flush() == V.VBH_OK
    for i in (len(poses) - 2, len(poses) - 1):
        last = outs[i % 3]
        assert last.done and last.c_struct().frame_id == i + 1
        same_stream(last.to_host(), ref[i])
    assert sum(len(r) for r in ref) > 1000
    assert va.counters().error_flags == 0
    va.close()
    vb.close()


def test_small_host_capacity_is_reported(room):
    from paper_1805_03709_b300.volume import HostStream
    cam, poses, depth = room
    va, vb = volume(cam), volume(cam)
    small = HostStream.allocate(64, 1000)
    host_depth = torch.from_numpy(depth).pin_memory()
    assert va.process_frame_host(host_depth[0], poses[0], 1, 0.0, small) == V.VBH_OK
    assert va.process_frame_host_flush() == V.VBH_ERR_BUFFER_TOO_SMALL
    vb.process_frame(torch.from_numpy(depth[0]).cuda(), poses[0], 1, 0.0)
    ref = vb.stream.to_host()
    nb, ne = small.n
    assert small.done and nb == len(ref) > 64 and ne == sum(len(v[1]) for v in ref.values())
    keys = small.keys3[:64].numpy()
    info = small.info[:64].numpy().view(np.uint32)
    for k, inf in zip(map(tuple, keys.tolist()), info.tolist()):
        assert ref[k][0] == inf   # the records that fit are real records of the frame
    va.close()
    vb.close()
