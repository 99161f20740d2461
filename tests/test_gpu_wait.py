"""Failure detection of the fusion kernel's bounded wait, without a GPU fault: the handle's wait
limit set to 0 makes every wait for a block's asynchronous voxel copy give up at once (a flag
that never comes in time).  The kernel raises the sticky timeout flag, drains its copy and
returns; vbh_integrate_frame reports VBH_ERR_TIMEOUT; nothing hangs, the CUDA context stays
usable, and after vbh_clear_errors the same handle fuses further frames exactly like the oracle
started from the handle's own (partly fused) state."""
import numpy as np
import pytest
import torch

import oracle
from paper_1805_03709_b300 import synth
from paper_1805_03709_b300 import vbh as V

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1805_03709_b300 import build
    build.build()
    assert torch.cuda.is_available()


def test_zero_wait_limit_times_out_and_the_handle_recovers():
    from paper_1805_03709_b300.volume import Volume
    cam, poses, depth = synth.tiny_sequence(n_frames=4)
    args = dict(voxel_size=0.01, trunc=0.04, width=cam.width, height=cam.height, fx=cam.fx,
                fy=cam.fy, cx=cam.cx, cy=cam.cy)
    vol = Volume(n_buckets=1 << 14, max_blocks=1 << 14, **args)
    d = [torch.from_numpy(x).cuda() for x in depth]
    # frame 1: every block is new, so no copy is waited for even with a zero limit
    vol.set_wait_limit(0)
    st = vol.integrate(d[0], poses[0], 1, stats=True)
    assert st.error_flags == 0 and st.touched > 100
    k1, F1, W1 = vol.dump()
    # frame 2 from the same pose: its blocks are live, every unit's copy wait gives up
    with pytest.raises(V.VbhError) as e:
        vol.integrate(d[0], poses[0], 2, stats=True)
    assert e.value.status == V.VBH_ERR_TIMEOUT
    assert vol.counters().error_flags & 8
    torch.cuda.synchronize()                       # the context is alive
    assert float(torch.ones(4, device="cuda").sum()) == 4.0
    k2, F2, W2 = vol.dump()
    np.testing.assert_array_equal(k2, k1)
    # a unit whose wait gave up was left untouched: nothing was fused by frame 2
    np.testing.assert_array_equal(W2, W1)
    np.testing.assert_array_equal(F2, F1)
    # the flag is sticky until cleared; with the default limit restored the handle recovers
    vol.set_wait_limit(1 << 24)
    vol.clear_errors()
    assert vol.counters().error_flags == 0
    orc = oracle.OracleVolume(0.01, 0.04, 64.0, 0.001, 0.0, cam.width, cam.height, cam.fx,
                              cam.fy, cam.cx, cam.cy)
    orc.load(k2, F2.astype(np.float64), W2.astype(np.float64))
    for i in (1, 2, 3):
        st = vol.integrate(d[i], poses[i], 10 + i, stats=True)
        assert st.error_flags == 0
        assert st.touched == orc.integrate(depth[i], poses[i])
    kg, Fg, Wg = vol.dump()
    ko, Fo, Wo = orc.dump()
    np.testing.assert_array_equal(kg, ko)
    np.testing.assert_array_equal(Wg, Wo.astype(np.float32))
    assert np.abs(Fg - Fo).max() <= 1e-5
    vol.close()
