"""mv_frame_host: the per-frame loop from and to host memory (Algorithm 1:
upload, integrate, raycast, download), pipelined inside the library over two
device buffer sets, checked bit for bit against mv_frame on device buffers."""
import numpy as np
import pytest

from paper_1511_07106_b300 import Mapper, synth
from parity_utils import dev, host

pytestmark = pytest.mark.gpu


def test_host_frames_equal_device_frames():
    """Six frames in flight two at a time (tickets waited on one frame
    late), pinned and pageable inputs mixed, one frame without colour: the
    host maps and the volume equal those of mv_frame on device buffers."""
    import torch
    wl = synth.single_volume_128(frames=6, res=96)
    (vs,) = wl.volumes
    frames = [wl.frame(i) for i in range(wl.n_frames)]
    a, b = Mapper(), Mapper()
    va = a.add_volume(vs.h, vs.r, vs.s)
    vb = b.add_volume(vs.h, vs.r, vs.s)
    outs, tickets, keep = [], [], []
    ref = []
    for i, (d, c) in enumerate(frames):
        use_rgb = i != 3
        dm = b.frame(dev(d), dev(c) if use_rgb else None, wl.cam, wl.poses[i])
        ref.append({k: host(v) for k, v in dm.items()})
        if i % 2 == 0:
            hd, hc = torch.from_numpy(d).pin_memory(), torch.from_numpy(c).pin_memory()
        else:
            hd, hc = torch.from_numpy(d.copy()), torch.from_numpy(c.copy())  # pageable
        out = a.alloc_host_maps(wl.cam, vertex=True, vol_id=True)
        tickets.append(a.frame_host(hd, hc if use_rgb else None, wl.cam, wl.poses[i], out))
        outs.append(out)
        keep.append((hd, hc))
        if i >= 1:
            a.frame_host_wait(tickets[i - 1])
    a.frame_host_wait(tickets[-1])
    assert tickets == list(range(len(frames)))
    for i in range(len(frames)):
        for k in ("depth", "normal", "rgba", "vertex", "vol_id"):
            np.testing.assert_array_equal(outs[i][k].numpy(), ref[i][k], err_msg=f"frame {i} {k}")
    assert (ref[-1]["depth"] > 0).mean() > 0.3
    Fa, Wa, ca = a.read_decoded(va)
    Fb, Wb, cb = b.read_decoded(vb)
    np.testing.assert_array_equal(Fa, Fb)
    np.testing.assert_array_equal(Wa, Wb)
    np.testing.assert_array_equal(ca, cb)
    a.close()
    b.close()


def test_host_frame_rejects_bad_arguments_and_unknown_tickets():
    import torch
    from paper_1511_07106_b300 import _abi
    wl = synth.single_volume_128(frames=1, res=32)
    (vs,) = wl.volumes
    m = Mapper()
    m.add_volume(vs.h, vs.r, vs.s)
    d, c = wl.frame(0)
    out = m.alloc_host_maps(wl.cam)
    with pytest.raises(_abi.MVError):
        m.frame_host_wait(0)  # nothing issued yet
    t = m.frame_host(torch.from_numpy(d), None, wl.cam, wl.poses[0], out)
    m.frame_host_wait(t)
    with pytest.raises(_abi.MVError):
        m.frame_host_wait(t + 1)
    with pytest.raises(ValueError):
        m.frame_host(torch.from_numpy(d).cuda(), None, wl.cam, wl.poses[0], out)
    m.close()
