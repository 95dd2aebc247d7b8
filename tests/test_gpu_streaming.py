"""Full-cover out-of-core frames (mv_frame_streamed): every swapped-out
volume is uploaded, integrated, raycast and downloaded again in every frame
(Sec. Volumetric Integration, Sec. Raycasting, Algorithm 1).  The maps of
every frame and the final volumes must equal, bit for bit, those of the same
volumes kept resident (mv_frame)."""
import numpy as np
import pytest

from paper_1511_07106_b300 import Mapper, MVError, synth
from parity_utils import dev, gpu_maps

pytestmark = pytest.mark.gpu

KEYS = ("depth", "normal", "rgba", "vertex", "vol_id")


@pytest.mark.parametrize("n_slots,fmt", [(1, "f32"), (3, "f32"), (2, "f16"), (2, "i16"), (2, "mixed")])
def test_streamed_frames_equal_resident_frames(n_slots, fmt):
    """Every storage format, and the three mixed in one frame (slots are
    sized in bytes, so one slot holds volumes of any format in turn)."""
    wl = synth.room_tiles(res=48, pitch=0.01, split=2, frames=6, width=160, height=120)
    fmts = [("f32", "f16", "i16")[k % 3] if fmt == "mixed" else fmt for k in range(len(wl.volumes))]
    a, b = Mapper(), Mapper()
    ida = [a.add_volume(v.h, v.r, v.s, f) for v, f in zip(wl.volumes, fmts)]
    idb = [b.add_volume(v.h, v.r, v.s, f) for v, f in zip(wl.volumes, fmts)]
    streamed = [idb[k] for k in (1, 2, 4, 6, 7)]  # more volumes than slots
    for vid in streamed:
        b.swap_out(vid)
    hits = 0
    for i in range(wl.n_frames):
        d, c = wl.frame(i)
        ga = gpu_maps(a.frame(dev(d), dev(c), wl.cam, wl.poses[i]))
        gb = gpu_maps(b.frame_streamed(dev(d), dev(c), wl.cam, wl.poses[i], n_slots=n_slots))
        for key in KEYS:
            np.testing.assert_array_equal(ga[key], gb[key], err_msg=f"frame {i} {key}")
        hits += int((np.isin(gb["vol_id"], streamed)).sum())
    assert hits > 0  # the streamed volumes do contribute hits
    for x, y in zip(ida, idb):
        Fa, Wa, Ca = a.read_decoded(x)
        Fb, Wb, Cb = b.read_decoded(y)
        np.testing.assert_array_equal(Fa, Fb)
        np.testing.assert_array_equal(Wa, Wb)
        np.testing.assert_array_equal(Ca, Cb)
        np.testing.assert_array_equal(a.read_brick_flags(x), b.read_brick_flags(y))
    assert all(not b.query(v)["resident"] for v in streamed)
    # back in HBM, the streamed volumes raycast like the resident ones
    for vid in streamed:
        b.swap_in(vid)
    T = wl.poses[-1]
    ga, gb = gpu_maps(a.raycast(wl.cam, T)), gpu_maps(b.raycast(wl.cam, T))
    for key in KEYS:
        np.testing.assert_array_equal(ga[key], gb[key])
    a.close()
    b.close()


def test_streamed_frame_without_swapped_out_volumes_equals_frame():
    wl = synth.room_tiles(res=48, pitch=0.01, split=2, frames=2, width=96, height=72)
    a, b = Mapper(), Mapper()
    for v in wl.volumes:
        a.add_volume(v.h, v.r, v.s)
        b.add_volume(v.h, v.r, v.s)
    for i in range(wl.n_frames):
        d, c = wl.frame(i)
        ga = gpu_maps(a.frame(dev(d), dev(c), wl.cam, wl.poses[i]))
        gb = gpu_maps(b.frame_streamed(dev(d), dev(c), wl.cam, wl.poses[i], n_slots=2))
        for key in KEYS:
            np.testing.assert_array_equal(ga[key], gb[key])
    with pytest.raises(MVError):
        b.frame_streamed(dev(d), dev(c), wl.cam, wl.poses[0], n_slots=0)
    with pytest.raises(MVError):
        b.frame_streamed(dev(d), dev(c), wl.cam, wl.poses[0], n_slots=5)
    # the context stays usable after the rejected calls
    gb = gpu_maps(b.frame_streamed(dev(d), dev(c), wl.cam, wl.poses[0], n_slots=1))
    assert (gb["depth"] > 0).any()
    a.close()
    b.close()
