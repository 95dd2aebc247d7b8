"""Surface points on the GPU (mv_extract_points) against the oracle on the
GPU's own volume: the same edges bit for bit (the decisions depend only on the
stored values), positions within FP32 rounding, colours within 1 LSB."""
import numpy as np
import pytest

import oracle
from paper_1511_07106_b300 import Mapper, MVError, synth
from parity_utils import dev, oracle_volume_from_gpu

pytestmark = pytest.mark.gpu


def integrated(wl, frames, fmt="f32"):
    m = Mapper()
    (vs,) = wl.volumes
    vid = m.add_volume(vs.h, vs.r, vs.s, fmt)
    for i in range(frames):
        d, c = wl.frame(i)
        m.integrate(dev(d), dev(c), wl.cam, wl.poses[i])
    return m, vid, vs


def compare(m, vid, vs):
    g = m.extract_points(vid)
    o = oracle.extract_points(oracle_volume_from_gpu(m, vid, vs))
    ge = g["edge"].cpu().numpy()
    order = np.argsort(ge)
    ge = ge[order]
    np.testing.assert_array_equal(ge, o["edge"])
    gx = g["xyz"].cpu().numpy()[order].astype(np.float64)
    scale = np.abs(o["xyz"]).max() + vs.s
    assert np.abs(gx - o["xyz"]).max() <= 1e-6 * scale
    gc = g["rgb"].cpu().numpy()[order].astype(np.int32)
    assert np.abs(gc - o["rgb"].astype(np.int32)).max() <= 1
    return len(ge)


@pytest.mark.parametrize("fmt", ["f32", "f16", "i16"])
def test_extract_matches_oracle(fmt):
    wl = synth.single_volume_128(frames=10)
    m, vid, vs = integrated(wl, 10, fmt)
    n = compare(m, vid, vs)
    assert n > 20000
    m.close()


def test_extract_ragged_volume_small_cap_and_swapped_out():
    wl = synth.single_volume_128(frames=6)
    m = Mapper()
    (vs,) = wl.volumes
    spec = synth.VolumeSpec((vs.h[0] + 3, vs.h[1] - 5, vs.h[2]), (77, 93, 61), vs.s)
    vid = m.add_volume(spec.h, spec.r, spec.s)
    for i in range(6):
        d, c = wl.frame(i)
        m.integrate(dev(d), dev(c), wl.cam, wl.poses[i])
    n = compare(m, vid, spec)
    g = m.extract_points(vid, cap=7)  # grows to the exact count
    assert g["xyz"].shape[0] == n
    empty = m.add_volume((10000, 0, 0), (16, 16, 16), vs.s)
    assert m.extract_points(empty)["xyz"].shape[0] == 0
    m.swap_out(vid)
    with pytest.raises(MVError):
        m.extract_points(vid)
    m.swap_in(vid)
    assert m.extract_points(vid)["xyz"].shape[0] == n
    m.close()
