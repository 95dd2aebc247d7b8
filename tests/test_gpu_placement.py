"""Dynamic volume placement on the GPU (mv_placer_*) against the oracle:
the endpoint histogram c(l) bit for bit (both sides evaluate the endpoint in
FP64 in the same operation order), the top-n / hysteresis policy step by
step, and the contents of the placed volumes against standalone volumes that
integrate exactly the frames during which each was resident (the paper's
tiling invariant under dynamic placement, Sec. Dynamic Mapping for SLAM)."""
import numpy as np
import pytest

import oracle
from paper_1511_07106_b300 import Config, Mapper, MVError, Placer, synth
from parity_utils import dev

pytestmark = pytest.mark.gpu


def small_room(frames=120):
    return synth.placement_room(frames=frames, width=160, height=120, volume_voxels=40, side_m=0.6,
                                max_volumes=5)


def test_histogram_bit_exact():
    pw = small_room(40)
    wl = pw.wl
    m = Mapper(Config(z_min=0.2, z_max=4.5))
    p = Placer(m, pw.cell_voxels, pw.volume_voxels, pw.voxel_size, pw.max_volumes)
    cell_m = pw.cell_voxels * float(np.float32(pw.voxel_size))
    for i in range(0, 40, 7):
        d, _ = wl.frame(i)
        d[::13, ::5] = np.nan
        g = p.histogram(dev(d), wl.cam, wl.poses[i])
        o = oracle.endpoint_histogram(d, wl.cam, wl.poses[i], cell_m, z_min=np.float32(0.2),
                                      z_max=np.float32(4.5))
        assert g == o
        assert len(g) > 3
    with pytest.raises(MVError):
        p.histogram(dev(d), wl.cam, wl.poses[0], cap=2)
    # a cell size small enough to push cell coordinates past 2^20 is refused
    tiny = Placer(m, 1, 2, 1e-7, 4)
    with pytest.raises(MVError):
        tiny.histogram(dev(d), wl.cam, wl.poses[0])
    p.close()
    tiny.close()
    m.close()


@pytest.mark.parametrize("fmt", ["f32", "f16", "i16"])
def test_placement_follows_oracle_policy_and_volumes_match_standalone(fmt):
    """In each storage format: placed volumes are created, evicted to host
    memory and restored in that format."""
    pw = small_room()
    wl = pw.wl
    m = Mapper()
    hyst = 1.2
    p = Placer(m, pw.cell_voxels, pw.volume_voxels, pw.voxel_size, pw.max_volumes, hysteresis=hyst, fmt=fmt)
    cell_m = pw.cell_voxels * float(np.float32(pw.voxel_size))
    st = oracle.PlacementState()
    frames = list(range(0, wl.n_frames, 2))
    resident_at = {}  # volume id -> frames integrated while resident
    totals = {"added": 0, "restored": 0, "evicted": 0}
    maps = m.alloc_maps(wl.cam)
    for i in frames:
        d, c = wl.frame(i)
        for vid, cell, res in p.volumes():
            if res:
                resident_at.setdefault(vid, []).append(i)
        m.frame(dev(d), dev(c), wl.cam, wl.poses[i], out=maps)
        r = p.update(dev(d), wl.cam, wl.poses[i])
        h = oracle.endpoint_histogram(d, wl.cam, wl.poses[i], cell_m)
        a, rs, e = oracle.place(st, h, pw.max_volumes, hyst)
        assert (r["added"], r["restored"], r["evicted"]) == (len(a), len(rs), len(e)), i
        placed = p.volumes()
        assert {cell for _, cell, res in placed if res} == st.resident, i
        assert {cell for _, cell, res in placed if not res} == st.evicted, i
        for k in totals:
            totals[k] += r[k]
    assert totals["evicted"] > 0 and totals["restored"] > 0, totals
    # each placed volume equals a standalone volume that integrated the same frames
    spec = {vid: cell for vid, cell, _ in p.volumes()}
    checked = 0
    for vid, fr in resident_at.items():
        solo = Mapper()
        cell = spec[vid]
        sid = solo.add_volume(tuple(k * pw.cell_voxels for k in cell), (pw.volume_voxels,) * 3, pw.voxel_size,
                              fmt)
        assert m.query(vid)["fmt"] == solo.query(sid)["fmt"]
        for i in fr:
            d, c = wl.frame(i)
            solo.integrate(dev(d), dev(c), wl.cam, wl.poses[i])
        Fa, Wa, Ca = m.read_decoded(vid)
        Fb, Wb, Cb = solo.read_decoded(sid)
        np.testing.assert_array_equal(Fa, Fb)
        np.testing.assert_array_equal(Wa, Wb)
        np.testing.assert_array_equal(Ca, Cb)
        checked += (Wa > 0).any()
        solo.close()
    assert checked >= pw.max_volumes
    p.close()
    m.close()


def test_placer_argument_errors():
    m = Mapper()
    for bad in (dict(cell_voxels=0), dict(volume_voxels=1), dict(voxel_size=0.0), dict(max_volumes=0),
                dict(hysteresis=0.5), dict(min_count=0)):
        kw = dict(cell_voxels=62, volume_voxels=64, voxel_size=0.01, max_volumes=4)
        kw.update(bad)
        with pytest.raises(MVError):
            Placer(m, **kw)
    m.close()
