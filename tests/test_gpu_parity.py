"""CUDA path vs FP64 oracle, through the C ABI (libmvtsdf.so), on a B300.

Integration is checked in lockstep: before each frame the GPU state is read
back and the oracle applies the same frame to it in FP64; the GPU's state
after the frame must match within the tolerances of parity_utils.  The
raycast is checked by raycasting the GPU's own final state in the oracle.
Sizes span several bricks and ragged tails; one test runs the full 512^3 /
640x480 workload on sampled voxels and pixels."""
import math

import numpy as np
import pytest

import oracle
from paper_1511_07106_b300 import Config, Mapper, MVError, synth
from parity_utils import (check_brick_flags, check_lockstep, compare_raycast, dev, gpu_maps,
                          host, oracle_volume_from_gpu)

pytestmark = pytest.mark.gpu


def ocfg(cfg: Config):
    return oracle.Config(trunc_vox=cfg.trunc_voxels, w_max=cfg.w_max, color_w_max=cfg.color_w_max,
                         z_min=cfg.z_min, z_max=cfg.z_max, step_vox=cfg.ray_step)


def run_lockstep(wl, fmt="f32", frames=None, cfg=Config(), with_colour=True):
    m = Mapper(cfg)
    (vs,) = wl.volumes
    vid = m.add_volume(vs.h, vs.r, vs.s, fmt)
    oc = ocfg(cfg)
    worst, flagged = 0.0, 0.0
    n = wl.n_frames if frames is None else frames
    for i in range(n):
        d, c = wl.frame(i)
        before = oracle_volume_from_gpu(m, vid, vs)
        counts, flags = oracle.integrate(before, d, c if with_colour else None, wl.cam, wl.poses[i],
                                         oc, want_flags=True)
        m.stats(reset=True)
        m.integrate(dev(d), dev(c) if with_colour else None, wl.cam, wl.poses[i])
        F, W, rgba = m.read_decoded(vid)
        w, fl = check_lockstep(before, F, W, rgba, flags, fmt=fmt, with_colour=with_colour)
        worst, flagged = max(worst, w), max(flagged, fl)
        st = m.stats()
        nflag = int((flags != 0).sum())
        assert abs(st["updated"] - counts[0]) <= nflag
        if with_colour:
            assert abs(st["band"] - counts[1]) <= nflag
    return m, vid, worst, flagged


@pytest.fixture(scope="module")
def c1_run():
    wl = synth.single_volume_128()
    m, vid, worst, flagged = run_lockstep(wl)
    yield wl, m, vid, worst, flagged
    m.close()


def test_integrate_lockstep_128(c1_run):
    wl, m, vid, worst, flagged = c1_run
    assert worst <= 1e-4
    assert flagged < 0.01
    F, W, _ = m.read_decoded(vid)
    assert (W > 0).mean() > 0.1


def test_brick_flags_sound_and_effective(c1_run):
    wl, m, vid, _, _ = c1_run
    (vs,) = wl.volumes
    recall = check_brick_flags(m, vid, vs, min_free_recall=0.5)
    assert recall > 0.5


@pytest.mark.parametrize("pose_index", [0, 11, 29])
def test_raycast_parity_128(c1_run, pose_index):
    wl, m, vid, _, _ = c1_run
    (vs,) = wl.volumes
    T = wl.poses[pose_index]
    g = gpu_maps(m.raycast(wl.cam, T))
    ov = oracle_volume_from_gpu(m, vid, vs)
    o = oracle.raycast([ov], wl.cam, T, ocfg(m.config), ids=[vid])
    summary = compare_raycast(g, o, wl.cam, T, vs.s, require_hits=0.3)
    assert summary["max_depth_err_vox"] < 0.02


@pytest.mark.parametrize("fmt", ["f16", "i16"])
def test_reduced_storage_lockstep_and_raycast(fmt):
    wl = synth.single_volume_128(frames=10, res=64)
    m, vid, worst, flagged = run_lockstep(wl, fmt=fmt)
    (vs,) = wl.volumes
    ov = oracle_volume_from_gpu(m, vid, vs)
    T = wl.poses[3]
    g = gpu_maps(m.raycast(wl.cam, T))
    o = oracle.raycast([ov], wl.cam, T, ocfg(m.config), ids=[vid])
    compare_raycast(g, o, wl.cam, T, vs.s, require_hits=0.3)
    m.close()


def test_ragged_volume_and_image():
    """Volume dims not multiples of the 8-voxel brick, image not a multiple of
    the 16x8 raycast tile, non-cubic volume."""
    base = synth.single_volume_128(frames=6, res=40)
    cam = synth.Camera(115.0, 115.0, 70.3, 52.1, 141, 103)
    vs = synth.VolumeSpec((-21, -13, -5), (45, 29, 37), 0.06)
    wl = synth.Workload("ragged", cam, base.scene, base.poses, [vs], base.seed)
    m, vid, worst, _ = run_lockstep(wl)
    ov = oracle_volume_from_gpu(m, vid, vs)
    for T in (wl.poses[0], wl.poses[4]):
        g = gpu_maps(m.raycast(cam, T))
        o = oracle.raycast([ov], cam, T, ocfg(m.config), ids=[vid])
        compare_raycast(g, o, cam, T, vs.s, require_hits=0.1)
    m.close()


def test_smallest_volume_and_invalid_depth():
    cam = synth.Camera(20.0, 20.0, 7.5, 5.5, 16, 12)
    m = Mapper()
    vid = m.add_volume((0, 0, 10), (2, 2, 2), 0.05)
    T = np.eye(4)
    for bad in (0.0, np.nan, -1.0):
        d = np.full((12, 16), bad, np.float32)
        m.integrate(dev(d), None, cam, T)
    assert m.stats()["updated"] == 0
    F, W, _ = m.read_decoded(vid)
    assert np.all(W == 0) and np.all(F == 0)
    d = np.full((12, 16), 0.53, np.float32)
    m.integrate(dev(d), None, cam, T)
    F, W, _ = m.read_decoded(vid)
    ov = oracle.Volume((0, 0, 10), (2, 2, 2), 0.05)
    oracle.integrate(ov, d, None, cam, T, oracle.Config())
    np.testing.assert_allclose(F, ov.F, atol=1e-6)
    np.testing.assert_array_equal(W, ov.W)
    m.close()


def test_axis_aligned_rays():
    """Degenerate ray directions: poses whose rotations are exact axis
    permutations (some entries -0.0) and an integral principal point, so the
    centre row, column and pixel of every view have rays with exactly zero
    direction components (the march's domain clip and the step-over DDA take
    their zero-direction branches), some of them lying in lattice planes.
    Lockstep integration and the raycast against the oracle."""
    res = 64
    s = float(np.float32(1.5 / res))
    scene = synth.Scene(planes=np.array([[0.0, 0.0, 1.0, 0.0]]),
                        spheres=np.array([[0.1, -0.05, 0.35, 0.3], [-0.3, 0.25, 0.2, 0.2]]),
                        boxes=np.array([[0.2, 0.2, 0.0, 0.5, 0.45, 0.4]]))
    cam = synth.Camera(100.0, 100.0, 40.0, 30.0, 81, 61)
    views = [((0.0, 0.0, 1.6), (0.0, 0.0, 0.0), (0.0, 1.0, 0.0)),
             ((-1.3, 0.0, 0.3), (0.0, 0.0, 0.3), (0.0, 0.0, 1.0)),
             ((0.0, 1.3, 0.25), (0.0, 0.0, 0.25), (0.0, 0.0, 1.0)),
             ((0.9, 0.0, 0.3), (0.0, 0.0, 0.3), (0.0, 0.0, 1.0))]
    poses = [synth.look_at(*views[i % 4]) for i in range(8)]
    for T in poses:
        assert set(np.unique(np.abs(T[:3, :3]))) == {0.0, 1.0}
    wl = synth.Workload("axis-aligned views of a 64^3 volume", cam, scene, poses,
                        [synth.VolumeSpec((-res // 2, -res // 2, -4), (res, res, res), s)], seed=9)
    m, vid, worst, flagged = run_lockstep(wl)
    assert worst <= 1e-4 and flagged < 0.01
    (vs,) = wl.volumes
    ov = oracle_volume_from_gpu(m, vid, vs)
    for T in poses[:4]:
        g = gpu_maps(m.raycast(cam, T))
        o = oracle.raycast([ov], cam, T, ocfg(m.config), ids=[vid])
        compare_raycast(g, o, cam, T, s, require_hits=0.3)
        # the centre pixel's ray runs exactly along an axis
        assert g["depth"][30, 40] > 0 and o["depth"][30, 40] > 0
    m.close()


@pytest.mark.parametrize("cfg", [
    Config(trunc_voxels=2.0, w_max=3, color_w_max=2),
    Config(z_min=0.9, z_max=1.7, ray_step=0.5),
    Config(trunc_voxels=7.5, w_max=65535, n_bisect=12),
], ids=["narrow-band-low-caps", "depth-range-half-step", "wide-band-high-cap"])
def test_nondefault_config_lockstep_and_raycast(cfg):
    """Configurations other than the default: a narrow truncation band with
    weight and colour caps reached within the frames (the capped running
    average), a depth range that gates measurements and clips the march with
    half-voxel samples, and a wide band with the largest weight cap."""
    wl = synth.single_volume_128(frames=8, res=64)
    m, vid, worst, flagged = run_lockstep(wl, cfg=cfg)
    assert worst <= 1e-4 and flagged < 0.01
    (vs,) = wl.volumes
    F, W, _ = m.read_decoded(vid)
    assert W.max() <= cfg.w_max
    if cfg.w_max < wl.n_frames:
        assert W.max() == cfg.w_max  # the cap was reached
    ov = oracle_volume_from_gpu(m, vid, vs)
    for T in (wl.poses[2], wl.poses[7]):
        g = gpu_maps(m.raycast(wl.cam, T))
        o = oracle.raycast([ov], wl.cam, T, ocfg(cfg), ids=[vid])
        compare_raycast(g, o, wl.cam, T, vs.s, require_hits=0.1)
        hit = g["depth"] > 0
        assert np.all((g["depth"][hit] >= cfg.z_min) & (g["depth"][hit] <= cfg.z_max))
    m.close()


@pytest.mark.parametrize("size", [(1920, 1080), (2048, 96)], ids=["1920x1080", "2048x96"])
def test_large_and_wide_images(size):
    """Image sizes beyond the benchmark's: 1920x1080 and an extreme 2048x96
    (a depth-tile pyramid three top-level tiles high).  Lockstep integration
    against the oracle, the raycast against the oracle on every 13th pixel,
    and the frame graph equal to separate calls, bit for bit."""
    W, H = size
    base = synth.single_volume_128(frames=4, res=64)
    f = 0.8 * W if H > 200 else 0.25 * W  # the strip sees a band of the scene
    # an integral principal point: with (W - 1) / 2 the voxel plane through the
    # optical axis would project onto pixel-rounding ties (flagged, not compared)
    cam = synth.Camera(f, f, W / 2.0, H / 2.0, W, H)
    wl = synth.Workload(f"64^3 volume at {W}x{H}", cam, base.scene, base.poses, base.volumes, base.seed)
    m, vid, worst, flagged = run_lockstep(wl)
    assert worst <= 1e-4 and flagged < 0.01
    (vs,) = wl.volumes
    ov = oracle_volume_from_gpu(m, vid, vs)
    T = wl.poses[3]
    g = gpu_maps(m.raycast(cam, T))
    idx = np.arange(0, W * H, 13)
    mask = np.zeros(W * H, bool)
    mask[idx] = True
    o = oracle.raycast([ov], cam, T, ocfg(m.config), ids=[vid], pixels=idx)
    compare_raycast(g, o, cam, T, vs.s, mask=mask.reshape(H, W), require_hits=0.05)
    # the same frames through the frame graph on a second mapper
    b = Mapper()
    bid = b.add_volume(vs.h, vs.r, vs.s)
    maps = b.alloc_maps(cam)
    for i in range(wl.n_frames):
        d, c = wl.frame(i)
        b.frame(dev(d), dev(c), cam, wl.poses[i], out=maps)
    fb = gpu_maps(maps)
    fa = gpu_maps(m.raycast(cam, wl.poses[-1]))
    for k in ("depth", "normal", "rgba", "vol_id"):
        np.testing.assert_array_equal(fa[k], fb[k])
    Fa, Wa, Ca = m.read_decoded(vid)
    Fb, Wb, Cb = b.read_decoded(bid)
    np.testing.assert_array_equal(Fa, Fb)
    np.testing.assert_array_equal(Wa, Wb)
    np.testing.assert_array_equal(Ca, Cb)
    m.close()
    b.close()


@pytest.mark.parametrize("size,split,res,fmt", [((160, 120), 12, 122, "f32"), ((16, 8), 16, 98, "f32"),
                                                ((160, 120), 12, 122, "f16"), ((160, 120), 12, 122, "i16")],
                         ids=["1728-volumes-160x120", "4096-volumes-16x8", "1728-volumes-f16", "1728-volumes-i16"])
def test_many_volumes_equal_one_volume(size, split, res, fmt):
    """1728 or 4096 volumes (tiles of one volume, two-voxel overlap): more
    than the 256 the frame set-up ranks nearest first (the unranked view
    list); at 16x8 with 16x8-pixel CTA tiles one CTA sees every volume in
    view, hundreds of them holding surface, more than the 256 candidates its
    shared-memory list holds (the CTA falls back to the view list).  Voxels
    and maps equal the single volume's bit for bit (tiling invariance, Sec.
    Comparison to KinectFusion)."""
    W, H = size
    base = synth.single_volume_128(frames=4, res=res)
    cam = synth.Camera(W / 2.0, W / 2.0, W / 2.0, H / 2.0, W, H)
    wl = synth.Workload(f"{res}^3 volume at {W}x{H}", cam, base.scene, base.poses, base.volumes, base.seed)
    tl = synth.tiled(wl, split)
    assert len(tl.volumes) == split ** 3
    (vs,) = wl.volumes
    single, tiles = Mapper(), Mapper()
    tiles.set_tuning(0, 8)  # 16x8-pixel CTA tiles
    sid = single.add_volume(vs.h, vs.r, vs.s, fmt)
    tids = [tiles.add_volume(t.h, t.r, t.s, fmt) for t in tl.volumes]
    for i in range(wl.n_frames):
        d, c = wl.frame(i)
        single.integrate(dev(d), dev(c), cam, wl.poses[i])
        tiles.integrate(dev(d), dev(c), cam, wl.poses[i])
    Fs, Ws, Cs = single.read_decoded(sid)
    assert (Ws > 0).mean() > 0.01
    for t, tid in zip(tl.volumes, tids):
        F, Wt, col = tiles.read_decoded(tid)
        o = [t.h[a] - vs.h[a] for a in range(3)]
        sl = (slice(o[2], o[2] + t.r[2]), slice(o[1], o[1] + t.r[1]), slice(o[0], o[0] + t.r[0]))
        np.testing.assert_array_equal(F, Fs[sl])
        np.testing.assert_array_equal(Wt, Ws[sl])
        np.testing.assert_array_equal(col, Cs[sl])
    for T in (wl.poses[1], wl.poses[3]):
        a = gpu_maps(single.raycast(cam, T))
        b = gpu_maps(tiles.raycast(cam, T))
        assert (a["depth"] > 0).mean() > 0.3
        for k in ("depth", "normal", "rgba"):
            np.testing.assert_array_equal(a[k], b[k])
    single.close()
    tiles.close()


def test_volume_capacity():
    """4096 volumes fit a context; one more is refused with a status, and a
    removal frees a slot again."""
    m = Mapper()
    ids = [m.add_volume((3 * k, 0, 0), (2, 2, 2), 0.01) for k in range(4096)]
    with pytest.raises(MVError) as e:
        m.add_volume((0, 5, 0), (2, 2, 2), 0.01)
    assert "CAPACITY" in str(e.value) or "volumes" in str(e.value)
    m.remove_volume(ids[100])
    m.add_volume((0, 5, 0), (2, 2, 2), 0.01)
    assert len(m.volumes()) == 4096
    m.close()


def test_far_from_the_origin():
    """The single-volume workload moved by (40000, -30000, 20000) voxels
    (about 0.9, 0.7 and 0.5 km) with its camera and scene: voxel positions
    are exact lattice differences from the camera's lattice point plus its
    sub-voxel fraction (the camera split in FP64), so lockstep integration and
    the raycast match the oracle, which works with the world coordinates in
    FP64, as they do at the origin."""
    base = synth.single_volume_128(frames=6, res=64)
    (vs,) = base.volumes
    N = np.array([40000, -30000, 20000])
    off = N * vs.s
    sc = base.scene
    scene = synth.Scene(planes=np.array([[*p[:3], p[3] + np.dot(p[:3], off)] for p in sc.planes]),
                        spheres=np.array([[*(p[:3] + off), p[3]] for p in sc.spheres]),
                        boxes=np.array([[*(b[:3] + off), *(b[3:] + off)] for b in sc.boxes]))
    poses = []
    for T in base.poses:
        T = T.copy()
        T[:3, 3] += off
        poses.append(T)
    far = synth.VolumeSpec(tuple(int(a) for a in np.array(vs.h) + N), vs.r, vs.s)
    wl = synth.Workload("64^3 volume 1 km from the origin", base.cam, scene, poses, [far], base.seed)
    m, vid, worst, flagged = run_lockstep(wl)
    assert worst <= 1e-4 and flagged < 0.01
    ov = oracle_volume_from_gpu(m, vid, far)
    for T in (poses[2], poses[5]):
        g = gpu_maps(m.raycast(wl.cam, T))
        o = oracle.raycast([ov], wl.cam, T, ocfg(m.config), ids=[vid])
        compare_raycast(g, o, wl.cam, T, vs.s, require_hits=0.3)
    m.close()


@pytest.mark.parametrize("size", [(1, 1), (1, 37), (53, 1), (3, 2)], ids=["1x1", "1x37", "53x1", "3x2"])
def test_tiny_images(size):
    """Images of one pixel, one column, one row and 3x2 (a depth-tile pyramid
    of a single partial tile, raycast tiles mostly outside the image):
    lockstep integration, the raycast against the oracle, and the frame graph
    equal to separate calls."""
    W, H = size
    base = synth.single_volume_128(frames=6, res=32)
    cam = synth.Camera(60.0, 60.0, (W - 1) / 2.0 + 0.25, (H - 1) / 2.0 - 0.125, W, H)
    wl = synth.Workload(f"32^3 volume at {W}x{H}", cam, base.scene, base.poses, base.volumes, base.seed)
    m, vid, worst, flagged = run_lockstep(wl)
    assert worst <= 1e-4
    assert m.read_decoded(vid)[1].max() > 0  # something was integrated
    (vs,) = wl.volumes
    # the raycast of a volume built from 160x120 frames, at the tiny image
    full = synth.Workload("32^3 volume", synth.Camera(100.0, 100.0, 80.0, 60.0, 160, 120), base.scene,
                          base.poses, base.volumes, base.seed)
    r = Mapper()
    rid = r.add_volume(vs.h, vs.r, vs.s)
    for i in range(full.n_frames):
        d, c = full.frame(i)
        r.integrate(dev(d), dev(c), full.cam, full.poses[i])
    ov = oracle_volume_from_gpu(r, rid, vs)
    hits = 0
    for T in wl.poses:
        g = gpu_maps(r.raycast(cam, T))
        o = oracle.raycast([ov], cam, T, ocfg(r.config), ids=[rid])
        compare_raycast(g, o, cam, T, vs.s, require_hits=0.0)
        hits += int((g["depth"] > 0).sum())
    assert hits > 0
    r.close()
    b = Mapper()
    bid = b.add_volume(vs.h, vs.r, vs.s)
    maps = b.alloc_maps(cam)
    for i in range(wl.n_frames):
        d, c = wl.frame(i)
        b.frame(dev(d), dev(c), cam, wl.poses[i], out=maps)
    fa = gpu_maps(m.raycast(cam, wl.poses[-1]))
    fb = gpu_maps(maps)
    for k in ("depth", "normal", "rgba", "vol_id"):
        np.testing.assert_array_equal(fa[k], fb[k])
    np.testing.assert_array_equal(m.read_decoded(vid)[0], b.read_decoded(bid)[0])
    m.close()
    b.close()


class _CorruptedFrames:
    """A workload whose depth frames have a tenth of their pixels replaced by
    invalid or extreme values."""

    def __init__(self, wl, z_min, z_max, seed=7):
        self.wl, self.cam, self.poses, self.volumes = wl, wl.cam, wl.poses, wl.volumes
        self.n_frames = wl.n_frames
        self.bad = np.array([0.0, -1.0, np.nan, np.inf, -np.inf, 1e30, z_min * 0.999, min(z_max * 1.001, 1e30)],
                            np.float32)
        self.seed = seed

    def frame(self, i):
        d, c = self.wl.frame(i)
        rng = np.random.default_rng(self.seed + i)
        sel = rng.random(d.shape) < 0.1
        d = d.copy()
        d[sel] = rng.choice(self.bad, size=int(sel.sum()))
        return d, c


@pytest.mark.parametrize("zr", [(0.0, float("inf")), (0.5, 3.0)], ids=["default-range", "range-0.5-3"])
def test_invalid_and_extreme_depths(zr):
    """A tenth of every frame's pixels set to 0, -1, NaN, +-inf, 1e30 and
    values just outside [z_min, z_max]: a depth counts when it is > 0 and
    inside the range (so +inf and 1e30 count when z_max is infinite, as free
    space along their rays); lockstep integration and the raycast against
    the oracle."""
    cfg = Config(z_min=zr[0], z_max=zr[1])
    base = synth.single_volume_128(frames=5, res=48)
    wl = _CorruptedFrames(base, max(zr[0], 1e-3), zr[1])
    m, vid, worst, flagged = run_lockstep(wl, cfg=cfg)
    assert worst <= 1e-4 and flagged < 0.01
    (vs,) = wl.volumes
    ov = oracle_volume_from_gpu(m, vid, vs)
    for T in (wl.poses[1], wl.poses[4]):
        g = gpu_maps(m.raycast(wl.cam, T))
        o = oracle.raycast([ov], wl.cam, T, ocfg(cfg), ids=[vid])
        compare_raycast(g, o, wl.cam, T, vs.s, require_hits=0.2)
    m.close()


def test_empty_context_raycast_is_all_miss():
    cam = synth.Camera(20.0, 20.0, 9.5, 7.5, 20, 15)
    m = Mapper()
    out = gpu_maps(m.raycast(cam, np.eye(4)))
    assert np.all(out["depth"] == 0) and np.all(out["vol_id"] == -1) and np.all(out["rgba"] == 0)
    m.integrate(dev(np.ones((15, 20), np.float32)), None, cam, np.eye(4))
    m.close()


def test_tiling_invariance_on_gpu():
    """2x2x2 subvolumes with the two-voxel overlap equal one volume covering
    them, bit for bit, after integration and in the merged raycast
    (Sec. Comparison to KinectFusion)."""
    wl = synth.single_volume_128(frames=8, res=34)
    tl = synth.tiled(wl, 2)
    (vs,) = wl.volumes
    single, tiles = Mapper(), Mapper()
    sid = single.add_volume(vs.h, vs.r, vs.s)
    tids = [tiles.add_volume(t.h, t.r, t.s) for t in tl.volumes]
    for i in range(wl.n_frames):
        d, c = wl.frame(i)
        single.integrate(dev(d), dev(c), wl.cam, wl.poses[i])
        tiles.integrate(dev(d), dev(c), wl.cam, wl.poses[i])
    Fs, Ws, Cs = single.read_decoded(sid)
    for t, tid in zip(tl.volumes, tids):
        F, W, C = tiles.read_decoded(tid)
        o = [t.h[a] - vs.h[a] for a in range(3)]
        sl = (slice(o[2], o[2] + t.r[2]), slice(o[1], o[1] + t.r[1]), slice(o[0], o[0] + t.r[0]))
        np.testing.assert_array_equal(F, Fs[sl])
        np.testing.assert_array_equal(W, Ws[sl])
        np.testing.assert_array_equal(C, Cs[sl])
    for T in (wl.poses[1], wl.poses[5]):
        a = gpu_maps(single.raycast(wl.cam, T))
        b = gpu_maps(tiles.raycast(wl.cam, T))
        assert (a["depth"] > 0).mean() > 0.3
        np.testing.assert_array_equal(a["depth"], b["depth"])
        np.testing.assert_array_equal(a["normal"], b["normal"])
        np.testing.assert_array_equal(a["rgba"], b["rgba"])
    # and the tiles against the oracle's multi-volume raycast
    ovs = [oracle_volume_from_gpu(tiles, tid, t) for t, tid in zip(tl.volumes, tids)]
    T = wl.poses[3]
    g = gpu_maps(tiles.raycast(wl.cam, T))
    o = oracle.raycast(ovs, wl.cam, T, ocfg(tiles.config), ids=tids)
    compare_raycast(g, o, wl.cam, T, vs.s, require_hits=0.3)
    single.close()
    tiles.close()


def test_per_volume_path_equals_batched_path():
    wl = synth.single_volume_128(frames=5, res=34)
    tl = synth.tiled(wl, 2)
    a, b = Mapper(), Mapper()
    ida = [a.add_volume(t.h, t.r, t.s) for t in tl.volumes]
    idb = [b.add_volume(t.h, t.r, t.s) for t in tl.volumes]
    for i in range(wl.n_frames):
        d, c = wl.frame(i)
        a.integrate(dev(d), dev(c), wl.cam, wl.poses[i])
        for vid in idb:
            b.integrate_volume(vid, dev(d), dev(c), wl.cam, wl.poses[i])
    for x, y in zip(ida, idb):
        Fa, Wa, Ca = a.read_decoded(x)
        Fb, Wb, Cb = b.read_decoded(y)
        np.testing.assert_array_equal(Fa, Fb)
        np.testing.assert_array_equal(Wa, Wb)
        np.testing.assert_array_equal(Ca, Cb)
    T = wl.poses[2]
    ga = gpu_maps(a.raycast(wl.cam, T))
    out = b.alloc_maps(wl.cam)
    for k, vid in enumerate(idb):
        b.raycast_volume(vid, k == 0, wl.cam, T, out)
    gb = gpu_maps(out)
    for key in ("depth", "normal", "rgba", "vertex", "vol_id"):
        np.testing.assert_array_equal(ga[key], gb[key])
    a.close()
    b.close()


def test_plane_filled_volume_raycast_is_exact():
    """A linear signed distance written into the volume: the GPU hit equals the
    analytic ray--plane intersection within FP32 rounding."""
    m = Mapper()
    h, r, s = (-30, -30, -30), (60, 60, 60), 0.02
    vid = m.add_volume(h, r, s)
    rng = np.random.default_rng(7)
    n = rng.normal(size=3)
    n /= np.linalg.norm(n)
    dd = 0.03
    z, y, x = np.meshgrid(*[np.arange(k) for k in r[::-1]], indexing="ij")
    p = np.stack([(h[0] + x) * s, (h[1] + y) * s, (h[2] + z) * s], -1)
    F = np.clip((dd - p @ n) / (4 * s), -1, 1)
    m.write_decoded(vid, F, np.ones_like(F))
    eye = -0.9 * n
    T = synth.look_at(eye, eye + n + np.array([0.05, -0.03, 0.02]))
    cam = synth.Camera(50.0, 50.0, 31.5, 23.5, 64, 48)
    g = gpu_maps(m.raycast(cam, T))
    o, d = synth.pixel_rays(cam, T)
    tau = (dd - o @ n) / (d @ n)
    pt = o + tau[..., None] * d
    inside = np.all((pt > (np.array(h) + 1) * s) & (pt < (np.array(h) + np.array(r) - 2) * s), -1)
    assert inside.mean() > 0.5
    err = np.abs(g["depth"] - tau) * np.linalg.norm(d, axis=-1) / s
    assert err[inside].max() < 2e-3
    cosang = g["normal"][inside] @ (-n)
    assert cosang.min() > math.cos(math.radians(0.1))
    m.close()


def test_sphere_filled_volume_outside_and_inside():
    """A sphere's signed distance written into the volume (radius 0.4 m,
    1.6 cm voxels).  From outside: the hit within the trilinear error bound
    of the analytic ray--sphere intersection (3 s^2 / (8 rho) over the incidence
    cosine, plus the refinement)
    and equal to the oracle's raycast of the same volume.  From inside: every
    ray's first valid sample is <= 0 and it leaves through a -/+ crossing, so
    no pixel has a hit (Sec. Raycasting: only a +/- change of sign is a
    surface), on the GPU and in the oracle."""
    m = Mapper()
    h, r, s = (-40, -40, -40), (80, 80, 80), 0.016
    vid = m.add_volume(h, r, s)
    c, rho, mu = np.array([0.02, -0.03, 0.01]), 0.4, 4 * s
    z, y, x = np.meshgrid(*[np.arange(k) for k in r[::-1]], indexing="ij")
    p = np.stack([(h[0] + x) * s, (h[1] + y) * s, (h[2] + z) * s], -1)
    F = np.clip((np.linalg.norm(p - c, axis=-1) - rho) / mu, -1, 1)
    m.write_decoded(vid, F, np.ones_like(F))
    ov = oracle_volume_from_gpu(m, vid, synth.VolumeSpec(h, r, s))
    cam = synth.Camera(40.0, 40.0, 31.5, 23.5, 64, 48)
    # outside
    eye = np.array([0.1, -0.55, 0.45])
    T = synth.look_at(eye, c + np.array([0.03, 0.0, -0.02]))
    g = gpu_maps(m.raycast(cam, T))
    o_ray, d = synth.pixel_rays(cam, T)
    oc = o_ray - c
    a2, b2, c2 = np.sum(d * d, -1), 2 * (d @ oc), oc @ oc - rho * rho
    disc = b2 * b2 - 4 * a2 * c2
    tau = np.where(disc > 0, (-b2 - np.sqrt(np.maximum(disc, 0))) / (2 * a2), np.nan)
    hit = np.isfinite(tau)
    cosi = np.abs(np.sum((o_ray + np.nan_to_num(tau)[..., None] * d - c) / rho * d, -1)) / np.linalg.norm(d, axis=-1)
    safe = hit & (cosi > 0.3)  # away from grazing rays
    assert safe.mean() > 0.2 and np.all(g["depth"][safe] > 0)
    # trilinear interpolation of the distance errs by at most 3 s^2 / (8 rho) (s^2 / 8 times
    # the curvature 1 / rho on each axis), a depth error of that over the incidence cosine;
    # plus the refinement (0.002 voxel)
    err = np.abs(g["depth"] - np.nan_to_num(tau)) * np.linalg.norm(d, axis=-1) / s
    bound = 3 * s / (8 * rho) / np.maximum(cosi, 1e-9) + 0.002
    assert np.all(err[safe] <= bound[safe]), float((err - bound)[safe].max())
    o = oracle.raycast([ov], cam, T, ocfg(m.config), ids=[vid])
    compare_raycast(g, o, cam, T, s, require_hits=0.2)
    # inside, near the centre
    T = synth.look_at(c + np.array([0.05, 0.02, -0.03]), c + np.array([0.5, 0.3, 0.1]))
    g = gpu_maps(m.raycast(cam, T))
    o = oracle.raycast([ov], cam, T, ocfg(m.config), ids=[vid])
    assert not (g["depth"] > 0).any() and not (o["depth"] > 0).any()
    m.close()


def test_swap_out_in_roundtrip():
    wl = synth.single_volume_128(frames=6, res=34)
    tl = synth.tiled(wl, 2)
    m = Mapper()
    ids = [m.add_volume(t.h, t.r, t.s) for t in tl.volumes]
    for i in range(3):
        d, c = wl.frame(i)
        m.integrate(dev(d), dev(c), wl.cam, wl.poses[i])
    keep = ids[0]
    F0, W0, C0 = m.read_decoded(keep)
    m.swap_out(keep)
    q = m.query(keep)
    assert not q["resident"] and q["host_bytes"] > 0 and q["device_bytes"] == 0
    with pytest.raises(MVError):
        m.integrate_volume(keep, dev(wl.frame(3)[0]), None, wl.cam, wl.poses[3])
    for i in range(3, 6):
        d, c = wl.frame(i)
        m.integrate(dev(d), dev(c), wl.cam, wl.poses[i])  # skips the swapped-out volume
    F1, W1, C1 = m.read_decoded(keep)  # read from host memory
    np.testing.assert_array_equal(F0, F1)
    np.testing.assert_array_equal(W0, W1)
    np.testing.assert_array_equal(C0, C1)
    out = gpu_maps(m.raycast(wl.cam, wl.poses[0]))
    assert not np.any(out["vol_id"] == keep)
    m.swap_in(keep)
    assert m.query(keep)["resident"]
    F2, W2, C2 = m.read_decoded(keep)
    np.testing.assert_array_equal(F0, F2)
    np.testing.assert_array_equal(W0, W2)
    # the volume takes part again
    d, c = wl.frame(0)
    m.integrate(dev(d), dev(c), wl.cam, wl.poses[0])
    F3, W3, _ = m.read_decoded(keep)
    assert np.any(W3 != W2)
    m.remove_volume(ids[1])
    assert ids[1] not in m.volumes()
    m.close()


def test_raycast_unchanged_by_swap_and_host_write():
    """The raycast's derived cell masks are rebuilt from the voxels after a
    swap-in and after a host write: the maps of the same view stay identical
    bit for bit."""
    wl = synth.single_volume_128(frames=5, res=64)
    (vs,) = wl.volumes
    m = Mapper()
    vid = m.add_volume(vs.h, vs.r, vs.s)
    for i in range(5):
        d, c = wl.frame(i)
        m.integrate(dev(d), dev(c), wl.cam, wl.poses[i])
    a = gpu_maps(m.raycast(wl.cam, wl.poses[2]))
    assert (a["depth"] > 0).mean() > 0.2
    m.swap_out(vid)
    m.swap_in(vid)
    b = gpu_maps(m.raycast(wl.cam, wl.poses[2]))
    F, W, rgba = m.read_decoded(vid)
    m.write_decoded(vid, F, W, rgba)
    c = gpu_maps(m.raycast(wl.cam, wl.poses[2]))
    for k in ("depth", "normal", "rgba", "vol_id"):
        np.testing.assert_array_equal(a[k], b[k])
        np.testing.assert_array_equal(a[k], c[k])
    m.close()


def test_errors_leave_context_usable():
    m = Mapper()
    with pytest.raises(MVError) as e:
        m.add_volume((0, 0, 0), (8192, 8192, 8192), 0.001)  # ~4.4 TB
    assert "OOM" in str(e.value)
    with pytest.raises(MVError):
        m.remove_volume(12345)
    with pytest.raises(MVError):
        m.integrate_volume(77, dev(np.zeros((4, 4), np.float32)), None,
                           synth.Camera(4.0, 4.0, 1.5, 1.5, 4, 4), np.eye(4))
    vid = m.add_volume((0, 0, 0), (16, 16, 16), 0.01)
    m.integrate(dev(np.ones((4, 4), np.float32)), None, synth.Camera(4.0, 4.0, 1.5, 1.5, 4, 4), np.eye(4))
    m.synchronize()
    assert vid in m.volumes()
    m.close()


@pytest.mark.parametrize("fmt", ["f32", "f16", "i16"])
def test_full_size_512_sampled_parity(fmt):
    """The 512^3 / 640x480 room workload in the benchmark's launch
    configuration, in each storage format: lockstep parity of frame 4 on 2 M
    sampled voxels and the raycast on every 11th pixel."""
    wl = synth.room_512(frames=5)
    (vs,) = wl.volumes
    m = Mapper()
    vid = m.add_volume(vs.h, vs.r, vs.s, fmt)
    for i in range(4):
        d, c = wl.frame(i)
        m.integrate(dev(d), dev(c), wl.cam, wl.poses[i])
    before = oracle_volume_from_gpu(m, vid, vs)
    rng = np.random.default_rng(0)
    # sample half from updated-looking voxels (W > 0) and half uniformly
    seen = np.flatnonzero(before.W.reshape(-1) > 0)
    idx = np.unique(np.concatenate([rng.choice(seen, 1_000_000), rng.integers(0, before.F.size, 1_000_000)]))
    d, c = wl.frame(4)
    _, flags = oracle.integrate_voxels(before, idx, d, c, wl.cam, wl.poses[4], ocfg(m.config))
    m.integrate(dev(d), dev(c), wl.cam, wl.poses[4])
    F, W, rgba = m.read_decoded(vid)
    sel = np.zeros(before.F.shape, bool)
    sel.reshape(-1)[idx] = True
    fl = np.where(sel, flags, 255)  # unsampled voxels are excluded via the flag
    check_lockstep(before, F, W, rgba, fl, fmt=fmt)
    after = oracle_volume_from_gpu(m, vid, vs)
    T = wl.poses[4]
    pix = np.arange(0, wl.cam.width * wl.cam.height, 11)
    o = oracle.raycast([after], wl.cam, T, ocfg(m.config), ids=[vid], pixels=pix)
    g = gpu_maps(m.raycast(wl.cam, T))
    mask = np.zeros((wl.cam.height, wl.cam.width), bool)
    mask.reshape(-1)[pix] = True
    compare_raycast(g, o, wl.cam, T, vs.s, mask=mask, require_hits=0.5)
    m.close()


def test_frame_graph_equals_separate_calls():
    """mv_frame (one CUDA graph per frame, parameters updated in place) gives
    the same volumes and maps as mv_integrate + mv_raycast, also across a
    change of the resident set (graph rebuilt)."""
    wl = synth.single_volume_128(frames=6, res=34)
    tl = synth.tiled(wl, 2)
    a, b = Mapper(), Mapper()
    ida = [a.add_volume(t.h, t.r, t.s) for t in tl.volumes[:4]]
    idb = [b.add_volume(t.h, t.r, t.s) for t in tl.volumes[:4]]
    for i in range(wl.n_frames):
        if i == 3:  # change the resident set mid-sequence
            ida.append(a.add_volume(*_spec(tl.volumes[4])))
            idb.append(b.add_volume(*_spec(tl.volumes[4])))
            b.swap_out(idb[0])
            a.swap_out(ida[0])
        d, c = wl.frame(i)
        a.integrate(dev(d), dev(c), wl.cam, wl.poses[i])
        ga = gpu_maps(a.raycast(wl.cam, wl.poses[i]))
        gb = gpu_maps(b.frame(dev(d), dev(c), wl.cam, wl.poses[i]))
        for key in ("depth", "normal", "rgba", "vertex", "vol_id"):
            np.testing.assert_array_equal(ga[key], gb[key])
    for x, y in zip(ida, idb):
        Fa, Wa, Ca = a.read_decoded(x)
        Fb, Wb, Cb = b.read_decoded(y)
        np.testing.assert_array_equal(Fa, Fb)
        np.testing.assert_array_equal(Wa, Wb)
        np.testing.assert_array_equal(Ca, Cb)
    assert b.timings()["frame_graph"][0] == wl.n_frames
    a.close()
    b.close()


def _spec(t):
    return t.h, t.r, t.s


def test_autotune_changes_speed_not_results():
    """mv_autotune leaves the map untouched, and every launch shape gives
    bit-identical volumes and maps."""
    wl = synth.single_volume_128(frames=4, res=64)
    (vs,) = wl.volumes
    a, b = Mapper(), Mapper()
    va, vb = a.add_volume(vs.h, vs.r, vs.s), b.add_volume(vs.h, vs.r, vs.s)
    d, c = wl.frame(0)
    a.integrate(dev(d), dev(c), wl.cam, wl.poses[0])
    b.integrate(dev(d), dev(c), wl.cam, wl.poses[0])
    before = b.read_decoded(vb)
    d1, c1 = wl.frame(1)
    tun = b.autotune(dev(d1), dev(c1), wl.cam, wl.poses[1])
    assert tun["raycast_tile"] in range(4) and tun["integrate_ctas_per_sm"] >= 1
    assert all(t > 0 for t in tun["raycast_ms"])
    after = b.read_decoded(vb)
    for x, y in zip(before, after):
        np.testing.assert_array_equal(x, y)
    for i in range(1, 4):
        d, c = wl.frame(i)
        a.integrate(dev(d), dev(c), wl.cam, wl.poses[i])
        b.frame(dev(d), dev(c), wl.cam, wl.poses[i])
    for x, y in zip(a.read_decoded(va), b.read_decoded(vb)):
        np.testing.assert_array_equal(x, y)
    ref = gpu_maps(a.raycast(wl.cam, wl.poses[2]))
    for tile in range(4):
        b.set_tuning(tile, 2)
        got = gpu_maps(b.raycast(wl.cam, wl.poses[2]))
        for key in ("depth", "normal", "rgba", "vertex", "vol_id"):
            np.testing.assert_array_equal(ref[key], got[key])
    a.close()
    b.close()


@pytest.mark.parametrize("levels", [1, 2])
def test_uneven_volumes_batched_equals_per_volume_and_oracle(levels):
    """Volumes of different sizes and pitches, some out of view: the batched
    graph (view list, nearest first; work list built per brick or from the
    super bricks in view first) equals the per-volume loop bit for bit, and
    the merged raycast matches the oracle."""
    wl = synth.uneven_volumes(n_volumes=12, frames=6, edges=(16, 24, 40), pitch_mm=(15.0, 40.0),
                              half_extent=1.6, height_m=2.2, width=160, height=120)
    a, b = Mapper(), Mapper()
    t = a.tuning()
    a.set_tuning(t["raycast_tile"], t["integrate_ctas_per_sm"], levels)
    assert a.tuning()["work_list_levels"] == levels
    ida = [a.add_volume(v.h, v.r, v.s) for v in wl.volumes]
    idb = [b.add_volume(v.h, v.r, v.s) for v in wl.volumes]
    for i in range(wl.n_frames):
        d, c = wl.frame(i)
        ga = gpu_maps(a.frame(dev(d), dev(c), wl.cam, wl.poses[i]))
        for vid in idb:
            b.integrate_volume(vid, dev(d), dev(c), wl.cam, wl.poses[i])
        out = b.alloc_maps(wl.cam)
        for k, vid in enumerate(idb):
            b.raycast_volume(vid, k == 0, wl.cam, wl.poses[i], out)
        gb = gpu_maps(out)
        for key in ("depth", "normal", "rgba", "vertex", "vol_id"):
            np.testing.assert_array_equal(ga[key], gb[key])
    seen = 0
    for x, y, v in zip(ida, idb, wl.volumes):
        Fa, Wa, Ca = a.read_decoded(x)
        Fb, Wb, Cb = b.read_decoded(y)
        np.testing.assert_array_equal(Fa, Fb)
        np.testing.assert_array_equal(Wa, Wb)
        seen += (Wa > 0).any()
    assert 0 < seen < len(ida)  # some volumes were in view, some never
    ovs = [oracle_volume_from_gpu(a, i, v) for i, v in zip(ida, wl.volumes)]
    T = wl.poses[3]
    g = gpu_maps(a.raycast(wl.cam, T))
    o = oracle.raycast(ovs, wl.cam, T, ocfg(a.config), ids=ida)
    pitch = min(v.s for v in wl.volumes)
    compare_raycast(g, o, wl.cam, T, pitch, require_hits=0.05)
    a.close()
    b.close()


@pytest.mark.parametrize("fmt", ["f32", "f16", "i16"])
def test_full_size_uneven_volumes_sampled_parity(fmt):
    """The 64 uneven volumes at full size (edges 128-768, pitches 1-8 mm, 7.3 G
    voxels) at 640x480, through the batched frame graph in each storage
    format: lockstep parity of frame 5 on up to 2 M sampled voxels of every
    observed volume, and the merged raycast of that frame on every 2nd
    pixel.  Each volume is read (mv_read_box) over the box of its observed
    bricks joined with the part of the view frustum that frame 5 can update
    (depths up to its largest depth + mu), widened by 2 voxels: outside it no
    voxel is observed, so samples there lie in cells with an unobserved
    corner (invalid: they cannot bracket) and the oracle, given the box as a
    volume, finds the same hits; volumes with nothing observed cannot hold a
    hit and are left out."""
    from parity_utils import frustum_box, observed_box, union_box
    wl = synth.uneven_volumes(frames=6)
    m = Mapper()
    ids = [m.add_volume(v.h, v.r, v.s, fmt) for v in wl.volumes]
    k = 5
    for i in range(k):
        d, c = wl.frame(i)
        m.frame(dev(d), dev(c), wl.cam, wl.poses[i])
    m.synchronize()
    d, c = wl.frame(k)
    T = wl.poses[k]
    z_far = float(d.max()) + 0.05  # mu is 4 voxels of at most 8 mm
    boxes, before = {}, {}
    for vid, v in zip(ids, wl.volumes):
        box = union_box(observed_box(m, vid, v), frustum_box(v, wl.cam, T, z_far))
        if box is not None:
            boxes[vid] = box
            before[vid] = m.read_box_decoded(vid, *box)
    maps = gpu_maps(m.frame(dev(d), dev(c), wl.cam, T))
    rng = np.random.default_rng(7)
    crops, checked = [], 0
    for vid, v in zip(ids, wl.volumes):
        if vid not in boxes:
            assert observed_box(m, vid, v) is None  # frame k observed nothing outside the frustum box
            continue
        lo, n = boxes[vid]
        F1, W1, c1 = m.read_box_decoded(vid, lo, n)
        if not (W1 > 0).any():
            continue
        h = tuple(int(v.h[a] + lo[a]) for a in range(3))
        after = oracle.Volume(h, tuple(n), float(v.s), F1, W1, c1)
        crops.append((vid, after))
        F0, W0, c0 = before[vid]
        prior = oracle.Volume(h, tuple(n), float(v.s), F0.copy(), W0.copy(), c0.copy())
        seen = np.flatnonzero(after.W.reshape(-1) > 0)
        nsm = min(1_000_000, seen.size)
        idx = np.unique(np.concatenate([rng.choice(seen, nsm, replace=False),
                                        rng.integers(0, prior.F.size, nsm)]))
        _, flags = oracle.integrate_voxels(prior, idx, d, c, wl.cam, T, ocfg(m.config))
        sel = np.zeros(prior.F.shape, bool)
        sel.reshape(-1)[idx] = True
        check_lockstep(prior, after.F, after.W, after.rgba, np.where(sel, flags, 255), fmt=fmt)
        checked += int(sel.sum())
    assert len(crops) >= 2 and checked > 1_000_000
    pix = np.arange(0, wl.cam.width * wl.cam.height, 2)
    o = oracle.raycast([v for _, v in crops], wl.cam, T, ocfg(m.config), ids=[i for i, _ in crops], pixels=pix)
    mask = np.zeros((wl.cam.height, wl.cam.width), bool)
    mask.reshape(-1)[pix] = True
    pitch = min(v.s for _, v in crops)
    # the observed volumes cover a small part of this early view (about 1.4 %
    # of the pixels hit): every 2nd pixel gives a few thousand hits
    res = compare_raycast(maps, o, wl.cam, T, pitch, mask=mask, require_hits=0.01)
    assert res["hits"] > 1000
    m.close()


def test_read_box_equals_the_whole_volume_cropped():
    """mv_read_box returns the box of mv_read_volume, resident or swapped out."""
    wl = synth.single_volume_128(frames=3, res=40)
    (vs,) = wl.volumes
    for fmt in ("f32", "i16"):
        m = Mapper()
        vid = m.add_volume(vs.h, vs.r, vs.s, fmt)
        for i in range(wl.n_frames):
            d, c = wl.frame(i)
            m.integrate(dev(d), dev(c), wl.cam, wl.poses[i])
        raw, col = m.read_volume(vid)
        for lo, n in (((0, 0, 0), tuple(vs.r)), ((3, 9, 17), (20, 5, 11)), ((39, 0, 7), (1, 40, 1))):
            sl = (slice(lo[2], lo[2] + n[2]), slice(lo[1], lo[1] + n[1]), slice(lo[0], lo[0] + n[0]))
            for swapped in (False, True):
                if swapped:
                    m.swap_out(vid)
                r2, c2 = m.read_box(vid, lo, n)
                np.testing.assert_array_equal(r2, raw[sl])
                np.testing.assert_array_equal(c2, col[sl])
                if swapped:
                    m.swap_in(vid)
        with pytest.raises(MVError):
            m.read_box(vid, (0, 0, 0), (41, 1, 1))
        m.close()


def test_two_level_list_at_scale_equals_one_level():
    """Eight 512^3 tiles (2.1 M resident bricks, above the automatic
    threshold): the frame graph's two-level work list (super bricks in view,
    then their bricks) gives the same volumes' brick flags, the same counts
    of listed bricks and updated voxels, and the same maps as the one-level
    list, frame after frame."""
    wl = synth.room_tiles(res=512, pitch=0.003, split=2, frames=4)
    a, b = Mapper(), Mapper()
    ida = [a.add_volume(v.h, v.r, v.s) for v in wl.volumes]
    idb = [b.add_volume(v.h, v.r, v.s) for v in wl.volumes]
    t = b.tuning()
    b.set_tuning(t["raycast_tile"], t["integrate_ctas_per_sm"], 1)
    assert a.tuning()["work_list_levels"] == 0  # automatic: two levels at this size
    for i in range(wl.n_frames):
        d, c = wl.frame(i)
        a.timings(reset=True)
        ga = gpu_maps(a.frame(dev(d), dev(c), wl.cam, wl.poses[i]))
        gb = gpu_maps(b.frame(dev(d), dev(c), wl.cam, wl.poses[i]))
        assert a.timings()["brick_list"][0] == 2  # super bricks, then their bricks
        for key in ("depth", "normal", "rgba", "vertex", "vol_id"):
            np.testing.assert_array_equal(ga[key], gb[key])
        sa, sb = a.stats(reset=True), b.stats(reset=True)
        for key in ("swept", "updated", "band", "bricks", "ray_hits"):
            assert sa[key] == sb[key], key
        assert sa["updated"] > 0 and sa["ray_hits"] > 0
    for x, y in zip(ida, idb):
        np.testing.assert_array_equal(a.read_brick_flags(x), b.read_brick_flags(y))
    a.close()
    b.close()


def test_surface_count_skip_and_far_cull_are_exact():
    """Two exact shortcuts.  (1) A volume in which no brick holds an observed
    voxel at or behind a surface (every brick flag NO-NEGATIVE) cannot end a
    bracket; the raycast skips it whole (no samples) and the maps equal those
    without it.  The per-volume count behind the skip follows every path that
    changes the flags: integration, device writes, host writes to a swapped-out
    volume, and the swap.  (2) Bricks farther than the frame's farthest valid
    depth plus mu are never updated, so they are not listed at all."""
    s = 0.01
    scene = synth.Scene()
    scene.planes = np.array([[0.0, 0.0, 1.0, 1.0]])  # wall z = 1 m
    cam = synth.Camera(100.0, 100.0, 39.5, 29.5, 80, 60)
    poses = [synth.look_at((0.01 * i, -0.005 * i, 0.0), (0.0, 0.0, 1.0), up=(0.0, 1.0, 0.0)) for i in range(6)]
    air = synth.VolumeSpec((-30, -25, 35), (60, 50, 20), s)      # z in [0.35, 0.54]: free space only
    wall = synth.VolumeSpec((-40, -32, 90), (80, 64, 20), s)     # z in [0.90, 1.09]: holds the wall
    far = synth.VolumeSpec((-60, -50, 150), (120, 100, 16), s)   # z in [1.50, 1.65]: behind the wall
    wl = synth.Workload("wall", cam, scene, poses, [air, wall, far], seed=3)
    m = Mapper()
    ia, ib, ic = (m.add_volume(v.h, v.r, v.s) for v in wl.volumes)
    for i in range(wl.n_frames):
        d, c = wl.frame(i)
        assert np.nanmax(np.where(d > 0, d, np.nan)) < 1.05
        m.stats(reset=True)
        m.integrate_volume(ic, dev(d), dev(c), cam, poses[i])
        assert m.stats()["bricks"] == 0  # every brick of `far` lies beyond max depth + mu
        m.integrate(dev(d), dev(c), cam, poses[i])
    assert (m.read_decoded(ic)[1] == 0).all()
    Fa, Wa, _ = m.read_decoded(ia)
    assert (Wa > 0).mean() > 0.3 and (Fa[Wa > 0] > 0).all()
    assert (m.read_brick_flags(ia) & 4).all() and not (m.read_brick_flags(ib) & 4).all()
    T = poses[2]

    def alone(vid):
        out = m.alloc_maps(cam)
        m.stats(reset=True)
        m.raycast_volume(vid, True, cam, T, out)
        return m.stats()["ray_samples"], gpu_maps(out)

    sa, ga = alone(ia)
    assert sa == 0 and (ga["vol_id"] < 0).all()
    sb, gb = alone(ib)
    assert sb > 0 and (gb["vol_id"] == ib).mean() > 0.9
    m.stats(reset=True)
    g = gpu_maps(m.raycast(cam, T))
    assert m.stats()["ray_samples"] == sb
    for key in ("depth", "normal", "rgba", "vertex", "vol_id"):
        np.testing.assert_array_equal(g[key], gb[key])

    # a plane z = 0.45 m written into `air`: now it must be marched and hit
    z = (air.h[2] + np.arange(air.r[2]))[:, None, None] * s
    F_plane = np.broadcast_to(np.clip((0.45 - z) / (4 * s), -1, 1), Fa.shape).astype(np.float32)
    ones = np.ones_like(F_plane)
    o, dirs = synth.pixel_rays(cam, T)
    tau = (0.45 - o[..., 2]) / dirs[..., 2]

    def check_plane_hit():
        sa, ga = alone(ia)
        assert sa > 0
        hit = ga["vol_id"] == ia
        assert hit.mean() > 0.9
        err = np.abs(ga["depth"] - tau) * np.linalg.norm(dirs, axis=-1) / s
        assert err[hit].max() < 2e-3
        np.testing.assert_array_equal(gpu_maps(m.raycast(cam, T))["vol_id"][hit], ia)

    m.write_decoded(ia, F_plane, ones)            # resident: flags recomputed on the device
    check_plane_hit()
    m.swap_out(ia)
    m.write_decoded(ia, np.ones_like(F_plane), ones)  # swapped out: flags recomputed on the host
    m.swap_in(ia)
    assert alone(ia)[0] == 0
    m.swap_out(ia)
    m.write_decoded(ia, F_plane, ones)
    m.swap_in(ia)
    check_plane_hit()
    m.swap_out(ia)                                # the count travels with the swap
    m.swap_in(ia)
    check_plane_hit()
    m.close()


def test_reserved_pinned_buffers_roundtrip():
    """Swap-outs served from reserved pinned buffers (and from buffers that
    removed volumes gave back) keep the volumes bit for bit."""
    wl = synth.single_volume_128(frames=4, res=64)
    (vs,) = wl.volumes
    m = Mapper()
    m.reserve_host(vs.r, "f32", 1)
    ids = [m.add_volume(vs.h, vs.r, vs.s) for _ in range(3)]
    for i in range(4):
        d, c = wl.frame(i)
        m.integrate(dev(d), dev(c), wl.cam, wl.poses[i])
    ref = m.read_decoded(ids[0])
    for vid in ids:
        m.swap_out(vid)
    m.remove_volume(ids[2])  # its host buffers go back to the spares
    extra = m.add_volume(vs.h, vs.r, vs.s)
    m.write_decoded(extra, *ref)
    m.swap_out(extra)
    for vid in (ids[0], ids[1], extra):
        m.swap_in(vid)
        for a, b in zip(m.read_decoded(vid), ref):
            np.testing.assert_array_equal(a, b)
    m.reserve_host(vs.r, "f32", 0)
    m.close()


@pytest.mark.parametrize("fmts", ["f32", "mixed"])
def test_raycast_batch_equals_single_views(fmts):
    """mv_raycast_batch (every view in one launch) gives each view the maps of
    mv_raycast at that pose, bit for bit, on uneven volumes (view lists,
    merge across volumes; F32 only, or the three storage formats mixed) and
    on an empty context."""
    import torch
    wl = synth.uneven_volumes(n_volumes=12, frames=6, edges=(16, 24, 40), pitch_mm=(15.0, 40.0),
                              half_extent=1.6, height_m=2.2, width=160, height=120)
    m = Mapper()
    for k, v in enumerate(wl.volumes):
        m.add_volume(v.h, v.r, v.s, "f32" if fmts == "f32" else ("f32", "f16", "i16")[k % 3])
    for i in range(4):
        d, c = wl.frame(i)
        m.integrate(dev(d), dev(c), wl.cam, wl.poses[i])
    poses = np.stack([wl.poses[i] for i in (0, 2, 3, 5, 1)])
    n, H, W = len(poses), wl.cam.height, wl.cam.width
    out = dict(depth=torch.empty((n, H, W), dtype=torch.float32, device="cuda"),
               normal=torch.empty((n, H, W, 3), dtype=torch.float32, device="cuda"),
               rgba=torch.empty((n, H, W, 4), dtype=torch.uint8, device="cuda"),
               vertex=torch.empty((n, H, W, 3), dtype=torch.float32, device="cuda"),
               vol_id=torch.empty((n, H, W), dtype=torch.int32, device="cuda"))
    m.raycast_batch(wl.cam, poses, out=out)
    got = gpu_maps(out)
    for k in range(n):
        ref = gpu_maps(m.raycast(wl.cam, poses[k]))
        for key in ("depth", "normal", "rgba", "vertex", "vol_id"):
            np.testing.assert_array_equal(got[key][k], ref[key], err_msg=f"view {k} {key}")
    assert (got["depth"] > 0).mean() > 0.05
    m.close()
    e = Mapper()
    emp = e.raycast_batch(wl.cam, poses[:2])
    assert np.all(host(emp["depth"]) == 0) and np.all(host(emp["vol_id"]) == -1)
    e.close()
