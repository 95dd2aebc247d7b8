"""Volumes at the size limits of the library, through the C ABI, on a B300.

Two limits are exercised: a volume of more than 2^32 voxels (the kernels'
64-bit voxel offsets; every other test stays below 2^32) and volumes 8192
voxels long on one axis (brick index 1023, the largest the 10-bit fields of
a work-list entry hold).  Each is checked against a small volume on the same
lattice: the global-lattice positions make overlapping volumes of one pitch
see bit-identical samples (Sec. Comparison to KinectFusion), so the large
volume's voxels in the small one's box, and its maps where both volumes hold
the hit well inside, must equal the small volume's bit for bit; the small
volume is checked against the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_1511_07106_b300 import Config, Mapper, synth
from parity_utils import compare_raycast, dev, gpu_maps, oracle_volume_from_gpu

pytestmark = pytest.mark.gpu


def _ocfg(cfg: Config):
    return oracle.Config(trunc_vox=cfg.trunc_voxels, w_max=cfg.w_max, color_w_max=cfg.color_w_max,
                         z_min=cfg.z_min, z_max=cfg.z_max, step_vox=cfg.ray_step)


def _poses(centre, n, seed):
    """n camera poses looking along +z from near `centre` (mm jitter, < 1 degree)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        T = np.eye(4)
        R = synth.rotation((1.0, 0.0, 0.0), np.deg2rad(rng.uniform(-0.8, 0.8))) @ \
            synth.rotation((0.0, 1.0, 0.0), np.deg2rad(rng.uniform(-0.8, 0.8)))
        T[:3, :3] = R
        T[:3, 3] = np.asarray(centre, float) + rng.uniform(-0.004, 0.004, 3)
        out.append(T)
    return out


def _hits_inside(maps, cam, T, spec, pitch, margin):
    """Pixels whose hit point lies inside the box of `spec` by `margin` voxels."""
    o, d = synth.pixel_rays(cam, T)
    p = o + maps["depth"][..., None].astype(np.float64) * d
    q = p / pitch - np.asarray(spec.h, float)
    inside = np.all((q >= margin) & (q <= np.asarray(spec.r, float) - 1 - margin), axis=-1)
    return inside & (maps["depth"] > 0)


def _check_against_small(big_spec, small_spec, scene, cam, poses, min_pixels, cfg=Config()):
    big, small = Mapper(cfg), Mapper(cfg)
    bid = big.add_volume(big_spec.h, big_spec.r, big_spec.s)
    sid = small.add_volume(small_spec.h, small_spec.r, small_spec.s)
    for i, T in enumerate(poses):
        d, c = synth.render(scene, cam, T, seed=11, frame=i)
        big.integrate(dev(d), dev(c), cam, T)
        small.integrate(dev(d), dev(c), cam, T)
    lo = [small_spec.h[a] - big_spec.h[a] for a in range(3)]
    raw_b, col_b = big.read_box(bid, lo, small_spec.r)
    raw_s, col_s = small.read_volume(sid)
    assert (raw_s[..., 1] > 0).sum() > 1000, "the small volume saw too little"
    np.testing.assert_array_equal(raw_b, raw_s)
    np.testing.assert_array_equal(col_b, col_s)
    T = poses[-1]
    a = gpu_maps(big.raycast(cam, T))
    b = gpu_maps(small.raycast(cam, T))
    sel = _hits_inside(b, cam, T, small_spec, small_spec.s, 3.0)
    assert sel.sum() >= min_pixels, f"only {sel.sum()} pixels hit inside the small volume"
    for k in ("depth", "normal", "rgba"):
        np.testing.assert_array_equal(a[k][sel], b[k][sel])
    # the small volume against the FP64 oracle on the same state
    ov = oracle_volume_from_gpu(small, sid, small_spec)
    o = oracle.raycast([ov], cam, T, _ocfg(small.config), ids=[sid])
    compare_raycast(b, o, cam, T, small_spec.s, require_hits=0.5 * min_pixels / (cam.width * cam.height))
    big.close()
    small.close()


def test_volume_beyond_2_32_voxels_equals_small_volume():
    """2048 x 2048 x 1040 voxels (4.36 G voxels, 52 GB at F32 with colour):
    its raycast takes the 64-bit offset path."""
    s = 0.005
    big = synth.VolumeSpec((-1024, -1024, 0), (2048, 2048, 1040), s)
    assert np.prod(big.r, dtype=np.int64) > 2 ** 32
    small = synth.VolumeSpec((-32, -32, 470), (64, 64, 64), s)
    n = np.array([0.15, -0.10, 1.0])
    n /= np.linalg.norm(n)
    scene = synth.Scene(planes=np.array([[*n, n @ np.array([0.0, 0.0, 2.5])]]),
                        spheres=np.array([[0.05, 0.03, 2.42, 0.06]]))
    cam = synth.Camera(300.0, 300.0, 79.5, 59.5, 160, 120)
    _check_against_small(big, small, scene, cam, _poses((0.0, 0.0, 0.0), 4, 21), min_pixels=500)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_8192_voxel_long_volume_equals_small_volume(axis):
    """8192 x 16 x 16 voxels along `axis` at 1 mm, seen at its far end (brick
    index 1023 on that axis); a fronto-parallel plane crosses it."""
    s = 0.001
    f = 600.0 if axis < 2 else 1200.0
    cam = synth.Camera(f, f, 79.5, 59.5, 160, 120)
    if axis < 2:
        # the strip lies across the view at 1 m; the camera looks at its far end
        r = [16, 16, 16]
        r[axis] = 8192
        h = [-8, -8, 992]
        h[axis] = -4096
        rs = [16, 16, 16]
        rs[axis] = 64
        hs = list(h)
        hs[axis] = 4000
        centre = [0.0, 0.0, 0.0]
        centre[axis] = 4.03
        plane_z = 1.0
    else:
        # the tube runs along the view; the camera sits inside it, 1 m before the plane
        r, h = [16, 16, 8192], [-8, -8, 0]
        rs, hs = [16, 16, 64], [-8, -8, 8128]
        centre = [0.0, 0.0, 7.184]
        plane_z = 8.184  # voxel 8184: brick 1023
    big = synth.VolumeSpec(tuple(h), tuple(r), s)
    small = synth.VolumeSpec(tuple(hs), tuple(rs), s)
    assert big.r[axis] == 8192  # 1024 bricks: indices 0 .. 1023
    scene = synth.Scene(planes=np.array([[0.0, 0.0, 1.0, plane_z]]))
    poses = _poses(centre, 4, 31 + axis)
    _check_against_small(big, small, scene, cam, poses, min_pixels=40 if axis == 2 else 100)


def test_misaligned_buffers_are_refused_before_any_launch():
    """Device buffers the kernels access as 4-byte words must start on a
    4-byte boundary: the entry points return MV_ERR_ARG for a depth frame or
    a map one or two bytes off, launch nothing, and the context keeps
    working."""
    import ctypes as C
    import torch
    from paper_1511_07106_b300 import _abi
    from paper_1511_07106_b300.mapper import intrinsics
    cam = synth.Camera(40.0, 40.0, 15.5, 11.5, 32, 24)
    m = Mapper()
    m.add_volume((-8, -8, 20), (16, 16, 16), 0.02)
    K = intrinsics(cam)
    T = np.ascontiguousarray(np.eye(4).reshape(16))
    Tp = T.ctypes.data_as(C.POINTER(C.c_double))
    buf = torch.zeros(4 * cam.width * cam.height + 16, dtype=torch.uint8, device="cuda")
    base = buf.data_ptr()
    assert m._lib.mv_integrate(m._h, C.c_void_p(base + 1), None, C.byref(K), Tp, None) == _abi.MV_ERR_ARG
    assert m._lib.mv_raycast(m._h, C.byref(K), Tp, None, None, C.c_void_p(base + 2), None, None,
                             None) == _abi.MV_ERR_ARG
    assert m._lib.mv_depth_to_maps(m._h, C.c_void_p(base + 2), C.byref(K), None, C.c_void_p(base),
                                   C.c_void_p(base), None) == _abi.MV_ERR_ARG
    depth = torch.full((cam.height, cam.width), 0.5, dtype=torch.float32, device="cuda")
    rgb = torch.zeros((cam.height, cam.width, 3), dtype=torch.uint8, device="cuda")
    m.integrate(depth, rgb, cam, np.eye(4))
    maps = m.raycast(cam, np.eye(4))
    assert maps["depth"].shape == (cam.height, cam.width)
    m.close()
