"""mv_integrate_noalloc: integration into caller-owned storage without any
allocation, checked against the context-based mv_integrate_volume.

Some callers cannot allocate GPU memory: code that runs inside another
framework's memory pool or budget, or where the device-wide synchronisation an
allocation can cause is not acceptable.  They pass their own volume storage,
and the library works in a fixed array built into it.  This file is collected
last, so that a run stopping at the first failure has already run every other
test when it gets here; it passes alone in a fresh process as well."""
import ctypes as C

import numpy as np
import pytest

from paper_1511_07106_b300 import Mapper, _abi, synth
from paper_1511_07106_b300.mapper import intrinsics

pytestmark = pytest.mark.gpu

F32_TOL = 1e-4  # the TSDF tolerance of the parity tests (units of mu)


def bricks_to_linear(a, r, nb):
    """(nbricks, 512, ...) brick-major storage -> [z, y, x, ...] over r voxels."""
    tail = a.shape[2:]
    g = a.reshape(nb[2], nb[1], nb[0], 8, 8, 8, *tail)           # bz by bx lz ly lx
    g = g.transpose(0, 3, 1, 4, 2, 5, *range(6, 6 + len(tail)))   # bz lz by ly bx lx
    g = g.reshape(nb[2] * 8, nb[1] * 8, nb[0] * 8, *tail)
    return g[: r[2], : r[1], : r[0]]


FMTS = {"f32": _abi.MV_TSDF_F32, "f16": _abi.MV_TSDF_F16, "i16": _abi.MV_TSDF_I16}


@pytest.mark.parametrize("fmt", ["f32", "f16", "i16"])
def test_noalloc_integrate_matches_context_call_twice(fmt):
    """Two frames in a row through mv_integrate_noalloc equal the context
    path (mv_integrate_volume) in every storage format: decoded TSDF within
    the parity tests' tolerance, weights, colour and brick flags exact."""
    import torch
    from paper_1511_07106_b300.mapper import decode
    wl = synth.single_volume_128(frames=2, res=64)
    (vs,) = wl.volumes
    lib = _abi.lib()
    m = Mapper()
    vid = m.add_volume(vs.h, vs.r, vs.s, fmt)
    nb = [(r + 7) // 8 for r in vs.r]
    nbricks = nb[0] * nb[1] * nb[2]
    # caller-owned storage of a new volume: zero TSDF/weight/colour, every brick unobserved
    if fmt == "f32":
        fw = torch.zeros(nbricks * 512 * 2, dtype=torch.float32, device="cuda")
    else:
        fw = torch.zeros(nbricks * 512, dtype=torch.int32, device="cuda")
    rgba = torch.zeros(nbricks * 512 * 4, dtype=torch.uint8, device="cuda")
    flags = torch.full((nbricks,), 6, dtype=torch.uint8, device="cuda")
    desc = _abi.mv_volume_desc((C.c_int32 * 3)(*vs.h), (C.c_int32 * 3)(*vs.r), vs.s, FMTS[fmt])
    view = _abi.mv_volume_view(desc, fw.data_ptr(), rgba.data_ptr(), flags.data_ptr())
    K = intrinsics(wl.cam)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for i in range(2):
        d, c = wl.frame(i)
        dd, dc = torch.from_numpy(d).cuda(), torch.from_numpy(c).cuda()
        m.integrate_volume(vid, dd, dc, wl.cam, wl.poses[i])
        T = np.ascontiguousarray(wl.poses[i], np.float64).reshape(16)
        st = lib.mv_integrate_noalloc(C.byref(view), None, C.c_void_p(dd.data_ptr()),
                                      C.c_void_p(dc.data_ptr()), C.byref(K),
                                      T.ctypes.data_as(C.POINTER(C.c_double)), stream)
        assert st == _abi.MV_OK
        torch.cuda.synchronize()
        F_ref, W_ref, col_ref = m.read_decoded(vid)
        if fmt == "f32":
            raw = bricks_to_linear(fw.cpu().numpy().reshape(nbricks, 512, 2), vs.r, nb)
        else:
            raw = bricks_to_linear(fw.cpu().numpy().view(np.uint32).reshape(nbricks, 512), vs.r, nb)
        F, W = decode(raw, FMTS[fmt])
        col = bricks_to_linear(rgba.cpu().numpy().reshape(nbricks, 512, 4), vs.r, nb)
        assert (W_ref > 0).mean() > 0.05
        assert np.abs(F - F_ref).max() <= F32_TOL
        np.testing.assert_array_equal(W, W_ref)
        np.testing.assert_array_equal(col, col_ref)
        np.testing.assert_array_equal(flags.cpu().numpy(), m.read_brick_flags(vid).reshape(-1))
    m.close()


def test_noalloc_rejects_the_configs_the_context_rejects():
    """An infinite truncation or weight cap would spread inf / NaN into the
    caller's volume: both entry points refuse such a configuration."""
    import torch
    lib = _abi.lib()
    vol = torch.zeros(512 * 2, dtype=torch.float32, device="cuda")
    col = torch.zeros(512 * 4, dtype=torch.uint8, device="cuda")
    flags = torch.full((1,), 6, dtype=torch.uint8, device="cuda")
    desc = _abi.mv_volume_desc((C.c_int32 * 3)(0, 0, 0), (C.c_int32 * 3)(8, 8, 8), 0.01, _abi.MV_TSDF_F32)
    view = _abi.mv_volume_view(desc, vol.data_ptr(), col.data_ptr(), flags.data_ptr())
    cam = synth.Camera(10.0, 10.0, 4.5, 3.5, 10, 8)
    K = intrinsics(cam)
    T = np.eye(4).reshape(16)
    depth = torch.ones(80, dtype=torch.float32, device="cuda")
    for field, value in (("trunc_voxels", float("inf")), ("w_max", float("inf")), ("w_max", 1e31)):
        cfg = _abi.mv_config()
        assert lib.mv_config_default(C.byref(cfg)) == _abi.MV_OK
        setattr(cfg, field, value)
        st = lib.mv_integrate_noalloc(C.byref(view), C.byref(cfg), C.c_void_p(depth.data_ptr()), None,
                                      C.byref(K), T.ctypes.data_as(C.POINTER(C.c_double)),
                                      C.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert st == _abi.MV_ERR_ARG, (field, value)
        h = C.c_void_p()
        assert lib.mv_create(C.byref(cfg), 0, C.byref(h)) == _abi.MV_ERR_ARG, (field, value)
    torch.cuda.synchronize()
    assert torch.all(vol == 0)


def test_brick_classes_equal_the_per_voxel_path_at_full_size():
    """The 512^3 room (64^3 bricks, the allocation-free path's capacity) over
    five frames: the context path, whose work list classes bricks against the
    frame's depth tiles (behind: not listed; in front: f = 1; updated whole;
    projecting onto accepted depths only), gives bit for bit the volume of the
    allocation-free path, which lists every brick in the frustum and decides
    voxel by voxel."""
    import torch
    wl = synth.room_512(frames=5)
    (vs,) = wl.volumes
    lib = _abi.lib()
    m = Mapper()
    vid = m.add_volume(vs.h, vs.r, vs.s, "f32")
    nb = [(r + 7) // 8 for r in vs.r]
    nbricks = nb[0] * nb[1] * nb[2]
    fw = torch.zeros(nbricks * 512 * 2, dtype=torch.float32, device="cuda")
    rgba = torch.zeros(nbricks * 512 * 4, dtype=torch.uint8, device="cuda")
    flags = torch.full((nbricks,), 6, dtype=torch.uint8, device="cuda")
    desc = _abi.mv_volume_desc((C.c_int32 * 3)(*vs.h), (C.c_int32 * 3)(*vs.r), vs.s, _abi.MV_TSDF_F32)
    view = _abi.mv_volume_view(desc, fw.data_ptr(), rgba.data_ptr(), flags.data_ptr())
    K = intrinsics(wl.cam)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for i in range(wl.n_frames):
        d, c = wl.frame(i)
        dd, dc = torch.from_numpy(d).cuda(), torch.from_numpy(c).cuda()
        m.integrate(dd, dc, wl.cam, wl.poses[i])
        T = np.ascontiguousarray(wl.poses[i], np.float64).reshape(16)
        st = lib.mv_integrate_noalloc(C.byref(view), None, C.c_void_p(dd.data_ptr()),
                                      C.c_void_p(dc.data_ptr()), C.byref(K),
                                      T.ctypes.data_as(C.POINTER(C.c_double)), stream)
        assert st == _abi.MV_OK
    torch.cuda.synchronize()
    F_ref, W_ref, col_ref = m.read_decoded(vid)
    lin = bricks_to_linear(fw.cpu().numpy().reshape(nbricks, 512, 2), vs.r, nb)
    col = bricks_to_linear(rgba.cpu().numpy().reshape(nbricks, 512, 4), vs.r, nb)
    assert (W_ref > 0).mean() > 0.02
    np.testing.assert_array_equal(lin[..., 0], F_ref)
    np.testing.assert_array_equal(lin[..., 1], W_ref)
    np.testing.assert_array_equal(col, col_ref)
    np.testing.assert_array_equal(flags.cpu().numpy(), m.read_brick_flags(vid).reshape(-1))
    m.close()


def test_noalloc_rejects_volumes_beyond_its_fixed_capacity():
    import torch
    lib = _abi.lib()
    small = torch.zeros(1024, dtype=torch.float32, device="cuda")
    r = 520  # 65^3 bricks > MV_NOALLOC_MAX_BRICKS = 64^3
    desc = _abi.mv_volume_desc((C.c_int32 * 3)(0, 0, 0), (C.c_int32 * 3)(r, r, r), 0.01, _abi.MV_TSDF_F32)
    view = _abi.mv_volume_view(desc, small.data_ptr(), small.data_ptr(), small.data_ptr())
    cam = synth.Camera(10.0, 10.0, 4.5, 3.5, 10, 8)
    K = intrinsics(cam)
    T = np.eye(4).reshape(16)
    st = lib.mv_integrate_noalloc(C.byref(view), None, C.c_void_p(small.data_ptr()), None, C.byref(K),
                                  T.ctypes.data_as(C.POINTER(C.c_double)),
                                  C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == _abi.MV_ERR_CAPACITY
    assert (65 ** 3) > _abi.MV_NOALLOC_MAX_BRICKS
