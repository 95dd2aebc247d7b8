"""Raycast gradients on the GPU (mv_raycast_backward) against the FP64
oracle's analytic gradients, a loose FP32 finite-difference check, and
Adam pose refinement through the torch.autograd.Function."""
import numpy as np
import pytest

import oracle
from paper_1511_07106_b300 import Config, Mapper, diff, synth
from parity_utils import dev, gpu_maps, oracle_volume_from_gpu

pytestmark = pytest.mark.gpu

EXACT = Config(n_bisect=30)  # the differentiable forward wants the exact root


def prefilled(wl, frames, cfg=EXACT, fmt="f32"):
    m = Mapper(cfg)
    ids = [m.add_volume(v.h, v.r, v.s, fmt) for v in wl.volumes]
    for i in range(frames):
        d, c = wl.frame(i)
        m.integrate(dev(d), dev(c), wl.cam, wl.poses[i])
    return m, ids


def safe_pixels(ovs, ids, cam, T, margin=0.02):
    """Pixels whose oracle hit is included and lies well inside its cell."""
    g = oracle.raycast_grad(ovs, cam, T, ids=ids, want_tsdf=False)
    o, d = synth.pixel_rays(cam, T)
    vol_of = {i: v for i, v in zip(ids, ovs)}
    raw = oracle.raycast(ovs, cam, T, ids=ids)
    ok = (g["excluded"] == 0) & (raw["vol"] >= 0)
    out = np.zeros_like(ok)
    for y, x in zip(*np.nonzero(ok)):
        v = vol_of[raw["vol"][y, x]]
        q = (o + g["depth"][y, x] * d[y, x]) / v.s - np.array(v.h)
        fr = q - np.floor(q)
        out[y, x] = np.all((fr > margin) & (fr < 1 - margin))
    return out, g


def random_colours(m, ids, seed):
    """Replace the volumes' RGB by random per-voxel colours (TSDF, weights and
    colour weights kept): the scene's colours are constant on each primitive,
    which leaves almost no hit with a colour gradient to check."""
    rng = np.random.default_rng(seed)
    for vid in ids:
        raw, col = m.read_volume(vid)
        col[..., :3] = rng.integers(0, 256, size=col[..., :3].shape, dtype=np.uint8)
        m.write_volume(vid, raw, col)


def incidence(ovs, ids, cam, T):
    """|cos| of the angle between each pixel's ray and the oracle's normal."""
    o = oracle.raycast(ovs, cam, T, ids=ids)
    _, d = synth.pixel_rays(cam, T)
    dn = d / np.linalg.norm(d, axis=-1, keepdims=True)
    return np.abs(np.sum(o["normal"] * dn, -1))


def per_pixel_pose_jacobians(m, cam, T, maps, pix, channel=None):
    """GPU dL/dxi of single pixels: one view per listed pixel (the same pose
    and forward maps), each with a one-hot upstream gradient on its pixel --
    on the depth (channel None) or on one colour channel.  Returns (n, 6)."""
    import torch
    n = len(pix)
    H, W = cam.height, cam.width
    depth = maps["depth"][None].expand(n, H, W).contiguous()
    vid = maps["vol_id"][None].expand(n, H, W).contiguous()
    ys = torch.tensor([p[0] for p in pix], device="cuda")
    xs = torch.tensor([p[1] for p in pix], device="cuda")
    k = torch.arange(n, device="cuda")
    gd = gc = None
    if channel is None:
        gd = torch.zeros((n, H, W), dtype=torch.float32, device="cuda")
        gd[k, ys, xs] = 1.0
    else:
        gc = torch.zeros((n, H, W, 3), dtype=torch.float32, device="cuda")
        gc[k, ys, xs, channel] = 1.0
    gp = torch.zeros((n, 6), dtype=torch.float32, device="cuda")
    m.raycast_backward(cam, np.repeat(np.asarray(T)[None], n, 0), depth, vid, gd, gc, gp, {})
    return gp.cpu().numpy().astype(np.float64)


def check_pixel_jacobians(g, o, what):
    """Per pixel: |g - o| <= 1e-3 |o| + 1e-4 median |o| (6-vectors; FP32
    gradient arithmetic at the FP32-refined root against the FP64 exact root,
    on pixels whose hit is away from cell faces and not grazing; the second
    term covers pixels whose Jacobian nearly cancels, e.g. a colour gradient
    summed from eight corner colours)."""
    err = np.linalg.norm(g - o, axis=-1)
    on = np.linalg.norm(o, axis=-1)
    lim = 1e-3 * on + 1e-4 * np.median(on) + 1e-9
    bad = err > lim
    assert not bad.any(), (f"{what}: {bad.sum()} of {len(err)} pixels off; worst relative "
                           f"{(err / np.maximum(np.linalg.norm(o, axis=-1), 1e-30)).max():.3g}")


def check_voxel_gradients(gts, ids, o_gF, what, rel=1e-3, floor=1e-5):
    """Per voxel: |g - o| <= rel |o| + floor max |o| over all volumes.  The
    floor covers the FP32 hit position's error in the small trilinear weights
    of far corners: about r 2^-24 voxel for coordinates up to r voxels (1e-5
    of the largest gradient at 64^3, 1e-4 at 256^3)."""
    top = max(np.abs(a).max() for a in o_gF)
    assert top > 0, f"{what}: no TSDF gradient"
    nz = 0
    for k, i in enumerate(ids):
        g = gts[i].cpu().numpy().astype(np.float64)
        o = o_gF[k]
        bad = np.abs(g - o) > rel * np.abs(o) + floor * top
        assert not bad.any(), (f"{what}: volume {i}: {bad.sum()} voxels off, e.g. "
                               f"{[(tuple(int(v) for v in q), g[tuple(q)], o[tuple(q)]) for q in np.argwhere(bad)[:3]]}")
        # every voxel that receives a gradient on one side receives it on the other
        assert np.array_equal(g != 0, o != 0), f"{what}: volume {i}: gradient support differs"
        nz += int((o != 0).sum())
    return nz


@pytest.mark.parametrize("fmt", ["f32", "f16", "i16"])
def test_backward_pose_jacobians_match_oracle_per_pixel(fmt):
    """dtau/dxi and dC/dxi pixel by pixel (not summed over the image, where
    errors of opposite sign could cancel) against the FP64 oracle, in each
    storage format (the oracle reads the same stored values, decoded)."""
    wl = synth.room_tiles(res=64, pitch=0.008, frames=12, width=160, height=120)
    m, ids = prefilled(wl, 12, fmt=fmt)
    random_colours(m, ids, 11)
    ovs = [oracle_volume_from_gpu(m, i, v) for i, v in zip(ids, wl.volumes)]
    T = wl.poses[5]
    safe, o = safe_pixels(ovs, ids, wl.cam, T)
    safe &= incidence(ovs, ids, wl.cam, T) > 0.05
    assert safe.mean() > 0.3
    rng = np.random.default_rng(0)
    cand = np.argwhere(safe)
    pix = [tuple(p) for p in cand[rng.choice(len(cand), size=192, replace=False)]]
    maps = m.alloc_maps(wl.cam)
    m.raycast(wl.cam, T, out=maps)
    g = per_pixel_pose_jacobians(m, wl.cam, T, maps, pix)
    check_pixel_jacobians(g, np.stack([o["jac_tau"][p] for p in pix]), "dtau/dxi")
    for ch in range(3):
        g = per_pixel_pose_jacobians(m, wl.cam, T, maps, pix, channel=ch)
        o_c = np.stack([o["jac_rgb"][p][ch] for p in pix])
        assert np.all(np.linalg.norm(o_c, axis=-1) > 0)
        check_pixel_jacobians(g, o_c, f"dC{ch}/dxi")
    m.close()


@pytest.mark.parametrize("fmt", ["f32", "f16", "i16"])
def test_backward_tsdf_gradients_match_oracle_per_voxel(fmt):
    """dL/dF voxel by voxel: (a) depth path, positive upstream weights on
    every safe pixel (the terms of one voxel share a sign, so a relative
    tolerance per voxel is meaningful); (b) colour path, random upstream on
    pixels 9 apart (cells of different pixels rarely share voxels).  A
    gradient scattered to the wrong corner, a dropped colour term or a wrong
    scale fails here even where the image-wide norm would agree."""
    import torch
    wl = synth.room_tiles(res=64, pitch=0.008, frames=12, width=160, height=120)
    m, ids = prefilled(wl, 12, fmt=fmt)
    random_colours(m, ids, 12)
    ovs = [oracle_volume_from_gpu(m, i, v) for i, v in zip(ids, wl.volumes)]
    T = wl.poses[5]
    safe, _ = safe_pixels(ovs, ids, wl.cam, T)
    safe &= incidence(ovs, ids, wl.cam, T) > 0.05
    rng = np.random.default_rng(3)
    maps = m.alloc_maps(wl.cam)
    m.raycast(wl.cam, T, out=maps)
    H, W = wl.cam.height, wl.cam.width
    sparse = np.zeros((H, W), bool)
    sparse[::9, ::9] = True
    cases = (("depth path", np.where(safe, rng.uniform(0.5, 1.5, size=safe.shape), 0.0), None),
             ("colour path", None, np.where((safe & sparse)[..., None], rng.normal(size=(H, W, 3)), 0.0)))
    for what, gd, gc in cases:
        o = oracle.raycast_grad(ovs, wl.cam, T, grad_depth=gd, grad_rgb=gc, ids=ids)
        gp = torch.zeros((1, 6), dtype=torch.float32, device="cuda")
        gts = {i: torch.zeros(tuple(v.r[::-1]), dtype=torch.float32, device="cuda")
               for i, v in zip(ids, wl.volumes)}
        m.raycast_backward(wl.cam, T[None], maps["depth"][None].contiguous(), maps["vol_id"][None].contiguous(),
                           None if gd is None else dev(gd.astype(np.float32))[None].contiguous(),
                           None if gc is None else dev(gc.astype(np.float32))[None].contiguous(), gp, gts)
        nz = check_voxel_gradients(gts, ids, o["grad_F"], what)
        assert nz > (1000 if gd is not None else 100), f"{what}: only {nz} voxels with a gradient"
        g_pose = gp.cpu().numpy()[0].astype(np.float64)
        assert np.linalg.norm(g_pose - o["grad_pose"]) <= 1e-3 * np.linalg.norm(o["grad_pose"])
    m.close()


def test_backward_matches_float32_finite_differences():
    """Loose check (FP32 forward noise): d/dxi of sum_p w_p depth_p over pixels
    whose hits stay in their cells."""
    import torch
    wl = synth.room_tiles(res=64, pitch=0.008, frames=12, width=160, height=120, seed=7)
    m, ids = prefilled(wl, 12)
    ovs = [oracle_volume_from_gpu(m, i, v) for i, v in zip(ids, wl.volumes)]
    T = wl.poses[3]
    safe, _ = safe_pixels(ovs, ids, wl.cam, T, margin=0.1)
    rng = np.random.default_rng(1)
    wgt = np.where(safe, rng.uniform(0.5, 1.5, size=safe.shape), 0.0)
    maps = m.alloc_maps(wl.cam)
    m.raycast(wl.cam, T, out=maps)
    gp = torch.zeros((1, 6), dtype=torch.float32, device="cuda")
    m.raycast_backward(wl.cam, T[None], maps["depth"][None].contiguous(), maps["vol_id"][None].contiguous(),
                       dev(wgt.astype(np.float32))[None].contiguous(), None, gp, {})
    an = gp.cpu().numpy()[0]
    h = 1e-4
    fd = np.zeros(6)
    for k in range(6):
        e = np.zeros(6)
        e[k] = h
        dp = gpu_maps(m.raycast(wl.cam, oracle.se3_exp(e) @ T))["depth"].astype(np.float64)
        dm = gpu_maps(m.raycast(wl.cam, oracle.se3_exp(-e) @ T))["depth"].astype(np.float64)
        fd[k] = np.sum(wgt * (dp - dm)) / (2 * h)
    rel = np.linalg.norm(an - fd) / np.linalg.norm(fd)
    assert rel < 5e-2, (an, fd)
    m.close()


def test_adam_pose_refinement_reduces_pose_error():
    import torch
    wl = synth.room_tiles(res=64, pitch=0.008, frames=40, width=160, height=120, seed=5)
    m, ids = prefilled(wl, 40)
    idx = [4, 14, 24, 34]
    T_true = [wl.poses[i] for i in idx]
    T_init = synth.perturb_poses(T_true, seed=6, sigma_t=0.02, sigma_r_deg=1.0)
    with torch.no_grad():
        ref_d, ref_c = diff.render(m, wl.cam, torch.tensor(np.stack(T_true)))

    def err(Ts):
        t = np.mean([np.linalg.norm(a[:3, 3] - b[:3, 3]) for a, b in zip(Ts, T_true)])
        r = np.mean([np.degrees(np.arccos(np.clip((np.trace(a[:3, :3].T @ b[:3, :3]) - 1) / 2, -1, 1)))
                     for a, b in zip(Ts, T_true)])
        return t, r

    t0, r0 = err(T_init)
    T_fin, losses = diff.refine_poses(m, wl.cam, np.stack(T_init), ref_d, ref_c, steps=50)
    t1, r1 = err(T_fin)
    assert losses[-1] < 0.5 * losses[0]
    assert t1 < 0.5 * t0 and r1 < 0.5 * r0, (t0, t1, r0, r1)
    m.close()


@pytest.mark.parametrize("fmt", ["f32", "i16"])
def test_fused_l1_backward_equals_loss_grad_then_backward(fmt):
    """mv_raycast_backward_l1 against the Python closed form (l1_loss_grad)
    followed by mv_raycast_backward on the same renders: the same pose-gradient
    bits and the loss to float rounding; the fused and unfused refinement then
    take the same steps (the same poses, bit for bit); with no pixel valid in
    both renders the gradient and the loss are 0."""
    import torch
    wl = synth.room_tiles(res=64, pitch=0.008, frames=40, width=160, height=120, seed=5)
    m, ids = prefilled(wl, 40, fmt=fmt)
    random_colours(m, ids, 3)
    cam = wl.cam
    T_true = np.stack([wl.poses[i] for i in (4, 14, 24, 34)])
    T = np.stack(synth.perturb_poses(list(T_true), seed=6, sigma_t=0.02, sigma_r_deg=1.0))
    n = T.shape[0]
    ref = m.raycast_batch(cam, T_true)
    ref_d, ref_rgba = ref["depth"], ref["rgba"]
    ref_c = ref_rgba[..., :3].float() / 255.0
    out = m.raycast_batch(cam, T)
    colour = out["rgba"][..., :3].float() / 255.0
    loss, gd, gc = diff.l1_loss_grad(out["depth"], colour, ref_d, ref_c, 0.1)
    g1 = torch.zeros((n, 6), dtype=torch.float32, device="cuda")
    m.raycast_backward(cam, T, out["depth"], out["vol_id"], gd.contiguous(), gc.contiguous(), g1, {})
    g2 = torch.zeros_like(g1)
    l2 = torch.zeros(1, dtype=torch.float32, device="cuda")
    m.raycast_backward_l1(cam, T, out["depth"], out["rgba"], out["vol_id"], ref_d, ref_rgba, 0.1, g2, l2)
    assert torch.count_nonzero(g1) == 6 * n
    assert torch.equal(g1, g2)
    assert abs(float(l2) - float(loss)) <= 1e-5 * abs(float(loss))

    Ta, la = diff.refine_poses(m, cam, T, ref_d, ref_c, steps=3, fused=True)
    Tb, lb = diff.refine_poses(m, cam, T, ref_d, ref_c, steps=3, fused=False)
    np.testing.assert_array_equal(Ta, Tb)
    np.testing.assert_allclose(la, lb, rtol=1e-5)

    none = torch.zeros_like(ref_d)
    m.raycast_backward_l1(cam, T, out["depth"], out["rgba"], out["vol_id"], none, ref_rgba, 0.1, g2, l2)
    assert torch.count_nonzero(g2) == 0 and float(l2) == 0.0

    # a colour buffer that does not start on a 4-byte boundary is refused on
    # the host before any launch
    import ctypes as C
    from paper_1511_07106_b300 import _abi
    from paper_1511_07106_b300.mapper import intrinsics
    shifted = torch.zeros(ref_rgba.numel() + 4, dtype=torch.uint8, device="cuda")
    P = np.ascontiguousarray(T.reshape(-1, 16))
    K = intrinsics(cam)
    st = m._lib.mv_raycast_backward_l1(
        m._h, C.byref(K), P.ctypes.data_as(C.POINTER(C.c_double)), n, C.c_void_p(out["depth"].data_ptr()),
        C.c_void_p(shifted.data_ptr() + 1), C.c_void_p(out["vol_id"].data_ptr()), C.c_void_p(ref_d.data_ptr()),
        C.c_void_p(ref_rgba.data_ptr()), 0.1, C.c_void_p(g2.data_ptr()), C.c_void_p(l2.data_ptr()), None)
    assert st == _abi.MV_ERR_ARG
    m.close()


def test_full_size_tiles_gradients_sampled():
    """The differentiable-raycast workload at full size: 8 x 256^3 tiles at
    2 mm, 640x480, two poses perturbed by N(0, 2 cm) / N(0, 1 deg).  On a
    sample of pixels (every 13th): per-pixel pose Jacobians of depth and
    colour and per-voxel TSDF gradients against the FP64 oracle, and the
    pose gradient against FP32 central differences."""
    import torch
    wl = synth.room_tiles(frames=30)
    m, ids = prefilled(wl, 30)
    random_colours(m, ids, 13)
    ovs = [oracle_volume_from_gpu(m, i, v) for i, v in zip(ids, wl.volumes)]
    cam = wl.cam
    H, W = cam.height, cam.width
    pix = np.arange(0, H * W, 13)
    sel = np.zeros((H, W), bool)
    sel.reshape(-1)[pix] = True
    T_init = synth.perturb_poses([wl.poses[8], wl.poses[22]], seed=6)
    rng = np.random.default_rng(21)
    maps = m.alloc_maps(cam)
    for T in T_init:
        g0 = oracle.raycast_grad(ovs, cam, T, ids=ids, want_tsdf=False, pixels=pix)
        o, d = synth.pixel_rays(cam, T)
        dn = d / np.linalg.norm(d, axis=-1, keepdims=True)
        raw = oracle.raycast(ovs, cam, T, ids=ids, pixels=pix)
        safe = sel & (g0["excluded"] == 0) & (raw["vol"] >= 0)
        safe &= np.abs(np.sum(raw["normal"] * dn, -1)) > 0.05
        vol_of = {i: v for i, v in zip(ids, ovs)}
        for y, x in zip(*np.nonzero(safe)):
            v = vol_of[raw["vol"][y, x]]
            q = (o + g0["depth"][y, x] * d[y, x]) / v.s - np.array(v.h)
            fr = q - np.floor(q)
            safe[y, x] = np.all((fr > 0.02) & (fr < 0.98))
        assert safe.sum() > 0.3 * sel.sum()
        m.raycast(cam, T, out=maps)
        cand = np.argwhere(safe)
        pp = [tuple(p) for p in cand[rng.choice(len(cand), size=96, replace=False)]]
        g = per_pixel_pose_jacobians(m, cam, T, maps, pp)
        check_pixel_jacobians(g, np.stack([g0["jac_tau"][p] for p in pp]), "dtau/dxi")
        for ch in range(3):
            g = per_pixel_pose_jacobians(m, cam, T, maps, pp, channel=ch)
            check_pixel_jacobians(g, np.stack([g0["jac_rgb"][p][ch] for p in pp]), f"dC{ch}/dxi")
        # FP32 central differences of sum_p w_p depth_p on the GPU forward;
        # pixels whose hit jumps to another surface under a perturbation of
        # 1e-4 (a silhouette nearer than the step) are left out of the sum
        h = 1e-4
        w = np.where(safe, rng.uniform(0.5, 1.5, size=safe.shape), 0.0)
        pm = []
        for k in range(6):
            e = np.zeros(6)
            e[k] = h
            dp = gpu_maps(m.raycast(cam, oracle.se3_exp(e) @ T))["depth"].astype(np.float64)
            dm = gpu_maps(m.raycast(cam, oracle.se3_exp(-e) @ T))["depth"].astype(np.float64)
            pm.append((dp, dm))
            w = np.where((dp > 0) & (dm > 0) & (np.abs(dp - dm) < 2e-3), w, 0.0)
        assert (w > 0).sum() > 0.9 * safe.sum()
        fd = np.array([np.sum(w * (dp - dm)) / (2 * h) for dp, dm in pm])
        m.raycast(cam, T, out=maps)
        # TSDF gradients of the depth path, per voxel, over all 8 volumes
        ob = oracle.raycast_grad(ovs, cam, T, grad_depth=w, ids=ids, pixels=np.flatnonzero(w > 0))
        gp = torch.zeros((1, 6), dtype=torch.float32, device="cuda")
        gts = {i: torch.zeros(tuple(v.r[::-1]), dtype=torch.float32, device="cuda")
               for i, v in zip(ids, wl.volumes)}
        m.raycast_backward(cam, T[None], maps["depth"][None].contiguous(), maps["vol_id"][None].contiguous(),
                           dev(w.astype(np.float32))[None].contiguous(), None, gp, gts)
        nz = check_voxel_gradients(gts, ids, ob["grad_F"], "depth path", floor=1e-4)
        assert nz > 10000
        an = gp.cpu().numpy()[0].astype(np.float64)
        assert np.linalg.norm(an - ob["grad_pose"]) <= 1e-3 * np.linalg.norm(ob["grad_pose"])
        assert np.linalg.norm(an - fd) <= 5e-2 * np.linalg.norm(fd), (an, fd)
        del gts
    m.close()
