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


def prefilled(wl, frames, cfg=EXACT):
    m = Mapper(cfg)
    ids = [m.add_volume(v.h, v.r, v.s) for v in wl.volumes]
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


def test_backward_matches_oracle_gradients():
    import torch
    wl = synth.room_tiles(res=64, pitch=0.008, frames=12, width=160, height=120)
    m, ids = prefilled(wl, 12)
    ovs = [oracle_volume_from_gpu(m, i, v) for i, v in zip(ids, wl.volumes)]
    T = wl.poses[5]
    safe, _ = safe_pixels(ovs, ids, wl.cam, T)
    assert safe.mean() > 0.3
    rng = np.random.default_rng(0)
    gd = np.where(safe, rng.normal(size=safe.shape), 0.0)
    gc = np.where(safe[..., None], rng.normal(size=safe.shape + (3,)), 0.0)
    o = oracle.raycast_grad(ovs, wl.cam, T, grad_depth=gd, grad_rgb=gc, ids=ids)
    maps = m.alloc_maps(wl.cam)
    m.raycast(wl.cam, T, out=maps)
    gp = torch.zeros((1, 6), dtype=torch.float32, device="cuda")
    gts = {i: torch.zeros(tuple(v.r[::-1]), dtype=torch.float32, device="cuda")
           for i, v in zip(ids, wl.volumes)}
    m.raycast_backward(wl.cam, T[None], maps["depth"][None].contiguous(), maps["vol_id"][None].contiguous(),
                       dev(gd.astype(np.float32))[None].contiguous(),
                       dev(gc.astype(np.float32))[None].contiguous(), gp, gts)
    g_pose = gp.cpu().numpy()[0].astype(np.float64)
    rel = np.linalg.norm(g_pose - o["grad_pose"]) / np.linalg.norm(o["grad_pose"])
    assert rel < 1e-3, (g_pose, o["grad_pose"])
    num = sum(np.linalg.norm(gts[i].cpu().numpy() - o["grad_F"][k]) ** 2 for k, i in enumerate(ids))
    den = sum(np.linalg.norm(o["grad_F"][k]) ** 2 for k in range(len(ids)))
    assert np.sqrt(num / den) < 1e-3
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
    T_fin, losses = diff.refine_poses(m, wl.cam, np.stack(T_init), ref_d, ref_c, steps=50, lr=2e-3)
    t1, r1 = err(T_fin)
    assert losses[-1] < 0.5 * losses[0]
    assert t1 < 0.5 * t0 and r1 < 0.5 * r0, (t0, t1, r0, r1)
    m.close()
