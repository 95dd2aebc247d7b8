"""Pins for the oracle's raycast gradients (left se(3) pose perturbation
T(xi) = exp(xi^) T, xi = (rho, phi) in the world frame, and TSDF voxel values):
the plane's closed form, central finite differences of the (separately pinned)
FP64 forward, and the chain rule.  CPU only."""
import numpy as np
import pytest

import oracle
from paper_1511_07106_b300 import synth

CAM = synth.Camera(40.0, 40.0, 15.5, 11.5, 32, 24)


def voxel_positions(vol):
    rx, ry, rz = vol.r
    z, y, x = np.meshgrid(np.arange(rz), np.arange(ry), np.arange(rx), indexing="ij")
    return np.stack([(vol.h[0] + x) * vol.s, (vol.h[1] + y) * vol.s, (vol.h[2] + z) * vol.s], -1)


def test_se3_exp_properties():
    assert np.allclose(oracle.se3_exp(np.zeros(6)), np.eye(4))
    rng = np.random.default_rng(0)
    xi = rng.normal(size=6) * 0.3
    E = oracle.se3_exp(xi)
    Rm = E[:3, :3]
    assert np.allclose(Rm @ Rm.T, np.eye(3), atol=1e-12) and np.isclose(np.linalg.det(Rm), 1.0)
    # rotation about z by theta is the textbook rotation matrix
    th = 0.7
    assert np.allclose(oracle.se3_exp([0, 0, 0, 0, 0, th])[:3, :3], synth.rotation([0, 0, 1], th), atol=1e-12)
    # first order: exp(h xi) = I + h xi^ + O(h^2)
    h = 1e-6
    Eh = oracle.se3_exp(h * xi)
    hat = np.zeros((4, 4))
    hat[:3, :3] = [[0, -xi[5], xi[4]], [xi[5], 0, -xi[3]], [-xi[4], xi[3], 0]]
    hat[:3, 3] = xi[:3]
    assert np.allclose((Eh - np.eye(4)) / h, hat, atol=1e-5)


def plane_volume(n, dd):
    vol = oracle.Volume(h=(-25, -25, -25), r=(50, 50, 50), s=0.02)
    mu = 4 * vol.s
    vol.F[:] = np.clip((dd - voxel_positions(vol) @ n) / mu, -1, 1)
    vol.W[:] = 1.0
    return vol


def test_plane_depth_gradient_closed_form():
    """tau* = (dd - n.o) / (n.d): d tau/d rho = -n / (n.d) and
    d tau/d phi = -(x* x n) / (n.d), from differentiating the intersection."""
    rng = np.random.default_rng(1)
    n = rng.normal(size=3)
    n /= np.linalg.norm(n)
    dd = 0.05
    vol = plane_volume(n, dd)
    eye = -0.6 * n + rng.normal(scale=0.03, size=3)
    T = synth.look_at(eye, eye + n + rng.normal(scale=0.1, size=3))
    out = oracle.raycast_grad([vol], CAM, T)
    o, d = synth.pixel_rays(CAM, T)
    nd = d @ n
    tau = (dd - o @ n) / nd
    x = o + tau[..., None] * d
    ok = out["excluded"] == 0
    assert ok.mean() > 0.5
    exp_rho = -n[None, None, :] / nd[..., None]
    exp_phi = -np.cross(x, n) / nd[..., None]
    np.testing.assert_allclose(out["jac_tau"][ok][:, :3], exp_rho[ok], rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(out["jac_tau"][ok][:, 3:], exp_phi[ok], rtol=1e-9, atol=1e-12)


def sphere_volume_with_colour(seed=2):
    rng = np.random.default_rng(seed)
    vol = oracle.Volume(h=(-25, -25, -25), r=(50, 50, 50), s=0.02)
    p = voxel_positions(vol)
    c, rho = np.array([0.02, -0.01, 0.03]), 0.3
    vol.F[:] = np.clip((np.linalg.norm(p - c, axis=-1) - rho) / (4 * vol.s), -1, 1)
    vol.W[:] = 1.0
    # smooth colour field
    vol.rgba[..., 0] = np.clip(128 + 300 * p[..., 0], 0, 255).astype(np.uint8)
    vol.rgba[..., 1] = np.clip(128 + 300 * p[..., 1], 0, 255).astype(np.uint8)
    vol.rgba[..., 2] = np.clip(128 + 300 * p[..., 2], 0, 255).astype(np.uint8)
    vol.rgba[..., 3] = 1
    T = synth.look_at((0.15, -0.1, -0.55), c + rng.normal(scale=0.02, size=3))
    return vol, T


def trilinear_rgb(vol, x):
    q = x / vol.s - np.array(vol.h)
    c = np.clip(np.floor(q), 0, np.array(vol.r) - 2).astype(int)
    f = q - c
    out = np.zeros(3)
    for k in range(8):
        dx, dy, dz = k & 1, (k >> 1) & 1, (k >> 2) & 1
        w = (f[0] if dx else 1 - f[0]) * (f[1] if dy else 1 - f[1]) * (f[2] if dz else 1 - f[2])
        out += w * vol.rgba[c[2] + dz, c[1] + dy, c[0] + dx, :3] / 255.0
    return out


def interior(vol, out, margin=0.05):
    """Pixels whose hit lies well inside a cell (FD steps stay in one cell)."""
    ok = out["excluded"] == 0
    o, d = synth.pixel_rays(CAM, out["T"])
    x = o + out["depth"][..., None] * d
    q = x / vol.s - np.array(vol.h)
    fr = q - np.floor(q)
    return ok & np.all((fr > margin) & (fr < 1 - margin), -1)


@pytest.mark.parametrize("k", range(6))
def test_pose_gradient_matches_central_differences(k):
    vol, T = sphere_volume_with_colour()
    out = oracle.raycast_grad([vol], CAM, T)
    out["T"] = T
    sel = interior(vol, out)
    assert sel.sum() > 40
    h = 1e-5
    e = np.zeros(6)
    e[k] = h
    Tp, Tm = oracle.se3_exp(e) @ T, oracle.se3_exp(-e) @ T
    rp = oracle.raycast([vol], CAM, Tp)
    rm = oracle.raycast([vol], CAM, Tm)
    fd = (rp["depth"] - rm["depth"]) / (2 * h)
    an = out["jac_tau"][..., k]
    err = np.abs(fd - an)[sel] / (np.abs(an[sel]) + 1e-3)
    assert np.median(err) < 1e-6 and err.max() < 1e-4
    # colour: C(x*(xi)) through an independent trilinear evaluation of the hit point
    ys, xs = np.nonzero(sel)
    for y, x in list(zip(ys, xs))[::7]:
        cp = trilinear_rgb(vol, rp["vertex"][y, x])
        cm = trilinear_rgb(vol, rm["vertex"][y, x])
        fdc = (cp - cm) / (2 * h)
        anc = out["jac_rgb"][y, x, :, k]
        assert np.all(np.abs(fdc - anc) <= 1e-4 * (np.abs(anc) + 1e-2))


def test_tsdf_gradient_matches_central_differences():
    """d tau / dF_j at single pixels: one-hot upstream gradient, FD of the
    forward with each of the hit cell's 8 corner values perturbed."""
    vol, T = sphere_volume_with_colour(3)
    base = oracle.raycast_grad([vol], CAM, T)
    base["T"] = T
    sel = interior(vol, base)
    ys, xs = np.nonzero(sel)
    checked = 0
    for y, x in list(zip(ys, xs))[::25][:6]:
        gd = np.zeros((CAM.height, CAM.width))
        gd[y, x] = 1.0
        g = oracle.raycast_grad([vol], CAM, T, grad_depth=gd)["grad_F"][0]
        idx = np.argwhere(g != 0)
        assert len(idx) == 8
        for z, yy, xx in idx:
            h = 1e-5
            v2 = vol.copy()
            v2.F[z, yy, xx] += h
            tp = oracle.raycast([v2], CAM, T)["depth"][y, x]
            v2.F[z, yy, xx] -= 2 * h
            tm = oracle.raycast([v2], CAM, T)["depth"][y, x]
            fd = (tp - tm) / (2 * h)
            assert abs(fd - g[z, yy, xx]) <= 1e-4 * abs(g[z, yy, xx]) + 1e-9
            checked += 1
    assert checked >= 24


def test_upstream_gradients_follow_the_chain_rule():
    vol, T = sphere_volume_with_colour(4)
    rng = np.random.default_rng(5)
    gd = rng.normal(size=(CAM.height, CAM.width))
    gc = rng.normal(size=(CAM.height, CAM.width, 3))
    out = oracle.raycast_grad([vol], CAM, T, grad_depth=gd, grad_rgb=gc)
    exp = np.einsum("hw,hwk->k", gd, out["jac_tau"]) + np.einsum("hwc,hwck->k", gc, out["jac_rgb"])
    np.testing.assert_allclose(out["grad_pose"], exp, rtol=1e-10, atol=1e-10)
    assert np.all(out["jac_tau"][out["excluded"] != 0] == 0)


def test_colour_tsdf_gradient_matches_central_differences():
    """dC/dF_j (colour of the hit moves with the hit point): one-hot colour
    upstream gradient against FD of the independently interpolated colour at
    the forward's hit vertex."""
    vol, T = sphere_volume_with_colour(6)
    base = oracle.raycast_grad([vol], CAM, T)
    base["T"] = T
    sel = interior(vol, base)
    ys, xs = np.nonzero(sel)
    checked = 0
    for y, x in list(zip(ys, xs))[::31][:4]:
        for ch in range(3):
            gc = np.zeros((CAM.height, CAM.width, 3))
            gc[y, x, ch] = 1.0
            g = oracle.raycast_grad([vol], CAM, T, grad_rgb=gc)["grad_F"][0]
            for z, yy, xx in np.argwhere(g != 0)[::3]:
                h = 1e-5
                v2 = vol.copy()
                v2.F[z, yy, xx] += h
                cp = trilinear_rgb(vol, oracle.raycast([v2], CAM, T)["vertex"][y, x])[ch]
                v2.F[z, yy, xx] -= 2 * h
                cm = trilinear_rgb(vol, oracle.raycast([v2], CAM, T)["vertex"][y, x])[ch]
                fd = (cp - cm) / (2 * h)
                assert abs(fd - g[z, yy, xx]) <= 1e-4 * abs(g[z, yy, xx]) + 1e-7
                checked += 1
    assert checked >= 12


def test_pixel_subset_gradients_equal_the_full_image_restricted():
    """The pixel-list form computes exactly the listed pixels of the full
    image's per-pixel outputs, and its sums run over those pixels only."""
    vol, T = sphere_volume_with_colour(seed=4)
    rng = np.random.default_rng(5)
    gd = rng.normal(size=(CAM.height, CAM.width))
    gc = rng.normal(size=(CAM.height, CAM.width, 3))
    pix = np.arange(0, CAM.width * CAM.height, 5)
    sel = np.zeros((CAM.height, CAM.width), bool)
    sel.reshape(-1)[pix] = True
    full = oracle.raycast_grad([vol], CAM, T, grad_depth=np.where(sel, gd, 0.0),
                               grad_rgb=np.where(sel[..., None], gc, 0.0))
    sub = oracle.raycast_grad([vol], CAM, T, grad_depth=gd, grad_rgb=gc, pixels=pix)
    for k in ("depth", "jac_tau", "jac_rgb", "excluded"):
        np.testing.assert_array_equal(sub[k][sel], full[k][sel])
        assert not np.any(sub[k][~sel])
    assert (sub["depth"][sel] > 0).mean() > 0.3
    np.testing.assert_allclose(sub["grad_pose"], full["grad_pose"], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(sub["grad_F"][0], full["grad_F"][0], rtol=1e-12, atol=1e-15)
