"""Pins for the oracle's depth-map conversion and point-to-plane ICP
(Sec. Depth Map Conversion; Sec. Camera Tracking): plane normals in closed
form, zero residual at the true pose, and convergence to a known pose on a
scene of planes.  CPU only."""
import numpy as np

import oracle
from paper_1511_07106_b300 import synth

CAM = synth.Camera(60.0, 60.0, 31.5, 23.5, 64, 48)


def test_fronto_parallel_plane_maps():
    D = 1.25
    depth = np.full((CAM.height, CAM.width), D, np.float32)
    depth[10, 20] = 0.0  # a hole
    v, n = oracle.depth_maps(depth, CAM)
    xs = (np.arange(CAM.width) - CAM.cx) / CAM.fx * D
    np.testing.assert_allclose(v[5, :, 0], xs, rtol=1e-15)
    assert np.all(v[..., 2][depth > 0] == D) and np.all(v[10, 20] == 0)
    inner = np.zeros(depth.shape, bool)
    inner[:-1, :-1] = True
    inner[10, 20] = inner[9, 20] = inner[10, 19] = False  # the hole and the two pixels that use it
    np.testing.assert_allclose(n[inner], np.broadcast_to([0.0, 0.0, -1.0], n[inner].shape), atol=1e-15)
    assert np.all(n[~inner] == 0)
    # world frame: rotated normal, moved vertex
    T = synth.look_at((0.3, -0.2, 1.0), (0.5, 2.0, 0.8))
    vw, nw = oracle.depth_maps(depth, CAM, T)
    np.testing.assert_allclose(vw[inner], v[inner] @ T[:3, :3].T + T[:3, 3], atol=1e-12)
    np.testing.assert_allclose(nw[inner], n[inner] @ T[:3, :3].T, atol=1e-12)


def test_tilted_plane_normals_are_the_plane_normal():
    scene = synth.Scene()
    nrm = np.array([0.3, -0.2, 1.0])
    nrm /= np.linalg.norm(nrm)
    scene.planes = np.array([list(nrm) + [2.0]])
    T = synth.look_at((0.1, 0.2, 0.0), (0.2, 0.1, 3.0), up=(0.0, 1.0, 0.0))
    depth, _ = synth.render(scene, CAM, T, noise=False)
    _, nw = oracle.depth_maps(depth, CAM, T)
    ok = np.any(nw != 0, -1)
    assert ok.mean() > 0.9
    # facing the camera: the plane normal oriented against the viewing direction
    want = nrm if nrm @ (T[:3, 3] - 2.0 * nrm) > 0 else -nrm
    assert np.abs(nw[ok] - want).max() < 1e-5  # float32 depths


def corner_scene():
    scene = synth.Scene()
    scene.planes = np.array([[0.0, 0.0, 1.0, 0.0], [1.0, 0.0, 0.0, 2.0], [0.0, 1.0, 0.0, 1.5]])
    T_true = synth.look_at((0.2, -0.4, 1.1), (1.6, 1.2, 0.3))
    depth, _ = synth.render(scene, CAM, T_true, noise=False)
    return scene, T_true, depth


def test_zero_residual_at_the_true_pose():
    _, T, depth = corner_scene()
    v, n = oracle.depth_maps(depth, CAM)
    mv, mn = oracle.depth_maps(depth, CAM, T)
    out = oracle.icp_system(v, n, CAM, T, mv.astype(np.float32), mn.astype(np.float32), T, 0.1, 0.8)
    assert out["count"] > 0.8 * (CAM.width - 1) * (CAM.height - 1)
    # the model maps are float32: residuals of their rounding only (|r| < 4e-7 m)
    assert out["error"] < out["count"] * 1.6e-13 and np.abs(out["b"]).max() < out["count"] * 3 * 4e-7
    np.testing.assert_allclose(out["A"], out["A"].T)
    assert np.linalg.eigvalsh(out["A"]).min() > 0  # three planes constrain all six directions


def test_icp_converges_to_the_true_pose():
    _, T_true, depth = corner_scene()
    mv, mn = oracle.depth_maps(depth, CAM, T_true)
    delta = np.array([0.012, -0.008, 0.01, 0.01, -0.015, 0.008])
    T0 = oracle.se3_exp(delta) @ T_true
    T, last = oracle.track(depth, CAM, mv.astype(np.float32), mn.astype(np.float32), T_true, T0, 15, 0.2,
                           0.5)
    # the model maps are float32: the fixed point is T_true to within their rounding
    assert np.abs(T[:3, 3] - T_true[:3, 3]).max() < 1e-5
    R = T[:3, :3] @ T_true[:3, :3].T
    assert np.degrees(np.arccos(np.clip((np.trace(R) - 1) / 2, -1, 1))) < 1e-3
    # the first step moves most of the way (a sign error in J would diverge)
    T1, _ = oracle.track(depth, CAM, mv.astype(np.float32), mn.astype(np.float32), T_true, T0, 1, 0.2, 0.5)
    e0 = np.linalg.norm(T0[:3, 3] - T_true[:3, 3])
    e1 = np.linalg.norm(T1[:3, 3] - T_true[:3, 3])
    assert e1 < 0.3 * e0
