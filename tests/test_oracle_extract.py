"""Pins for the oracle's surface points (the point cloud of a volume and its
vertex count, Sec. Insertion and Removal, Table 1): closed forms for planes and
spheres, unobserved voxels, and interpolated colour.  CPU only."""
import math

import numpy as np

import oracle


def grid(vol):
    rx, ry, rz = vol.r
    z, y, x = np.meshgrid(np.arange(rz), np.arange(ry), np.arange(rx), indexing="ij")
    return np.stack([(vol.h[0] + x) * vol.s, (vol.h[1] + y) * vol.s, (vol.h[2] + z) * vol.s], -1)


def test_axis_plane_gives_one_point_per_column_on_the_plane():
    vol = oracle.Volume(h=(-5, -4, -6), r=(11, 9, 13), s=0.1)
    z0 = 0.037  # between voxel planes z = 0.0 and 0.1
    p = grid(vol)
    vol.F[:] = np.clip((z0 - p[..., 2]) / 0.4, -1, 1)
    vol.W[:] = 1.0
    out = oracle.extract_points(vol)
    assert len(out["xyz"]) == 11 * 9
    assert np.all(out["edge"] % 3 == 2)  # all on z edges
    np.testing.assert_allclose(out["xyz"][:, 2], z0, atol=1e-15)
    assert np.all(np.diff(out["edge"]) > 0)


def test_oblique_plane_points_lie_exactly_on_the_plane():
    rng = np.random.default_rng(3)
    n = rng.normal(size=3)
    n /= np.linalg.norm(n)
    vol = oracle.Volume(h=(-10, -10, -10), r=(21, 21, 21), s=0.05)
    d = 0.013
    # |F| < 1 near the plane: the clamp never touches an edge that crosses it
    vol.F[:] = np.clip((d - grid(vol) @ n) / 0.2, -1, 1)
    vol.W[:] = 1.0
    out = oracle.extract_points(vol)
    assert len(out["xyz"]) > 500
    np.testing.assert_allclose(out["xyz"] @ n, d, atol=1e-12)


def test_sphere_point_count_and_distance():
    """Edges crossing a sphere of radius rho: the integral of |n_x|+|n_y|+|n_z|
    over it divided by s^2, i.e. 3 * 2 pi rho^2 / s^2; every point within the
    interpolation error s^2 / (8 rho) (+ clamp-free band) of the sphere."""
    s, rho = 0.01, 0.3
    r = 71
    vol = oracle.Volume(h=(-35, -35, -35), r=(r, r, r), s=s)
    vol.F[:] = np.clip((np.linalg.norm(grid(vol), axis=-1) - rho) / (4 * s), -1, 1)
    vol.W[:] = 1.0
    out = oracle.extract_points(vol)
    want = 6 * math.pi * rho ** 2 / s ** 2
    assert abs(len(out["xyz"]) - want) < 0.01 * want
    dist = np.abs(np.linalg.norm(out["xyz"], axis=-1) - rho)
    assert dist.max() <= s * s / (8 * (rho - s)) + 1e-12


def test_unobserved_voxels_give_no_points():
    vol = oracle.Volume(h=(0, 0, 0), r=(8, 8, 8), s=0.1)
    vol.F[:] = np.where(np.arange(8)[None, None, :] < 4, 0.5, -0.5)  # crossing between x = 3 and 4
    vol.W[:] = 1.0
    assert len(oracle.extract_points(vol)["xyz"]) == 64
    vol.W[:, :2, :] = 0.0   # rows y = 0, 1 unobserved
    vol.W[5, :, 4] = 0.0    # one voxel line on the far side
    out = oracle.extract_points(vol)
    assert len(out["xyz"]) == 8 * 6 - 6
    assert np.all(out["edge"] % 3 == 0)


def test_colour_is_linearly_interpolated_and_rounded_half_up():
    vol = oracle.Volume(h=(0, 0, 0), r=(4, 3, 3), s=1.0)
    vol.W[:] = 1.0
    vol.F[:] = np.array([0.75, -0.25, -1.0, -1.0])[None, None, :]  # zero at x = 0.75
    vol.rgba[..., 0] = np.array([0, 100, 0, 0], np.uint8)[None, None, :]
    vol.rgba[..., 1] = np.array([200, 10, 0, 0], np.uint8)[None, None, :]
    vol.rgba[..., 2] = np.array([3, 5, 0, 0], np.uint8)[None, None, :]
    out = oracle.extract_points(vol)
    assert len(out["xyz"]) == 9
    np.testing.assert_allclose(out["xyz"][:, 0], 0.75)
    # 0 + 0.75 * 100 = 75; 200 - 0.75 * 190 = 57.5 -> 58; 3 + 0.75 * 2 = 4.5 -> 5
    assert np.all(out["rgb"] == np.array([75, 58, 5], np.uint8))
