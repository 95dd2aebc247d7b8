"""Pins for the FP64 oracle, each against something other than the oracle:
ray--plane geometry, textbook closed forms, special cases where the update
must leave a voxel untouched, analytic ray--primitive intersections on volumes
filled with closed-form signed distances, dense brute-force sampling with an
independent trilinear evaluation, and the paper's tiling invariant
(Sec. Comparison to KinectFusion).  CPU only."""
import math

import numpy as np
import pytest

import oracle
from paper_1511_07106_b300 import synth

CAM_S = synth.Camera(50.0, 50.0, 31.5, 23.5, 64, 48)


def identity_pose():
    return np.eye(4)


def frontal_volume():
    # every voxel of this volume projects inside CAM_S's image from the origin
    return oracle.Volume(h=(-12, -12, 28), r=(25, 25, 24), s=0.025)


def voxel_positions(vol):
    rx, ry, rz = vol.r
    z, y, x = np.meshgrid(np.arange(rz), np.arange(ry), np.arange(rx), indexing="ij")
    return np.stack([(vol.h[0] + x) * vol.s, (vol.h[1] + y) * vol.s, (vol.h[2] + z) * vol.s], -1)


# ---------------------------------------------------------------------------
# integration
# ---------------------------------------------------------------------------

def test_frontal_plane_single_frame_is_distance_along_ray(oracle_lib):
    """One frame of a fronto-parallel plane z = z0 seen from the origin: each
    voxel's value is the signed distance from the voxel to the plane measured
    along the camera ray through it (intersection point minus voxel, by
    geometry), truncated at mu and skipped beyond -mu."""
    vol = frontal_volume()
    z0, mu = 0.9, 4 * vol.s
    depth = np.full((CAM_S.height, CAM_S.width), z0, np.float32)
    cfg = oracle.Config(trunc_vox=4.0)
    oracle.integrate(vol, depth, None, CAM_S, identity_pose(), cfg)
    z0 = float(np.float32(z0))
    p = voxel_positions(vol)
    # ray from the camera centre through the voxel meets the plane at P = p * z0 / p_z
    P = p * (z0 / p[..., 2:3])
    # signed: positive while the plane lies beyond the voxel
    alpha = np.linalg.norm(P, axis=-1) - np.linalg.norm(p, axis=-1)
    upd = alpha >= -mu
    expect_F = np.where(upd, np.minimum(1.0, alpha / mu), 0.0)
    np.testing.assert_allclose(vol.F, expect_F, atol=1e-12)
    np.testing.assert_array_equal(vol.W, upd.astype(np.float64))


def test_optical_axis_is_textbook_truncated_distance(oracle_lib):
    """On the optical axis the projective distance is the Euclidean one:
    F = clamp((z0 - z) / mu, ., 1)."""
    vol = oracle.Volume(h=(0, 0, 10), r=(2, 2, 60), s=0.02)
    z0 = float(np.float32(0.7))
    depth = np.full((CAM_S.height, CAM_S.width), z0, np.float32)
    oracle.integrate(vol, depth, None, CAM_S, identity_pose(), oracle.Config(trunc_vox=3.0))
    z = (vol.h[2] + np.arange(60)) * vol.s
    mu = 3.0 * vol.s
    d = z0 - z
    exp = np.where(d >= -mu, np.minimum(1.0, d / mu), 0.0)
    np.testing.assert_allclose(vol.F[:, 0, 0], exp, atol=1e-12)


def test_running_average_is_arithmetic_mean(oracle_lib):
    """Below the weight cap, n frames give the arithmetic mean of the n
    per-frame truncated distances and W = n (weighted running average with
    unit per-frame weight, Sec. Volumetric Integration)."""
    vol = oracle.Volume(h=(0, 0, 30), r=(2, 2, 20), s=0.02)
    mu = 4 * vol.s
    zs = [0.75, 0.78, 0.76, 0.80, 0.77, 0.79]
    for z0 in zs:
        depth = np.full((CAM_S.height, CAM_S.width), z0, np.float32)
        oracle.integrate(vol, depth, None, CAM_S, identity_pose(), oracle.Config())
    z = (vol.h[2] + np.arange(20)) * vol.s
    per = np.array([[min(1.0, (float(np.float32(z0)) - zz) / mu) for zz in z] for z0 in zs])
    always = np.all(per >= -1.0, axis=0)
    np.testing.assert_allclose(vol.F[always, 0, 0], per[:, always].mean(0), atol=1e-12)
    assert np.all(vol.W[always, 0, 0] == len(zs))


def test_weight_cap_fixed_point_and_moving_average(oracle_lib):
    """At the cap W_max the update is an exponential moving average with
    factor W_max / (W_max + 1); a constant input is its fixed point."""
    wmax = 5.0
    cfg = oracle.Config(w_max=wmax)
    vol = oracle.Volume(h=(0, 0, 30), r=(2, 2, 4), s=0.02)
    d_a = np.full((CAM_S.height, CAM_S.width), 0.65, np.float32)
    for _ in range(12):
        oracle.integrate(vol, d_a, None, CAM_S, identity_pose(), cfg)
    z = (vol.h[2] + np.arange(4)) * vol.s
    mu = 4 * vol.s
    fa = np.minimum(1.0, (float(np.float32(0.65)) - z) / mu)
    np.testing.assert_allclose(vol.F[:, 0, 0], fa, atol=1e-12)
    assert np.all(vol.W == wmax)
    d_b = np.full((CAM_S.height, CAM_S.width), 0.62, np.float32)
    fb = np.minimum(1.0, (float(np.float32(0.62)) - z) / mu)
    for m in range(1, 8):
        oracle.integrate(vol, d_b, None, CAM_S, identity_pose(), cfg)
        exp = fb + (fa - fb) * (wmax / (wmax + 1.0)) ** m
        np.testing.assert_allclose(vol.F[:, 0, 0], exp, atol=1e-12)


def test_voxels_that_must_not_change(oracle_lib):
    """Behind the camera, outside the image, invalid depth (0, negative, NaN),
    depth outside [z_min, z_max] and sdf < -mu: the voxel keeps its state."""
    rng = np.random.default_rng(0)
    vol = oracle.Volume(h=(-40, -40, -40), r=(80, 80, 80), s=0.02)
    vol.F[:] = rng.uniform(-1, 1, vol.F.shape)
    vol.W[:] = rng.integers(1, 9, vol.W.shape)
    F0, W0 = vol.F.copy(), vol.W.copy()
    p = voxel_positions(vol)
    # 1) depth everywhere invalid -> nothing changes
    for bad in (0.0, -1.0, np.nan):
        d = np.full((CAM_S.height, CAM_S.width), bad, np.float32)
        cnt, _ = oracle.integrate(vol, d, None, CAM_S, identity_pose(), oracle.Config())
        assert cnt[0] == 0
    # 2) depth outside [z_min, z_max]
    d = np.full((CAM_S.height, CAM_S.width), 0.5, np.float32)
    cnt, _ = oracle.integrate(vol, d, None, CAM_S, identity_pose(), oracle.Config(z_min=0.6, z_max=2.0))
    assert cnt[0] == 0
    np.testing.assert_array_equal(vol.F, F0)
    np.testing.assert_array_equal(vol.W, W0)
    # 3) valid depth: voxels behind the camera, outside the view cone, or more
    #    than mu behind the surface keep their state
    d = np.full((CAM_S.height, CAM_S.width), 0.4, np.float32)
    oracle.integrate(vol, d, None, CAM_S, identity_pose(), oracle.Config())
    behind = p[..., 2] <= 0
    outside = (np.abs(p[..., 0]) / np.maximum(p[..., 2], 1e-9) > 33.0 / 50.0) | \
              (np.abs(p[..., 1]) / np.maximum(p[..., 2], 1e-9) > 25.0 / 50.0)
    # a point more than mu behind the plane along its ray: z > z0 * (1 + mu / |P|) is sufficient
    deep = p[..., 2] > 0.4 + 4 * vol.s * 2
    keep = behind | outside | deep
    np.testing.assert_array_equal(vol.F[keep], F0[keep])
    np.testing.assert_array_equal(vol.W[keep], W0[keep])
    assert np.any(vol.W != W0)


def test_colour_band_and_half_up_rounding(oracle_lib):
    """Colour is averaged only inside the band |sdf| < mu, rounded half up, and
    its weight saturates at color_w_max."""
    vol = oracle.Volume(h=(0, 0, 30), r=(2, 2, 20), s=0.02)
    z = (vol.h[2] + np.arange(20)) * vol.s
    z0 = 0.7
    vol.rgba[:, 0, 0] = (100, 0, 255, 1)
    d = np.full((CAM_S.height, CAM_S.width), z0, np.float32)
    rgb = np.zeros((CAM_S.height, CAM_S.width, 3), np.uint8)
    rgb[..., 0], rgb[..., 1], rgb[..., 2] = 201, 1, 0
    oracle.integrate(vol, d, rgb, CAM_S, identity_pose(), oracle.Config())
    mu = 4 * vol.s
    sd = float(np.float32(z0)) - z
    band = np.abs(sd) < mu
    assert band.any() and (~band).any()
    # (100*1 + 201)/2 = 150.5 -> 151, (0 + 1)/2 = 0.5 -> 1, (255 + 0)/2 = 127.5 -> 128
    np.testing.assert_array_equal(vol.rgba[band, 0, 0], np.tile([151, 1, 128, 2], (band.sum(), 1)))
    np.testing.assert_array_equal(vol.rgba[~band, 0, 0], np.tile([100, 0, 255, 1], ((~band).sum(), 1)))
    # saturation of the colour weight
    vol.rgba[:, 0, 0] = (10, 10, 10, 255)
    oracle.integrate(vol, d, rgb, CAM_S, identity_pose(), oracle.Config(color_w_max=255))
    # (10*255 + 201)/256 = 10.746 -> 11; (10*255+1)/256 = 9.96 -> 10; 2550/256 = 9.96 -> 10
    np.testing.assert_array_equal(vol.rgba[band, 0, 0], np.tile([11, 10, 10, 255], (band.sum(), 1)))


def test_counts_match_changed_voxels(oracle_lib):
    wl = synth.single_volume_128(frames=2, res=24)
    (vs,) = wl.volumes
    vol = oracle.Volume(vs.h, vs.r, vs.s)
    d, c = wl.frame(0)
    cnt, _ = oracle.integrate(vol, d, c, wl.cam, wl.poses[0], oracle.Config())
    assert cnt[0] == int((vol.W > 0).sum()) > 0
    assert cnt[1] == int((vol.rgba[..., 3] > 0).sum()) > 0


# ---------------------------------------------------------------------------
# raycast on volumes filled with closed-form signed distances
# ---------------------------------------------------------------------------

def fill(vol, sdf_metres, mu):
    p = voxel_positions(vol)
    vol.F[:] = np.clip(sdf_metres(p) / mu, -1.0, 1.0)
    vol.W[:] = 1.0


def rays(cam, T):
    o, d = synth.pixel_rays(cam, T)
    return o, d


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_raycast_plane_is_exact(oracle_lib, seed):
    """A linear signed distance is reproduced exactly by trilinear
    interpolation, so the hit is the analytic ray--plane intersection and the
    normal is the plane normal facing the camera."""
    rng = np.random.default_rng(seed)
    vol = oracle.Volume(h=(-30, -30, -30), r=(60, 60, 60), s=0.02)
    mu = 4 * vol.s
    n = rng.normal(size=3)
    n /= np.linalg.norm(n)
    dd = float(rng.uniform(-0.1, 0.1))
    fill(vol, lambda p: dd - p @ n, mu)  # positive where n.p < dd
    eye = -0.9 * n + rng.normal(scale=0.05, size=3)
    T = synth.look_at(eye, eye + n + rng.normal(scale=0.1, size=3))
    cfg = oracle.Config(trunc_vox=4.0)
    out = oracle.raycast([vol], CAM_S, T, cfg)
    o, d = rays(CAM_S, T)
    tau = (dd - o @ n) / (d @ n)
    hit_pt = o + tau[..., None] * d
    inside = np.all((hit_pt > (np.array(vol.h) + 1) * vol.s) & (hit_pt < (np.array(vol.h) + np.array(vol.r) - 2) * vol.s), -1)
    assert inside.sum() > 0.5 * inside.size
    hit = out["depth"] > 0
    assert np.all(hit[inside])
    np.testing.assert_allclose(out["depth"][inside], tau[inside], atol=1e-10)
    np.testing.assert_allclose(out["normal"][inside], np.broadcast_to(-n, out["normal"][inside].shape), atol=1e-9)
    np.testing.assert_allclose(out["vertex"][inside], hit_pt[inside], atol=1e-9)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_raycast_hit_colour_is_the_affine_colour_at_the_hit(oracle_lib, seed):
    """Hit colour (trilinear RGB of the hit cell, rounded half up): with a
    linear signed distance (exact hit, as above) and a colour that is affine
    in the voxel index -- which trilinear interpolation reproduces exactly --
    each channel must equal the affine colour at the analytic ray--plane hit,
    rounded half up.  Distinct signed gradients per channel catch a wrong
    corner weight, a swapped axis or channel, a floor instead of rounding and
    a colour taken from another cell than the hit's."""
    rng = np.random.default_rng(10 + seed)
    vol = oracle.Volume(h=(-30, -30, -30), r=(60, 60, 60), s=0.02)
    mu = 4 * vol.s
    n = rng.normal(size=3)
    n /= np.linalg.norm(n)
    dd = float(rng.uniform(-0.1, 0.1))
    fill(vol, lambda p: dd - p @ n, mu)
    # colour_ch(i) = c0_ch + g_ch . i over local voxel indices i = (x, y, z), inside [0, 255]
    c0 = np.array([10.0, 20.0, 200.0])
    g = np.array([[2.0, 1.0, 0.0], [0.0, 2.0, 1.0], [-1.0, 0.0, -2.0]])  # rows: channel; cols: x, y, z
    z, y, x = np.meshgrid(*(np.arange(r) for r in vol.r[::-1]), indexing="ij")
    idx = np.stack([x, y, z], -1).astype(np.float64)
    col = c0 + idx @ g.T
    assert col.min() >= 0 and col.max() <= 255
    vol.rgba[..., :3] = col.astype(np.uint8)
    vol.rgba[..., 3] = 1
    eye = -0.9 * n + rng.normal(scale=0.05, size=3)
    T = synth.look_at(eye, eye + n + rng.normal(scale=0.1, size=3))
    out = oracle.raycast([vol], CAM_S, T, oracle.Config(trunc_vox=4.0))
    o, d = rays(CAM_S, T)
    tau = (dd - o @ n) / (d @ n)
    hit_pt = o + tau[..., None] * d
    inside = np.all((hit_pt > (np.array(vol.h) + 1) * vol.s) &
                    (hit_pt < (np.array(vol.h) + np.array(vol.r) - 2) * vol.s), -1)
    q = hit_pt / vol.s - np.array(vol.h)          # local voxel coordinates of the hit
    want = c0 + q @ g.T                           # exact affine colour there
    frac = want - np.floor(want)
    safe = inside & np.all(np.abs(frac - 0.5) > 1e-6, -1)
    assert safe.sum() > 0.5 * safe.size
    got = out["rgba"][..., :3].astype(np.float64)
    np.testing.assert_array_equal(got[safe], np.floor(want[safe] + 0.5))
    assert np.all(out["rgba"][..., 3][inside] == 255)


def test_raycast_sphere_within_interpolation_bound(oracle_lib):
    """Sphere of radius rho: trilinear interpolation of its distance function
    errs by at most s^2 / (4 rho) near the surface, which bounds the hit
    error along the ray; normals point radially outward."""
    vol = oracle.Volume(h=(-25, -25, -25), r=(50, 50, 50), s=0.02)
    mu, rho = 4 * vol.s, 0.3
    c = np.array([0.01, -0.02, 0.03])
    fill(vol, lambda p: np.linalg.norm(p - c, axis=-1) - rho, mu)
    T = synth.look_at((0.2, -0.1, -0.45), c)
    out = oracle.raycast([vol], CAM_S, T, oracle.Config())
    o, d = rays(CAM_S, T)
    oc = o - c
    a = np.einsum("...k,...k", d, d)
    b = 2 * d @ oc
    cc = oc @ oc - rho * rho
    disc = b * b - 4 * a * cc
    tau = np.where(disc > 0, (-b - np.sqrt(np.maximum(disc, 0))) / (2 * a), np.nan)
    # only pixels whose ray meets the sphere well away from the silhouette
    good = disc > 0.3 * (b * b)
    assert good.sum() > 100
    hit = out["depth"] > 0
    assert np.all(hit[good])
    err = np.abs(out["depth"][good] - tau[good]) * np.sqrt(a[good])
    # tensor-product linear interpolation errs by <= (s^2/8) sum_i |f_ii|; for
    # |p - c| - rho that sum is 2/|p - c| >= ... taken at the cell's nearest
    # corner (rho - sqrt(3) s); the hit moves by that over cos(incidence)
    pts = o + tau[..., None] * d
    radial = (pts - c) / rho
    cos_inc = np.abs(np.einsum("...k,...k", d / np.sqrt(a)[..., None], radial))
    bound = (vol.s ** 2 / 8) * 2 / (rho - math.sqrt(3) * vol.s) / cos_inc[good]
    assert np.all(err <= 1.1 * bound + 1e-12)
    cosang = np.einsum("...k,...k", out["normal"][good], radial[good])
    assert cosang.min() > math.cos(math.radians(3.0))


def test_raycast_box_faces_exact(oracle_lib):
    """Axis-aligned box: its signed distance is linear near the middle of a
    face, so hits there are exact."""
    vol = oracle.Volume(h=(-30, -30, -30), r=(60, 60, 60), s=0.02)
    mu = 4 * vol.s
    lo, hi = np.array([-0.25, -0.2, -0.15]), np.array([0.2, 0.25, 0.3])

    def box_sdf(p):
        q = np.abs(p - (lo + hi) / 2) - (hi - lo) / 2
        return np.linalg.norm(np.maximum(q, 0), axis=-1) + np.minimum(q.max(-1), 0)

    fill(vol, box_sdf, mu)
    T = synth.look_at((0.0, 0.0, -0.5), (0.0, 0.0, 0.0))
    out = oracle.raycast([vol], CAM_S, T, oracle.Config())
    o, d = rays(CAM_S, T)
    tau = (lo[2] - o[2]) / d[..., 2]
    pt = o + tau[..., None] * d
    face = np.all((pt[..., :2] > lo[:2] + mu + 2 * vol.s) & (pt[..., :2] < hi[:2] - mu - 2 * vol.s), -1)
    assert face.sum() > 50
    np.testing.assert_allclose(out["depth"][face], tau[face], atol=1e-10)
    np.testing.assert_allclose(out["normal"][face], np.broadcast_to([0, 0, -1.0], out["normal"][face].shape), atol=1e-9)


# ---------------------------------------------------------------------------
# the march's semantics on hand-built fields
# ---------------------------------------------------------------------------

def axis_cam():
    return synth.Camera(10.0, 10.0, 0.0, 0.0, 1, 1)


def x_ray_pose(y=0.0, z=0.0):
    # camera looking along +x: z_cam = +x_world
    T = np.eye(4)
    T[:3, 0], T[:3, 1], T[:3, 2] = (0, 1, 0), (0, 0, 1), (1, 0, 0)
    T[:3, 3] = (-0.5, y, z)
    return T


def row_volume(values, valid=None):
    n = len(values)
    vol = oracle.Volume(h=(0, -2, -2), r=(n, 4, 4), s=0.1)
    vol.F[:] = np.asarray(values, np.float64)[None, None, :]
    vol.W[:] = 1.0 if valid is None else np.asarray(valid, np.float64)[None, None, :]
    return vol


def test_march_all_invalid_has_no_hit(oracle_lib):
    vol = row_volume([1, 1, -1, -1, 1, -1], valid=[0] * 6)
    out = oracle.raycast([vol], axis_cam(), x_ray_pose(0.05, 0.05), oracle.Config())
    assert out["depth"][0, 0] == 0 and out["vol"][0, 0] == -1


def test_march_first_positive_to_nonpositive_pair(oracle_lib):
    # voxels at x = 0, .1, .2 ...: roots at x = 0.25 and 0.65 -> first one wins
    vol = row_volume([1, 0.5, 0.5, -0.5, -0.5, 0.5, 0.5, -0.5, -0.5, -1])
    out = oracle.raycast([vol], axis_cam(), x_ray_pose(0.05, 0.05), oracle.Config(step_vox=0.5))
    assert abs(out["depth"][0, 0] - (0.5 + 0.25)) < 1e-12


def test_march_starting_inside_finds_later_front_face(oracle_lib):
    # first valid sample negative, then a back face (- to +), then a front face
    vol = row_volume([-0.5, -0.5, 0.5, 0.5, 0.5, -0.5, -0.5])
    out = oracle.raycast([vol], axis_cam(), x_ray_pose(0.05, 0.05), oracle.Config(step_vox=0.5))
    assert abs(out["depth"][0, 0] - (0.5 + 0.45)) < 1e-12


def test_march_invalid_sample_breaks_the_pair(oracle_lib):
    # positive, invalid cell, negative: no valid consecutive pair -> no hit
    vol = row_volume([1, 1, 1, 1, -1, -1, -1, -1], valid=[1, 1, 1, 0, 1, 1, 1, 1])
    out = oracle.raycast([vol], axis_cam(), x_ray_pose(0.05, 0.05), oracle.Config(step_vox=1.0))
    assert out["depth"][0, 0] == 0
    # the same field fully valid has its root at x = 0.35
    vol2 = row_volume([1, 1, 1, 1, -1, -1, -1, -1])
    out2 = oracle.raycast([vol2], axis_cam(), x_ray_pose(0.05, 0.05), oracle.Config(step_vox=1.0))
    assert abs(out2["depth"][0, 0] - (0.5 + 0.35)) < 1e-12


def test_footprint_of_an_axis_ray(oracle_lib):
    """Voxels a dense march reads, counted by hand on a row: samples at every
    voxel plane x = 0 .. n-1 (step 1 voxel), each reading its cell's 2x2x2
    corners (the last plane's cell clamps to n-2).  No surface: all n x 2 x 2
    voxels.  A root at x = 3.5: cells 0..4 are sampled (corners x = 0..5), the
    bisection stays in cell 3, and the hit reads the colour of cell 3."""
    vol = row_volume([1.0] * 10)
    (fp,) = oracle.raycast_footprint([vol], axis_cam(), x_ray_pose(0.05, 0.05), oracle.Config(step_vox=1.0))
    assert fp == (4 * 10, 0)
    vol2 = row_volume([1, 1, 1, 1, -1, -1, -1, -1, -1, -1])
    (fp2,) = oracle.raycast_footprint([vol2], axis_cam(), x_ray_pose(0.05, 0.05), oracle.Config(step_vox=1.0))
    assert fp2 == (4 * 6, 8)


@pytest.mark.parametrize("seed", [0, 1])
def test_footprint_matches_brute_force_sample_cells(oracle_lib, seed):
    """A volume with no surface (F > 0 wherever observed, random observation
    pattern) has no hit, so every sample on the global grid inside the domain
    is read: the footprint is the union of the 2x2x2 corner sets of all those
    samples' cells, enumerated here ray by ray from the grid definition."""
    rng = np.random.default_rng(seed)
    vol = oracle.Volume(h=(-5, -4, 20), r=(9, 8, 7), s=0.05)
    vol.F[:] = rng.uniform(0.1, 1.0, size=vol.F.shape)
    vol.W[:] = (rng.uniform(size=vol.W.shape) < 0.7).astype(np.float64)
    cam = synth.Camera(12.0, 12.0, 5.5, 4.5, 12, 10)
    T = synth.look_at(rng.normal(scale=0.05, size=3), (0.0, 0.0, 1.2))
    step = 0.7
    (fp,) = oracle.raycast_footprint([vol], cam, T, oracle.Config(step_vox=step))
    o, d = synth.pixel_rays(cam, T)
    h, r, s = np.array(vol.h), np.array(vol.r), vol.s
    seen = np.zeros(vol.F.shape, bool)
    for y in range(cam.height):
        for x in range(cam.width):
            q0, dv = o / s, d[y, x] / s
            lo, hi = 0.0, np.inf
            for a in range(3):
                t0, t1 = (h[a] - q0[a]) / dv[a], (h[a] + r[a] - 1 - q0[a]) / dv[a]
                lo, hi = max(lo, min(t0, t1)), min(hi, max(t0, t1))
            if lo > hi:
                continue
            delta = step * s / np.linalg.norm(d[y, x])
            for k in range(int(np.ceil(lo / delta)), int(np.floor(hi / delta)) + 1):
                q = q0 + k * delta * dv
                c = np.clip(np.floor(q).astype(int) - h, 0, r - 2)
                seen[c[2]:c[2] + 2, c[1]:c[1] + 2, c[0]:c[0] + 2] = True
    assert seen.sum() > 50
    assert fp == (int(seen.sum()), 0)


def test_footprint_of_a_pixel_subset_is_not_larger(oracle_lib):
    """Reading fewer rays reads no new voxels: the footprint of every other
    pixel is at most that of all pixels, and the two halves together cover at
    least the whole."""
    vol = oracle.Volume(h=(-30, -30, -30), r=(60, 60, 60), s=0.02)
    n = np.array([0.2, -0.1, 1.0])
    n /= np.linalg.norm(n)
    fill(vol, lambda p: 0.05 - p @ n, 4 * vol.s)
    T = synth.look_at(-0.9 * n, n)
    full = oracle.raycast_footprint([vol], CAM_S, T)[0]
    npx = CAM_S.width * CAM_S.height
    even = oracle.raycast_footprint([vol], CAM_S, T, pixels=np.arange(0, npx, 2))[0]
    odd = oracle.raycast_footprint([vol], CAM_S, T, pixels=np.arange(1, npx, 2))[0]
    assert full[0] > 0 and full[1] > 0
    for a in range(2):
        assert even[a] <= full[a] and odd[a] <= full[a] <= even[a] + odd[a]


def test_merge_takes_nearest_and_breaks_ties_by_id(oracle_lib):
    a = row_volume([1, 1, -1, -1, -1, -1])            # root x = 0.15
    b = row_volume([1, 1, 1, 1, -1, -1])              # root x = 0.35
    out = oracle.raycast([b, a], axis_cam(), x_ray_pose(0.05, 0.05), oracle.Config(), ids=[7, 9])
    assert out["vol"][0, 0] == 9 and abs(out["depth"][0, 0] - 0.65) < 1e-12
    c = a.copy()
    out = oracle.raycast([c, a], axis_cam(), x_ray_pose(0.05, 0.05), oracle.Config(), ids=[5, 3])
    assert out["vol"][0, 0] == 3


# ---------------------------------------------------------------------------
# brute force: dense sampling with an independent trilinear evaluation
# ---------------------------------------------------------------------------

def trilinear_np(F, W, q):
    r = np.array(F.shape[::-1])
    c = np.clip(np.floor(q), 0, r - 2).astype(np.int64)
    f = q - c
    val = np.zeros(q.shape[:-1])
    ok = np.ones(q.shape[:-1], bool)
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                w = (f[..., 0] if dx else 1 - f[..., 0]) * (f[..., 1] if dy else 1 - f[..., 1]) * \
                    (f[..., 2] if dz else 1 - f[..., 2])
                idx = (c[..., 2] + dz, c[..., 1] + dy, c[..., 0] + dx)
                val += w * F[idx]
                ok &= W[idx] > 0
    return val, ok


@pytest.mark.parametrize("seed", [3, 4])
def test_raycast_matches_dense_brute_force(oracle_lib, seed):
    """Random smooth fields on a 12^3 grid, all voxels valid: the first
    positive-to-nonpositive crossing found by sampling every ray at 1/200
    voxel and bisecting equals the oracle's hit, wherever the dense
    sampling sees a single crossing per voxel of ray length."""
    rng = np.random.default_rng(seed)
    vol = oracle.Volume(h=(-6, -6, -6), r=(12, 12, 12), s=0.05)
    p = voxel_positions(vol)
    cs = rng.uniform(-0.15, 0.15, size=(3, 3))
    rs = rng.uniform(0.08, 0.18, size=3)
    sd = np.min([np.linalg.norm(p - c, axis=-1) - r for c, r in zip(cs, rs)], axis=0)
    vol.F[:] = np.clip(sd / (4 * vol.s), -1, 1)
    vol.W[:] = 1.0
    cam = synth.Camera(12.0, 12.0, 3.5, 2.5, 8, 6)
    T = synth.look_at((0.05, -0.1, -0.6), (0.0, 0.0, 0.0))
    out = oracle.raycast([vol], cam, T, oracle.Config(step_vox=1.0))
    o, d = synth.pixel_rays(cam, T)
    q0 = (o - np.array(vol.h) * vol.s) / vol.s
    checked = 0
    for y in range(cam.height):
        for x in range(cam.width):
            dv = d[y, x] / vol.s
            lo, hi = 0.0, np.inf
            for a in range(3):
                t0, t1 = (0 - q0[a]) / dv[a], (11 - q0[a]) / dv[a]
                lo, hi = max(lo, min(t0, t1)), min(hi, max(t0, t1))
            if not lo < hi:
                assert out["depth"][y, x] == 0
                continue
            nd = np.linalg.norm(dv)
            ts = np.arange(lo, hi, 0.005 / nd)
            val, ok = trilinear_np(vol.F, vol.W, q0 + ts[:, None] * dv)
            sgn = val > 0
            cross = np.nonzero(sgn[:-1] & ~sgn[1:])[0]
            any_change = np.nonzero(sgn[:-1] != sgn[1:])[0]
            if len(cross) == 0:
                assert out["depth"][y, x] == 0
                continue
            k = cross[0]
            # skip rays where two sign changes lie within one voxel of the crossing
            near = np.abs(ts[any_change] - ts[k]) * nd < 1.5
            if near.sum() > 1 or ts[k] * nd < 1.5:
                continue
            a_, b_ = ts[k], ts[k + 1]
            for _ in range(60):
                m = 0.5 * (a_ + b_)
                vm, _ = trilinear_np(vol.F, vol.W, (q0 + m * dv)[None])
                if vm[0] > 0:
                    a_ = m
                else:
                    b_ = m
            assert abs(out["depth"][y, x] - 0.5 * (a_ + b_)) * nd < 1e-8
            checked += 1
    assert checked > 10


# ---------------------------------------------------------------------------
# the paper's invariant: volumes tiling a region equal one volume over it
# ---------------------------------------------------------------------------

def test_tiling_invariance_integration_and_raycast(oracle_lib):
    """2x2x2 subvolumes of r^3 on the lattice h_t = k (r - 2) (two-voxel
    overlap) against one volume of (2r - 2)^3: bit-identical TSDF, weight and
    colour on every voxel after integration, and the same merged raycast
    (Sec. Comparison to KinectFusion)."""
    wl = synth.single_volume_128(frames=4, res=34)
    tl = synth.tiled(wl, 2)
    (vs,) = wl.volumes
    single = oracle.Volume(vs.h, vs.r, vs.s)
    tiles = [oracle.Volume(t.h, t.r, t.s) for t in tl.volumes]
    cfg = oracle.Config()
    for i in range(wl.n_frames):
        d, c = wl.frame(i)
        oracle.integrate(single, d, c, wl.cam, wl.poses[i], cfg)
        for t in tiles:
            oracle.integrate(t, d, c, wl.cam, wl.poses[i], cfg)
    for t in tiles:
        o = [t.h[a] - vs.h[a] for a in range(3)]
        sl = (slice(o[2], o[2] + t.r[2]), slice(o[1], o[1] + t.r[1]), slice(o[0], o[0] + t.r[0]))
        np.testing.assert_array_equal(t.F, single.F[sl])
        np.testing.assert_array_equal(t.W, single.W[sl])
        np.testing.assert_array_equal(t.rgba, single.rgba[sl])
    assert (single.W > 0).mean() > 0.05
    T = wl.poses[1]
    a = oracle.raycast([single], wl.cam, T, cfg)
    b = oracle.raycast(tiles, wl.cam, T, cfg)
    np.testing.assert_array_equal(a["depth"] > 0, b["depth"] > 0)
    assert (a["depth"] > 0).mean() > 0.3
    np.testing.assert_allclose(b["depth"], a["depth"], atol=1e-9 * vs.s)
    np.testing.assert_allclose(b["normal"], a["normal"], atol=1e-9)
    np.testing.assert_array_equal(b["rgba"], a["rgba"])


@pytest.mark.parametrize("seed", [5, 6])
def test_rotated_camera_plane_is_distance_along_ray(oracle_lib, seed):
    """A rotated, translated camera facing a plane perpendicular to its view
    axis sees a constant depth z0; every voxel's value is again the signed
    distance along its camera ray to that plane, computed in world
    coordinates by ray--plane intersection."""
    rng = np.random.default_rng(seed)
    vol = oracle.Volume(h=(-4, -4, -4), r=(9, 9, 9), s=0.025)
    centre = np.zeros(3)
    eye = rng.normal(size=3)
    eye = 1.0 * eye / np.linalg.norm(eye)
    T = synth.look_at(eye, centre + rng.normal(scale=0.02, size=3))
    f = T[:3, 2]
    z0 = float(np.float32(1.0 + rng.uniform(-0.05, 0.05)))
    depth = np.full((CAM_S.height, CAM_S.width), z0, np.float32)
    oracle.integrate(vol, depth, None, CAM_S, T, oracle.Config())
    p = voxel_positions(vol)
    rel = p - eye
    P = eye + rel * (z0 / (rel @ f))[..., None]
    alpha = np.linalg.norm(P - eye, axis=-1) - np.linalg.norm(rel, axis=-1)
    mu = 4 * vol.s
    upd = alpha >= -mu
    assert upd.any() and (~upd).any()
    np.testing.assert_allclose(vol.F, np.where(upd, np.minimum(1, alpha / mu), 0.0), atol=1e-12)
    np.testing.assert_array_equal(vol.W, upd.astype(float))


def test_nearest_pixel_lookup(oracle_lib):
    """Each voxel reads the depth of the pixel whose centre is nearest to its
    projection (found here by brute force over all pixel centres).  The
    depth image encodes the pixel index, and a huge truncation distance keeps
    the value unclamped, so the stored TSDF reveals which pixel was read."""
    vol = oracle.Volume(h=(-9, -7, 33), r=(19, 15, 3), s=0.0237)
    uu, vv = np.meshgrid(np.arange(CAM_S.width), np.arange(CAM_S.height))
    depth = (0.95 + 0.0005 * (uu + CAM_S.width * vv)).astype(np.float32)
    cfg = oracle.Config(trunc_vox=1000.0)
    T = identity_pose()
    T[:3, 3] = (0.0031, -0.0047, 0.0)  # off the lattice: no projection falls exactly between pixels
    oracle.integrate(vol, depth, None, CAM_S, T, cfg)
    p = voxel_positions(vol).reshape(-1, 3) - T[:3, 3]
    mu = 1000.0 * vol.s
    up = CAM_S.fx * p[:, 0] / p[:, 2] + CAM_S.cx
    vp = CAM_S.fy * p[:, 1] / p[:, 2] + CAM_S.cy
    d2 = (uu.reshape(1, -1) - up[:, None]) ** 2 + (vv.reshape(1, -1) - vp[:, None]) ** 2
    nearest = d2.argmin(1)
    D = depth.reshape(-1)[nearest].astype(np.float64)
    exp = (D - p[:, 2]) * np.linalg.norm(p, axis=1) / p[:, 2] / mu
    np.testing.assert_allclose(vol.F.reshape(-1), exp, atol=1e-12)
    # the lookup is not plain truncation of the projection
    floor_pix = np.floor(vp).astype(int) * CAM_S.width + np.floor(up).astype(int)
    assert np.any(floor_pix != nearest)


def test_decision_flags_are_rare_on_a_typical_view(oracle_lib):
    """The margins flag only decisions an FP32 implementation could take the
    other way; on an ordinary view they must leave almost every pixel and
    voxel comparable."""
    wl = synth.single_volume_128(frames=3, res=48)
    (vs,) = wl.volumes
    vol = oracle.Volume(vs.h, vs.r, vs.s)
    for i in range(3):
        d, c = wl.frame(i)
        _, fl = oracle.integrate(vol, d, c, wl.cam, wl.poses[i], oracle.Config(), want_flags=True)
        assert (fl != 0).mean() < 0.01
    out = oracle.raycast([vol], wl.cam, wl.poses[1], oracle.Config())
    hard = out["flags"] & (oracle.RF_SIGN | oracle.RF_CELL | oracle.RF_RANGE | oracle.RF_TIE)
    assert (hard != 0).mean() < 0.03
    assert (out["depth"] > 0).mean() > 0.3
