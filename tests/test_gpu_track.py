"""Depth-map conversion and point-to-plane ICP on the GPU against the FP64
oracle (Sec. Depth Map Conversion; Sec. Camera Tracking).  Each side computes
its own maps from the same float32 depth frames; the model maps, the same
oracle-made float32 arrays on both sides, stand for the previous raycast."""
import numpy as np
import pytest

import oracle
from paper_1511_07106_b300 import Mapper, synth
from parity_utils import dev

pytestmark = pytest.mark.gpu

DIST, COS = 0.1, 0.8


def room(frames=8):
    return synth.room_512(frames=frames, width=160, height=120)


def model_maps(wl, i):
    d, _ = wl.frame(i)
    mv, mn = oracle.depth_maps(d, wl.cam, wl.poses[i])
    return mv.astype(np.float32), mn.astype(np.float32)


def test_depth_maps_match_oracle():
    wl = room(3)
    m = Mapper()
    d, _ = wl.frame(2)
    d[::17, ::5] = 0.0
    d[3::23, 1::7] = np.nan  # invalid depths of other kinds: no vertex, no normal
    d[5::29, 2::3] = -1.0
    d[7::31, 4::11] = -np.inf
    for T in (None, wl.poses[2]):
        gv, gn = (t.cpu().numpy().astype(np.float64) for t in m.depth_to_maps(dev(d), wl.cam, T))
        ov, on = oracle.depth_maps(d, wl.cam, T)
        np.testing.assert_array_equal(np.any(gv != 0, -1), d > 0)
        np.testing.assert_array_equal(np.any(gn != 0, -1), np.any(on != 0, -1))
        assert np.abs(gv - ov).max() <= 1e-6 * (np.abs(ov).max() + 1)
        ok = np.any(on != 0, -1)
        cosang = np.sum(gn[ok] * on[ok], -1)
        assert cosang.min() > np.cos(2e-3)
    m.close()


def test_icp_system_matches_oracle():
    wl = room(6)
    m = Mapper()
    mv, mn = model_maps(wl, 4)
    d, _ = wl.frame(5)
    T_est = oracle.se3_exp([0.004, -0.003, 0.002, 0.002, 0.001, -0.003]) @ wl.poses[4]
    gv, gn = m.depth_to_maps(dev(d), wl.cam)
    g = m.icp_linearize(gv, gn, wl.cam, T_est, dev(mv), dev(mn), wl.poses[4], DIST, COS)
    ov, on = oracle.depth_maps(d, wl.cam)
    o = oracle.icp_system(ov, on, wl.cam, T_est, mv, mn, wl.poses[4], DIST, COS)
    assert o["count"] > 5000
    assert abs(g["count"] - o["count"]) <= o["abse"][1]
    diag = np.sqrt(np.outer(np.diag(o["A"]), np.diag(o["A"])))
    assert np.all(np.abs(g["A"] - o["A"]) <= o["absA"] + 2e-4 * diag + 1e-9)
    bb = np.sqrt(np.diag(o["A"]) * o["error"])
    assert np.all(np.abs(g["b"] - o["b"]) <= o["absb"] + 2e-4 * bb + 1e-12)
    assert abs(g["error"] - o["error"]) <= o["abse"][0] + 2e-4 * o["error"] + 1e-15
    m.close()


def test_track_matches_oracle_and_ground_truth():
    wl = room(8)
    m = Mapper()
    for i in (3, 6):
        mv, mn = model_maps(wl, i - 1)
        d, _ = wl.frame(i)
        T_prev = wl.poses[i - 1]
        Tg, last = m.track(dev(d), wl.cam, dev(mv), dev(mn), T_prev, T_prev, iterations=10, dist=DIST,
                           cos_min=COS)
        To, _ = oracle.track(d, wl.cam, mv, mn, T_prev, T_prev, 10, DIST, COS)
        assert np.abs(Tg[:3, 3] - To[:3, 3]).max() < 2e-5
        R = Tg[:3, :3] @ To[:3, :3].T
        assert np.arccos(np.clip((np.trace(R) - 1) / 2, -1, 1)) < 2e-4
        T_true = wl.poses[i]
        moved = np.linalg.norm(T_prev[:3, 3] - T_true[:3, 3])
        err = np.linalg.norm(Tg[:3, 3] - T_true[:3, 3])
        assert err < 3e-3 and err < 0.5 * moved + 1e-3, (err, moved)
        Re = Tg[:3, :3] @ T_true[:3, :3].T
        assert np.degrees(np.arccos(np.clip((np.trace(Re) - 1) / 2, -1, 1))) < 0.2
        assert last["count"] > 5000
    m.close()


def test_track_stops_without_inliers_and_iterates_on_the_device():
    """The Gauss-Newton loop runs on the device: with model maps that hold no
    surface the first linearisation has no inliers, the loop stops there and
    the estimate is returned unchanged (bit for bit); with zero iterations
    the estimate is returned as given.  A tracked frame launches one
    linearisation kernel per iteration and nothing else."""
    wl = room(4)
    m = Mapper()
    d, _ = wl.frame(2)
    empty = np.zeros((wl.cam.height, wl.cam.width, 3), np.float32)
    T0 = wl.poses[1].copy()
    T0[:3, 3] += (0.0123, -0.0045, 0.0067)
    Tg, last = m.track(dev(d), wl.cam, dev(empty), dev(empty), wl.poses[1], T0, iterations=10, dist=DIST,
                       cos_min=COS)
    np.testing.assert_array_equal(Tg, T0)
    assert last["count"] == 0 and last["error"] == 0.0
    Tz, lz = m.track(dev(d), wl.cam, dev(empty), dev(empty), wl.poses[1], T0, iterations=0, dist=DIST,
                     cos_min=COS)
    np.testing.assert_array_equal(Tz, T0)
    assert lz["count"] == 0
    mv, mn = model_maps(wl, 1)
    m.timings(reset=True)
    Tg, last = m.track(dev(d), wl.cam, dev(mv), dev(mn), wl.poses[1], wl.poses[1], iterations=7, dist=DIST,
                       cos_min=COS)
    t = m.timings()
    assert t["icp"][0] == 7 and t["depth_maps"][0] == 1
    To, _ = oracle.track(d, wl.cam, mv, mn, wl.poses[1], wl.poses[1], 7, DIST, COS)
    assert np.abs(Tg[:3, 3] - To[:3, 3]).max() < 2e-5
    m.close()
