"""Pins for the oracle of dynamic placement (Sec. Dynamic Mapping for SLAM;
Sec. Insertion and Removal): the ray-endpoint histogram c(l) against closed
forms, and the top-n / hysteresis policy against hand-worked cases.  CPU only."""
import math

import numpy as np

import oracle
from paper_1511_07106_b300 import synth

CAM = synth.Camera(100.0, 100.0, 39.5, 29.5, 80, 60)


def interval_counts(n, c, f, D, cell, offset=0.0):
    """Pixels u in [0, n) per cell k of floor((D (u - c) / f + offset) / cell),
    counted from the cell boundaries: u lies in cell k iff
    c + f (k cell - offset) / D <= u < c + f ((k + 1) cell - offset) / D."""
    out = {}
    lo = math.floor(((0 - c) * D / f + offset) / cell) - 1
    hi = math.floor(((n - 1 - c) * D / f + offset) / cell) + 1
    for k in range(lo, hi + 1):
        a = c + f * (k * cell - offset) / D
        b = c + f * ((k + 1) * cell - offset) / D
        m = sum(1 for u in range(n) if a <= u < b)
        if m:
            out[k] = m
    return out


def test_fronto_parallel_plane_counts_are_products_of_interval_counts():
    D, cell = 2.0, 0.5
    depth = np.full((CAM.height, CAM.width), D, np.float32)
    h = oracle.endpoint_histogram(depth, CAM, np.eye(4), cell)
    cx = interval_counts(CAM.width, CAM.cx, CAM.fx, D, cell)
    cy = interval_counts(CAM.height, CAM.cy, CAM.fy, D, cell)
    kz = math.floor(D / cell)
    want = {(i, j, kz): cx[i] * cy[j] for i in cx for j in cy}
    assert h == want
    assert h[(-2, -2, 4)] == 15 * 5 and h[(-1, -1, 4)] == 25 * 25


def test_rotated_and_translated_camera():
    """Camera looking along world +x (axes permuted exactly), moved by whole
    cells plus a fraction: world x = D + tx, world y = -(camera x) + ty,
    world z = -(camera y) + tz."""
    D, cell = 1.7, 0.4
    T = np.eye(4)
    T[:3, :3] = [[0, 0, 1], [-1, 0, 0], [0, -1, 0]]
    t = np.array([3 * cell + 0.05, -2 * cell + 0.11, 5 * cell + 0.07])
    T[:3, 3] = t
    depth = np.full((CAM.height, CAM.width), D, np.float32)
    h = oracle.endpoint_histogram(depth, CAM, T, cell)
    kx = math.floor((D + t[0]) / cell)
    # world y = -(D (u - cx) / fx) + ty: count by the cell of -(camera x)
    cy_ = {}
    for u in range(CAM.width):
        k = math.floor((-(D * (u - CAM.cx) / CAM.fx) + t[1]) / cell)
        cy_[k] = cy_.get(k, 0) + 1
    cz_ = {}
    for v in range(CAM.height):
        k = math.floor((-(D * (v - CAM.cy) / CAM.fy) + t[2]) / cell)
        cz_[k] = cz_.get(k, 0) + 1
    want = {(kx, j, k): cy_[j] * cz_[k] for j in cy_ for k in cz_}
    assert h == want


def test_invalid_depths_are_not_counted():
    rng = np.random.default_rng(0)
    depth = rng.uniform(0.5, 4.0, size=(CAM.height, CAM.width)).astype(np.float32)
    depth[::7, ::3] = 0.0
    depth[1::11, 2::5] = np.nan
    depth[5, :] = -1.0
    depth[9, :] = 4.5  # beyond z_max
    h = oracle.endpoint_histogram(depth, CAM, np.eye(4), 0.3, z_min=0.4, z_max=4.2)
    valid = (depth > 0) & (depth >= 0.4) & (depth <= 4.2)
    assert sum(h.values()) == int(valid.sum())
    cells, ok = oracle.endpoint_cells(depth, CAM, np.eye(4), 0.3, z_min=0.4, z_max=4.2)
    assert np.array_equal(ok, valid)
    # z cell of each valid pixel is floor(D / cell) for the identity pose
    assert np.array_equal(cells[ok][:, 2], np.floor(depth[ok].astype(np.float64) / 0.3).astype(np.int64))


def test_policy_fills_free_slots_by_count_then_cell_order():
    st = oracle.PlacementState()
    hist = {(0, 0, 0): 5, (1, 0, 0): 50, (0, 1, 0): 50, (0, 0, 1): 20, (2, 2, 2): 1}
    added, restored, evicted = oracle.place(st, hist, max_volumes=3, hysteresis=1.5)
    # 50, 50 (tie: (1,0,0) has z=0,y=0 before (0,1,0) with y=1), then 20
    assert added == [(1, 0, 0), (0, 1, 0), (0, 0, 1)] and not restored and not evicted
    assert st.resident == {(1, 0, 0), (0, 1, 0), (0, 0, 1)}


def test_policy_hysteresis_and_restore():
    st = oracle.PlacementState()
    oracle.place(st, {(0, 0, 0): 100, (1, 0, 0): 60}, max_volumes=2, hysteresis=1.5)
    # 80 is not larger than 1.5 * 60 = 90: nothing changes
    assert oracle.place(st, {(0, 0, 0): 100, (1, 0, 0): 60, (2, 0, 0): 80}, 2, 1.5) == ([], [], [])
    # 91 > 90: (1,0,0) (lowest) leaves, (2,0,0) enters
    a, r, e = oracle.place(st, {(0, 0, 0): 100, (1, 0, 0): 60, (2, 0, 0): 91}, 2, 1.5)
    assert a == [(2, 0, 0)] and e == [(1, 0, 0)] and st.resident == {(0, 0, 0), (2, 0, 0)}
    # a resident cell without endpoints counts 0: any candidate displaces it, and
    # a cell seen before comes back as a restore
    a, r, e = oracle.place(st, {(0, 0, 0): 10, (1, 0, 0): 1}, 2, 1.5)
    assert r == [(1, 0, 0)] and e == [(2, 0, 0)] and not a
    assert st.evicted == {(2, 0, 0)}


def test_policy_min_count_and_stop_at_first_refusal():
    st = oracle.PlacementState()
    oracle.place(st, {(0, 0, 0): 10}, 1, 1.0, min_count=5)
    assert st.resident == {(0, 0, 0)}
    # below min_count never enters even with a free slot
    st2 = oracle.PlacementState()
    assert oracle.place(st2, {(0, 0, 0): 4}, 3, 1.0, min_count=5) == ([], [], [])
    # hysteresis 1.0 still needs strictly more than the lowest count
    assert oracle.place(st, {(0, 0, 0): 10, (1, 0, 0): 10}, 1, 1.0) == ([], [], [])
    a, r, e = oracle.place(st, {(0, 0, 0): 10, (1, 0, 0): 11}, 1, 1.0)
    assert a == [(1, 0, 0)] and e == [(0, 0, 0)]
