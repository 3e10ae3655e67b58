"""Pins of the oracle's box geometries (sphere-box distance, box-box
separating-axis test, box poses of the robot) against closed forms and brute
force sampling. CPU only."""
import math

import numpy as np

from oracle import ezo_oracle as orc
from paper_2504_10783_gb300 import workloads as wl


def test_sphere_box_distance_closed_forms():
    bc, bR, bh = np.zeros(3), np.eye(3), np.array([1.0, 2.0, 3.0])
    f = lambda c, r: float(orc.sphere_box_distance(np.asarray(c, float), r, bc, bR, bh))
    assert abs(f([3, 0, 0], 0.5) - 1.5) < 1e-15            # face region
    assert abs(f([2, 3, 0], 0.0) - math.sqrt(2)) < 1e-15    # edge region
    assert abs(f([2, 3, 4], 0.1) - (math.sqrt(3) - 0.1)) < 1e-15  # corner region
    assert abs(f([0.5, 0, 0], 0.0) + 0.5) < 1e-15           # inside: nearest face 0.5 away
    assert f([1.0, 0, 0], 0.0) == 0.0                       # on the surface, a point does not overlap
    # invariance under a common rigid motion
    rng = np.random.default_rng(0)
    R = wl.rot_zyx(*rng.uniform(-3, 3, 3))
    t = rng.normal(size=3)
    for c in rng.uniform(-4, 4, size=(50, 3)):
        a = float(orc.sphere_box_distance(c, 0.2, bc, bR, bh))
        b = float(orc.sphere_box_distance(R @ c + t, 0.2, t, R, bh))
        assert abs(a - b) < 1e-12


def _box_points(c, R, h, k, surface):
    g = np.linspace(-1, 1, k)
    P = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    if surface:
        P = P[np.abs(P).max(axis=1) == 1.0]
    return c + (P * h) @ R.T


def test_box_box_separation_axis_aligned():
    I = np.eye(3)
    h = np.array([0.5, 0.5, 0.5])
    # gap of 0.3 along x: separation 0.3; overlap of 0.2: -0.2 (the smallest depth)
    assert abs(float(orc.box_box_separation(np.zeros(3), I, h, np.array([1.3, 0.1, 0.0]), I, h)) - 0.3) < 1e-12
    assert abs(float(orc.box_box_separation(np.zeros(3), I, h, np.array([0.8, 0.1, 0.0]), I, h)) + 0.2) < 1e-12


def test_box_box_separation_against_sampling():
    """Random oriented pairs away from contact (|sep| > 0.05): a positive
    separation never exceeds the distance from sampled points of B's surface
    to A; a negative one comes with sampled points of B inside A."""
    rng = np.random.default_rng(1)
    n_sep = n_ovl = 0
    for _ in range(300):
        ha, hb = rng.uniform(0.1, 0.6, 3), rng.uniform(0.1, 0.6, 3)
        Ra, Rb = wl.rot_zyx(*rng.uniform(-3, 3, 3)), wl.rot_zyx(*rng.uniform(-3, 3, 3))
        cb = rng.uniform(-1.2, 1.2, 3)
        sep = float(orc.box_box_separation(np.zeros(3), Ra, ha, cb, Rb, hb))
        if abs(sep) < 0.05:
            continue
        if sep > 0:
            P = _box_points(cb, Rb, hb, 25, True)
            d = orc.sphere_box_distance(P, 0.0, np.zeros(3), Ra, ha)
            assert d.min() >= sep - 1e-9
            n_sep += 1
        else:
            P = _box_points(cb, Rb, hb, 15, False)
            assert (orc.sphere_box_distance(P, 0.0, np.zeros(3), Ra, ha) < 0).any()
            n_ovl += 1
    assert n_sep > 50 and n_ovl > 50


def test_box_box_edge_axis_separates():
    """Two unit cubes whose edges cross: A's vertical edge at (0.5, 0.5) and a
    horizontal ridge of B along (1, -1, 0) / sqrt 2 (B's other axes at 45
    degrees between u = (1, 1, 0) / sqrt 2 and z), B just beyond A along u.
    Only the cross-product axis z x b_0 (= u) separates them; the six face
    axes alone would report an overlap."""
    h = np.full(3, 0.5)
    u = np.array([1.0, 1.0, 0.0]) / math.sqrt(2)
    z = np.array([0.0, 0.0, 1.0])
    b0 = np.array([1.0, -1.0, 0.0]) / math.sqrt(2)
    b1 = (u + z) / math.sqrt(2)
    Rb = np.column_stack([b0, b1, np.cross(b0, b1)])
    for gap, want_sep in ((0.05, True), (-0.05, False)):
        # B's nearest point to A along u: its support in direction -u
        sup = float(np.sum(h * np.abs(Rb.T @ u)))
        cb = u * (0.5 * math.sqrt(2) + sup + gap)
        sep = float(orc.box_box_separation(np.zeros(3), np.eye(3), h, cb, Rb, h))
        assert (sep > 0) == want_sep
        faces = max(
            float(np.abs(cb @ L) - np.sum(h * np.abs(L)) - np.sum(h * np.abs(Rb.T @ L)))
            for L in list(np.eye(3)) + list(Rb.T))
        if want_sep:
            assert faces < 0 < sep  # the separating axis is an edge-edge one
            P = _box_points(cb, Rb, h, 41, True)
            assert orc.sphere_box_distance(P, 0.0, np.zeros(3), np.eye(3), h).min() > 0


def test_box_arm_poses_and_labels():
    r = wl.box_arm_robot()
    assert r.n_boxes == 11 and r.self_bb.shape[0] == 26
    c, R = orc.box_poses(r, np.zeros((1, 7)))
    # arm straight up: segment boxes centred half way up their segments
    np.testing.assert_allclose(c[0, :4], [[0, 0, 0.17], [0, 0, 0.54], [0, 0, 0.94], [0, 0, 1.203]], atol=1e-12)
    np.testing.assert_allclose(c[0, 4:, :2], 0.0, atol=1e-12)
    np.testing.assert_allclose(c[0, 4:, 2], [0.34, 0.34, 0.74, 0.74, 1.14, 1.14, 1.266], atol=1e-12)
    env = wl.tabletop_box_env(3)
    assert env.n_boxes == 3 and env.n_obs > 50
    q = wl.uniform_configs(2, r, 300)
    lab = orc.in_collision(r, env, q)
    sd = orc.signed_distance(r, env, q)
    np.testing.assert_array_equal(lab, sd < 0)
    assert 0.2 < lab.mean() < 0.9
    # the arm straight up misses everything: the table top is at z = 0 and 0.2 m away
    assert not orc.in_collision(r, env, np.zeros((1, 7)))[0]


def test_box_seed_path_is_collision_free():
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "workloads.json")) as f:
        s = json.load(f)["boxes"]
    r = wl.box_arm_robot()
    env = wl.tabletop_box_env(s["env_seed"])
    V = np.asarray(s["path"])
    for k in range(V.shape[0] - 1):
        t = np.linspace(0.0, 1.0, 200)[:, None]
        assert orc.signed_distance(r, env, V[k] + t * (V[k + 1] - V[k])).min() >= 0.02
