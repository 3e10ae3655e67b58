"""Pins of the FP64 oracle against what the paper and the mathematics fix:
published vectors, closed forms, brute force and invariants. CPU only."""
import json
import math
import os

import numpy as np
import pytest
from scipy import stats

from oracle import ezo_oracle as orc
from paper_2504_10783_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def load_scene():
    with open(os.path.join(GOLDEN, "workloads.json")) as f:
        return json.load(f)


# --------------------------------------------------------------- Philox ----
def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = orc.philox4x32_10(np.array(v[:4], dtype=np.uint64), v[4:6])
        assert [int(x) for x in out] == v[6:10]


def test_uniform_conversions_exact_ends():
    assert orc.u01_closed_open(0) == 0.0
    assert orc.u01_closed_open(0xFFFFFFFF) == 1.0 - 2.0 ** -24
    assert orc.u01_open_closed(0) == 2.0 ** -24
    assert orc.u01_open_closed(0xFFFFFFFF) == 1.0
    assert orc.blocks_per_step(1) == 1 and orc.blocks_per_step(3) == 1 and orc.blocks_per_step(7) == 2
    assert orc.blocks_per_step(8) == 2 and orc.blocks_per_step(9) == 3 and orc.blocks_per_step(16) == 4
    # the step uniform: low bytes as one 24-bit integer, w0 lowest
    assert orc.step_uniform(0xFFFFFF00, 0x000000FF, 0x12345600) == 0xFF00 * 2.0 ** -24
    assert orc.step_uniform(0xFF, 0xFF, 0xFF) == 1.0 - 2.0 ** -24


def test_philox_uniforms_are_uniform():
    ctr = np.zeros((50000, 4), dtype=np.uint64)
    ctr[:, 0] = np.arange(50000)
    u = orc.u01_closed_open(orc.philox4x32_10(ctr, (5, 9)).ravel())
    h, _ = np.histogram(u, bins=20, range=(0, 1))
    assert stats.chisquare(h).pvalue > 1e-4


# ----------------------------------------------------------- kinematics ----
def test_dh7_home_and_bent_poses():
    """Closed forms of the 7-DOF chain: at q = 0 all links stack on the z axis
    (origins at 0, 0.34, 0.34, 0.74, 0.74, 1.14, 1.14, 1.266); q2 = pi/2 folds
    the arm from joint 2 onto +x; q4 = pi/2 folds it from joint 4 onto -x."""
    r = wl.dh7_robot()
    _, o = orc.dh_frames(r, np.zeros((1, 7)))
    z = [0, 0.34, 0.34, 0.74, 0.74, 1.14, 1.14, 1.266]
    np.testing.assert_allclose(o[0], np.column_stack([np.zeros(8), np.zeros(8), z]), atol=1e-12)
    q = np.zeros((2, 7))
    q[0, 1] = math.pi / 2
    q[1, 3] = math.pi / 2
    _, o = orc.dh_frames(r, q)
    np.testing.assert_allclose(o[0, -1], [0.926, 0, 0.34], atol=1e-12)
    np.testing.assert_allclose(o[1, -1], [-0.526, 0, 0.74], atol=1e-12)


def _elementary_chain(r, q):
    """Independent construction: 4x4 products of the four elementary moves."""
    T = np.eye(4)
    out = [T.copy()]
    prism = r.prismatic
    for i in range(r.n):
        th = r.theta_off[i] + (0.0 if prism[i] else q[i])
        Rz = np.eye(4)
        Rz[:2, :2] = [[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]]
        Tz = np.eye(4)
        Tz[2, 3] = r.d[i] + (q[i] if prism[i] else 0.0)
        Tx = np.eye(4)
        Tx[0, 3] = r.a[i]
        al = r.alpha[i]
        Rx = np.eye(4)
        Rx[1:3, 1:3] = [[math.cos(al), -math.sin(al)], [math.sin(al), math.cos(al)]]
        T = T @ Rz @ Tz @ Tx @ Rx
        out.append(T.copy())
    return out


def _mixed_robot():
    """A 4-joint chain with prismatic joints 2 and 4 and non-zero offsets."""
    r = wl.dh7_robot()
    return wl.Robot(name="mixed", a=np.array([0.1, 0.0, 0.3, 0.05]), alpha=np.array([0.4, -1.2, 0.0, 0.7]),
                    d=np.array([0.2, 0.1, 0.0, 0.3]), theta_off=np.array([0.3, -0.5, 0.1, 0.0]),
                    q_lo=np.array([-2.0, 0.0, -2.0, -0.5]), q_hi=np.array([2.0, 1.0, 2.0, 0.5]),
                    sphere_frame=r.sphere_frame[:0], sphere_xyz=r.sphere_xyz[:0], sphere_r=r.sphere_r[:0],
                    sphere_link=r.sphere_link[:0], self_pairs=r.self_pairs[:0],
                    joint_type=np.array([0, 1, 0, 1], dtype=np.int32))


@pytest.mark.parametrize("robot", [wl.dh7_robot(), wl.planar3_robot(), _mixed_robot(), wl.point2_robot(),
                                   wl.chain_robot(10)], ids=lambda r: r.name)
def test_dh_frames_match_elementary_products(robot):
    q = wl.uniform_configs(3, robot, 20)
    R, o = orc.dh_frames(robot, q)
    for k in range(q.shape[0]):
        Ts = _elementary_chain(robot, q[k])
        for i, T in enumerate(Ts):
            np.testing.assert_allclose(R[k, i], T[:3, :3], atol=1e-12)
            np.testing.assert_allclose(o[k, i], T[:3, 3], atol=1e-12)


def test_planar_sphere_centres_sum_of_angles():
    """Planar arm: the point a fraction f along link k is
    sum_{i<k} (cos, sin)(theta_1 + .. + theta_i) + f (cos, sin)(theta_1 + .. + theta_k)."""
    r = wl.planar3_robot()
    q = wl.uniform_configs(4, r, 50)
    c = orc.sphere_centres(r, q)
    for k in range(q.shape[0]):
        cum = np.cumsum(q[k])
        s = 0
        for link in range(3):
            base = np.array([sum(math.cos(cum[i]) for i in range(link)),
                             sum(math.sin(cum[i]) for i in range(link))])
            for j in range(4):
                f = (j + 0.5) / 4
                p = base + f * np.array([math.cos(cum[link]), math.sin(cum[link])])
                np.testing.assert_allclose(c[k, s, :2], p, atol=1e-12)
                assert abs(c[k, s, 2]) < 1e-15
                s += 1


def test_chain_robot_layout():
    """The n-joint chain: two spheres per link on its distal frame k at
    o_k - (1 - f) a x_k (f = 1/4, 3/4), which for the links without a d
    offset (k >= 2) lies between the origins of frames k - 1 and k, and self
    pairs between links at least three apart (4 sphere pairs per link
    pair)."""
    n = 10
    r = wl.chain_robot(n)
    assert r.sphere_frame.tolist() == [k for k in range(1, n + 1) for _ in range(2)]
    link_pairs = sum(max(0, n - (i + 2)) for i in range(1, n + 1))
    assert r.self_pairs.shape == (4 * link_pairs, 2) == (112, 2)
    assert np.all(np.abs(r.sphere_link[r.self_pairs[:, 0]] - r.sphere_link[r.self_pairs[:, 1]]) >= 3)
    q = wl.uniform_configs(5, r, 10)
    R, o = orc.dh_frames(r, q)
    c = orc.sphere_centres(r, q)
    for k in range(1, n + 1):
        for j, f in ((2 * (k - 1), 0.25), (2 * (k - 1) + 1, 0.75)):
            np.testing.assert_allclose(c[:, j], o[:, k] - (1 - f) * 0.15 * R[:, k][:, :, 0], atol=1e-12)
            if k >= 2:
                np.testing.assert_allclose(c[:, j], o[:, k - 1] + f * (o[:, k] - o[:, k - 1]), atol=1e-12)
    # the largest robot the library takes: 16 links of 16 spheres, f = (i + 1/2) / 16
    m = wl.chain_robot(16, r=0.02, per_link=16)
    assert m.sphere_r.shape == (256,) and np.all(m.sphere_r == 0.02)
    assert m.self_pairs.shape == (16 * 16 * sum(max(0, 16 - (i + 2)) for i in range(1, 17)), 2) == (23296, 2)
    q = wl.uniform_configs(6, m, 4)
    R, o = orc.dh_frames(m, q)
    c = orc.sphere_centres(m, q)
    for k in (2, 9, 16):
        for i in (0, 7, 15):
            f = (i + 0.5) / 16
            np.testing.assert_allclose(c[:, 16 * (k - 1) + i], o[:, k - 1] + f * (o[:, k] - o[:, k - 1]), atol=1e-12)


def test_dh7_sphere_layout():
    r = wl.dh7_robot()
    assert r.n_spheres == 40 and r.self_pairs.shape == (228, 2)
    assert r.sphere_r.max() <= 0.08 and r.sphere_r.min() >= 0.04
    # at q = 0 every sphere lies on the z axis between 0 and 1.266
    c = orc.sphere_centres(r, np.zeros((1, 7)))[0]
    np.testing.assert_allclose(c[:, :2], 0, atol=1e-12)
    assert np.all(np.diff(c[:, 2]) > 0) and c[-1, 2] < 1.266


# ------------------------------------------------------------ collision ----
def _brute(robot, env, q):
    c = orc.sphere_centres(robot, q[None])[0]
    hit, sd = False, math.inf
    for i in range(robot.n_spheres):
        for o in env.spheres:
            d = math.dist(c[i], o[:3])
            hit |= d * d < (robot.sphere_r[i] + o[3]) ** 2
            sd = min(sd, d - robot.sphere_r[i] - o[3])
    for i, j in robot.self_pairs:
        d = math.dist(c[i], c[j])
        hit |= d * d < (robot.sphere_r[i] + robot.sphere_r[j]) ** 2
        sd = min(sd, d - robot.sphere_r[i] - robot.sphere_r[j])
    return hit, sd


def test_collision_matches_brute_force_loops():
    r = wl.dh7_robot()
    env = wl.box_obstacles(2, 10, box_lo=(0.2, -0.6, 0.3), box_hi=(0.8, 0.6, 1.2), r_lo=0.05, r_hi=0.15)
    q = wl.uniform_configs(5, r, 60)
    lab = orc.in_collision(r, env, q)
    sd = orc.signed_distance(r, env, q)
    for k in range(q.shape[0]):
        h, s = _brute(r, env, q[k])
        assert lab[k] == h
        assert abs(sd[k] - s) < 1e-12
    assert 0 < lab.sum() < q.shape[0]


def test_collision_touching_cases():
    """An obstacle tangent to a robot sphere at home pose, nudged by +-1e-4."""
    r = wl.dh7_robot()
    c = orc.sphere_centres(r, np.zeros((1, 7)))[0]
    i = 20
    for gap, expect in [(1e-4, False), (-1e-4, True)]:
        R = 0.05
        x = c[i, 0] + r.sphere_r[i] + R + gap
        env = wl.Env("t", np.array([[x, c[i, 1], c[i, 2], R]]))
        assert orc.in_collision(r, env, np.zeros((1, 7)))[0] == expect
        assert abs(orc.signed_distance(r, env, np.zeros((1, 7)))[0] - gap) < 1e-12


def test_self_collision_planar_fold():
    """Planar arm folded so link 3 comes back over link 1: links 1 and 3 touch."""
    r = wl.planar3_robot()
    env = wl.Env("none", np.zeros((0, 4)))
    folded = np.array([[0.0, math.pi - 0.05, math.pi - 0.05]])
    straight = np.array([[0.0, 0.0, 0.0]])
    assert orc.in_collision(r, env, folded)[0]
    assert not orc.in_collision(r, env, straight)[0]


def test_signed_distance_sign_matches_label():
    r = wl.dh7_robot()
    env = wl.box_obstacles(11, 64)
    q = wl.uniform_configs(6, r, 3000)
    assert np.array_equal(orc.in_collision(r, env, q), orc.signed_distance(r, env, q) < 0)


# ------------------------------------------------- round size and test ----
@pytest.mark.parametrize("eps,delta", [(0.1, 0.05), (0.05, 0.05), (0.01, 0.05), (0.005, 0.005)])
def test_round_size_meets_binomial_guarantee(eps, delta):
    """With M from the paper's formula, a region whose collision fraction is
    exactly eps passes the unadaptive test with probability <= delta_k
    (exact binomial tail), and M is the smallest size whose Chernoff bound
    exp(-tau^2 eps M / 2) reaches delta_k."""
    tau = 0.5
    total = 0.0
    for k in range(1, 51):
        dk = orc.delta_k(k, delta)
        M = orc.test_size(k, eps, delta, tau)
        thr = math.floor(M * (1 - tau) * eps)
        assert stats.binom.cdf(thr, M, eps) <= dk
        assert math.exp(-tau * tau * eps * M / 2) <= dk * (1 + 1e-12)
        assert math.exp(-tau * tau * eps * (M - 1) / 2) > dk
        total += dk
    assert total <= delta


def test_round_size_values():
    """Sizes quoted for eps=0.1/delta=0.05 and eps=delta=0.05 with tau=0.5."""
    assert [orc.test_size(k, 0.1, 0.05, 0.5) for k in (1, 2, 5)] == [280, 391, 537]
    assert [orc.test_size(k, 0.05, 0.05, 0.5) for k in (1, 2, 10)] == [559, 781, 1296]
    assert orc.batch_size(1, 0.05, 0.05, 0.5, 10000) == 10000
    assert orc.batch_size(1, 0.05, 0.05, 0.5, 100) == 559


def test_unadaptive_test_threshold():
    M = 559
    thr = M * 0.5 * 0.05  # 13.975
    assert orc.unadaptive_test(13, M, 0.05, 0.5)
    assert not orc.unadaptive_test(14, M, 0.05, 0.5)
    assert orc.unadaptive_test(0, M, 0.05, 0.5)
    assert thr == pytest.approx(13.975)


# ------------------------------------------------ distance to a segment ----
def test_projection_cases():
    v1 = np.array([0.0, 0.0, 0.0])
    v2 = np.array([2.0, 0.0, 0.0])
    c = np.array([[1.0, 1.0, 0.0], [-1.0, 1.0, 0.0], [3.0, -1.0, 2.0]])
    p = orc.project_onto_segment(c, v1, v2)
    np.testing.assert_allclose(p, [[1, 0, 0], [0, 0, 0], [2, 0, 0]])
    np.testing.assert_allclose(orc.project_onto_segment(c, v1, v1), np.zeros((3, 3)))
    np.testing.assert_allclose(orc.dist_to_segment(c, v1, v2), [1.0, math.sqrt(2), math.sqrt(6)])


def test_distance_equals_brute_force_minimum():
    rng = np.random.default_rng(0)
    v1, v2 = rng.standard_normal(7), rng.standard_normal(7)
    c = rng.standard_normal((30, 7)) * 2
    t = np.linspace(0, 1, 200001)[:, None]
    pts = (1 - t) * v1 + t * v2
    d = orc.dist_to_segment(c, v1, v2)
    for k in range(c.shape[0]):
        bf = np.linalg.norm(pts - c[k], axis=1).min()
        assert d[k] <= bf + 1e-12 and bf - d[k] < 1e-7


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(1)
    v1, v2 = rng.standard_normal(5), rng.standard_normal(5)
    for _ in range(20):
        c = rng.standard_normal(5) * 2
        g = orc.dist_gradient(c, v1, v2)[0]
        h = 1e-6
        fd = np.array([(orc.dist_to_segment(c + h * e, v1, v2)[0] - orc.dist_to_segment(c - h * e, v1, v2)[0])
                       / (2 * h) for e in np.eye(5)])
        np.testing.assert_allclose(g, fd, atol=1e-6)
        assert abs(np.linalg.norm(g) - 1) < 1e-12


def test_distance_is_convex_jensen():
    """App. A: dist_L is convex."""
    rng = np.random.default_rng(2)
    v1, v2 = rng.standard_normal(4), rng.standard_normal(4)
    x1, x2 = rng.standard_normal((500, 4)) * 3, rng.standard_normal((500, 4)) * 3
    lam = rng.uniform(size=(500, 1))
    lhs = orc.dist_to_segment(lam * x1 + (1 - lam) * x2, v1, v2)
    rhs = lam[:, 0] * orc.dist_to_segment(x1, v1, v2) + (1 - lam[:, 0]) * orc.dist_to_segment(x2, v1, v2)
    assert np.all(lhs <= rhs + 1e-12)


def test_tangent_plane_never_cuts_segment():
    """Eq. (4): the plane through c with normal grad dist_L(c) supports the
    sub-level set at dist_L(c), so a^T v <= a^T c - dist_L(c) on L."""
    rng = np.random.default_rng(3)
    v1, v2 = rng.standard_normal(6), rng.standard_normal(6)
    c = rng.standard_normal((200, 6)) * 2
    a = orc.dist_gradient(c, v1, v2)
    b = np.einsum("ij,ij->i", a, c)
    d = orc.dist_to_segment(c, v1, v2)
    t = np.linspace(0, 1, 101)[:, None]
    L = (1 - t) * v1 + t * v2
    assert np.all((L @ a.T).max(axis=0) <= b - d + 1e-12)


# ---------------------------------------------------------- placement ----
def test_placement_hand_worked_example():
    g = json.load(open(os.path.join(GOLDEN, "placement_example.json")))
    c = np.array(g["candidates"])
    res = orc.place_hyperplanes(c, np.arange(c.shape[0]), np.array(g["v1"]), np.array(g["v2"]),
                                g["n_f"], g["step_back_max"], g["t_col"])
    assert res.status == orc.STATUS_OK
    assert res.order == g["expected_order"]
    np.testing.assert_allclose(res.rows_a, g["expected_rows_a"], atol=1e-15)
    np.testing.assert_allclose(res.rows_b, g["expected_rows_b"], atol=1e-15)
    np.testing.assert_allclose(res.deltas, g["expected_deltas"], atol=1e-15)


def test_placement_invariants_random():
    rng = np.random.default_rng(4)
    for trial in range(20):
        n = 3 + trial % 5
        v1, v2 = rng.standard_normal(n), rng.standard_normal(n)
        c = rng.standard_normal((300, n)) * 1.5
        c = c[orc.dist_to_segment(c, v1, v2) > 2e-3]
        res = orc.place_hyperplanes(c, np.arange(c.shape[0]), v1, v2, 10, 0.05, 1e-3)
        H = res.rows_a.shape[0]
        assert res.status == 0 and 1 <= H <= 10
        # L stays inside every new half space
        assert np.all(res.rows_a @ v1 <= res.rows_b + 1e-12)
        assert np.all(res.rows_a @ v2 <= res.rows_b + 1e-12)
        assert all(0 < d <= 0.05 + 1e-15 for d in res.deltas)
        # every placed candidate lies outside its own half space and inside
        # the earlier ones; the order is by distance
        dist = orc.dist_to_segment(c, v1, v2)
        for h, i in enumerate(res.order):
            assert res.rows_a[h] @ c[i] > res.rows_b[h]
            assert np.all(res.rows_a[:h] @ c[i] <= res.rows_b[:h])
        assert np.all(np.diff(dist[res.order]) >= 0)
        if H < 10:
            # nothing placed is left inside all rows
            inside = np.all(c @ res.rows_a.T <= res.rows_b, axis=1)
            assert not inside.any()


def test_placement_tcol_reports_collision():
    v1, v2 = np.zeros(3), np.array([1.0, 0, 0])
    c = np.array([[0.5, 5e-4, 0.0], [0.5, 0.3, 0.0]])
    res = orc.place_hyperplanes(c, np.arange(2), v1, v2, 10, 0.01, 1e-3)
    assert res.status == orc.STATUS_SEGMENT_IN_COLLISION and res.rows_a.shape[0] == 0


# ---------------------------------------------------------- hit-and-run ----
def test_hit_and_run_uniform_on_box():
    n = 3
    A = np.vstack([np.eye(n), -np.eye(n)])
    b = np.concatenate([np.ones(n), np.zeros(n)])
    x = orc.hit_and_run(A, b, np.full(n, 0.2), np.full(n, 0.7), 6000, 40, seed=3, stream=0, k=1)
    assert np.all(x @ A.T <= b + 1e-12)
    for d in range(n):
        h, _ = np.histogram(x[:, d], bins=10, range=(0, 1))
        assert stats.chisquare(h).pvalue > 1e-4
    h2, _, _ = np.histogram2d(x[:, 0], x[:, 1], bins=5, range=[[0, 1], [0, 1]])
    assert stats.chisquare(h2.ravel()).pvalue > 1e-4


def test_hit_and_run_uniform_on_cut_box():
    """Unit square cut by x + y <= 1: the marginal density of x is 2 (1 - x)."""
    A = np.array([[1.0, 0], [0, 1.0], [-1.0, 0], [0, -1.0], [1.0, 1.0]])
    b = np.array([1.0, 1.0, 0.0, 0.0, 1.0])
    x = orc.hit_and_run(A, b, np.array([0.1, 0.1]), np.array([0.5, 0.3]), 8000, 40, seed=4, stream=2, k=3)
    assert np.all(x @ A.T <= b + 1e-12)
    edges = np.linspace(0, 1, 11)
    h, _ = np.histogram(x[:, 0], bins=edges)
    cdf = 1 - (1 - edges) ** 2
    assert stats.chisquare(h, np.diff(cdf) * x.shape[0]).pvalue > 1e-4


def test_hit_and_run_streams_are_reproducible_and_distinct():
    A, b = orc.joint_box(wl.dh7_robot())
    v1, v2 = np.zeros(7), np.full(7, 0.3)
    x1 = orc.hit_and_run(A, b, v1, v2, 50, 5, seed=9, stream=1, k=1)
    x2 = orc.hit_and_run(A, b, v1, v2, 50, 5, seed=9, stream=1, k=1)
    x3 = orc.hit_and_run(A, b, v1, v2, 50, 5, seed=9, stream=2, k=1)
    part = orc.hit_and_run(A, b, v1, v2, 20, 5, seed=9, stream=1, k=1, first_walk=30)
    assert np.array_equal(x1, x2) and not np.allclose(x1, x3)
    np.testing.assert_array_equal(part, x1[30:])


# ------------------------------------------------------------ bisection ----
def test_bisection_brackets_the_boundary():
    s = load_scene()["planar3"]
    r = wl.planar3_robot()
    env = wl.Env("p", np.array(s["obstacles"]))
    v1, v2 = np.array(s["v1"]), np.array(s["v2"])
    q = wl.uniform_configs(8, r, 4000)
    c = q[orc.in_collision(r, env, q)][:200]
    res = orc.bisect(r, env, c, v1, v2, 10)
    p = orc.project_onto_segment(c, v1, v2)
    assert orc.in_collision(r, env, res.c_star).all()
    # c* lies on [p, c], no farther than c, and the free end of the final
    # bracket is one step of |c - p| / 2^N_b closer to p
    dc = np.linalg.norm(c - p, axis=1)
    ds = np.linalg.norm(res.c_star - p, axis=1)
    assert np.all(ds <= dc + 1e-12)
    cross = (res.c_star - p) - (ds / dc)[:, None] * (c - p)
    assert np.abs(cross).max() < 1e-12
    free_end = res.c_star - (c - p) / 2 ** 10
    assert not orc.in_collision(r, env, free_end).any()
    # the fraction along [p, c] is the dyadic number the decisions spell
    frac = np.ones(c.shape[0])
    lo = np.zeros(c.shape[0])
    for k in range(10):
        mid = 0.5 * (lo + frac)
        frac = np.where(res.decisions[:, k], mid, frac)
        lo = np.where(res.decisions[:, k], lo, mid)
    np.testing.assert_allclose(ds / dc, frac, atol=1e-12)


# ------------------------------------------------------ whole algorithm ----
def _uniform_in_polytope_by_rejection(robot, A, b, count, seed):
    rng = np.random.default_rng(seed)
    out = []
    while sum(len(o) for o in out) < count:
        x = rng.uniform(robot.q_lo, robot.q_hi, size=(20000, robot.n))
        out.append(x[np.all(x @ A.T <= b, axis=1)])
    return np.concatenate(out)[:count]


def test_eizo_planar_contains_segment_and_is_certified():
    s = load_scene()["planar3"]
    r = wl.planar3_robot()
    env = wl.Env("p", np.array(s["obstacles"]))
    v1, v2 = np.array(s["v1"]), np.array(s["v2"])
    A0, b0 = orc.joint_box(r)
    prm = orc.Params(eps=0.1, delta=0.05, n_p=1000, n_f=10, n_b=10, n_mix=30, seed=1)
    res = orc.eizo(r, env, v1, v2, A0, b0, prm)
    assert res.status == 0 and res.planes > 0
    assert orc.segment_contained(res.A, res.b, v1, v2, tol=1e-12)
    x = _uniform_in_polytope_by_rejection(r, res.A, res.b, 20000, 5)
    assert orc.in_collision(r, env, x).mean() <= prm.eps


def test_eizo_planar_collision_fraction_on_a_dense_grid():
    """The planar polytope's collision fraction by brute force: the centres
    of a 96^3 grid over the joint box that lie in P, checked one by one. It
    is within eps, and within 0.02 of the rejection-sampling estimate."""
    s = load_scene()["planar3"]
    r = wl.planar3_robot()
    env = wl.Env("p", np.array(s["obstacles"]))
    v1, v2 = np.array(s["v1"]), np.array(s["v2"])
    A0, b0 = orc.joint_box(r)
    prm = orc.Params(eps=0.1, delta=0.05, n_p=1000, n_f=10, n_b=10, n_mix=30, seed=1)
    res = orc.eizo(r, env, v1, v2, A0, b0, prm)
    g = 96
    axes = [np.linspace(lo, hi, g, endpoint=False) + (hi - lo) / (2 * g) for lo, hi in zip(r.q_lo, r.q_hi)]
    X = np.stack(np.meshgrid(*axes, indexing="ij"), -1).reshape(-1, 3)
    X = X[np.all(X @ res.A.T <= res.b, axis=1)]
    assert X.shape[0] > 10000
    grid = orc.in_collision(r, env, X).mean()
    mc = orc.in_collision(r, env, _uniform_in_polytope_by_rejection(r, res.A, res.b, 20000, 5)).mean()
    assert grid <= prm.eps
    assert abs(grid - mc) <= 0.02, (grid, mc)


def test_eizo_certificate_holds_over_seeds():
    """The guarantee of Sec. III-A: P[collision fraction > eps] <= delta.
    Over 100 seeds at eps = 0.1, delta = 0.05 the number of polytopes whose
    estimated collision fraction exceeds eps must be plausible under
    Binomial(100, 0.05)."""
    s = load_scene()["planar3"]
    r = wl.planar3_robot()
    env = wl.Env("p", np.array(s["obstacles"]))
    v1, v2 = np.array(s["v1"]), np.array(s["v2"])
    A0, b0 = orc.joint_box(r)
    bad = 0
    n_seeds = 100
    for seed in range(1, n_seeds + 1):
        prm = orc.Params(eps=0.1, delta=0.05, n_p=300, n_f=10, n_b=8, n_mix=20, seed=seed)
        res = orc.eizo(r, env, v1, v2, A0, b0, prm)
        x = _uniform_in_polytope_by_rejection(r, res.A, res.b, 4000, seed)
        bad += orc.in_collision(r, env, x).mean() > prm.eps
    assert stats.binom.sf(bad - 1, n_seeds, 0.05) > 1e-3, bad


def test_inflate_path_skips_contained_segment():
    """Sec. VI-A: a segment inside an earlier polytope is not inflated again."""
    s = load_scene()["planar3"]
    r = wl.planar3_robot()
    env = wl.Env("p", np.array(s["obstacles"]))
    v1, v2 = np.array(s["v1"]), np.array(s["v2"])
    verts = np.array([v1, 0.5 * (v1 + v2), v2])
    prm = orc.Params(eps=0.1, delta=0.05, n_p=500, n_f=10, n_b=10, n_mix=20, seed=2)
    out = orc.inflate_path(r, env, verts, prm)
    assert [k for k, _ in out] == [0]
    assert orc.segment_contained(out[0][1].A, out[0][1].b, verts[1], verts[2])


def test_inflate_dh7_path_covers_every_segment():
    d = load_scene()["dh7"]
    r = wl.dh7_robot()
    env = wl.box_obstacles(d["env_seed"], d["n_obs"])
    verts = np.array(d["path"])[:4]
    prm = orc.Params(eps=0.05, delta=0.05, n_p=1000, n_f=10, n_b=10, n_mix=30, seed=3)
    out = orc.inflate_path(r, env, verts, prm)
    for k in range(verts.shape[0] - 1):
        assert any(orc.segment_contained(res.A, res.b, verts[k], verts[k + 1]) for _, res in out)
    for k, res in out:
        assert res.status == 0
        assert orc.segment_contained(res.A, res.b, verts[k], verts[k + 1], tol=1e-12)


# ------------------------------------------------------- Forest (Sec. V) ----
def test_point_robot_and_forest_closed_forms():
    """The point robot sits at (0, q_1, q_0); a configuration collides iff
    its distance to a disk centre is below 0.35 (brute force over disks)."""
    r = wl.point2_robot()
    env = wl.forest_obstacles(41)
    assert env.n_obs == 15 and np.all(env.spheres[:, 3] == 0.35)
    assert np.all((env.spheres[:, 1:3] >= 1.5) & (env.spheres[:, 1:3] <= 8.5)) and np.all(env.spheres[:, 0] == 0)
    q = wl.uniform_configs(5, r, 4000)
    c = orc.sphere_centres(r, q)[:, 0, :]
    np.testing.assert_allclose(c, np.column_stack([np.zeros(4000), q[:, 1], q[:, 0]]), atol=1e-12)
    brute = np.zeros(4000, dtype=bool)
    for i in range(4000):
        for o in env.spheres:
            if (q[i, 0] - o[2]) ** 2 + (q[i, 1] - o[1]) ** 2 < o[3] ** 2:
                brute[i] = True
    lab = orc.in_collision(r, env, q)
    np.testing.assert_array_equal(lab, brute)
    assert 0.05 < lab.mean() < 0.3


def test_forest_seed_path_is_collision_free():
    s = load_scene()["forest"]
    r = wl.point2_robot()
    env = wl.forest_obstacles(s["forest_seed"])
    V = np.asarray(s["path"])
    assert np.allclose(V[0], [0.5, 0.5]) and np.allclose(V[-1], [9.5, 9.5])
    for k in range(V.shape[0] - 1):
        t = np.linspace(0.0, 1.0, 2000)[:, None]
        assert orc.signed_distance(r, env, V[k] + t * (V[k + 1] - V[k])).min() >= 0.02
