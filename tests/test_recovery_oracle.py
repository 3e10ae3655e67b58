"""Pins of the oracle's recovery steps (Sec. VI-B): fine discretisation of a
path, its collision check, set editing with the last steps of Algorithm 1 and
the coverage test, against closed forms, constructions and invariants. CPU."""
import math

import numpy as np

from oracle import ezo_oracle as orc
from paper_2504_10783_gb300 import workloads as wl


def test_path_points_counts_and_spacing():
    # |e| = 0.5 at step 0.1 -> 5 pieces, 6 points on the 3-4-5 line
    P, e = orc.path_points([[0.0, 0.0], [0.3, 0.4]], 0.1)
    assert P.shape == (6, 2) and np.all(e == 0)
    np.testing.assert_allclose(P, np.column_stack([0.06 * np.arange(6), 0.08 * np.arange(6)]), atol=1e-15)
    # a point edge is one piece (both ends), an edge of length 1.05 needs 11
    P, e = orc.path_points([[1.0, 1.0], [1.0, 1.0], [1.0, 2.05]], 0.1)
    assert list(np.bincount(e)) == [2, 12]
    # N_k is the least piece count with pieces no longer than the step
    rng = np.random.default_rng(3)
    V = rng.uniform(-2, 2, size=(9, 7))
    P, e = orc.path_points(V, 0.1)
    for k in range(8):
        pk = P[e == k]
        L = np.linalg.norm(V[k + 1] - V[k])
        N = pk.shape[0] - 1
        assert L / N <= 0.1 + 1e-12 and (N == 1 or L / (N - 1) > 0.1)
        np.testing.assert_allclose(pk[0], V[k], atol=1e-15)
        np.testing.assert_allclose(pk[-1], V[k + 1], atol=1e-12)
        np.testing.assert_allclose(np.linalg.norm(np.diff(pk, axis=0), axis=1), L / N, rtol=1e-9)


def _sweep_scene():
    """Planar 3R arm (links 1, spheres r = 0.1 at 1/8, 3/8, .. of each link)
    stretched along angle theta (q = (theta, 0, 0)), one disk of r = 0.1 at
    (1.5, 0). The spheres 1.375 and 1.625 from the base come closest; by the
    cosine rule the arm collides iff cos(theta) > min over those two of
    (d^2 + 1.5^2 - 0.2^2) / (2 d 1.5), i.e. |theta| < theta_c."""
    rd = wl.planar3_robot()
    env = wl.Env("disk", np.array([[1.5, 0.0, 0.0, 0.1]]))
    th_c = max(math.acos((d * d + 2.25 - 0.04) / (3.0 * d)) for d in (1.375, 1.625))
    return rd, env, th_c


def test_check_path_closed_form_sweep():
    rd, env, th_c = _sweep_scene()
    assert 0.10 < th_c < 0.11
    verts = np.array([[-0.5, 0.0, 0.0], [0.5, 0.0, 0.0], [1.0, 0.0, 0.0], [1.5, 0.0, 0.0]])
    edge, lab, P, eid = orc.check_path(rd, env, verts, 0.1)
    np.testing.assert_array_equal(lab, np.abs(P[:, 0]) < th_c)
    assert list(edge) == [True, False, False]
    # the endpoints of the first edge are free: only the interior points find it
    assert not lab[0] and not lab[np.nonzero(eid == 0)[0][-1]]
    # one piece per edge checks the endpoints only and misses the collision
    edge1, lab1, _, _ = orc.check_path(rd, env, verts, 10.0)
    assert not edge1.any() and lab1.shape == (6,)


def test_path_coverage_boxes():
    box = lambda lo, hi: (np.vstack([np.eye(2), -np.eye(2)]), np.concatenate([hi, -np.asarray(lo)]))
    polys = [box([0, 0], [1, 1]), box([1, 0], [2, 1])]
    # each endpoint in a different box: not covered; both in one: covered
    assert list(orc.path_coverage(polys, [[0.5, 0.5], [1.5, 0.5], [1.8, 0.9]])) == [False, True]
    assert list(orc.path_coverage(polys, [[0.2, 0.2], [0.8, 0.8], [2.5, 0.5]])) == [True, False]
    # a shared face counts as inside (tolerance 1e-9)
    assert list(orc.path_coverage(polys, [[1.0, 0.2], [1.0 + 1e-10, 0.7]])) == [True]
    assert not orc.path_coverage([], [[0, 0], [1, 1]]).any()


def test_edit_excludes_every_given_collision_and_keeps_the_segment():
    """With N_f and N_p at least the number of colliding configurations in P,
    each of them ends outside the edited polytope: a plane through c* (with
    step back) separates the segment from c*, and c lies beyond c* on the ray
    from its projection. Configurations outside P or free are never used,
    the old rows are kept and the seed segment stays inside."""
    rd, env, th_c = _sweep_scene()
    env = wl.Env("disks", np.array([[1.5, 0.0, 0.0, 0.1], [0.0, 1.6, 0.0, 0.15]]))
    A = np.vstack([np.eye(3), -np.eye(3)])
    b = np.full(6, 2.0)  # P: |q_i| <= 2
    v1, v2 = np.array([-1.2, 0.3, -0.2]), np.array([-0.8, -0.3, 0.2])
    t = np.linspace(0, 1, 400)[:, None]
    assert not orc.in_collision(rd, env, v1 + t * (v2 - v1)).any()
    rng = np.random.default_rng(5)
    X = rng.uniform(-2.0, 2.0, size=(300, 3))
    X[::7, 1] = 2.4  # outside P by construction
    lab = orc.in_collision(rd, env, X)
    inside = np.abs(X).max(axis=1) <= 2.0
    assert (lab & ~inside).any() and (lab & inside).sum() >= 20 and (~lab & inside).any()
    prm = orc.Params(n_p=1000, n_f=1000, n_b=12, step_back_max=0.01, t_col=1e-3)
    ed = orc.edit_polytope(rd, env, A, b, v1, v2, X, prm)
    np.testing.assert_array_equal(ed.inside, inside)
    np.testing.assert_array_equal(ed.cand_index, np.nonzero(lab & inside)[0])
    assert ed.place.status == orc.STATUS_OK
    H = ed.place.rows_a.shape[0]
    assert 1 <= H <= len(ed.cand_index)
    np.testing.assert_array_equal(ed.A[:6], A)
    np.testing.assert_array_equal(ed.b[:6], b)
    assert orc.segment_contained(ed.A, ed.b, v1, v2, tol=0.0)
    new_viol = (X @ ed.A[6:].T > ed.b[6:][None, :]).any(axis=1)
    assert new_viol[ed.cand_index].all()
    # c* is colliding and each plane passes Delta in (0, Delta_max] below it
    assert orc.in_collision(rd, env, ed.bisect.c_star).all()
    for row, i, dl in zip(range(H), ed.place.order, ed.place.deltas):
        a = ed.place.rows_a[row]
        assert abs(np.linalg.norm(a) - 1.0) < 1e-12 and 0.0 < dl <= 0.01
        assert abs(a @ ed.bisect.c_star[i] - ed.place.rows_b[row] - dl) < 1e-12


def test_edit_with_a_small_face_budget_stops_at_n_f():
    rd, env, _ = _sweep_scene()
    A = np.vstack([np.eye(3), -np.eye(3)])
    b = np.full(6, 2.0)
    v1, v2 = np.array([-1.2, 0.3, -0.2]), np.array([-0.8, -0.3, 0.2])
    X = np.column_stack([np.linspace(-0.09, 0.09, 40), np.linspace(-1.5, 1.5, 40), np.zeros(40)])
    prm = orc.Params(n_p=1000, n_f=2, n_b=8)
    ed = orc.edit_polytope(rd, env, A, b, v1, v2, X, prm)
    assert ed.labels.any() and ed.place.rows_a.shape[0] <= 2
    prm1 = orc.Params(n_p=3, n_f=100, n_b=8)
    ed1 = orc.edit_polytope(rd, env, A, b, v1, v2, X, prm1)
    assert ed1.cand_index.shape[0] == 3
