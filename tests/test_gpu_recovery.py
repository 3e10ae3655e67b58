"""GPU parity of the recovery steps (Sec. VI-B) through the C ABI against the
FP64 oracle: the discretised path check, set editing, the coverage test and
re-inflation. Tolerances as in test_gpu_parity: labels exact outside the
1e-5 m band, bisection decisions followed inside it, c* within 1e-9, planes
within 1e-6 relative, counts and indices exact."""
import json
import math
import os

import numpy as np
import pytest

from oracle import ezo_oracle as orc
from paper_2504_10783_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

AMB = 1e-5
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def ezo():
    from paper_2504_10783_gb300 import build, ezo as e
    build.build()
    return e


def dh7_scene():
    with open(os.path.join(GOLDEN, "workloads.json")) as f:
        s = json.load(f)["dh7"]
    return wl.dh7_robot(), wl.box_obstacles(s["env_seed"], s["n_obs"]), np.asarray(s["path"])


def labels_agree(rd, env_np, P, got, ref):
    diff = got != ref
    if diff.any():
        sd = orc.signed_distance(rd, env_np, P[diff].astype(np.float32).astype(np.float64))
        assert np.all(np.abs(sd) < AMB), f"{int((np.abs(sd) >= AMB).sum())} labels differ outside the band"


# ------------------------------------------------------- path discretisation --
def test_path_points_match_oracle(ezo):
    rng = np.random.default_rng(2)
    V = rng.uniform(-2, 2, size=(17, 7))
    V[5] = V[4]  # a point edge
    cnt, tot = ezo.path_points(V, 0.1)
    _, eid = orc.path_points(V, 0.1)
    np.testing.assert_array_equal(cnt, np.bincount(eid, minlength=16))
    assert tot == eid.shape[0]
    c1, t1 = ezo.path_points(V[:1], 0.1)
    assert c1.shape == (0,) and t1 == 0
    with pytest.raises(RuntimeError):
        ezo.path_points(V, 0.0)
    with pytest.raises(RuntimeError):
        ezo.path_points(V, float("nan"))


def test_check_path_closed_form_sweep(ezo):
    """Planar 3R arm swept through one disk: a point collides iff |theta| is
    below the closed-form angle (see the oracle pins), so the GPU labels are
    compared with the formula as well as with the oracle."""
    rd = wl.planar3_robot()
    env_np = wl.Env("disk", np.array([[1.5, 0.0, 0.0, 0.1]]))
    th_c = max(math.acos((d * d + 2.25 - 0.04) / (3.0 * d)) for d in (1.375, 1.625))
    verts = np.array([[-0.5, 0.0, 0.0], [0.5, 0.0, 0.0], [1.0, 0.0, 0.0], [1.5, 0.0, 0.0]])
    robot, env = ezo.Robot(rd), ezo.Env(env_np)
    pf = torch.zeros(64, dtype=torch.uint8, device="cuda")
    edge, npts = ezo.check_path(robot, env, verts, 0.1, pf)
    torch.cuda.synchronize()
    e_ref, lab_ref, P, _ = orc.check_path(rd, env_np, verts, 0.1)
    got = pf[:npts].cpu().numpy().astype(bool)
    assert npts == P.shape[0]
    np.testing.assert_array_equal(got, np.abs(P[:, 0]) < th_c)
    np.testing.assert_array_equal(got, lab_ref)
    np.testing.assert_array_equal(edge, e_ref)
    assert list(edge) == [True, False, False]


def test_check_path_matches_oracle_dh7(ezo):
    rd, env_np, _ = dh7_scene()
    rng = np.random.default_rng(9)
    V = rng.uniform(0.8 * rd.q_lo, 0.8 * rd.q_hi, size=(25, 7))
    robot, env = ezo.Robot(rd), ezo.Env(env_np)
    _, tot = ezo.path_points(V, 0.1)
    pf = torch.zeros(tot, dtype=torch.uint8, device="cuda")
    edge, npts = ezo.check_path(robot, env, V, 0.1, pf)
    torch.cuda.synchronize()
    e_ref, lab_ref, P, eid = orc.check_path(rd, env_np, V, 0.1)
    assert npts == tot == P.shape[0]
    got = pf.cpu().numpy().astype(bool)
    assert lab_ref.any() and not lab_ref.all()
    labels_agree(rd, env_np, P, got, lab_ref)
    for k in range(24):
        assert edge[k] == got[eid == k].any()
    # edge flags without the per-point buffer, and the error cases
    edge2, _ = ezo.check_path(robot, env, V, 0.1)
    np.testing.assert_array_equal(edge2, edge)
    e1, n1 = ezo.check_path(robot, env, V[:1], 0.1)
    assert e1.shape == (0,) and n1 == 0
    small = torch.zeros(tot - 1, dtype=torch.uint8, device="cuda")
    with pytest.raises(RuntimeError):
        ezo.check_path(robot, env, V, 0.1, small)


# ------------------------------------------------------------ set editing --
def _edit_replay(ezo, rd, env_np, v1, v2, A, b, X, prm_kw):
    """Runs the batch on [v1, v2] to a final polytope, replaces it with
    (A, b), edits it with X on the GPU and replays the edit in the oracle
    (following the GPU's bisection decisions inside the ambiguity band)."""
    robot, env = ezo.Robot(rd), ezo.Env(env_np)
    prm = ezo.Params.make(**prm_kw)
    oprm = orc.Params(eps=prm.eps, delta=prm.delta, tau=prm.tau, step_back_max=prm.step_back_max, t_col=prm.t_col,
                      n_p=prm.n_p, n_f=prm.n_f, n_b=prm.n_b, n_mix=prm.n_mix, n_it_max=prm.n_it_max, seed=prm.seed)
    bt = ezo.Batch(robot, [env], v1, v2, prm)
    bt.run()
    st0 = bt.state(0)
    assert st0["status"] in (ezo.SEG_ACCEPTED, ezo.SEG_MAX_ITER)
    bt.set_polytope(0, A, b)
    X = np.asarray(X, dtype=np.float32).astype(np.float64)
    bt.edit(X)
    st = bt.state(0)
    ref_in = orc.points_inside(A, b, X)
    lab = bt.read(0, "labels")[: X.shape[0]].astype(bool)
    labels_agree(rd, env_np, X, lab, orc.in_collision(rd, env_np, X))
    idx = np.nonzero(ref_in & lab)[0][: oprm.n_p]
    assert st["count"] == int((ref_in & lab).sum())
    assert st["n_cand"] == idx.size
    np.testing.assert_array_equal(bt.read(0, "cand_idx")[: idx.size], idx)
    bits = bt.read(0, "bits")[: idx.size]
    follow = ((bits[:, None] >> np.arange(oprm.n_b)[None, :]) & 1).astype(bool)
    ed = orc.edit_polytope(rd, env_np, A, b, v1, v2, X, oprm, follow=follow, band=AMB)
    # the oracle's own labels may differ from the GPU's inside the band only
    np.testing.assert_array_equal(ed.cand_index, idx)
    np.testing.assert_array_equal(ed.bisect.decisions, follow)
    cst = bt.read(0, "c_star")[:, : idx.size].T
    assert np.abs(cst - ed.bisect.c_star).max(initial=0.0) < 1e-9
    res = bt.segment(0)
    m0 = A.shape[0]
    H = ed.place.rows_a.shape[0]
    assert res.A.shape[0] == m0 + H and st["n_placed"] == H
    np.testing.assert_array_equal(res.A[:m0], A)
    np.testing.assert_allclose(res.A[m0:], ed.place.rows_a, rtol=1e-6, atol=1e-12)
    np.testing.assert_allclose(res.b[m0:], ed.place.rows_b, rtol=1e-6, atol=1e-12)
    np.testing.assert_array_equal(bt.read(0, "placed_idx")[:H], ed.place.order)
    if ed.place.status == orc.STATUS_OK:
        assert st["status"] == st0["status"]
    else:
        assert st["status"] == ezo.SEG_IN_COLLISION
    return bt, st, ed, X, idx


def test_edit_matches_oracle_planar(ezo):
    rd = wl.planar3_robot()
    env_np = wl.Env("disks", np.array([[1.5, 0.0, 0.0, 0.1], [0.0, 1.6, 0.0, 0.15]]))
    A = np.vstack([np.eye(3), -np.eye(3)])
    b = np.full(6, 2.0)
    v1, v2 = np.array([-1.2, 0.3, -0.2]), np.array([-0.8, -0.3, 0.2])
    rng = np.random.default_rng(5)
    X = rng.uniform(-2.0, 2.0, size=(300, 3))
    X[::7, 1] = 2.4
    bt, st, ed, X, idx = _edit_replay(ezo, rd, env_np, v1, v2, A, b, X,
                                      dict(eps=0.1, delta=0.05, n_p=1000, n_f=40, n_b=12, n_mix=20, n_it_max=3,
                                           seed=4))
    assert idx.size >= 20 and ed.place.status == orc.STATUS_OK
    res = bt.segment(0)
    assert orc.segment_contained(res.A, res.b, v1, v2, tol=0.0)
    if ed.place.rows_a.shape[0] < 40:  # the face budget was not the limit: every collision in P is cut off
        assert (X[idx] @ res.A[6:].T > res.b[6:][None, :]).any(axis=1).all()


def test_edit_matches_oracle_dh7(ezo):
    """A polytope of the 7-DOF path inflated on the GPU, edited with the
    colliding configurations among 1800 points drawn inside it and 200
    uniform ones (mostly outside it)."""
    rd, env_np, path = dh7_scene()
    robot, env = ezo.Robot(rd), ezo.Env(env_np)
    prm_kw = dict(n_p=2000, n_f=30, n_b=10, n_mix=30, n_it_max=6, seed=3)
    bt = ezo.Batch(robot, [env], path[0], path[1], ezo.Params.make(**prm_kw))
    bt.run()
    P = bt.segment(0)
    inside = orc.hit_and_run(P.A, P.b, path[0], path[1], 1800, 30, 77, 0, 1)
    X = np.vstack([inside, wl.uniform_configs(8, rd, 200)])
    assert X.shape[0] <= bt.s_cap
    bt2, st, ed, X, idx = _edit_replay(ezo, rd, env_np, path[0], path[1], P.A, P.b, X, prm_kw)
    assert idx.size >= 1


def test_edit_errors(ezo):
    rd, env_np, path = dh7_scene()
    robot, env = ezo.Robot(rd), ezo.Env(env_np)
    bt = ezo.Batch(robot, [env], path[0], path[1], ezo.Params.make(n_p=500, n_it_max=2, n_mix=10))
    bt.step(0)
    bt.sync()
    with pytest.raises(RuntimeError):
        bt.edit(np.zeros((3, 7)))  # segment still active
    bt.reset()
    bt.run()
    with pytest.raises(RuntimeError):
        bt.edit(np.zeros((bt.s_cap + 1, 7)))
    with pytest.raises(RuntimeError):
        bt.set_polytope(0, np.zeros((bt.m_cap + 1, 7)), np.zeros(bt.m_cap + 1))


# ------------------------------------------------- coverage and re-inflation --
def test_coverage_and_reinflate_match_oracle(ezo):
    rd, env_np, path = dh7_scene()
    robot, env = ezo.Robot(rd), ezo.Env(env_np)
    K = path.shape[0] - 1
    prm = ezo.Params.make(n_p=2000, n_f=10, n_b=10, n_mix=30, n_it_max=20, seed=2)
    bt = ezo.Batch(robot, [env], path[:-1], path[1:], prm, seg_stream=np.arange(K, dtype=np.uint32),
                   path_first=np.zeros(K, np.int32))
    bt.run_path(sequential=False)

    def polys():
        out = []
        for g in range(K):
            r = bt.segment(g)
            if r.status in (ezo.SEG_ACCEPTED, ezo.SEG_MAX_ITER):
                out.append((r.A, r.b))
        return out

    cov = bt.coverage()
    np.testing.assert_array_equal(cov, orc.path_coverage(polys(), path))
    assert cov.all()
    # move the first kept polytope far away; the segments it alone covered
    # are no longer covered, and inflating them again (same Philox streams)
    # gives them back the same polytopes, bit for bit
    g0 = next(g for g in range(K) if bt.segment(g).status == ezo.SEG_ACCEPTED)
    orig = {g: bt.segment(g) for g in range(K)}
    A = np.vstack([np.eye(7), -np.eye(7)])
    b = np.concatenate([np.full(7, 10.0), np.full(7, -9.0)])  # 9 <= q_i <= 10
    bt.set_polytope(g0, A, b)
    cov = bt.coverage()
    np.testing.assert_array_equal(cov, orc.path_coverage(polys(), path))
    bt.reinflate(~cov)
    for g in range(K):
        r = bt.segment(g)
        if cov[g]:  # untouched
            assert r.status == orig[g].status
            if g != g0:
                np.testing.assert_array_equal(r.A, orig[g].A)
        else:
            assert r.status in (ezo.SEG_ACCEPTED, ezo.SEG_MAX_ITER)
            assert orc.segment_contained(r.A, r.b, path[g], path[g + 1])
            if orig[g].status != ezo.SEG_SKIPPED:
                np.testing.assert_array_equal(r.A, orig[g].A)
                np.testing.assert_array_equal(r.b, orig[g].b)
    cov2 = bt.coverage()
    np.testing.assert_array_equal(cov2, orc.path_coverage(polys(), path))
    assert cov2.all()


def test_recovery_loop_excludes_found_collisions(ezo):
    """Sec. VI-B end to end: a trajectory through the sets (points drawn in
    each polytope, joined in order) is checked at 0.1 rad; the colliding
    points that lie in a set are excluded from it by editing; the seed
    segments stay inside their sets and every segment stays covered."""
    rd, env_np, path = dh7_scene()
    robot, env = ezo.Robot(rd), ezo.Env(env_np)
    K = path.shape[0] - 1
    prm = ezo.Params.make(eps=0.2, delta=0.2, n_p=1000, n_f=40, n_b=10, n_mix=30, n_it_max=3, seed=5)
    bt = ezo.Batch(robot, [env], path[:-1], path[1:], prm, seg_stream=np.arange(K, dtype=np.uint32),
                   path_first=np.zeros(K, np.int32))
    bt.run_path(sequential=False)
    kept = [g for g in range(K) if bt.segment(g).status in (ezo.SEG_ACCEPTED, ezo.SEG_MAX_ITER)]
    traj = [path[0]]
    for g in kept:
        r = bt.segment(g)
        traj.extend(orc.hit_and_run(r.A, r.b, path[g], path[g + 1], 6, 30, 11, g, 1))
    traj.append(path[-1])
    traj = np.asarray(traj)
    _, tot = ezo.path_points(traj, 0.1)
    pf = torch.zeros(tot, dtype=torch.uint8, device="cuda")
    edge, npts = ezo.check_path(robot, env, traj, 0.1, pf)
    torch.cuda.synchronize()
    P, _ = orc.path_points(traj, 0.1)
    cols = P[pf.cpu().numpy().astype(bool)][: bt.s_cap]
    assert cols.shape[0] > 0
    before = {g: bt.segment(g) for g in kept}
    bt.edit(cols)
    cols32 = cols.astype(np.float32).astype(np.float64)
    for g in kept:
        r = bt.segment(g)
        assert orc.segment_contained(r.A, r.b, path[g], path[g + 1])
        st = bt.state(g)
        was_in = orc.points_inside(before[g].A, before[g].b, cols32)
        assert st["count"] <= int(was_in.sum())
        if st["n_placed"] < prm.n_f and st["status"] != ezo.SEG_IN_COLLISION:
            col_in = np.nonzero(was_in)[0]
            lab = bt.read(g, "labels")[: cols.shape[0]].astype(bool)
            cut = col_in[lab[col_in]][: prm.n_p]
            assert not orc.points_inside(r.A, r.b, cols32[cut]).any()
    cov = bt.coverage()
    if not cov.all():
        bt.reinflate(~cov)
    assert bt.coverage().all()
