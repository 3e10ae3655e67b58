"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the
same seeded inputs.

Tolerances (stated here, derived in the design notes):
* collision labels: bit-exact except where the oracle's signed distance is
  within AMB = 1e-5 m of zero (FP32 forward kinematics);
* signed distance: |GPU - oracle| <= 2e-5 m;
* round size, test count, accept bit, candidate indices: exact;
* bisection: same decisions except ambiguous midpoints (the oracle follows
  the GPU there), c* within 1e-9;
* hyperplanes: rows and offsets within 1e-6 relative, same placement order;
* hit-and-run: start points within FP32 rounding; walks within 1e-3 for at
  least 99% of samples; every sample inside P up to 1e-5 (1 + |b|).
"""
import functools
import json
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


def scenes():
    with open(os.path.join(GOLDEN, "workloads.json")) as f:
        return json.load(f)


def planar_scene():
    s = scenes()["planar3"]
    return wl.planar3_robot(), wl.Env("planar", np.asarray(s["obstacles"])), np.asarray(s["v1"]), np.asarray(s["v2"])


def dh7_scene():
    s = scenes()["dh7"]
    return wl.dh7_robot(), wl.box_obstacles(s["env_seed"], s["n_obs"]), np.asarray(s["path"])


def table_env():
    return wl.table_cloud_obstacles(31)


def to_dev(q):
    return torch.from_numpy(np.asarray(q, dtype=np.float32).T.copy()).cuda().contiguous()


def gpu_labels(ezo, robot, env, q, lanes=0):
    qd = to_dev(q)
    flags = torch.empty(q.shape[0], dtype=torch.uint8, device="cuda")
    ezo.check_collision(robot, env, qd, flags, lanes=lanes)
    torch.cuda.synchronize()
    return flags.cpu().numpy().astype(bool)


def assert_labels_match(rd, env_np, q32, got, band=AMB):
    q64 = q32.astype(np.float64)
    ref = orc.in_collision(rd, env_np, q64)
    diff = got != ref
    if diff.any():
        sd = orc.signed_distance(rd, env_np, q64[diff])
        assert np.all(np.abs(sd) < band), f"{int((np.abs(sd) >= band).sum())} labels differ outside the band"
    return ref


# ------------------------------------------------------- collision labels --
@pytest.mark.parametrize("lanes", [1, 2, 4, 8])
@pytest.mark.parametrize("which", ["planar", "dh7", "table"])
def test_check_collision_matches_oracle(ezo, which, lanes):
    if which == "planar":
        rd, env_np, _, _ = planar_scene()
    elif which == "dh7":
        rd, env_np, _ = dh7_scene()
    else:
        rd, env_np = wl.dh7_robot(), table_env()
    robot, env = ezo.Robot(rd), ezo.Env(env_np)
    N = 3001  # several blocks and a ragged tail
    q32 = wl.uniform_configs(17, rd, N).astype(np.float32)
    got = gpu_labels(ezo, robot, env, q32, lanes)
    ref = assert_labels_match(rd, env_np, q32, got)
    assert 0 < ref.sum() < N


@pytest.mark.parametrize("lanes", [1, 2, 8])
def test_base_spheres_skipped_only_when_clear(ezo, lanes):
    """The 7-DOF arm's first eight spheres sit on the fixed base frame; the
    obstacle sweep skips them only when every base sphere clears every
    obstacle by more than 1e-4 m (their pairs are the same for every
    configuration). With one obstacle added far away the sweep starts past
    8 spheres; with the obstacle overlapping a base sphere (every
    configuration collides) or 5e-5 m from one the full sweep runs. The
    algorithmic flop count is the same in all three sets. Labels match the
    oracle in all three sets. (The bisection's wide check takes the same start; the
    round replays on this scene compare its decisions with the oracle.)"""
    rd, env_np, _ = dh7_scene()
    base = np.flatnonzero(np.asarray(rd.sphere_frame) == 0)
    assert base.size >= 8
    c0 = np.asarray(rd.sphere_xyz)[base[0]]
    r0 = float(np.asarray(rd.sphere_r)[base[0]])
    R = 0.05
    extra = {"far": [3.0, 3.0, 3.0, R], "touch": [c0[0] + 0.5 * (r0 + R), c0[1], c0[2], R],
             "near": [c0[0] + r0 + R + 5e-5, c0[1], c0[2], R]}
    robot = ezo.Robot(rd)
    N = 3001
    q32 = wl.uniform_configs(19, rd, N).astype(np.float32)
    flops, static = {}, {}
    for name, ob in extra.items():
        envw = wl.Env(name, np.vstack([env_np.spheres, [ob]]))
        env = ezo.Env(envw)
        flops[name] = ezo.check_flops(robot, env)
        static[name] = ezo.check_static_spheres(robot, env)
        got = gpu_labels(ezo, robot, env, q32, lanes)
        ref = assert_labels_match(rd, envw, q32, got)
        if name == "touch":
            assert ref.all() and got.all()
    assert static == {"far": 8, "touch": 0, "near": 0}
    assert flops["far"] == flops["touch"] == flops["near"]


def near_boundary_configs(rd, env_np, seed, n_seg=120, steps=(9, 17)):
    """Configurations close to the collision boundary, where the FP32 fast form
    is inside its rounding band and the direct re-check decides: the midpoints
    of FP64 bisections between free and colliding uniform configurations
    (oracle labels), from bisection step steps[0] to steps[1] - 1, so the
    distances to tangency range from ~1e-3 m down to ~1e-6 m."""
    q = wl.uniform_configs(seed, rd, 20 * n_seg)
    lab = orc.in_collision(rd, env_np, q)
    free, col = q[~lab][:n_seg], q[lab][:n_seg]
    k = min(free.shape[0], col.shape[0])
    lo, hi = free[:k].copy(), col[:k].copy()
    out = []
    for s in range(steps[1]):
        mid = 0.5 * (lo + hi)
        c = orc.in_collision(rd, env_np, mid)
        if s >= steps[0]:
            out.append(mid)
        hi = np.where(c[:, None], mid, hi)
        lo = np.where(c[:, None], lo, mid)
    return np.concatenate(out).astype(np.float32)


@functools.lru_cache(maxsize=None)
def _near_boundary_case(which):
    if which == "planar":
        rd, env_np, _, _ = planar_scene()
    elif which == "dh7":
        rd, env_np, _ = dh7_scene()
    else:
        rd, env_np = wl.dh7_robot(), table_env()
    return rd, env_np, near_boundary_configs(rd, env_np, 23)


@pytest.mark.parametrize("lanes", [1, 2, 4, 8])
@pytest.mark.parametrize("which", ["planar", "dh7", "table"])
def test_check_collision_near_boundary(ezo, which, lanes):
    """Labels of configurations within ~1e-3 m of tangency (many of them
    inside the fast form's rounding band, where every lane re-checks its own
    obstacles with the difference form) against the oracle, at every lane
    count."""
    rd, env_np, q32 = _near_boundary_case(which)
    robot, env = ezo.Robot(rd), ezo.Env(env_np)
    got = gpu_labels(ezo, robot, env, q32, lanes)
    sd = orc.signed_distance(rd, env_np, q32.astype(np.float64))
    near = np.abs(sd) < 1e-4
    assert near.sum() > 100  # the case this test is for
    assert_labels_match(rd, env_np, q32, got)


def test_check_collision_full_batch_sampled(ezo):
    """The bench's batch size (2e6 configurations) in the bench's launch
    shape, checked on 3000 sampled configurations."""
    rd, env_np, _ = dh7_scene()
    robot, env = ezo.Robot(rd), ezo.Env(env_np)
    N = 2_000_000
    g = torch.Generator(device="cuda").manual_seed(3)
    lo = torch.tensor(rd.q_lo, dtype=torch.float32, device="cuda")[:, None]
    hi = torch.tensor(rd.q_hi, dtype=torch.float32, device="cuda")[:, None]
    q = lo + (hi - lo) * torch.rand((rd.n, N), generator=g, device="cuda")
    flags = torch.empty(N, dtype=torch.uint8, device="cuda")
    ezo.check_collision(robot, env, q, flags)
    torch.cuda.synchronize()
    idx = np.random.default_rng(0).choice(N, 3000, replace=False)
    idx[:3] = [0, N - 1, N // 2]
    q32 = q[:, idx].T.cpu().numpy()
    got = flags[idx].cpu().numpy().astype(bool)
    assert_labels_match(rd, env_np, q32, got)


def test_check_collision_edge_cases(ezo):
    rd, env_np, _ = dh7_scene()
    robot = ezo.Robot(rd)
    empty = ezo.Env(np.zeros((0, 4)))
    q32 = wl.uniform_configs(4, rd, 500).astype(np.float32)
    got = gpu_labels(ezo, robot, empty, q32)
    assert_labels_match(rd, wl.Env("none", np.zeros((0, 4))), q32, got)
    # N = 0 is a no-op
    flags = torch.zeros(1, dtype=torch.uint8, device="cuda")
    ezo.check_collision(robot, empty, torch.zeros((7, 0), device="cuda"), flags)
    # touching cases at home pose: +-2e-5 m around tangency
    c = orc.sphere_centres(rd, np.zeros((1, 7)))[0]
    for gap, expect in [(2e-5, False), (-2e-5, True)]:
        o = np.array([[c[20, 0] + rd.sphere_r[20] + 0.05 + gap, c[20, 1], c[20, 2], 0.05]])
        assert gpu_labels(ezo, robot, ezo.Env(o), np.zeros((1, 7), dtype=np.float32))[0] == expect
    # a wrong lanes value is rejected
    with pytest.raises(ezo.EzoError):
        ezo.check_collision(robot, empty, to_dev(q32), torch.empty(500, dtype=torch.uint8, device="cuda"), lanes=3)


def test_signed_distance_matches_oracle(ezo):
    rd, env_np, _ = dh7_scene()
    robot, env = ezo.Robot(rd), ezo.Env(env_np)
    q32 = wl.uniform_configs(21, rd, 2000).astype(np.float32)
    sd = torch.empty(2000, device="cuda")
    ezo.signed_distance(robot, env, to_dev(q32), sd)
    torch.cuda.synchronize()
    ref = orc.signed_distance(rd, env_np, q32.astype(np.float64))
    assert np.abs(sd.cpu().numpy() - ref).max() <= 2e-5


# --------------------------------------------------------------- sampling --
def _gpu_hnr(ezo, A, b, v1, v2, N, n_mix, seed, stream, k):
    Ad = torch.from_numpy(np.ascontiguousarray(A)).cuda()
    bd = torch.from_numpy(np.ascontiguousarray(b)).cuda()
    out = torch.empty((A.shape[1], N), dtype=torch.float32, device="cuda")
    ezo.hit_and_run(Ad, bd, v1, v2, N, n_mix, seed, stream, k, out)
    torch.cuda.synchronize()
    return out.cpu().numpy().T.astype(np.float64)


def test_hit_and_run_start_points_pin_philox(ezo):
    rd = wl.dh7_robot()
    A, b = orc.joint_box(rd)
    v1, v2 = np.full(7, -0.5), np.full(7, 0.8)
    x = _gpu_hnr(ezo, A, b, v1, v2, 4099, 0, seed=77, stream=5, k=3)
    ref = orc.hit_and_run(A, b, v1, v2, 4099, 0, seed=77, stream=5, k=3)
    assert np.abs(x - ref).max() < 1e-6


@pytest.mark.parametrize("which", ["box", "polytope"])
def test_hit_and_run_matches_oracle_walks(ezo, which):
    rd = wl.dh7_robot()
    A, b = orc.joint_box(rd)
    v1, v2 = np.full(7, -0.5), np.full(7, 0.8)
    if which == "polytope":
        rng = np.random.default_rng(1)
        G = rng.standard_normal((30, 7))
        G /= np.linalg.norm(G, axis=1, keepdims=True)
        h = np.maximum(G @ v1, G @ v2) + rng.uniform(0.05, 1.0, 30)
        A, b = np.vstack([A, G]), np.concatenate([b, h])
    N = 3000
    x = _gpu_hnr(ezo, A, b, v1, v2, N, 40, seed=9, stream=2, k=1)
    ref = orc.hit_and_run(A, b, v1, v2, N, 40, seed=9, stream=2, k=1)
    err = np.abs(x - ref).max(axis=1)
    assert np.quantile(err, 0.99) < 1e-3, np.quantile(err, [0.5, 0.9, 0.99])
    assert np.median(err) < 1e-4
    assert np.all(x @ A.T <= b + 1e-5 * (1 + np.abs(b)))


@pytest.mark.parametrize("lanes", [0, 1, 2, 4, 8])
def test_round_walks_equal_flat_walks(ezo, lanes):
    """The round sampler gives the flat sampler's samples bit for bit for
    every number of lanes per walk (same Philox draws, same per-row
    arithmetic), in round 1 (the joint box) and in round 2, whose polytope
    carries the planes placed in round 1."""
    rd, env_np, path = dh7_scene()
    robot, env = ezo.Robot(rd), ezo.Env(env_np)
    prm = ezo.Params.make(n_p=3000, seed=13)
    bt = ezo.Batch(robot, [env], path[2], path[3], prm, seg_stream=[7])
    bt.set_sample_lanes(lanes)
    seen_planes = False
    for k in (1, 2):
        bt.step(0)
        bt.step(1)
        bt.sync()
        st = bt.state(0)
        if st["k"] != k:
            break  # accepted in round 1
        seg = bt.segment(0)
        seen_planes |= seg.A.shape[0] > 14
        S = bt.read(0, "samples")[:, : st["n_samples"]].T.astype(np.float64)
        x = _gpu_hnr(ezo, seg.A, seg.b, path[2], path[3], st["n_samples"], prm.n_mix, 13, 7, k)
        np.testing.assert_array_equal(S, x)
        for step in range(2, 7):
            bt.step(step)
        bt.sync()
    assert seen_planes
    with pytest.raises(RuntimeError):
        bt.set_sample_lanes(3)


# ----------------------------------------------------- round-by-round replay --
def _replay_rounds(ezo, rd, env_np, v1, v2, prm_kw, max_rounds=6, band=AMB):
    robot, env = ezo.Robot(rd), ezo.Env(env_np)
    prm = ezo.Params.make(**prm_kw)
    oprm = orc.Params(eps=prm.eps, delta=prm.delta, tau=prm.tau, step_back_max=prm.step_back_max,
                      t_col=prm.t_col, n_p=prm.n_p, n_f=prm.n_f, n_b=prm.n_b, n_mix=prm.n_mix,
                      n_it_max=prm.n_it_max, seed=prm.seed)
    bt = ezo.Batch(robot, [env], v1, v2, prm)
    A, b = orc.joint_box(rd)
    rounds = 0
    total_amb = 0
    for k in range(1, max_rounds + 1):
        for step in range(3):
            bt.step(step)
        bt.sync()
        st = bt.state(0)
        assert st["k"] == k
        assert st["m_test"] == orc.test_size(k, oprm.eps, oprm.delta, oprm.tau)
        assert st["n_samples"] == orc.batch_size(k, oprm.eps, oprm.delta, oprm.tau, oprm.n_p)
        S = bt.read(0, "samples")[:, : st["n_samples"]].T.astype(np.float64)
        assert np.all(S @ A.T <= b + 1e-5 * (1 + np.abs(b)))
        # the round's walks (several lanes per walk here) follow the FP64 walks
        ref = orc.hit_and_run(A, b, v1, v2, 600, oprm.n_mix, oprm.seed, 0, k)
        err = np.abs(S[:600] - ref).max(axis=1)
        assert np.quantile(err, 0.99) < 1e-3 and np.median(err) < 1e-4, np.quantile(err, [0.5, 0.99])
        lab = bt.read(0, "labels")[: st["n_samples"]].astype(bool)
        assert_labels_match(rd, env_np, S.astype(np.float32), lab, band)
        bt.step(3)
        bt.sync()
        st = bt.state(0)
        M = st["m_test"]
        count = int(lab[:M].sum())
        assert st["count"] == count
        accept = orc.unadaptive_test(count, M, oprm.eps, oprm.tau)
        assert (st["status"] == ezo.SEG_ACCEPTED) == accept
        rounds = k
        if accept:
            break
        idx = np.nonzero(lab)[0][: oprm.n_p]
        assert st["n_cand"] == idx.size
        np.testing.assert_array_equal(bt.read(0, "cand_idx")[: idx.size], idx)
        bt.step(4)
        bt.sync()
        nc = idx.size
        bits = bt.read(0, "bits")[:nc]
        follow = ((bits[:, None] >> np.arange(oprm.n_b)[None, :]) & 1).astype(bool)
        br = orc.bisect(rd, env_np, S[idx], v1, v2, oprm.n_b, follow=follow, band=band)
        total_amb += br.ambiguous
        np.testing.assert_array_equal(br.decisions, follow)
        cst = bt.read(0, "c_star")[:, :nc].T
        assert np.abs(cst - br.c_star).max() < 1e-9
        dist = bt.read(0, "dist")[:nc]
        np.testing.assert_allclose(dist, orc.dist_to_segment(br.c_star, v1, v2), rtol=1e-12, atol=1e-14)
        m_before = st["m"]
        bt.step(5)
        bt.sync()
        st = bt.state(0)
        pl = orc.place_hyperplanes(cst, idx, v1, v2, oprm.n_f, oprm.step_back_max, oprm.t_col)
        H = st["m"] - m_before
        assert H == pl.rows_a.shape[0] == st["n_placed"]
        res = bt.segment(0)
        np.testing.assert_allclose(res.A[m_before:], pl.rows_a, rtol=1e-6, atol=1e-12)
        np.testing.assert_allclose(res.b[m_before:], pl.rows_b, rtol=1e-6, atol=1e-12)
        np.testing.assert_array_equal(bt.read(0, "placed_idx")[:H], pl.order)
        np.testing.assert_allclose(bt.read(0, "placed_delta")[:H], pl.deltas, rtol=1e-9)
        assert orc.segment_contained(res.A, res.b, v1, v2, tol=1e-12)
        A, b = res.A, res.b
        bt.step(6)
        bt.sync()
    return rounds, total_amb


def test_round_replay_planar(ezo):
    rd, env_np, v1, v2 = planar_scene()
    rounds, _ = _replay_rounds(ezo, rd, env_np, v1, v2,
                               dict(eps=0.1, delta=0.05, n_p=1000, n_f=10, n_b=10, n_mix=30, seed=1))
    assert rounds >= 2


def test_round_replay_dh7(ezo):
    rd, env_np, path = dh7_scene()
    rounds, _ = _replay_rounds(ezo, rd, env_np, path[0], path[1],
                               dict(eps=0.05, delta=0.05, n_p=2000, n_f=10, n_b=10, n_mix=60, seed=1), max_rounds=4)
    assert rounds >= 2


# ------------------------------------------ longer chains (16-joint kernels) --
def chain10_robot():
    return wl.chain_robot(10)


CHAIN10_V1 = np.array([0.8861, 0.0227, 0.9525, -0.8383, 0.2147, -0.247, 0.6038, -0.6509, 0.7433, 0.0879])
CHAIN10_V2 = np.array([1.1274, 0.0089, 0.9108, -0.665, 0.5052, -0.3252, 0.8852, -0.3935, 0.5499, 0.1532])


@pytest.mark.parametrize("lanes", [1, 2, 8])
def test_chain10_labels_match_oracle(ezo, lanes):
    rd, env_np = chain10_robot(), wl.box_obstacles(5, 32)
    q32 = wl.uniform_configs(17, rd, 3001).astype(np.float32)
    got = gpu_labels(ezo, ezo.Robot(rd), ezo.Env(env_np), q32, lanes)
    ref = assert_labels_match(rd, env_np, q32, got)
    assert 0 < ref.sum() < q32.shape[0]


def test_maximum_sizes_labels_match_oracle(ezo):
    """The largest robot and obstacle set the library takes: 16 joints, 256
    robot spheres (16 per link, 23,296 self pairs) and 4,096 obstacle
    spheres. Each group of lanes keeps its sphere centres in shared memory,
    so only 4 and 8 lanes per configuration fit; those (and the automatic
    choice) match the oracle, while 1 and 2 lanes and the one-lane signed
    distance are refused on the host with nothing launched, and the next
    CUDA work runs normally."""
    rd = wl.chain_robot(16, r=0.02, per_link=16)
    env_np = wl.box_obstacles(41, 4096, box_lo=(-2.5, -2.5, -2.5), box_hi=(2.5, 2.5, 2.5), r_lo=0.02, r_hi=0.05)
    assert rd.sphere_r.shape[0] == 256 and rd.self_pairs.shape[0] == 23296
    robot, env = ezo.Robot(rd), ezo.Env(env_np)
    q32 = wl.uniform_configs(23, rd, 96).astype(np.float32)
    q64 = q32.astype(np.float64)
    ref = orc.in_collision(rd, env_np, q64, chunk=4)  # 4 x 256 x 4096 pairs per chunk
    assert 0 < ref.sum() < ref.size
    sd = orc.signed_distance(rd, env_np, q64, chunk=4)
    for lanes in (4, 8, 0):
        got = gpu_labels(ezo, robot, env, q32, lanes)
        diff = got != ref
        assert np.all(np.abs(sd[diff]) < AMB), f"lanes {lanes}: {int(diff.sum())} labels differ outside the band"
    for lanes in (1, 2):
        with pytest.raises(ezo.EzoError):
            gpu_labels(ezo, robot, env, q32, lanes)
    with pytest.raises(ezo.EzoError):
        ezo.signed_distance(robot, env, to_dev(q32), torch.empty(96, device="cuda"))
    x = torch.full((1024,), 2.0, device="cuda")
    assert float(x.sum()) == 2048.0


# a collision-free seed segment of the maximum-size scene (oracle clearance
# above 0.05 m at 41 points along it)
MAX_V1 = np.array([-1.4826, -1.746, -2.3949, 2.4696, 1.6865, 1.8756, -1.3964, -2.1476, 2.3273, 1.6844, 1.2096,
                   0.2345, 0.7711, 1.3283, 0.1993, 1.0377])
MAX_V2 = np.array([-1.5623, -1.8776, -2.4, 2.4, 1.7994, 1.8865, -1.4513, -2.2256, 2.4, 1.8468, 1.2367, 0.112,
                   0.6759, 1.4873, 0.2195, 0.8656])


def test_maximum_sizes_segment_inflation(ezo):
    """Algorithm 1 on the maximum-size scene (16 joints, 256 robot spheres,
    4,096 obstacles): the batch raises its label and bisection lanes to the
    fewest whose sphere centres fit in shared memory and refuses a shape
    below them; the polytope contains the segment, the last round's sample
    labels match the oracle outside the band, and 8 lanes give the same
    polytope bit for bit."""
    rd = wl.chain_robot(16, r=0.02, per_link=16)
    env_np = wl.box_obstacles(41, 4096, box_lo=(-2.5, -2.5, -2.5), box_hi=(2.5, 2.5, 2.5), r_lo=0.02, r_hi=0.05)
    line = MAX_V1[None, :] + np.linspace(0, 1, 41)[:, None] * (MAX_V2 - MAX_V1)[None, :]
    assert orc.signed_distance(rd, env_np, line, chunk=4).min() > 0.05
    robot, env = ezo.Robot(rd), ezo.Env(env_np)
    prm = ezo.Params.make(eps=0.1, delta=0.05, n_p=1000, n_f=10, n_b=10, n_mix=30, seed=2)
    bt = ezo.Batch(robot, [env], MAX_V1, MAX_V2, prm)
    sh = bt.shape()
    assert sh["check_lanes"] >= 4 and sh["bisect_lanes"] >= 4
    with pytest.raises(ezo.EzoError):
        bt.set_shape(sh["sample_fill_tiles"], 2, sh["bisect_lanes"])
    bt.run()
    ref = bt.segment(0)
    assert ref.status in (ezo.SEG_ACCEPTED, ezo.SEG_MAX_ITER)
    assert orc.segment_contained(ref.A, ref.b, MAX_V1, MAX_V2, tol=1e-12)
    S = bt.read(0, "samples")[:, :48].T.astype(np.float64)
    lab = bt.read(0, "labels")[:48].astype(bool)
    want = orc.in_collision(rd, env_np, S, chunk=4)
    diff = lab != want
    if diff.any():
        assert np.all(np.abs(orc.signed_distance(rd, env_np, S[diff], chunk=4)) < AMB)
    bt.set_shape(sh["sample_fill_tiles"], 8, 8)
    bt.reset()
    bt.run()
    got = bt.segment(0)
    assert (got.status, got.rounds, got.checks) == (ref.status, ref.rounds, ref.checks)
    np.testing.assert_array_equal(got.A, ref.A)
    np.testing.assert_array_equal(got.b, ref.b)


def test_round_replay_chain10(ezo):
    """Rounds of a 10-joint chain replayed step by step against the oracle
    (walks, labels, test, candidates, bisection, planes)."""
    rd, env_np = chain10_robot(), wl.box_obstacles(5, 32)
    assert orc.signed_distance(rd, env_np, CHAIN10_V1[None, :] + np.linspace(0, 1, 200)[:, None]
                               * (CHAIN10_V2 - CHAIN10_V1)[None, :]).min() > 0.1
    rounds, _ = _replay_rounds(ezo, rd, env_np, CHAIN10_V1, CHAIN10_V2,
                               dict(eps=0.1, delta=0.05, n_p=1000, n_f=10, n_b=10, n_mix=30, seed=3), max_rounds=3)
    assert rounds >= 2


# ------------------------------------------------------- Forest (Sec. V) --
FOREST_PRM = dict(eps=0.01, delta=0.05, n_p=1000, n_f=10, n_b=10, n_mix=30, step_back_max=0.01)


def forest_scene():
    s = scenes()["forest"]
    return wl.point2_robot(), wl.forest_obstacles(s["forest_seed"]), np.asarray(s["path"])


@pytest.mark.parametrize("lanes", [1, 2, 8])
def test_forest_labels_match_oracle(ezo, lanes):
    """Point robot (two prismatic joints) among 15 disks: labels exact
    except within 1e-5 of a disk boundary."""
    rd, env_np, _ = forest_scene()
    q = wl.uniform_configs(21, rd, 200000)
    got = gpu_labels(ezo, ezo.Robot(rd), ezo.Env(env_np), q, lanes=lanes)
    ref = assert_labels_match(rd, env_np, q.astype(np.float32), got)
    assert 0.05 < ref.mean() < 0.3


def test_prismatic_chain_signed_distance_matches_oracle(ezo):
    """A 4-joint chain with two prismatic joints and offsets: the GPU's
    forward kinematics, through the signed distance, against the oracle."""
    base = wl.dh7_robot()
    rd = wl.Robot(name="mixed", a=np.array([0.1, 0.0, 0.3, 0.05]), alpha=np.array([0.4, -1.2, 0.0, 0.7]),
                  d=np.array([0.2, 0.1, 0.0, 0.3]), theta_off=np.array([0.3, -0.5, 0.1, 0.0]),
                  q_lo=np.array([-2.0, 0.0, -2.0, -0.5]), q_hi=np.array([2.0, 1.0, 2.0, 0.5]),
                  sphere_frame=np.array([1, 2, 2, 3, 4, 4], dtype=np.int32),
                  sphere_xyz=np.array([[0, 0, 0.1], [0.1, 0, 0], [0, 0.1, 0], [0, 0, 0], [0.05, 0, 0], [0, 0, 0.05]]),
                  sphere_r=np.full(6, 0.05), sphere_link=np.array([1, 2, 2, 3, 4, 4], dtype=np.int32),
                  self_pairs=np.array([[0, 4], [0, 5]], dtype=np.int32),
                  joint_type=np.array([0, 1, 0, 1], dtype=np.int32))
    env_np = wl.box_obstacles(4, 64, box_lo=(-0.6, -0.6, -0.2), box_hi=(0.6, 0.6, 1.0))
    robot, env = ezo.Robot(rd), ezo.Env(env_np)
    q = wl.uniform_configs(22, rd, 20000)
    sd = torch.empty(q.shape[0], device="cuda")
    ezo.signed_distance(robot, env, to_dev(q), sd)
    torch.cuda.synchronize()
    ref = orc.signed_distance(rd, env_np, q.astype(np.float32).astype(np.float64))
    assert np.abs(sd.cpu().numpy() - ref).max() <= 2e-5
    got = gpu_labels(ezo, robot, env, q)
    lab = assert_labels_match(rd, env_np, q.astype(np.float32), got)
    assert 0.05 < lab.mean() < 0.95


def test_round_replay_forest(ezo):
    rd, env_np, path = forest_scene()
    k = int(np.argmax(np.linalg.norm(np.diff(path, axis=0), axis=1)))
    rounds, _ = _replay_rounds(ezo, rd, env_np, path[k], path[k + 1], dict(FOREST_PRM, seed=3), max_rounds=5)
    assert rounds >= 1


def test_forest_path_polytopes_contain_segments_and_certify(ezo):
    """The whole Forest seed path with the paper's Forest parameters: every
    kept polytope is accepted, holds its segment, and an independent uniform
    sample of it collides at a rate within eps (binomial 4-sigma margin)."""
    rd, env_np, path = forest_scene()
    robot, env = ezo.Robot(rd), ezo.Env(env_np)
    K = path.shape[0] - 1
    bt = ezo.Batch(robot, [env], path[:-1], path[1:], ezo.Params.make(**dict(FOREST_PRM, seed=7)),
                   seg_stream=np.arange(K, dtype=np.uint32), path_first=np.zeros(K, np.int32))
    bt.run_path(sequential=False, mode=ezo.RUN_GRAPH)
    rng = np.random.default_rng(8)
    kept = 0
    for g in range(K):
        r = bt.segment(g)
        if r.status == ezo.SEG_SKIPPED:
            continue
        kept += 1
        assert r.status == ezo.SEG_ACCEPTED
        assert orc.segment_contained(r.A, r.b, path[g], path[g + 1], tol=1e-12)
        x = rng.uniform(rd.q_lo, rd.q_hi, size=(200000, 2))
        x = x[np.all(x @ r.A.T <= r.b, axis=1)][:20000]
        rate = orc.in_collision(rd, env_np, x).mean()
        assert rate <= FOREST_PRM["eps"] + 4 * np.sqrt(FOREST_PRM["eps"] / x.shape[0])
    assert bt.coverage().all() and kept >= 1


# ---------------------------------------------------- box geometries (IV-D) --
# Box pairs are decided in FP32 by a separating-axis test whose cross-product
# axes are not normalised; the label band for scenes with boxes is 5e-5 m on
# the oracle's FP64 value (its error bound for the largest skipped-axis angle).
AMB_BOX = 5e-5


def box_scene():
    s = scenes()["boxes"]
    return wl.box_arm_robot(), wl.tabletop_box_env(s["env_seed"]), np.asarray(s["path"])


@pytest.mark.parametrize("lanes", [1, 2, 4, 8])
def test_box_arm_labels_match_oracle(ezo, lanes):
    """11-box arm (26 box-box self pairs) over a table box, two rotated boxes
    and voxel spheres: every pair type with a box, against the FP64 oracle."""
    rd, env_np, _ = box_scene()
    q = wl.uniform_configs(31, rd, 20000)
    got = gpu_labels(ezo, ezo.Robot(rd), ezo.Env(env_np), q, lanes=lanes)
    ref = assert_labels_match(rd, env_np, q.astype(np.float32), got, AMB_BOX)
    assert 0.2 < ref.mean() < 0.9


def test_sphere_arm_with_boxes_and_self_box_pairs(ezo):
    """The 40-sphere arm with the 11 boxes added, sphere-box self pairs
    between the first link's spheres and the boxes of frames >= 4, over the
    table-top scene: sphere x box, box x sphere, box x box, both self kinds."""
    base, env_np, _ = box_scene()
    sph = wl.dh7_robot()
    link1 = np.nonzero(sph.sphere_link == sph.sphere_link.min())[0]
    far = np.nonzero(base.box_frame >= 4)[0]
    sb = np.array([(i, k) for i in link1 for k in far], dtype=np.int32)
    rd = wl.Robot(name="mixed_boxes", a=sph.a, alpha=sph.alpha, d=sph.d, theta_off=sph.theta_off, q_lo=sph.q_lo,
                  q_hi=sph.q_hi, sphere_frame=sph.sphere_frame, sphere_xyz=sph.sphere_xyz, sphere_r=sph.sphere_r,
                  sphere_link=sph.sphere_link, self_pairs=sph.self_pairs, box_frame=base.box_frame,
                  box_xyz=base.box_xyz, box_rot=base.box_rot, box_half=base.box_half, self_sb=sb,
                  self_bb=base.self_bb)
    q = wl.uniform_configs(32, rd, 20000)
    got = gpu_labels(ezo, ezo.Robot(rd), ezo.Env(env_np), q)
    ref = assert_labels_match(rd, env_np, q.astype(np.float32), got, AMB_BOX)
    assert 0.2 < ref.mean() < 0.95
    # sphere geometries only: the signed distance refuses boxes
    sd = torch.empty(16, device="cuda")
    with pytest.raises(RuntimeError):
        ezo.signed_distance(ezo.Robot(rd), ezo.Env(env_np), to_dev(q[:16]), sd)


def test_round_replay_boxes(ezo):
    rd, env_np, path = box_scene()
    rounds, _ = _replay_rounds(ezo, rd, env_np, path[0], path[1],
                               dict(eps=0.1, delta=0.05, n_p=1000, n_f=10, n_b=10, n_mix=30, seed=2),
                               max_rounds=3, band=AMB_BOX)
    assert rounds >= 1


def test_box_path_polytopes_contain_segments(ezo):
    rd, env_np, path = box_scene()
    robot, env = ezo.Robot(rd), ezo.Env(env_np)
    K = path.shape[0] - 1
    bt = ezo.Batch(robot, [env], path[:-1], path[1:],
                   ezo.Params.make(eps=0.1, delta=0.05, n_p=2000, n_f=10, n_b=10, n_mix=30, n_it_max=20, seed=3),
                   seg_stream=np.arange(K, dtype=np.uint32), path_first=np.zeros(K, np.int32))
    bt.run_path(sequential=False, mode=ezo.RUN_GRAPH)
    for g in range(K):
        r = bt.segment(g)
        if r.status != ezo.SEG_SKIPPED:
            assert r.status in (ezo.SEG_ACCEPTED, ezo.SEG_MAX_ITER)
            assert orc.segment_contained(r.A, r.b, path[g], path[g + 1], tol=1e-12)
    assert bt.coverage().all()


# ------------------------------------------------------------- end to end --
def test_inflate_segment_certified_planar(ezo):
    rd, env_np, v1, v2 = planar_scene()
    robot, env = ezo.Robot(rd), ezo.Env(env_np)
    prm = ezo.Params.make(eps=0.1, delta=0.05, n_p=1000, n_f=10, n_b=10, n_mix=30, seed=4)
    res = ezo.inflate_segment(robot, env, v1, v2, prm)
    assert res.status == ezo.SEG_ACCEPTED and res.planes > 0
    assert orc.segment_contained(res.A, res.b, v1, v2, tol=1e-12)
    rng = np.random.default_rng(2)
    x = rng.uniform(rd.q_lo, rd.q_hi, size=(400000, 3))
    x = x[np.all(x @ res.A.T <= res.b, axis=1)][:20000]
    assert orc.in_collision(rd, env_np, x).mean() <= prm.eps


def test_graph_mode_equals_host_loop(ezo):
    rd, env_np, path = dh7_scene()
    robot, env = ezo.Robot(rd), ezo.Env(env_np)
    prm = ezo.Params.make(n_p=3000, seed=5)
    outs = []
    for mode in (ezo.RUN_HOST_LOOP, ezo.RUN_GRAPH):
        bt = ezo.Batch(robot, [env], path[:-1], path[1:], prm)
        bt.run(mode)
        outs.append([bt.segment(g) for g in range(bt.B)])
    for a, b in zip(*outs):
        assert (a.status, a.rounds, a.m, a.checks) == (b.status, b.rounds, b.m, b.checks)
        np.testing.assert_array_equal(a.A, b.A)
        np.testing.assert_array_equal(a.b, b.b)


def test_batched_segments_equal_single_segments(ezo):
    """Per-segment Philox streams make a segment's result independent of the
    batch it runs in."""
    rd, env_np, path = dh7_scene()
    robot, env = ezo.Robot(rd), ezo.Env(env_np)
    prm = ezo.Params.make(n_p=2000, seed=6)
    bt = ezo.Batch(robot, [env], path[:4], path[1:5], prm)
    bt.run()
    for g in range(4):
        one = ezo.inflate_segment(robot, env, path[g], path[g + 1], prm, stream_id=g)
        many = bt.segment(g)
        np.testing.assert_array_equal(one.A, many.A)
        assert one.rounds == many.rounds


def test_iteration_cap_capacity_and_invalid_parameters(ezo):
    """Sec. IV-C "Maximum iterations": with N_it = 1 a segment that the first
    round does not certify ends EZO_SEG_MAX_ITER with the round's planes, as
    in the oracle; a polytope without room for N_f more rows ends
    EZO_SEG_CAPACITY; parameters outside their ranges are refused."""
    rd, env_np, path = dh7_scene()
    robot, env = ezo.Robot(rd), ezo.Env(env_np)
    kw = dict(n_p=2000, n_f=10, n_b=10, n_mix=30, n_it_max=1, seed=5)
    bt = ezo.Batch(robot, [env], path[0], path[1], ezo.Params.make(**kw))
    bt.run()
    r = bt.segment(0)
    oprm = orc.Params(**{k: v for k, v in kw.items()})
    A0, b0 = orc.joint_box(rd)
    S = bt.read(0, "samples")[:, : bt.state(0)["n_samples"]].T.astype(np.float64)
    rr = orc.eizo_round(rd, env_np, A0, b0, path[0], path[1], 1, oprm, S)
    assert not rr.accept
    assert r.status == ezo.SEG_MAX_ITER and r.rounds == 1
    assert r.A.shape[0] == 14 + rr.place.rows_a.shape[0]
    assert orc.segment_contained(r.A, r.b, path[0], path[1], tol=1e-12)
    # no room for another plane: the edit stops with EZO_SEG_CAPACITY
    full = np.vstack([r.A] * 64)[: bt.m_cap]
    bfull = np.concatenate([r.b] * 64)[: bt.m_cap]
    bt.set_polytope(0, full, bfull)
    inside = orc.hit_and_run(full, bfull, path[0], path[1], 1500, 30, 9, 0, 1)
    bt.edit(inside)
    st = bt.state(0)
    if st["count"] > 0:
        assert st["status"] == ezo.SEG_CAPACITY and st["n_placed"] == 0
    # parameters out of range
    for bad in (dict(eps=0.0), dict(eps=1.0), dict(delta=-0.1), dict(n_p=0), dict(n_b=33), dict(n_f=0),
                dict(n_it_max=0), dict(n_f=100, n_it_max=30)):
        with pytest.raises(RuntimeError):
            ezo.Batch(robot, [env], path[0], path[1], ezo.Params.make(**dict(kw, **bad)))


def test_bulk_polytope_read_equals_per_segment_reads(ezo):
    rd, env_np, path = dh7_scene()
    robot, env = ezo.Robot(rd), ezo.Env(env_np)
    K = path.shape[0] - 1
    bt = ezo.Batch(robot, [env], path[:-1], path[1:], ezo.Params.make(n_p=2000, n_mix=30, seed=4),
                   seg_stream=np.arange(K, dtype=np.uint32), path_first=np.zeros(K, np.int32))
    bt.run_path(sequential=False, mode=ezo.RUN_GRAPH)
    st, As, bs = bt.polytopes()
    for g in range(K):
        r = bt.segment(g)
        assert st[g] == r.status
        np.testing.assert_array_equal(As[g], r.A)
        np.testing.assert_array_equal(bs[g], r.b)


def test_inflate_path_sequential_equals_speculative(ezo):
    rd, env_np, path = dh7_scene()
    robot, env = ezo.Robot(rd), ezo.Env(env_np)
    prm = ezo.Params.make(n_p=3000, seed=7)
    seq = ezo.inflate_path(robot, env, path, prm, sequential=True)
    spec = ezo.inflate_path(robot, env, path, prm, sequential=False)
    wave = ezo.inflate_path(robot, env, path, prm, sequential=2)
    assert [k for k, _ in seq] == [k for k, _ in spec] == [k for k, _ in wave]
    for (_, a), (_, b), (_, c) in zip(seq, spec, wave):
        np.testing.assert_array_equal(a.A, b.A)
        np.testing.assert_array_equal(a.A, c.A)
    K = path.shape[0] - 1
    for k in range(K):
        assert any(orc.segment_contained(r.A, r.b, path[k], path[k + 1]) for _, r in seq)
    for k, r in seq:
        assert r.status == ezo.SEG_ACCEPTED
        assert orc.segment_contained(r.A, r.b, path[k], path[k + 1], tol=1e-12)


@pytest.mark.parametrize("pieces", [20, 40])
def test_device_skip_rule_on_long_paths(ezo, pieces):
    """The skip rule after a speculative run runs on the device, one warp per
    path, with a sequential fallback for paths of more than 32 segments: a
    collision-free planar segment cut into 20 and into 40 pieces (most of
    them inside an earlier polytope) keeps, skips and inflates the same
    segments, with the same polytopes, as the paper's one-at-a-time order."""
    rd, env_np, v1, v2 = planar_scene()
    robot, env = ezo.Robot(rd), ezo.Env(env_np)
    t = np.linspace(0.0, 1.0, pieces + 1)[:, None]
    path = (1.0 - t) * v1[None, :] + t * v2[None, :]
    prm = ezo.Params.make(n_p=500, seed=23)
    res = {}
    for seq in (True, False):
        bt = ezo.Batch(robot, [env], path[:-1], path[1:], prm, path_first=np.zeros(pieces, np.int32))
        bt.run_path(sequential=seq, mode=ezo.RUN_HOST_LOOP if seq else ezo.RUN_GRAPH)
        res[seq] = [bt.segment(g) for g in range(pieces)]
    assert [r.status for r in res[True]] == [r.status for r in res[False]]
    assert sum(r.status == ezo.SEG_SKIPPED for r in res[False]) >= pieces // 2
    for a, b in zip(res[True], res[False]):
        if a.status != ezo.SEG_SKIPPED:
            np.testing.assert_array_equal(a.A, b.A)
            np.testing.assert_array_equal(a.b, b.b)


def test_inflate_path_matches_oracle_skip_rule(ezo):
    """Sec. VI-A on a planar path whose second half lies inside the first
    polytope and whose third segment leaves it: every segment is inflated
    speculatively, the oracle applies the skip rule (both endpoints inside an
    earlier kept polytope, 1e-9) to the GPU's polytopes in path order, and
    the segments the library keeps, in the speculative and in the
    sequential mode, are the ones the oracle keeps."""
    rd, env_np, v1, v2 = planar_scene()
    robot, env = ezo.Robot(rd), ezo.Env(env_np)
    v3 = v2 + np.array([0.0, 0.0, 0.6])
    assert orc.signed_distance(rd, env_np, v2[None, :] + np.linspace(0, 1, 100)[:, None] * (v3 - v2)[None, :]).min() > 0
    verts = np.array([v1, 0.5 * (v1 + v2), v2, v3])
    K = verts.shape[0] - 1
    prm = ezo.Params.make(eps=0.1, delta=0.05, n_p=500, n_f=10, n_b=10, n_mix=20, seed=2)
    bt = ezo.Batch(robot, [env], verts[:-1], verts[1:], prm, seg_stream=np.arange(K, dtype=np.uint32),
                   path_first=np.zeros(K, np.int32))
    bt.run_path(sequential=False, mode=ezo.RUN_GRAPH)
    res = [bt.segment(g) for g in range(K)]
    kept = []
    for k in range(K):
        if not any(orc.segment_contained(res[j].A, res[j].b, verts[k], verts[k + 1]) for j in kept):
            kept.append(k)
    assert [k for k in range(K) if res[k].status != ezo.SEG_SKIPPED] == kept
    assert kept[0] == 0 and 1 not in kept
    seq = ezo.inflate_path(robot, env, verts, prm, sequential=True)
    assert [k for k, _ in seq] == kept
    for (k, r) in seq:
        np.testing.assert_array_equal(r.A, res[k].A)


def test_segment_in_collision_reports_tcol(ezo):
    """A segment that passes through an obstacle: candidates land within
    t_col of L and the segment is reported in collision (Sec. IV-C)."""
    rd, env_np, v1, v2 = planar_scene()
    c = orc.sphere_centres(rd, (0.5 * (v1 + v2))[None])[0]
    blocked = np.vstack([env_np.spheres, [[c[10, 0], c[10, 1], 0.0, 0.15]]])
    robot, env = ezo.Robot(rd), ezo.Env(blocked)
    prm = ezo.Params.make(eps=0.1, delta=0.05, n_p=1000, n_f=10, n_b=20, n_mix=30, seed=3, t_col=1e-3)
    res = ezo.inflate_segment(robot, env, v1, v2, prm)
    assert res.status == ezo.SEG_IN_COLLISION


def test_degenerate_segment_point(ezo):
    """v1 = v2: the projection is v1 (Eq. 6) and inflation still works."""
    rd, env_np, v1, _ = planar_scene()
    robot, env = ezo.Robot(rd), ezo.Env(env_np)
    prm = ezo.Params.make(eps=0.1, delta=0.05, n_p=1000, n_f=10, n_b=10, n_mix=30, seed=8)
    res = ezo.inflate_segment(robot, env, v1, v1, prm)
    assert res.status == ezo.SEG_ACCEPTED
    assert np.all(res.A @ v1 <= res.b + 1e-12)


def test_wavefront_equals_sequential_on_several_paths(ezo):
    """Three seed paths over two obstacle sets with uneven N_p: the wavefront
    mode (one segment per path per batched wave) keeps the polytopes of the
    paper's one-segment-at-a-time order."""
    sc = scenes()["dh7_batched"]
    rd = wl.dh7_robot()
    robot = ezo.Robot(rd)
    use = [p for p in sc["paths"] if len(p["path"]) <= 6][:3]
    env_ids = sorted({p["env"] for p in use})
    envs = [ezo.Env(wl.box_obstacles(sc["envs"][e]["env_seed"], sc["envs"][e]["n_obs"])) for e in env_ids]
    v1, v2, seg_env, pf = [], [], [], []
    for p in use:
        verts = np.asarray(p["path"])
        first = len(v1)
        for k in range(verts.shape[0] - 1):
            v1.append(verts[k])
            v2.append(verts[k + 1])
            seg_env.append(env_ids.index(p["env"]))
            pf.append(first)
    B = len(v1)
    seg_np = np.asarray([1000 + 700 * (g % 4) for g in range(B)], dtype=np.int32)
    prm = ezo.Params.make(n_p=2000, seed=17)
    res = {}
    for seq in (1, 2):
        bt = ezo.Batch(robot, envs, np.asarray(v1), np.asarray(v2), prm, seg_env=seg_env, seg_np=seg_np,
                       path_first=pf)
        bt.run_path(sequential=seq, mode=ezo.RUN_GRAPH if seq == 2 else ezo.RUN_HOST_LOOP)
        res[seq] = [bt.segment(g) for g in range(B)]
    for a, b in zip(res[1], res[2]):
        assert a.status == b.status
        np.testing.assert_array_equal(a.A, b.A)


def test_wave_graph_equals_host_wavefront_and_oracle_order(ezo):
    """The wavefront order (Sec. VI-A) as one graph launch: two obstacle sets,
    three paths with uneven N_p, one of them running into an obstacle (t_col,
    Sec. IV-C) so that the rest of its path must stay idle. The single graph
    (the skip rule and the next segment of every path chosen on the device,
    waves and rounds as nested WHILE nodes) keeps, skips and stops the same
    segments with the same polytopes as the host-driven wavefront loop; the
    kept segments are the ones the oracle's skip rule picks from the GPU
    polytopes in path order; a second launch after a reset and a launch after
    the graph is rebuilt for another launch shape give the same bits."""
    rd, env_np, v1, v2 = planar_scene()
    c = orc.sphere_centres(rd, (0.5 * (v1 + v2))[None])[0]
    blocked = np.vstack([env_np.spheres, [[c[10, 0], c[10, 1], 0.0, 0.15]]])
    robot = ezo.Robot(rd)
    envs = [ezo.Env(env_np), ezo.Env(blocked)]
    # path 0: a free segment in six pieces (most of them skipped);
    # path 1 (blocked set, whose new sphere covers the first 65% of that
    # segment): a free step back from v2, then a segment ending at the
    # blocked midpoint, then one more segment (never run); path 2: three
    # pieces of path 0's segment
    q = v1 + 0.85 * (v2 - v1)
    assert orc.signed_distance(rd, wl.Env("b", blocked),
                               v2[None, :] + np.linspace(0, 1, 50)[:, None] * (q - v2)[None, :]).min() > 0
    t6 = np.linspace(0.0, 1.0, 7)[:, None]
    t3 = np.linspace(0.0, 1.0, 4)[:, None]
    paths = [((1.0 - t6) * v1 + t6 * v2, 0), (np.array([v2, q, 0.5 * (v1 + v2), v1 + 0.3 * (v2 - v1)]), 1),
             ((1.0 - t3) * v1 + t3 * v2, 0)]
    V1, V2, seg_env, pf, where = [], [], [], [], []
    for pi, (verts, e) in enumerate(paths):
        first = len(V1)
        for k in range(verts.shape[0] - 1):
            V1.append(verts[k])
            V2.append(verts[k + 1])
            seg_env.append(e)
            pf.append(first)
            where.append((pi, k))
    B = len(V1)
    seg_np = np.asarray([400 + 150 * (g % 3) for g in range(B)], dtype=np.int32)
    prm = ezo.Params.make(eps=0.1, delta=0.05, n_p=700, n_f=10, n_b=10, n_mix=20, seed=29, t_col=1e-3)

    def batch():
        return ezo.Batch(robot, envs, np.asarray(V1), np.asarray(V2), prm, seg_env=seg_env, seg_np=seg_np,
                         seg_stream=np.arange(B, dtype=np.uint32), path_first=pf)

    def run(bt, mode):
        bt.reset()
        bt.run_path(sequential=2, mode=mode)
        return [bt.segment(g) for g in range(B)]

    host = run(batch(), ezo.RUN_HOST_LOOP)
    bt = batch()
    graph = run(bt, ezo.RUN_GRAPH)
    again = run(bt, ezo.RUN_GRAPH)
    sh = bt.shape()
    bt.set_shape(sh["sample_fill_tiles"], 1 if sh["check_lanes"] != 1 else 2, sh["bisect_lanes"])
    rebuilt = run(bt, ezo.RUN_GRAPH)
    for other in (graph, again, rebuilt):
        assert [r.status for r in other] == [r.status for r in host]
        for a, b in zip(host, other):
            if a.status not in (ezo.SEG_SKIPPED, ezo.SEG_IDLE):
                np.testing.assert_array_equal(a.A, b.A)
                np.testing.assert_array_equal(a.b, b.b)
    st = [r.status for r in graph]
    # the oracle's order: per path, skip a segment inside a kept polytope,
    # stop after a collision
    for pi, (verts, _) in enumerate(paths):
        gs = [g for g in range(B) if where[g][0] == pi]
        kept, stopped = [], False
        for g in gs:
            k = where[g][1]
            if stopped:
                assert st[g] == ezo.SEG_IDLE
                continue
            if any(orc.segment_contained(graph[j].A, graph[j].b, verts[k], verts[k + 1]) for j in kept):
                assert st[g] == ezo.SEG_SKIPPED
                continue
            assert st[g] not in (ezo.SEG_SKIPPED, ezo.SEG_IDLE)
            kept.append(g)
            if st[g] == ezo.SEG_IN_COLLISION:
                stopped = True
            else:
                assert orc.segment_contained(graph[g].A, graph[g].b, verts[k], verts[k + 1], tol=1e-12)
    assert st[6 + 1] == ezo.SEG_IN_COLLISION and st[6 + 2] == ezo.SEG_IDLE
    assert sum(s == ezo.SEG_SKIPPED for s in st) >= 3


def test_fp32_fma_probe_within_the_nominal_peak(ezo):
    """The FMA calibration lies between half and 105% of the nominal FP32 rate
    (SMs x 128 lanes x 2 flops x the maximum SM clock)."""
    tf = ezo.probe_fp32_fma()
    prop = torch.cuda.get_device_properties(0)
    nominal = prop.multi_processor_count * 128 * 2 * 2.07e9 * 1e-12 if prop.major == 10 else None
    assert tf > 0
    if nominal is not None:
        assert 0.5 * nominal < tf < 1.05 * nominal, (tf, nominal)


# --------------------------------------- kinematics error of the FP32 checker --
@pytest.mark.parametrize("which", ["dh7", "chain10", "mixed"])
def test_sphere_centres_and_fk_error_against_oracle(ezo, which):
    """The checker's FP32 sphere centres and the library's FP64 ones against
    the oracle's FP64 forward kinematics (Sec. II), on the same FP32
    configurations: FP64 within 1e-12 m, FP32 within 1e-5 m (the label
    band), and ezo_fk_error equal to the largest FP32-FP64 distance per
    configuration."""
    if which == "dh7":
        rd = wl.dh7_robot()
    elif which == "chain10":
        rd = chain10_robot()
    else:
        rd = wl.Robot(name="mixed", a=np.array([0.1, 0.0, 0.3, 0.05]), alpha=np.array([0.4, -1.2, 0.0, 0.7]),
                      d=np.array([0.2, 0.1, 0.0, 0.3]), theta_off=np.array([0.3, -0.5, 0.1, 0.0]),
                      q_lo=np.array([-2.0, 0.0, -2.0, -0.5]), q_hi=np.array([2.0, 1.0, 2.0, 0.5]),
                      sphere_frame=np.array([4, 1, 2, 2, 3, 0], dtype=np.int32),
                      sphere_xyz=np.array([[0, 0, 0.1], [0.1, 0, 0], [0, 0.1, 0], [0, 0, 0], [0.05, 0, 0],
                                           [0, 0, 0.05]]),
                      sphere_r=np.full(6, 0.05), sphere_link=np.array([4, 1, 2, 2, 3, 0], dtype=np.int32),
                      self_pairs=np.zeros((0, 2), dtype=np.int32), joint_type=np.array([0, 1, 0, 1], dtype=np.int32))
    robot = ezo.Robot(rd)
    N = 1537  # several blocks and a ragged tail
    q32 = wl.uniform_configs(31, rd, N).astype(np.float32)
    qd = to_dev(q32)
    ns = rd.n_spheres
    c32 = torch.empty((ns, 3, N), dtype=torch.float64, device="cuda")
    c64 = torch.empty((ns, 3, N), dtype=torch.float64, device="cuda")
    err = torch.empty(N, dtype=torch.float32, device="cuda")
    ezo.sphere_centres(robot, qd, c32, fp64=False)
    ezo.sphere_centres(robot, qd, c64, fp64=True)
    ezo.fk_error(robot, qd, err)
    torch.cuda.synchronize()
    ref = orc.sphere_centres(rd, q32.astype(np.float64))[:, robot.sphere_order, :]  # [N, ns, 3]
    g32 = c32.cpu().numpy().transpose(2, 0, 1)
    g64 = c64.cpu().numpy().transpose(2, 0, 1)
    assert np.abs(g64 - ref).max() < 1e-12
    d32 = np.linalg.norm(g32 - ref, axis=2).max(axis=1)
    assert d32.max() < 1e-5 and d32.max() > 0
    np.testing.assert_allclose(err.cpu().numpy(), np.linalg.norm(g32 - g64, axis=2).max(axis=1), rtol=1e-6,
                               atol=1e-12)
    print(f"{which}: FP32 kinematics error max {d32.max():.2e} m, p99 {np.quantile(d32, 0.99):.2e} m")


# ---------------------------------------------- one-call entry points (C ABI) --
def test_one_call_segment_equals_batch_and_keeps_its_domain(ezo):
    """ezo_inflate_segment (Algorithm 1 in one call) against a one-segment
    batch with the same stream, bit for bit, from the joint box and from a
    caller's domain D (the joint box cut by one plane that keeps the
    segment); the result contains the segment and keeps D's rows."""
    rd, env_np, path = dh7_scene()
    robot, env = ezo.Robot(rd), ezo.Env(env_np)
    prm = ezo.Params.make(n_p=3000, seed=12)
    A0, b0 = orc.joint_box(rd)
    a = np.zeros(7)
    a[0] = 1.0
    A1 = np.vstack([A0, a])
    b1 = np.concatenate([b0, [max(path[2][0], path[3][0]) + 0.3]])
    for dom in (None, (A1, b1)):
        kw = {} if dom is None else dict(A0=dom[0], b0=dom[1])
        one = ezo.inflate_segment(robot, env, path[2], path[3], prm, stream_id=5, **kw)
        bt = ezo.Batch(robot, [env], path[2], path[3], prm, seg_stream=[5], **kw)
        bt.run()
        ref = bt.segment(0)
        assert (one.status, one.rounds, one.planes, one.checks) == (ref.status, ref.rounds, ref.planes, ref.checks)
        np.testing.assert_array_equal(one.A, ref.A)
        np.testing.assert_array_equal(one.b, ref.b)
        assert one.status == ezo.SEG_ACCEPTED
        assert orc.segment_contained(one.A, one.b, path[2], path[3], tol=1e-12)
        D = A0 if dom is None else dom[0]
        np.testing.assert_array_equal(one.A[: D.shape[0]], D)


def test_one_call_path_and_batch(ezo):
    """ezo_inflate_path in its three modes and ezo_inflate_batch over three
    paths in two obstacle sets with per-segment N_p, against batches built
    segment by segment with the same streams (bit for bit), with the oracle's
    skip rule (Sec. VI-A) and coverage of every seed segment."""
    sc = scenes()["dh7_batched"]
    rd = wl.dh7_robot()
    robot = ezo.Robot(rd)
    use = [p for p in sc["paths"] if 3 <= len(p["path"]) <= 5][:3]
    env_ids = sorted({p["env"] for p in use})[:2]
    use = [p for p in use if p["env"] in env_ids]
    envs_np = [wl.box_obstacles(sc["envs"][e]["env_seed"], sc["envs"][e]["n_obs"]) for e in env_ids]
    envs = [ezo.Env(e) for e in envs_np]
    prm = ezo.Params.make(n_p=2000, n_mix=30, seed=4)
    paths = [np.asarray(p["path"]) for p in use]
    pe = [env_ids.index(p["env"]) for p in use]
    nseg = [p.shape[0] - 1 for p in paths]
    seg_np = np.asarray([1000 + 500 * (g % 3) for g in range(sum(nseg))], np.int32)
    got = ezo.inflate_batch(robot, envs, paths, prm, path_env=pe, seg_np=seg_np, sequential=2, stream_base=40)
    # the same segments as one batch (wavefront mode)
    v1 = np.concatenate([p[:-1] for p in paths])
    v2 = np.concatenate([p[1:] for p in paths])
    first = np.concatenate([[sum(nseg[:i])] * nseg[i] for i in range(len(paths))]).astype(np.int32)
    seg_env = np.concatenate([[pe[i]] * nseg[i] for i in range(len(paths))]).astype(np.int32)
    bt = ezo.Batch(robot, envs, v1, v2, prm, seg_env=seg_env, seg_np=seg_np, path_first=first,
                   seg_stream=np.arange(40, 40 + v1.shape[0], dtype=np.uint32))
    bt.run_path(sequential=2, mode=ezo.RUN_GRAPH)
    for i, p in enumerate(paths):
        g0 = int(sum(nseg[:i]))
        kept = []
        for k in range(nseg[i]):
            r = bt.segment(g0 + k)
            if r.status not in (ezo.SEG_SKIPPED, ezo.SEG_IDLE):
                kept.append((k, r))
        assert [k for k, _ in got[i]] == [k for k, _ in kept]
        for (_, a), (_, b) in zip(got[i], kept):
            np.testing.assert_array_equal(a.A, b.A)
            np.testing.assert_array_equal(a.b, b.b)
        # the oracle's skip rule on these polytopes, and coverage
        okept = []
        for k in range(nseg[i]):
            if not any(orc.segment_contained(r.A, r.b, p[k], p[k + 1]) for _, r in okept):
                okept.append((k, dict(got[i])[k]))
        assert [k for k, _ in okept] == [k for k, _ in got[i]]
        assert orc.path_coverage([(r.A, r.b) for _, r in got[i]], p).all()
    # one path through ezo_inflate_path: the three modes agree with each other
    # and with the batch call's first path
    outs = [ezo.inflate_path(robot, envs[pe[0]], paths[0], prm, sequential=s_, stream_base=40) for s_ in (True, 2, False)]
    for o in outs:
        assert [k for k, _ in o] == [k for k, _ in outs[0]]
        for (_, a), (_, b) in zip(o, outs[0]):
            np.testing.assert_array_equal(a.A, b.A)
    with pytest.raises(ezo.EzoError):
        ezo.inflate_path(robot, envs[0], paths[0][:1], prm)


def test_round_kernel_shapes_are_bit_identical_and_tuned(ezo):
    """Every launch shape of the round kernels (the walks' lane rule, label
    lanes, bisection lanes) gives the same polytopes bit for bit; the
    autotuner picks one of them and the result is unchanged."""
    rd, env_np, path = dh7_scene()
    robot, env = ezo.Robot(rd), ezo.Env(env_np)
    K = 4
    prm = ezo.Params.make(n_p=3000, seed=14)
    bt = ezo.Batch(robot, [env], path[:K], path[1:K + 1], prm, seg_stream=np.arange(K, dtype=np.uint32))
    base = bt.shape()
    S = base["sample_fill_tiles"]

    def run():
        bt.reset()
        bt.run(ezo.RUN_GRAPH)
        return [bt.segment(g) for g in range(K)]

    ref = run()
    for sh in ((1, 1, 2), (S // 2, 4, 4), (2 * S, 8, 1), (100000, 2, 8), (S, 2, 16), (S, 4, 32), (S, 2, 96)):
        bt.set_shape(*sh)
        got = run()
        for a, b in zip(got, ref):
            assert (a.status, a.rounds, a.checks) == (b.status, b.rounds, b.checks), sh
            np.testing.assert_array_equal(a.A, b.A)
            np.testing.assert_array_equal(a.b, b.b)
    with pytest.raises(ezo.EzoError):
        bt.set_shape(S, 3, 8)
    with pytest.raises(ezo.EzoError):
        bt.set_shape(S, 2, 64)
    tuned = bt.tune(reps=1)
    assert tuned["check_lanes"] in (1, 2, 4, 8) and tuned["bisect_lanes"] in (2, 4, 8, 16, 32, 96)
    assert bt.shape() == tuned
    got = run()
    for a, b in zip(got, ref):
        np.testing.assert_array_equal(a.A, b.A)
    # a second batch of the same class takes the cached shape
    bt2 = ezo.Batch(robot, [env], path[:K], path[1:K + 1], prm, seg_stream=np.arange(K, dtype=np.uint32))
    assert bt2.tune(reps=1) == tuned
