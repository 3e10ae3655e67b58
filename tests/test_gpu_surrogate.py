"""The BF16 tensor-core MLP surrogate against its FP64 oracle: gradients of
one batch element by element (within a bound derived from the BF16
roundings of the training pass), predictions, and training progress on exact
signed-distance labels."""
import json
import os

import numpy as np
import pytest

from oracle import ezo_oracle as orc
from oracle import ezo_surrogate_oracle as so
from paper_2504_10783_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def ezo():
    from paper_2504_10783_gb300 import build, ezo as e
    build.build()
    return e


def bf16_round(x):
    """Round FP32 values to the nearest BF16 (ties to even), kept as FP64."""
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def gpu_weights_as_used(p):
    """The GPU multiplies BF16 copies of W1..W3; w4 and the biases stay FP32."""
    d = so.unpack(p)
    for k in ("W1", "W2", "W3"):
        d[k] = bf16_round(d[k])
    return so.pack(d)


def _scene():
    with open(os.path.join(GOLDEN, "workloads.json")) as f:
        s = json.load(f)["dh7"]
    return wl.dh7_robot(), wl.box_obstacles(s["env_seed"], s["n_obs"])


U_BF16 = 2.0 ** -8  # unit roundoff of BF16 (8-bit significand, round to nearest)


def bf16_gradient_sigma(p, X, t, u=U_BF16):
    """Standard deviation of g_GPU - g per parameter under the probabilistic
    model of rounding errors (each rounding an independent, mean-zero error,
    uniform within +-u |x|, so of variance u^2 x^2 / 3): the GPU's training
    pass rounds the activations H1..H3 and the pre-activation gradients
    dZ3..dZ1 to BF16; the weights and features the oracle uses are the GPU's
    BF16 values and add nothing. Variances are carried through the forward
    pass (Var z = sum_k W^2 Var h), the output and the backward pass (SiLU'
    and, for the perturbed pre-activation, SiLU'' <= 0.5) to every gradient,
    which is a sum over the batch of products of two perturbed factors."""
    P = so.unpack(p)
    _, c = so.forward(P, X)
    N = X.shape[0]
    sig = lambda z: 1.0 / (1.0 + np.exp(-z))
    dsilu = lambda z: sig(z) * (1.0 + z * (1.0 - sig(z)))
    r = u * u / 3.0
    W = {l: P[f"W{l}"] for l in (1, 2, 3)}
    W2 = {l: W[l] ** 2 for l in (1, 2, 3)}
    H = {0: X, 1: c["h1"], 2: c["h2"], 3: c["h3"]}
    Z = {l: c[f"z{l}"] for l in (1, 2, 3)}
    VH, VZ = {0: np.zeros_like(X)}, {}
    for l in (1, 2, 3):
        VZ[l] = VH[l - 1] @ W2[l].T
        VH[l] = r * H[l] ** 2 + dsilu(Z[l]) ** 2 * VZ[l]
    y = H[3] @ P["w4"] + P["b4"][0]
    dy = 2.0 * (y - t) / N
    Vdy = 4.0 * (VH[3] @ P["w4"] ** 2) / N ** 2
    gH, VgH = np.outer(dy, P["w4"]), np.outer(Vdy, P["w4"] ** 2)
    out = {"w4": np.sqrt(Vdy @ H[3] ** 2 + dy ** 2 @ VH[3]), "b4": np.array([np.sqrt(Vdy.sum())])}
    for l in (3, 2, 1):
        d = dsilu(Z[l])
        gZ = gH * d
        VgZ = r * gZ ** 2 + d ** 2 * VgH + (0.5 * gH) ** 2 * VZ[l]
        out[f"W{l}"] = np.sqrt(VgZ.T @ H[l - 1] ** 2 + (gZ ** 2).T @ VH[l - 1])
        out[f"b{l}"] = np.sqrt(VgZ.sum(axis=0))
        gH, VgH = gZ @ W[l], VgZ @ W2[l]
    return so.pack(out)


def test_surrogate_gradient_matches_oracle(ezo):
    """Gradient of the mean squared error on one batch, element by element:
    |g_GPU - g_oracle| <= 7 sigma of the BF16 rounding model + 1e-6 x the
    tensor's largest gradient (FP32 accumulation). A numpy model of the
    GPU's roundings stays within 4 sigma on every one of ~200k gradients over
    12 random networks; a wrong or missing term of the backward pass is
    ~1000 sigma away."""
    rd, _ = _scene()
    robot = ezo.Robot(rd)
    sur = ezo.Surrogate(robot, seed=3)
    rng = np.random.default_rng(1)
    N = 512
    q = rng.uniform(rd.q_lo, rd.q_hi, size=(N, 7)).astype(np.float32)
    t = rng.uniform(-0.1, 0.3, N).astype(np.float32)
    qd = torch.from_numpy(q.T.copy()).cuda()
    td = torch.from_numpy(t).cuda()
    loss, g = sur.grad(qd, td)
    p = gpu_weights_as_used(sur.params())
    X = bf16_round(so.features(q.astype(np.float64)))
    loss_ref, g_ref = so.loss_and_grad(p, X, t.astype(np.float64))
    assert abs(loss - loss_ref) <= 1e-2 * abs(loss_ref)
    sg = bf16_gradient_sigma(p, X, t.astype(np.float64))
    o = 0
    for name, shp in so.SHAPES:
        cnt = int(np.prod(shp))
        a, b, e = g[o:o + cnt].astype(np.float64), g_ref[o:o + cnt], sg[o:o + cnt]
        err = np.abs(a - b)
        lim = 7.0 * e + 1e-6 * np.abs(b).max()
        print(f"{name}: max |err| / sigma = {float(np.max(err / (e + 1e-300))):.2f}, max |err| = {err.max():.3e}")
        assert np.all(err <= lim), (name, float(np.max(err / lim)))
        o += cnt


@pytest.mark.parametrize("N", [1, 129, 1000, 40037])
def test_surrogate_predict_matches_oracle(ezo, N):
    """The tensor-core forward pass (128-row tiles, one persistent block per
    SM) against the FP64 oracle: a single row, a ragged second tile, several
    blocks, and several tiles per block with a ragged last tile."""
    rd, _ = _scene()
    robot = ezo.Robot(rd)
    sur = ezo.Surrogate(robot, seed=4)
    rng = np.random.default_rng(2)
    q = rng.uniform(rd.q_lo, rd.q_hi, size=(N, 7)).astype(np.float32)
    out = torch.empty(N, device="cuda")
    sur.predict(torch.from_numpy(q.T.copy()).cuda(), out)
    torch.cuda.synchronize()
    y_ref, _ = so.forward(gpu_weights_as_used(sur.params()), bf16_round(so.features(q.astype(np.float64))))
    y = out.cpu().numpy()
    assert not sur.timed_out()
    assert np.abs(y - y_ref).max() <= 1e-2 * max(1.0, np.abs(y_ref).max())


@pytest.mark.parametrize("which", ["planar3", "chain10"])
def test_surrogate_predict_other_chain_lengths(ezo, which):
    """Feature staging for 3 joints (6 features, one 16-byte chunk) and for
    10 joints (20 features over three chunks, written by all four column
    groups) against the FP64 oracle."""
    if which == "planar3":
        rd = wl.planar3_robot()
    else:
        rd = wl.chain_robot(10)
    sur = ezo.Surrogate(ezo.Robot(rd), seed=9)
    q = wl.uniform_configs(23, rd, 2051).astype(np.float32)
    out = torch.empty(q.shape[0], device="cuda")
    sur.predict(torch.from_numpy(q.T.copy()).cuda(), out)
    torch.cuda.synchronize()
    y_ref, _ = so.forward(gpu_weights_as_used(sur.params()), bf16_round(so.features(q.astype(np.float64))))
    y = out.cpu().numpy()
    assert np.abs(y - y_ref).max() <= 1e-2 * max(1.0, np.abs(y_ref).max())


def test_surrogate_predict_rows_do_not_depend_on_the_batch(ezo):
    """A row's prediction is the same bits whatever batch it is in: alone,
    in a ragged tile, or deep in a batch where each block runs several tiles
    (the same configuration placed at row 0, 130 and 39,000)."""
    rd, _ = _scene()
    sur = ezo.Surrogate(ezo.Robot(rd), seed=8)
    rng = np.random.default_rng(3)
    big = rng.uniform(rd.q_lo, rd.q_hi, size=(40037, 7)).astype(np.float32)
    probe = big[:5].copy()
    big[130:135] = probe
    big[39000:39005] = probe

    def run(q):
        out = torch.empty(q.shape[0], device="cuda")
        sur.predict(torch.from_numpy(q.T.copy()).cuda(), out)
        torch.cuda.synchronize()
        return out.cpu().numpy()

    alone = run(probe)
    y = run(big)
    np.testing.assert_array_equal(y[:5], alone)
    np.testing.assert_array_equal(y[130:135], alone)
    np.testing.assert_array_equal(y[39000:39005], alone)


def test_surrogate_training_learns_signed_distance(ezo):
    rd, env_np = _scene()
    robot, env = ezo.Robot(rd), ezo.Env(env_np)
    sur = ezo.Surrogate(robot, seed=5)
    # held-out configurations with exact labels
    q = wl.uniform_configs(9, rd, 4096).astype(np.float32)
    sd = np.clip(orc.signed_distance(rd, env_np, q.astype(np.float64)), -0.1, 0.3)
    qd = torch.from_numpy(q.T.copy()).cuda()
    out = torch.empty(q.shape[0], device="cuda")

    def rmse():
        sur.predict(qd, out)
        torch.cuda.synchronize()
        return float(np.sqrt(np.mean((out.cpu().numpy() - sd) ** 2)))

    before = rmse()
    losses = sur.train(env, n_samples=1 << 18, epochs=4, batch=4096, lr=1e-3, data_seed=11)
    after = rmse()
    assert np.all(np.isfinite(losses)) and losses[-1] <= losses[0]
    assert after < 0.5 * before and after < 0.7 * float(np.std(sd)), (before, after, float(np.std(sd)))


def test_surrogate_training_is_reproducible(ezo):
    """Two trainings from the same seeds (initial weights, data, labels) end
    with the same parameters bit for bit: every reduction of the training
    step (split-K weight gradients, column sums, the output layer's gradient
    and the loss) adds its partial sums in a fixed order. A ragged last
    mini-batch (2^16 samples in batches of 3200) is included."""
    rd, env_np = _scene()
    robot, env = ezo.Robot(rd), ezo.Env(env_np)
    params, losses = [], []
    for _ in range(2):
        sur = ezo.Surrogate(robot, seed=5)
        losses.append(sur.train(env, n_samples=1 << 16, epochs=2, batch=3200, lr=1e-3, data_seed=21))
        params.append(sur.params())
    np.testing.assert_array_equal(params[0], params[1])
    np.testing.assert_array_equal(losses[0], losses[1])


@pytest.fixture(scope="module")
def trained(ezo):
    rd, env_np = _scene()
    robot, env = ezo.Robot(rd), ezo.Env(env_np)
    sur = ezo.Surrogate(robot, seed=6)
    # 10^7 exact labels of uniform configurations in the joint box, mini-batches of 3200
    sur.train(env, n_samples=10_000_000, epochs=4, batch=3200, lr=1e-3, data_seed=12)
    return rd, env_np, robot, env, sur


def test_surrogate_false_negative_rate_reported(ezo, trained):
    """False negatives (in collision, predicted free) at margin 0 and at the
    margin that brings them to 1% on held-out configurations."""
    rd, env_np, robot, env, sur = trained
    q = wl.uniform_configs(10, rd, 40000).astype(np.float32)
    out = torch.empty(q.shape[0], device="cuda")
    sur.predict(torch.from_numpy(q.T.copy()).cuda(), out)
    torch.cuda.synchronize()
    y = out.cpu().numpy()
    col = orc.in_collision(rd, env_np, q.astype(np.float64))
    assert col.any() and (~col).any()
    fn0 = float(np.mean(y[col] >= 0.0))
    fp0 = float(np.mean(y[~col] < 0.0))
    m1 = float(np.quantile(y[col], 0.99))
    fp1 = float(np.mean(y[~col] < m1))
    print(f"surrogate: FN {fn0:.3f} / FP {fp0:.3f} at margin 0; margin {m1:.4f} for FN 1% gives FP {fp1:.3f}")
    assert fp1 < 0.5, "the surrogate does not separate colliding from free configurations"


def test_surrogate_bisection_round_replay(ezo, trained):
    """One round with surrogate-guided bisection: every candidate end point is
    exactly in collision on [c_proj, c]; candidates whose surrogate end point
    was free carry the exact bisection; placement equals the oracle's on the
    GPU's end points."""
    rd, env_np, robot, env, sur = trained
    with open(os.path.join(GOLDEN, "workloads.json")) as f:
        path = np.asarray(json.load(f)["dh7"]["path"])
    v1, v2 = path[3], path[4]
    prm = ezo.Params.make(n_p=2000, seed=21)
    bt = ezo.Batch(robot, [env], v1, v2, prm)
    bt.attach_surrogate(sur, 0.0)
    for step in range(4):
        bt.step(step)
    bt.sync()
    st = bt.state(0)
    assert st["status"] == ezo.SEG_ACTIVE and st["n_cand"] > 0
    nc = st["n_cand"]
    S = bt.read(0, "samples")[:, : st["n_samples"]].T.astype(np.float64)
    idx = bt.read(0, "cand_idx")[:nc]
    bt.step(4)
    bt.sync()
    cst = bt.read(0, "c_star")[:, :nc].T
    bits = bt.read(0, "bits")[:nc]
    c = S[idx]
    p = orc.project_onto_segment(c, v1, v2)
    # c* = p + f (c - p) with a dyadic f in (0, 1]
    f = np.einsum("ij,ij->i", cst - p, c - p) / np.einsum("ij,ij->i", c - p, c - p)
    np.testing.assert_allclose(cst, p + f[:, None] * (c - p), atol=1e-9)
    assert np.all((f > 0) & (f <= 1 + 1e-12))
    sd = orc.signed_distance(rd, env_np, cst)
    assert np.all(sd < 1e-5), "an end point is not in collision"
    follow = ((bits[:, None] >> np.arange(prm.n_b)[None, :]) & 1).astype(bool)
    ex = orc.bisect(rd, env_np, c, v1, v2, prm.n_b, follow=follow, band=1e-5)
    same = np.all(np.abs(ex.c_star - cst) < 1e-9, axis=1)
    print(f"{nc} candidates, {int(same.sum())} with the exact bisection's end point, "
          f"{bt.check_split(0)[1]} exact bisection checks vs {nc * prm.n_b} without the surrogate")
    m_before = st["m"]
    bt.step(5)
    bt.sync()
    st = bt.state(0)
    pl = orc.place_hyperplanes(cst, idx, v1, v2, prm.n_f, prm.step_back_max, prm.t_col)
    res = bt.segment(0)
    np.testing.assert_allclose(res.A[m_before:], pl.rows_a, rtol=1e-6, atol=1e-12)
    np.testing.assert_allclose(res.b[m_before:], pl.rows_b, rtol=1e-6, atol=1e-12)


def test_surrogate_path_gain_and_validity(ezo, trained):
    """The whole 10-segment path with and without the surrogate, Philox seeds
    1..5: every polytope contains its segment and is accepted by the exact
    test, and the surrogate cuts the exact checks spent in bisection to below
    0.6 of the exact method's on average (per seed the cut depends on the
    draw, how many surrogate end points verify in collision)."""
    rd, env_np, robot, env, sur = trained
    with open(os.path.join(GOLDEN, "workloads.json")) as f:
        path = np.asarray(json.load(f)["dh7"]["path"])
    K = path.shape[0] - 1
    ratios = []
    for seed in (1, 2, 3, 4, 5):
        prm = ezo.Params.make(n_p=10000, seed=seed)
        out = {}
        for use in (False, True):
            bt = ezo.Batch(robot, [env], path[:-1], path[1:], prm)
            if use:
                bt.attach_surrogate(sur, 0.0)
            bt.run(ezo.RUN_GRAPH)
            bis = sum(bt.check_split(g)[1] for g in range(K))
            for g in range(K):
                r = bt.segment(g)
                assert r.status == ezo.SEG_ACCEPTED
                assert orc.segment_contained(r.A, r.b, path[g], path[g + 1], tol=1e-12)
            out[use] = bis
        ratios.append(out[True] / out[False])
    print(f"exact bisection checks with / without the surrogate, seeds 1..5: {np.round(ratios, 3)}")
    assert np.mean(ratios) < 0.6, ratios


def test_surrogate_wavefront_graph_equals_host_loop(ezo, trained):
    """The wavefront order with surrogate-guided bisection as one graph
    launch (waves and rounds as nested WHILE nodes, the tensor-core
    bisection steps inside the round body) keeps, skips and inflates the
    same segments with the same polytopes, bit for bit, as the host-driven
    wavefront; the benchmark path is split into two paths of five segments."""
    rd, env_np, robot, env, sur = trained
    with open(os.path.join(GOLDEN, "workloads.json")) as f:
        path = np.asarray(json.load(f)["dh7"]["path"])
    K = path.shape[0] - 1
    pf = np.asarray([0] * 5 + [5] * (K - 5), dtype=np.int32)
    prm = ezo.Params.make(n_p=2000, seed=9)
    res = {}
    for mode in (ezo.RUN_HOST_LOOP, ezo.RUN_GRAPH):
        bt = ezo.Batch(robot, [env], path[:-1], path[1:], prm, seg_stream=np.arange(K, dtype=np.uint32),
                       path_first=pf)
        bt.attach_surrogate(sur, 0.0)
        bt.run_path(sequential=2, mode=mode)
        res[mode] = [bt.segment(g) for g in range(K)]
    assert [r.status for r in res[ezo.RUN_HOST_LOOP]] == [r.status for r in res[ezo.RUN_GRAPH]]
    for a, b in zip(res[ezo.RUN_HOST_LOOP], res[ezo.RUN_GRAPH]):
        if a.status not in (ezo.SEG_SKIPPED, ezo.SEG_IDLE):
            np.testing.assert_array_equal(a.A, b.A)
            np.testing.assert_array_equal(a.b, b.b)
    assert any(r.status == ezo.SEG_ACCEPTED for r in res[ezo.RUN_GRAPH])
