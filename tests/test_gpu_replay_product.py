"""Round-by-round replay of the product run loop against the FP64 oracle.

The batch is driven through ezo_batch_step with the kernel sequence of the
run loops (ezo_batch_run in either mode): the first round's sizing (step 0)
once, then per round sampling, labels, certification, bisection, placement
(steps 1-5) and the round close that ends the round and sizes the next one
(step 7), with the batch's own launch shapes (device lane rule for the
walks, the tuned lanes for the labels). The run loops launch steps 5 and 7
as one kernel (step 8: the placement's last block runs the close, the same
two device functions); stopping after step 5 lets the test read each
round's placement before the close. After each round
every segment that took part is replayed with the oracle (Algorithm 1,
Sec. IV-B, IV-C) on its own obstacle set, its own N_p and that round's GPU
samples and polytope, at the parity tolerances of tests/test_gpu_parity.py.
At the end a RUN_GRAPH run of an identical batch must give the same
polytopes bit for bit, and the skip rule of Sec. VI-A applied by the oracle
to those polytopes must keep the segments the library keeps.

Cases: the benchmarked path (7-DOF arm, 64 obstacles, 10 segments,
eps = delta = 0.05, N_p = 1e4, N_ms = 60, N_b = 10, seed 1, streams 0..9)
and a batch over three obstacle sets with per-segment N_p of 1000, 1700 and
2400.
"""
import json
import multiprocessing as mp
import os
from concurrent.futures import ProcessPoolExecutor

import numpy as np
import pytest

from oracle import ezo_oracle as orc
from paper_2504_10783_gb300 import workloads as wl

import _replay_jobs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

AMB = 1e-5
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
BENCH_PRM = dict(eps=0.05, delta=0.05, tau=0.5, step_back_max=0.01, t_col=1e-3, n_p=10000, n_f=10, n_b=10, n_mix=60,
                 n_it_max=50, seed=1)


@pytest.fixture(scope="module")
def ezo():
    from paper_2504_10783_gb300 import build, ezo as e
    build.build()
    return e


@pytest.fixture(scope="module")
def pool():
    workers = max(1, min(12, (os.cpu_count() or 2) - 1))
    with ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        yield ex


def scenes():
    with open(os.path.join(GOLDEN, "workloads.json")) as f:
        return json.load(f)


def drive_and_replay(ezo, pool, rd, envs_np, v1, v2, prm_kw, seg_env=None, seg_np=None, seg_stream=None,
                     path_first=None, n_walks=300):
    """Runs the batch round by round with the run loop's kernels and replays
    every round of every segment with the oracle. Returns the batch and the
    per-segment number of rounds."""
    robot = ezo.Robot(rd)
    envs = [ezo.Env(e) for e in envs_np]
    prm = ezo.Params.make(**prm_kw)
    B = v1.shape[0]
    seg_env = np.zeros(B, np.int32) if seg_env is None else np.asarray(seg_env, np.int32)
    seg_np = np.full(B, prm.n_p, np.int32) if seg_np is None else np.asarray(seg_np, np.int32)
    seg_stream = np.arange(B, dtype=np.uint32) if seg_stream is None else np.asarray(seg_stream, np.uint32)
    bt = ezo.Batch(robot, envs, v1, v2, prm, seg_env=seg_env, seg_np=seg_np, seg_stream=seg_stream,
                   path_first=path_first)
    A0, b0 = orc.joint_box(rd)
    poly = [(A0.copy(), b0.copy()) for _ in range(B)]
    active = list(range(B))
    rounds = np.zeros(B, np.int32)
    amb = 0
    bt.step(0)
    for k in range(1, prm.n_it_max + 1):
        for step in (1, 2, 3, 4, 5):
            bt.step(step)
        bt.sync()
        gpu, futs = {}, {}
        for g in active:
            st = bt.state(g)
            assert st["k"] == k and st["env"] == seg_env[g] and st["n_p"] == seg_np[g]
            ns, nc = st["n_samples"], st["n_cand"]
            S = bt.read(g, "samples")[:, :ns].T.copy()
            lab = bt.read(g, "labels")[:ns].astype(bool)
            bits = bt.read(g, "bits")[:nc]
            follow = ((bits[:, None] >> np.arange(prm.n_b)[None, :]) & 1).astype(bool) if nc else None
            res = bt.segment(g)
            gpu[g] = dict(st=st, cand=bt.read(g, "cand_idx")[:nc].copy(), c_star=bt.read(g, "c_star")[:, :nc].T.copy(),
                          dist=bt.read(g, "dist")[:nc].copy(), placed=bt.read(g, "placed_idx")[: st["n_placed"]].copy(),
                          deltas=bt.read(g, "placed_delta")[: st["n_placed"]].copy(), A=res.A, b=res.b, follow=follow)
            A, b = poly[g]
            job = dict(rd=rd, env=envs_np[seg_env[g]], A=A, b=b, v1=v1[g], v2=v2[g], k=k,
                       prm=dict(prm_kw, n_p=int(seg_np[g])), stream=int(seg_stream[g]), S=S, labels=lab,
                       follow=follow, band=AMB, n_walks=n_walks)
            futs[g] = pool.submit(_replay_jobs.replay_round, job)
        still = []
        for g in active:
            o, G = futs[g].result(), gpu[g]
            st = G["st"]
            A, b = poly[g]
            where = f"segment {g}, round {k}"
            assert st["m_test"] == o["m_test"] and st["n_samples"] == o["n_samples"], where
            assert o["inside"], where
            assert o["walk_q99"] < 1e-3 and o["walk_med"] < 1e-4, (where, o["walk_q99"], o["walk_med"])
            assert o["label_diff_outside_band"] == 0, (where, o["label_diff"])
            assert st["count"] == o["count"], where
            assert (st["status"] == ezo.SEG_ACCEPTED) == o["accept"], where
            rounds[g] = k
            m_before = A.shape[0]
            np.testing.assert_array_equal(G["A"][:m_before], A, err_msg=where)
            if o["accept"]:
                assert G["A"].shape[0] == m_before, where
                continue
            np.testing.assert_array_equal(G["cand"], o["cand"], err_msg=where)
            np.testing.assert_array_equal(G["follow"], o["decisions"], err_msg=where)
            amb += o["ambiguous"]
            assert np.abs(G["c_star"] - o["c_star"]).max() < 1e-9, where
            np.testing.assert_allclose(G["dist"], o["dist"], rtol=1e-12, atol=1e-14, err_msg=where)
            H = G["A"].shape[0] - m_before
            assert H == o["rows_a"].shape[0] == st["n_placed"], where
            np.testing.assert_allclose(G["A"][m_before:], o["rows_a"], rtol=1e-6, atol=1e-12, err_msg=where)
            np.testing.assert_allclose(G["b"][m_before:], o["rows_b"], rtol=1e-6, atol=1e-12, err_msg=where)
            np.testing.assert_array_equal(G["placed"], o["order"], err_msg=where)
            np.testing.assert_allclose(G["deltas"], o["deltas"], rtol=1e-9, err_msg=where)
            assert orc.segment_contained(G["A"], G["b"], v1[g], v2[g], tol=1e-12), where
            poly[g] = (G["A"], G["b"])
            if o["place_status"] == orc.STATUS_SEGMENT_IN_COLLISION:
                assert st["status"] == ezo.SEG_IN_COLLISION, where
            else:
                assert st["status"] == ezo.SEG_ACTIVE, where
                still.append(g)
        bt.step(7)
        active = still
        if not active:
            break
    bt.sync()
    for g in range(B):
        r = bt.segment(g)
        assert r.rounds == rounds[g]
        np.testing.assert_array_equal(r.A, poly[g][0])
    print(f"replayed {int(rounds.sum())} segment rounds, {amb} ambiguous bisection decisions followed")
    return bt, rounds


def graph_and_skip_rule(ezo, bt, rd, envs_np, v1, v2, prm_kw, path_first, **kw):
    """An identical batch run as the bench runs it (speculative path mode in
    one graph) keeps every polytope of the replayed run; the oracle's skip
    rule on those polytopes keeps the segments the library keeps."""
    robot = ezo.Robot(rd)
    envs = [ezo.Env(e) for e in envs_np]
    g2 = ezo.Batch(robot, envs, v1, v2, ezo.Params.make(**prm_kw), path_first=path_first, **kw)
    g2.run_path(sequential=False, mode=ezo.RUN_GRAPH)
    B = v1.shape[0]
    ref = [bt.segment(g) for g in range(B)]
    got = [g2.segment(g) for g in range(B)]
    kept = []
    for g in range(B):
        np.testing.assert_array_equal(got[g].A, ref[g].A)
        np.testing.assert_array_equal(got[g].b, ref[g].b)
        assert got[g].rounds == ref[g].rounds
        pf = path_first[g]
        skip = any(orc.segment_contained(ref[j].A, ref[j].b, v1[g], v2[g]) for j in kept if path_first[j] == pf)
        stopped = any(ref[j].status == ezo.SEG_IN_COLLISION for j in kept if path_first[j] == pf)
        if skip or stopped:
            assert got[g].status == (ezo.SEG_IDLE if stopped else ezo.SEG_SKIPPED), g
        else:
            assert got[g].status == ref[g].status, g
            kept.append(g)
    return kept


def test_replay_benchmarked_path(ezo, pool):
    """The benchmarked 10-segment path at N_p = 1e4, every round of every
    segment, through the run loop's kernels."""
    s = scenes()["dh7"]
    rd, env_np, path = wl.dh7_robot(), wl.box_obstacles(s["env_seed"], s["n_obs"]), np.asarray(s["path"])
    K = path.shape[0] - 1
    v1, v2 = path[:-1].copy(), path[1:].copy()
    pf = np.zeros(K, np.int32)
    bt, rounds = drive_and_replay(ezo, pool, rd, [env_np], v1, v2, BENCH_PRM, path_first=pf)
    assert rounds.max() >= 2
    kept = graph_and_skip_rule(ezo, bt, rd, [env_np], v1, v2, BENCH_PRM, pf,
                               seg_stream=np.arange(K, dtype=np.uint32))
    assert 0 < len(kept) <= K


def test_replay_multi_env_uneven_np(ezo, pool):
    """Six segments of three seed paths, each path in its own obstacle set
    (207, 398 and 436 spheres), with N_p of 1000, 1700 and 2400 in turn:
    each segment's rounds are replayed on its own obstacle set and N_p."""
    sc = scenes()["dh7_batched"]
    rd = wl.dh7_robot()
    env_ids = [7, 0, 6]
    envs_np = [wl.box_obstacles(sc["envs"][e]["env_seed"], sc["envs"][e]["n_obs"]) for e in env_ids]
    v1, v2, pf, seg_env = [], [], [], []
    for i, e in enumerate(env_ids):
        verts = np.asarray(next(p for p in sc["paths"] if p["env"] == e and len(p["path"]) >= 3)["path"])[:3]
        first = len(v1)
        for k in range(2):
            v1.append(verts[k])
            v2.append(verts[k + 1])
            pf.append(first)
            seg_env.append(i)
    v1, v2 = np.asarray(v1), np.asarray(v2)
    pf, seg_env = np.asarray(pf, np.int32), np.asarray(seg_env, np.int32)
    B = v1.shape[0]
    seg_np = np.asarray([(1000, 1700, 2400)[g % 3] for g in range(B)], np.int32)
    streams = np.arange(100, 100 + B, dtype=np.uint32)
    prm = dict(BENCH_PRM, n_p=2400, seed=9)
    bt, rounds = drive_and_replay(ezo, pool, rd, envs_np, v1, v2, prm, seg_env=seg_env, seg_np=seg_np,
                                  seg_stream=streams, path_first=pf)
    assert rounds.max() >= 2
    graph_and_skip_rule(ezo, bt, rd, envs_np, v1, v2, prm, pf, seg_env=seg_env, seg_np=seg_np, seg_stream=streams)
