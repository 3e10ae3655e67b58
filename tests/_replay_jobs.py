"""Oracle side of the round-by-round replays (test infrastructure).

One job replays one round of one segment with the FP64 oracle on the GPU's
inputs for that round (its polytope and its FP32 samples, widened) and
returns what the oracle computes, for the test to compare with the GPU's
outputs. Jobs run in a process pool started with `spawn`, so this module
imports only numpy and the oracle.
"""
from __future__ import annotations

import numpy as np

from oracle import ezo_oracle as orc


def replay_round(job: dict) -> dict:
    """job: rd, env, A, b, v1, v2, k, prm (orc.Params fields), stream, S (FP32
    samples [N, n]), labels (GPU, bool [N]), follow (GPU bisection decisions,
    bool [n_cand, n_b] or None), band, n_walks (walks compared with the FP64
    hit-and-run from the same Philox counters)."""
    rd, env = job["rd"], job["env"]
    prm = orc.Params(**job["prm"])
    A, b, v1, v2, k = job["A"], job["b"], job["v1"], job["v2"], job["k"]
    S = np.asarray(job["S"], dtype=np.float64)
    lab = np.asarray(job["labels"], dtype=bool)
    out = {"m_test": orc.test_size(k, prm.eps, prm.delta, prm.tau),
           "n_samples": orc.batch_size(k, prm.eps, prm.delta, prm.tau, prm.n_p)}
    # every sample inside P (FP32 samples against the FP64 polytope)
    out["inside"] = bool(np.all(S @ A.T <= b + 1e-5 * (1.0 + np.abs(b))))
    # the walks follow the FP64 walks of the same counters
    nw = min(job["n_walks"], S.shape[0])
    ref = orc.hit_and_run(A, b, v1, v2, nw, prm.n_mix, prm.seed, job["stream"], k)
    err = np.abs(S[:nw] - ref).max(axis=1)
    out["walk_q99"], out["walk_med"] = float(np.quantile(err, 0.99)), float(np.median(err))
    # labels: exact except within the band of the collision boundary
    col = orc.in_collision(rd, env, S)
    diff = np.nonzero(col != lab)[0]
    out["label_diff"] = int(diff.size)
    out["label_diff_outside_band"] = 0
    if diff.size:
        sd = orc.signed_distance(rd, env, S[diff])
        out["label_diff_outside_band"] = int(np.count_nonzero(np.abs(sd) >= job["band"]))
    # the rest of the round on the GPU's labels (identical outside the band)
    follow = job["follow"]
    rr = orc.eizo_round(rd, env, A, b, v1, v2, k, prm, S, labels=lab, follow=follow, band=job["band"])
    out.update(count=rr.n_col_first_m, accept=rr.accept, cand=rr.cand_index, decisions=rr.decisions,
               c_star=rr.c_star, ambiguous=rr.ambiguous)
    if rr.place is not None:
        pl = rr.place
        out.update(rows_a=pl.rows_a, rows_b=pl.rows_b, order=np.asarray(pl.order, dtype=np.int64),
                   deltas=np.asarray(pl.deltas), place_status=pl.status,
                   dist=orc.dist_to_segment(rr.c_star, v1, v2) if rr.c_star.shape[0] else np.zeros(0))
    return out
