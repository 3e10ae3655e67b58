"""FP64 CPU oracle for EI-ZO edge inflation.

TEST INFRASTRUCTURE ONLY. Nothing in the product path imports this module:
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may call it. It shares no code with
the CUDA library (no kernels, headers, tables or helpers); the only inputs the
two have in common come from ``paper_2504_10783_gb300.workloads``.

It follows "Superfast Configuration-Space Convex Set Computation on GPUs for
Online Motion Planning" (arXiv 2504.10783), Sec. IV, Algorithm 1 (EI-ZO), step
by step in float64, written for a reader to check against the paper:

* distance to a segment, its projection and gradient: Sec. IV-A, Eqs. (5)-(7);
* tangent plane with step back: Eqs. (4), (10) and Sec. IV-C, Eqs. (11)-(12);
* round size and unadaptive test: Sec. IV-B (|S| = max(N_p, M),
  M = ceil(2 log(1/delta_k) / (eps tau^2)), Eq. (9) for delta_k, accept iff
  the count in the first M samples is <= M (1 - tau) eps);
* hit-and-run sampling, one walk per sample with a fixed number of mixing
  steps: Sec. IV-B and IV-D;
* bisection with a fixed number of steps N_b along the negative gradient:
  Sec. IV-B, IV-C;
* greedy, sorted hyperplane placement with at most N_f faces per iteration:
  Sec. IV-B and the parameter tables of the appendix;
* path inflation with the containment skip: Sec. VI-A;
* box collision geometries (Sec. IV-D: the checker supports boxes and
  spheres; Sec. VII: an arm described by 11 boxes): sphere-box distance and
  the separating-axis test for box pairs, for robot boxes, obstacle boxes and
  listed self pairs;
* recovery from detected collisions: fine discretisation of a path and its
  collision check, set editing with the last steps of Algorithm 1 on given
  collisions that lie in the set, and the coverage test of the seed path:
  Sec. VI-B (step 0.1 rad from the appendix).

Where the paper is silent the oracle takes these readings (each one is also a
parameter or a documented choice of the CUDA library):

* natural log in M; tau = 0.5; k starts at 1;
* each hit-and-run walk starts at v1 + u (v2 - v1), u ~ U[0, 1);
* directions are n Box-Muller Gaussians, normalised; the chord [t_lo, t_hi]
  comes from the slack s = b - A x and q = A d, with t_lo <= 0 <= t_hi forced;
* random numbers come from Philox4x32-10 (Salmon et al., SC'11) with counter
  (walk, draw, round, stream) and key (seed low, seed high); a step's
  Gaussians use the top 24 bits of its words and its step length the low
  bytes of the first three, so 7 joints need two blocks per step;
* "the first N_p samples in S_col" are the colliding samples of lowest index;
* bisection runs on the segment [c_proj, c]; c* is its colliding end;
* candidates are sorted by (distance to L, sample index); a candidate is
  discarded when a^T c_j > b - Delta for a row added this round;
* a segment L_k is skipped when both its endpoints satisfy A x <= b + 1e-9 for
  an earlier polytope.
* box-box pairs skip cross-product axes of edges within ~0.6 degrees of
  parallel (|a x b|^2 < 1e-4); a point of radius 0 overlaps a box only when
  strictly inside it;
* a path edge is cut into N_k = max(1, ceil(|e|_2 / step)) equal pieces and
  checked at all N_k + 1 points; a set is edited with the given collisions
  that satisfy A c <= b + 1e-9, the first N_p by index, without a test.

Parity status: every function here is pinned by tests under ``tests/`` against
closed forms, invariants, brute force or published vectors, except the
free-running end-to-end polytope after the first ambiguous collision decision,
which is compared by statistics only ("parity unpinned" for that comparison).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# ---------------------------------------------------------------------------
# Counter-based random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw,
# "Parallel random numbers: as easy as 1, 2, 3", SC'11, Sec. 4.2).
# ---------------------------------------------------------------------------
_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = np.uint64(0x9E3779B9)
_W1 = np.uint64(0xBB67AE85)
_MASK = np.uint64(0xFFFFFFFF)
_S32 = np.uint64(32)


def philox4x32_10(counter, key) -> np.ndarray:
    """Ten Philox rounds on 4x32-bit counters ``counter[..., 4]`` with a
    2x32-bit key; the key is bumped by the Weyl constants between rounds.
    Each round multiplies words 0 and 2 by the two multipliers and mixes the
    high halves with words 1 and 3 and the key."""
    c = np.asarray(counter, dtype=np.uint64) & _MASK
    x0, x1, x2, x3 = c[..., 0], c[..., 1], c[..., 2], c[..., 3]
    k0 = np.uint64(int(key[0]) & 0xFFFFFFFF)
    k1 = np.uint64(int(key[1]) & 0xFFFFFFFF)
    for r in range(10):
        if r:
            k0 = (k0 + _W0) & _MASK
            k1 = (k1 + _W1) & _MASK
        p0 = _M0 * x0
        p1 = _M1 * x2
        x0, x1, x2, x3 = ((p1 >> _S32) ^ x1 ^ k0, p1 & _MASK, (p0 >> _S32) ^ x3 ^ k1, p0 & _MASK)
    return np.stack([x0, x1, x2, x3], axis=-1).astype(np.uint32)


def u01_closed_open(x) -> np.ndarray:
    """Top 24 bits of a 32-bit word as a float in [0, 1): (x >> 8) * 2^-24."""
    return (np.asarray(x, dtype=np.uint64) >> np.uint64(8)).astype(np.float64) * 2.0 ** -24


def u01_open_closed(x) -> np.ndarray:
    """Top 24 bits of a 32-bit word as a float in (0, 1]: ((x >> 8) + 1) * 2^-24."""
    return ((np.asarray(x, dtype=np.uint64) >> np.uint64(8)) + np.uint64(1)).astype(np.float64) * 2.0 ** -24


def seed_key(seed: int):
    return (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)


def blocks_per_step(n: int) -> int:
    """Philox blocks drawn per hit-and-run step: 2*ceil(n/2) words for the
    Box-Muller Gaussians of the direction (at least one block); the step
    length takes the low bytes of the first three words, which the 24-bit
    uniforms leave unused."""
    return max(1, (2 * ((n + 1) // 2) + 3) // 4)


def step_uniform(w0, w1, w2) -> np.ndarray:
    """The step length's uniform in [0, 1): the low bytes of three words
    as one 24-bit integer (w0 lowest), times 2^-24."""
    m = np.uint64(0xFF)
    w0, w1, w2 = (np.asarray(w, dtype=np.uint64) for w in (w0, w1, w2))
    t = (w0 & m) | ((w1 & m) << np.uint64(8)) | ((w2 & m) << np.uint64(16))
    return t.astype(np.float64) * 2.0 ** -24


# ---------------------------------------------------------------------------
# Robot kinematics and the sphere collision test (the collision checker the
# paper assumes, Sec. II; sphere geometries, Sec. IV-D and V-B).
# ---------------------------------------------------------------------------
def dh_frames(robot, q) -> tuple[np.ndarray, np.ndarray]:
    """Frames of a standard DH chain for configurations ``q[N, n]``.

    Returns rotations R[N, n+1, 3, 3] and origins o[N, n+1, 3]; frame 0 is the
    identity and T_i = T_{i-1} Rz(q_i + theta_off_i) Tz(d_i) Tx(a_i) Rx(alpha_i)
    for a revolute joint, T_i = T_{i-1} Rz(theta_off_i) Tz(d_i + q_i) Tx(a_i)
    Rx(alpha_i) for a prismatic one (``robot.prismatic``).
    """
    q = np.atleast_2d(np.asarray(q, dtype=np.float64))
    N, n = q.shape
    R = np.zeros((N, n + 1, 3, 3))
    o = np.zeros((N, n + 1, 3))
    R[:, 0] = np.eye(3)
    prism = np.zeros(n, dtype=bool) if getattr(robot, "joint_type", None) is None \
        else np.asarray(robot.joint_type) == 1
    for i in range(n):
        th = (0.0 * q[:, i] if prism[i] else q[:, i]) + robot.theta_off[i]
        dd = robot.d[i] + q[:, i] if prism[i] else np.full(N, robot.d[i])
        ct, st = np.cos(th), np.sin(th)
        ca, sa = math.cos(robot.alpha[i]), math.sin(robot.alpha[i])
        # Rz(th) Tz(d) Tx(a) Rx(alpha) as a rotation and a translation.
        L = np.zeros((N, 3, 3))
        L[:, 0, 0] = ct
        L[:, 0, 1] = -st * ca
        L[:, 0, 2] = st * sa
        L[:, 1, 0] = st
        L[:, 1, 1] = ct * ca
        L[:, 1, 2] = -ct * sa
        L[:, 2, 1] = sa
        L[:, 2, 2] = ca
        t = np.stack([robot.a[i] * ct, robot.a[i] * st, dd], axis=1)
        R[:, i + 1] = R[:, i] @ L
        o[:, i + 1] = o[:, i] + np.einsum("nij,nj->ni", R[:, i], t)
    return R, o


def sphere_centres(robot, q) -> np.ndarray:
    """World positions [N, N_s, 3] of the robot's collision spheres."""
    R, o = dh_frames(robot, q)
    f = robot.sphere_frame
    return np.einsum("nsij,sj->nsi", R[:, f], robot.sphere_xyz) + o[:, f]


def box_poses(robot, q):
    """World centres [N, B, 3] and rotations [N, B, 3, 3] (columns = box
    axes) of the robot's boxes."""
    R, o = dh_frames(robot, q)
    f = robot.box_frame
    c = np.einsum("nbij,bj->nbi", R[:, f], robot.box_xyz) + o[:, f]
    rot = np.einsum("nbij,bjk->nbik", R[:, f], robot.box_rot)
    return c, rot


def sphere_box_distance(c, r, bc, bR, bh):
    """Signed distance from a sphere (centre c, radius r) to an oriented box
    (centre bc, axes the columns of bR, half extents bh): the point's signed
    distance to the box minus r; broadcasts over leading dimensions. Outside
    the box the point distance is the norm of max(|p| - h, 0) with p the centre
    in box coordinates; inside it is the largest |p_i| - h_i (negative). The
    sphere and the box overlap iff the result is negative."""
    p = np.einsum("...ji,...j->...i", bR, c - bc)
    qv = np.abs(p) - bh
    outside = np.sqrt(np.sum(np.maximum(qv, 0.0) ** 2, axis=-1))
    inside = np.minimum(np.max(qv, axis=-1), 0.0)
    return outside + inside - r


BOX_EDGE_SKIP = 1e-4  # edge-edge axes with |a x b|^2 below this are not tested


def box_box_separation(ca, Ra, ha, cb, Rb, hb):
    """Separating-axis test of two oriented boxes (Gottschalk et al., OBBTree,
    SIGGRAPH'96): the largest over the candidate axes L (the three axes of
    each box and the nine cross products of one axis of each, normalised) of
    |(cb - ca) . L| - sum_k ha_k |a_k . L| - sum_k hb_k |b_k . L|. Cross
    products with |a x b|^2 < BOX_EDGE_SKIP (edges within ~0.6 degrees of
    parallel) are left out; the face axes cover those contacts up to a gap of
    edge length x 0.01. The boxes overlap iff the result is negative (then no
    axis separates them); when positive it is a lower bound of their
    distance. Broadcasts over leading dimensions."""
    T = cb - ca
    axes = [Ra[..., :, k] for k in range(3)] + [Rb[..., :, k] for k in range(3)]
    best = None
    cand = []
    for L in axes:
        cand.append((L, None))
    for i in range(3):
        for j in range(3):
            L = np.cross(Ra[..., :, i], Rb[..., :, j])
            n2 = np.sum(L * L, axis=-1)
            cand.append((L / np.sqrt(np.maximum(n2, 1e-300))[..., None], n2 >= BOX_EDGE_SKIP))
    for L, ok in cand:
        proj = np.abs(np.sum(T * L, axis=-1))
        ra = sum(ha[..., k] * np.abs(np.sum(Ra[..., :, k] * L, axis=-1)) for k in range(3))
        rb = sum(hb[..., k] * np.abs(np.sum(Rb[..., :, k] * L, axis=-1)) for k in range(3))
        sep = proj - ra - rb
        if ok is not None:
            sep = np.where(ok, sep, -np.inf)
        best = sep if best is None else np.maximum(best, sep)
    return best


def _box_pair_min(robot, env, c, rc, bc, bR):
    """Smallest pair value over the pairs that involve a box: robot spheres x
    obstacle boxes, robot boxes x obstacle spheres and boxes, and the listed
    sphere-box and box-box self pairs (sphere_box_distance and
    box_box_separation; negative iff that pair overlaps)."""
    N = c.shape[0]
    m = np.full(N, np.inf)
    eb = env.boxes if getattr(env, "boxes", None) is not None else np.zeros((0, 15))
    ec, eh, eR = eb[:, 0:3], eb[:, 3:6], eb[:, 6:15].reshape(-1, 3, 3)
    if c.shape[1] and eb.shape[0]:
        d = sphere_box_distance(c[:, :, None, :], rc[None, :, None], ec[None, None], eR[None, None], eh[None, None])
        m = np.minimum(m, d.min(axis=(1, 2)))
    if bc is not None and bc.shape[1]:
        bh = robot.box_half
        obs = np.asarray(env.spheres, dtype=np.float64)
        if obs.shape[0]:
            d = sphere_box_distance(obs[None, None, :, :3], obs[None, None, :, 3], bc[:, :, None, :],
                                    bR[:, :, None], bh[None, :, None, :])
            m = np.minimum(m, d.min(axis=(1, 2)))
        if eb.shape[0]:
            sep = box_box_separation(bc[:, :, None, :], bR[:, :, None], bh[None, :, None, :], ec[None, None],
                                     eR[None, None], eh[None, None])
            m = np.minimum(m, sep.min(axis=(1, 2)))
        sb = robot.self_sb if robot.self_sb is not None else np.zeros((0, 2), dtype=np.int32)
        if sb.shape[0]:
            d = sphere_box_distance(c[:, sb[:, 0]], rc[sb[:, 0]][None], bc[:, sb[:, 1]], bR[:, sb[:, 1]],
                                    bh[sb[:, 1]][None])
            m = np.minimum(m, d.min(axis=1))
        bbp = robot.self_bb if robot.self_bb is not None else np.zeros((0, 2), dtype=np.int32)
        if bbp.shape[0]:
            sep = box_box_separation(bc[:, bbp[:, 0]], bR[:, bbp[:, 0]], bh[bbp[:, 0]][None], bc[:, bbp[:, 1]],
                                     bR[:, bbp[:, 1]], bh[bbp[:, 1]][None])
            m = np.minimum(m, sep.min(axis=1))
    return m


def _has_boxes(robot, env) -> bool:
    return bool(getattr(robot, "n_boxes", 0)) or bool(getattr(env, "boxes", None) is not None and len(env.boxes))


def _chunks(N: int, size: int):
    for s in range(0, N, size):
        yield s, min(N, s + size)


def in_collision(robot, env, q, chunk: int = 512) -> np.ndarray:
    """Collision label per configuration: some robot sphere overlaps some
    obstacle sphere, or some listed self pair overlaps, i.e. a squared centre
    distance strictly below the squared sum of radii."""
    q = np.atleast_2d(np.asarray(q, dtype=np.float64))
    out = np.zeros(q.shape[0], dtype=bool)
    obs = np.asarray(env.spheres, dtype=np.float64)
    r = robot.sphere_r
    sp = robot.self_pairs
    for s, e in _chunks(q.shape[0], chunk):
        c = sphere_centres(robot, q[s:e])
        hit = np.zeros(e - s, dtype=bool)
        if obs.shape[0]:
            diff = c[:, :, None, :] - obs[None, None, :, :3]
            d2 = np.einsum("nsok,nsok->nso", diff, diff)
            rr = (r[:, None] + obs[None, :, 3]) ** 2
            hit |= (d2 < rr[None]).any(axis=(1, 2))
        if sp.shape[0]:
            diff = c[:, sp[:, 0]] - c[:, sp[:, 1]]
            d2 = np.einsum("npk,npk->np", diff, diff)
            hit |= (d2 < ((r[sp[:, 0]] + r[sp[:, 1]]) ** 2)[None]).any(axis=1)
        if _has_boxes(robot, env):
            bc, bR = box_poses(robot, q[s:e]) if getattr(robot, "n_boxes", 0) else (None, None)
            hit |= _box_pair_min(robot, env, c, r, bc, bR) < 0.0
        out[s:e] = hit
    return out


def signed_distance(robot, env, q, chunk: int = 512) -> np.ndarray:
    """Smallest ||c_i - c_j|| - r_i - r_j over all obstacle and self pairs
    (negative iff the configuration is in collision). Pairs with a box add
    sphere_box_distance (exact) and box_box_separation (its sign decides the
    label; when positive a lower bound of the distance)."""
    q = np.atleast_2d(np.asarray(q, dtype=np.float64))
    out = np.full(q.shape[0], np.inf)
    obs = np.asarray(env.spheres, dtype=np.float64)
    r = robot.sphere_r
    sp = robot.self_pairs
    for s, e in _chunks(q.shape[0], chunk):
        c = sphere_centres(robot, q[s:e])
        m = np.full(e - s, np.inf)
        if obs.shape[0] and c.shape[1]:
            diff = c[:, :, None, :] - obs[None, None, :, :3]
            dist = np.sqrt(np.einsum("nsok,nsok->nso", diff, diff))
            m = np.minimum(m, (dist - r[None, :, None] - obs[None, None, :, 3]).min(axis=(1, 2)))
        if sp.shape[0]:
            diff = c[:, sp[:, 0]] - c[:, sp[:, 1]]
            dist = np.sqrt(np.einsum("npk,npk->np", diff, diff))
            m = np.minimum(m, (dist - (r[sp[:, 0]] + r[sp[:, 1]])[None]).min(axis=1))
        if _has_boxes(robot, env):
            bc, bR = box_poses(robot, q[s:e]) if getattr(robot, "n_boxes", 0) else (None, None)
            m = np.minimum(m, _box_pair_min(robot, env, c, r, bc, bR))
        out[s:e] = m
    return out


# ---------------------------------------------------------------------------
# Distance to the seed segment L = conv{v1, v2}: Sec. IV-A, Eqs. (5)-(7).
# ---------------------------------------------------------------------------
def project_onto_segment(c, v1, v2) -> np.ndarray:
    """Eq. (6)/(7): c_proj = v1 if v1 = v2, else (1 - alpha) v1 + alpha v2 with
    alpha = min(max((c - v1)^T (v2 - v1) / ||v2 - v1||^2, 0), 1)."""
    c = np.atleast_2d(np.asarray(c, dtype=np.float64))
    v1 = np.asarray(v1, dtype=np.float64)
    v2 = np.asarray(v2, dtype=np.float64)
    e = v2 - v1
    ee = float(e @ e)
    if ee == 0.0:
        return np.broadcast_to(v1, c.shape).copy()
    alpha = np.clip(((c - v1) @ e) / ee, 0.0, 1.0)
    return (1.0 - alpha)[:, None] * v1 + alpha[:, None] * v2


def dist_to_segment(c, v1, v2) -> np.ndarray:
    """dist_L(c) = ||c - c_proj||_2 (the distance function of Sec. IV-A)."""
    c = np.atleast_2d(np.asarray(c, dtype=np.float64))
    return np.linalg.norm(c - project_onto_segment(c, v1, v2), axis=1)


def dist_gradient(c, v1, v2) -> np.ndarray:
    """Eq. (5): grad dist_L(c) = (c - c_proj) / ||c - c_proj||_2 (c not on L)."""
    c = np.atleast_2d(np.asarray(c, dtype=np.float64))
    g = c - project_onto_segment(c, v1, v2)
    return g / np.linalg.norm(g, axis=1, keepdims=True)


# ---------------------------------------------------------------------------
# Round size and the unadaptive test: Sec. IV-B, Eq. (9).
# ---------------------------------------------------------------------------
def delta_k(k: int, delta: float) -> float:
    """Eq. (9): delta_k = 6 delta / (pi^2 k^2)."""
    return 6.0 * delta / (math.pi ** 2 * k * k)


def test_size(k: int, eps: float, delta: float, tau: float) -> int:
    """M = ceil(2 log(1/delta_k) / (eps tau^2)) (natural log)."""
    return int(math.ceil(2.0 * math.log(1.0 / delta_k(k, delta)) / (eps * tau * tau)))


def batch_size(k: int, eps: float, delta: float, tau: float, n_p: int) -> int:
    """|S| = max(N_p, M)."""
    return max(int(n_p), test_size(k, eps, delta, tau))


def unadaptive_test(n_col_first_m: int, m: int, eps: float, tau: float) -> bool:
    """Accept iff the number of collisions among the first M samples is at
    most M (1 - tau) eps."""
    return float(n_col_first_m) <= m * (1.0 - tau) * eps


# ---------------------------------------------------------------------------
# Hit-and-run sampling (Sec. IV-B "UniformSample", Sec. IV-D: one walk per
# sample, accepted after a fixed number of mixing steps).
# ---------------------------------------------------------------------------
def hit_and_run(A, b, v1, v2, n_samples: int, n_mix: int, seed: int, stream: int, k: int,
                first_walk: int = 0) -> np.ndarray:
    """Samples [n_samples, n] of walks ``first_walk ..`` at round ``k``.

    Walk j draws Philox blocks with counter (j, draw, k, stream):
    draw 0 gives the start u (word 0): x = v1 + u (v2 - v1);
    step s uses draws 1 + s W .. 1 + s W + W - 1 (W = blocks_per_step(n)),
    whose words in order are w_0, w_1, ...; Gaussian pair i is
    sqrt(-2 ln u'(w_{2i})) (cos, sin)(2 pi u(w_{2i+1})) from the top 24 bits
    (u' in (0, 1], u in [0, 1)); the direction is the first n Gaussians
    normalised; the step is t = t_lo + u_t (t_hi - t_lo) on the chord of P
    through x, u_t = step_uniform(w_0, w_1, w_2) from the low bytes.
    """
    A = np.asarray(A, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    v1 = np.asarray(v1, dtype=np.float64)
    v2 = np.asarray(v2, dtype=np.float64)
    n = v1.shape[0]
    key = seed_key(seed)
    W = blocks_per_step(n)
    npair = (n + 1) // 2
    j = np.arange(first_walk, first_walk + n_samples, dtype=np.uint64)

    def draw(d):
        ctr = np.stack([j, np.full_like(j, d), np.full_like(j, k), np.full_like(j, stream)], axis=1)
        return philox4x32_10(ctr, key)

    u0 = u01_closed_open(draw(0)[:, 0])
    x = v1[None, :] + u0[:, None] * (v2 - v1)[None, :]
    for s in range(n_mix):
        words = np.concatenate([draw(1 + s * W + w) for w in range(W)], axis=1)
        z = np.empty((n_samples, 2 * npair))
        for i in range(npair):
            rho = np.sqrt(-2.0 * np.log(u01_open_closed(words[:, 2 * i])))
            phi = 2.0 * math.pi * u01_closed_open(words[:, 2 * i + 1])
            z[:, 2 * i] = rho * np.cos(phi)
            z[:, 2 * i + 1] = rho * np.sin(phi)
        dvec = z[:, :n]
        nrm = np.linalg.norm(dvec, axis=1)
        ok = nrm > 0.0
        dvec = np.where(ok[:, None], dvec / np.where(ok, nrm, 1.0)[:, None], 0.0)
        ut = step_uniform(words[:, 0], words[:, 1], words[:, 2])
        slack = b[None, :] - x @ A.T
        qd = dvec @ A.T
        with np.errstate(divide="ignore", invalid="ignore"):
            ratio = slack / qd
        t_hi = np.where(qd > 0.0, ratio, np.inf).min(axis=1)
        t_lo = np.where(qd < 0.0, ratio, -np.inf).max(axis=1)
        t_hi = np.maximum(t_hi, 0.0)
        t_lo = np.minimum(t_lo, 0.0)
        move = ok & np.isfinite(t_hi) & np.isfinite(t_lo) & ((t_hi - t_lo) >= 1e-12)
        t = np.where(move, t_lo + ut * (t_hi - t_lo), 0.0)
        x = x + t[:, None] * dvec
    return x


# ---------------------------------------------------------------------------
# Bisection toward the segment (Sec. IV-B "UpdatePointsViaBisection",
# Sec. IV-C "Choosing the number of bisection steps").
# ---------------------------------------------------------------------------
@dataclass
class BisectResult:
    c_star: np.ndarray  # [N, n]
    decisions: np.ndarray  # [N, n_b] bool, True = midpoint in collision
    ambiguous: int = 0  # decisions taken from the caller inside the band


def bisect(robot, env, c, v1, v2, n_b: int, follow=None, band: float = 0.0) -> BisectResult:
    """From each colliding sample c, bisect the segment [c_proj, c] N_b times
    keeping the colliding end (c_proj is free because L is collision-free).

    ``follow`` ([N, n_b] bool) makes the oracle take the caller's decision at
    midpoints whose signed distance lies within ``band`` of zero (replay of a
    run whose collision checks use another precision)."""
    c = np.atleast_2d(np.asarray(c, dtype=np.float64))
    lo = project_onto_segment(c, v1, v2)
    hi = c.copy()
    dec = np.zeros((c.shape[0], n_b), dtype=bool)
    amb = 0
    for s in range(n_b):
        mid = 0.5 * (lo + hi)
        col = in_collision(robot, env, mid)
        if follow is not None and band > 0.0:
            sd = signed_distance(robot, env, mid)
            near = np.abs(sd) < band
            amb += int(np.count_nonzero(near & (col != follow[:, s])))
            col = np.where(near, follow[:, s], col)
        dec[:, s] = col
        hi = np.where(col[:, None], mid, hi)
        lo = np.where(col[:, None], lo, mid)
    return BisectResult(c_star=hi, decisions=dec, ambiguous=amb)


# ---------------------------------------------------------------------------
# Ordering and placing hyperplanes (Sec. IV-B "OrderAndPlaceHyperplanes",
# Eq. (10); step back Sec. IV-C, Eqs. (11)-(12); t_col, Sec. IV-C).
# ---------------------------------------------------------------------------
STATUS_OK = 0
STATUS_SEGMENT_IN_COLLISION = 2


@dataclass
class PlaceResult:
    rows_a: np.ndarray  # [H, n]
    rows_b: np.ndarray  # [H] (already b_i - Delta_i)
    order: list = field(default_factory=list)  # candidate indices that received a plane
    deltas: list = field(default_factory=list)
    status: int = STATUS_OK


def place_hyperplanes(c_star, sample_index, v1, v2, n_f: int, step_back_max: float,
                      t_col: float) -> PlaceResult:
    """Sort candidates by (dist_L(c*), sample index); walk them in order; each
    one still inside the polytope gets the half space a^T x <= b - Delta with
    a = grad dist_L(c*), b = a^T c*, r = max(a^T v1, a^T v2) - b + Delta_max,
    Delta = Delta_max - r if r > 0 else Delta_max; candidates with
    a^T c_j > b - Delta are discarded; at most n_f planes. A candidate with
    dist_L <= t_col stops the round with "segment likely in collision"."""
    c_star = np.atleast_2d(np.asarray(c_star, dtype=np.float64))
    v1 = np.asarray(v1, dtype=np.float64)
    v2 = np.asarray(v2, dtype=np.float64)
    N, n = c_star.shape
    dist = dist_to_segment(c_star, v1, v2) if N else np.zeros(0)
    order = np.lexsort((np.asarray(sample_index), dist)) if N else np.zeros(0, dtype=int)
    alive = np.ones(N, dtype=bool)
    rows_a, rows_b, used, deltas = [], [], [], []
    for i in order:
        if len(rows_a) == n_f:
            break
        if not alive[i]:
            continue
        if dist[i] <= t_col:
            return PlaceResult(np.asarray(rows_a).reshape(-1, n), np.asarray(rows_b), used, deltas,
                               STATUS_SEGMENT_IN_COLLISION)
        a = dist_gradient(c_star[i], v1, v2)[0]
        bb = float(a @ c_star[i])
        r = max(float(a @ v1), float(a @ v2)) - bb + step_back_max
        delta = step_back_max - r if r > 0.0 else step_back_max
        rows_a.append(a)
        rows_b.append(bb - delta)
        used.append(int(i))
        deltas.append(delta)
        alive &= ~((c_star @ a) > bb - delta)
    return PlaceResult(np.asarray(rows_a).reshape(-1, n), np.asarray(rows_b), used, deltas, STATUS_OK)


# ---------------------------------------------------------------------------
# One EI-ZO iteration and the full loop (Algorithm 1).
# ---------------------------------------------------------------------------
@dataclass
class Params:
    eps: float = 0.05
    delta: float = 0.05
    tau: float = 0.5
    step_back_max: float = 0.01
    t_col: float = 1e-3
    n_p: int = 10000
    n_f: int = 10
    n_b: int = 10
    n_mix: int = 60
    n_it_max: int = 50
    seed: int = 1


@dataclass
class RoundResult:
    k: int
    m_test: int
    n_samples: int
    n_col_first_m: int
    accept: bool
    cand_index: np.ndarray  # sample indices of the candidates, ascending
    c_star: np.ndarray
    decisions: np.ndarray
    place: PlaceResult | None
    ambiguous: int = 0


def eizo_round(robot, env, A, b, v1, v2, k: int, prm: Params, samples, labels=None,
               follow=None, band: float = 0.0) -> RoundResult:
    """Lines of Algorithm 1 after sampling, for given samples S: labels,
    unadaptive test on the first M, the first N_p colliding samples, their
    projection and bisection, and hyperplane placement."""
    S = np.atleast_2d(np.asarray(samples, dtype=np.float64))
    m = test_size(k, prm.eps, prm.delta, prm.tau)
    col = in_collision(robot, env, S) if labels is None else np.asarray(labels, dtype=bool)
    n_col_m = int(np.count_nonzero(col[:m]))
    if unadaptive_test(n_col_m, m, prm.eps, prm.tau):
        return RoundResult(k, m, S.shape[0], n_col_m, True, np.zeros(0, dtype=np.int64),
                           np.zeros((0, S.shape[1])), np.zeros((0, prm.n_b), dtype=bool), None)
    idx = np.nonzero(col)[0][: prm.n_p]
    br = bisect(robot, env, S[idx], v1, v2, prm.n_b, follow=follow, band=band)
    pl = place_hyperplanes(br.c_star, idx, v1, v2, prm.n_f, prm.step_back_max, prm.t_col)
    return RoundResult(k, m, S.shape[0], n_col_m, False, idx, br.c_star, br.decisions, pl,
                       br.ambiguous)


@dataclass
class EizoResult:
    A: np.ndarray
    b: np.ndarray
    rounds: int
    status: int  # 0 ok, 2 segment in collision, 6 iteration cap reached
    planes: int
    checks: int  # exact collision checks performed


STATUS_MAX_ITER = 6


def eizo(robot, env, v1, v2, A0, b0, prm: Params, stream: int = 0) -> EizoResult:
    """Algorithm 1: P <- D; repeat sample / label / test / project / bisect /
    place until the test accepts, the segment is reported in collision, or
    N_it rounds ran (Sec. IV-C "Maximum iterations")."""
    A = np.asarray(A0, dtype=np.float64).copy()
    b = np.asarray(b0, dtype=np.float64).copy()
    checks = 0
    planes = 0
    for k in range(1, prm.n_it_max + 1):
        ns = batch_size(k, prm.eps, prm.delta, prm.tau, prm.n_p)
        S = hit_and_run(A, b, v1, v2, ns, prm.n_mix, prm.seed, stream, k)
        rr = eizo_round(robot, env, A, b, v1, v2, k, prm, S)
        checks += ns + rr.cand_index.shape[0] * prm.n_b
        if rr.accept:
            return EizoResult(A, b, k, STATUS_OK, planes, checks)
        pl = rr.place
        if pl.rows_a.shape[0]:
            A = np.vstack([A, pl.rows_a])
            b = np.concatenate([b, pl.rows_b])
            planes += pl.rows_a.shape[0]
        if pl.status != STATUS_OK:
            return EizoResult(A, b, k, pl.status, planes, checks)
    return EizoResult(A, b, prm.n_it_max, STATUS_MAX_ITER, planes, checks)


def joint_box(robot) -> tuple[np.ndarray, np.ndarray]:
    """The usual domain D: the joint-limit box as 2n half spaces
    (rows +e_i <= q_hi_i, then -e_i <= -q_lo_i)."""
    n = robot.n
    A = np.vstack([np.eye(n), -np.eye(n)])
    b = np.concatenate([robot.q_hi, -robot.q_lo])
    return A, b


def segment_contained(A, b, v1, v2, tol: float = 1e-9) -> bool:
    """Both endpoints of L satisfy A x <= b + tol (then all of L does, by
    convexity of the polytope)."""
    A = np.asarray(A)
    b = np.asarray(b)
    return bool(np.all(A @ v1 <= b + tol) and np.all(A @ v2 <= b + tol))


def inflate_path(robot, env, verts, prm: Params, A0=None, b0=None, stream_base: int = 0):
    """Sec. VI-A: inflate L_0 .. L_{K-1} in order, skipping L_k when an earlier
    polytope already contains it. Segment k draws its samples from stream
    ``stream_base + k``. Returns (list of (segment index, EizoResult), kept)."""
    verts = np.asarray(verts, dtype=np.float64)
    if A0 is None:
        A0, b0 = joint_box(robot)
    out = []
    for k in range(verts.shape[0] - 1):
        v1, v2 = verts[k], verts[k + 1]
        if any(segment_contained(r.A, r.b, v1, v2) for _, r in out):
            continue
        res = eizo(robot, env, v1, v2, A0, b0, prm, stream=stream_base + k)
        out.append((k, res))
        if res.status == STATUS_SEGMENT_IN_COLLISION:
            break
    return out


# ---------------------------------------------------------------------------
# Recovering from detected collisions (Sec. VI-B): a path or trajectory is
# checked at fine steps; the collisions that lie in a set are excluded from
# it with the last steps of Algorithm 1 (bisection, ordering, placement);
# then every segment of the seed path must still lie in some set, and a
# segment that does not is inflated again.
# ---------------------------------------------------------------------------
def path_points(verts, step: float):
    """Fine discretisation of a piecewise-linear path (Sec. VI-B; the
    appendix uses steps of 0.1 rad). Edge k, from v_k to v_{k+1}, is cut into
    N_k = max(1, ceil(|v_{k+1} - v_k|_2 / step)) equal pieces and its N_k + 1
    points v_k + (i / N_k)(v_{k+1} - v_k), i = 0..N_k, are checked (both
    ends, so a shared vertex is checked by both of its edges). |e|_2 is the
    square root of e_0^2 + e_1^2 + .. summed in that order.
    Returns (points [N, n], edge index of each point [N])."""
    verts = np.atleast_2d(np.asarray(verts, dtype=np.float64))
    pts, eid = [], []
    for k in range(verts.shape[0] - 1):
        e = verts[k + 1] - verts[k]
        ss = 0.0
        for x in e:
            ss += float(x) * float(x)
        nk = max(1, int(math.ceil(math.sqrt(ss) / step)))
        for i in range(nk + 1):
            pts.append(verts[k] + (i / nk) * e)
            eid.append(k)
    n = verts.shape[1]
    return np.asarray(pts, dtype=np.float64).reshape(-1, n), np.asarray(eid, dtype=np.int64)


def check_path(robot, env, verts, step: float):
    """Labels of the points of path_points and, per edge, whether any of its
    points collides. Returns (edge flags [K] bool, point labels [N] bool,
    points [N, n], edge index [N])."""
    P, eid = path_points(verts, step)
    lab = in_collision(robot, env, P) if P.shape[0] else np.zeros(0, dtype=bool)
    K = max(0, np.atleast_2d(verts).shape[0] - 1)
    edge = np.zeros(K, dtype=bool)
    for i in range(P.shape[0]):
        if lab[i]:
            edge[eid[i]] = True
    return edge, lab, P, eid


def points_inside(A, b, X, tol: float = 1e-9) -> np.ndarray:
    """Rows of X that satisfy A x <= b + tol."""
    X = np.atleast_2d(np.asarray(X, dtype=np.float64))
    A = np.asarray(A, dtype=np.float64)
    if A.shape[0] == 0:
        return np.ones(X.shape[0], dtype=bool)
    return np.all(X @ A.T <= np.asarray(b)[None, :] + tol, axis=1)


@dataclass
class EditResult:
    A: np.ndarray
    b: np.ndarray
    inside: np.ndarray  # [N] bool, the given configuration lies in P
    labels: np.ndarray  # [N] bool, in collision
    cand_index: np.ndarray  # indices of the configurations that were bisected
    bisect: BisectResult
    place: PlaceResult


def edit_polytope(robot, env, A, b, v1, v2, cfgs, prm: Params, follow=None, band: float = 0.0) -> EditResult:
    """Sec. VI-B set editing: the given configurations that lie in P
    (A c <= b + 1e-9) and collide form S_col; the first N_p of them by index
    are bisected toward the seed segment L = [v1, v2] and ordered, and
    hyperplanes are placed exactly as in a round of Algorithm 1 (no sampling
    and no test). The new rows are appended to P."""
    X = np.atleast_2d(np.asarray(cfgs, dtype=np.float64))
    inside = points_inside(A, b, X)
    lab = in_collision(robot, env, X) if X.shape[0] else np.zeros(0, dtype=bool)
    idx = np.nonzero(inside & lab)[0][: prm.n_p]
    br = bisect(robot, env, X[idx], v1, v2, prm.n_b, follow=follow, band=band)
    pl = place_hyperplanes(br.c_star, idx, v1, v2, prm.n_f, prm.step_back_max, prm.t_col)
    A2 = np.vstack([np.asarray(A, dtype=np.float64), pl.rows_a])
    b2 = np.concatenate([np.asarray(b, dtype=np.float64), pl.rows_b])
    return EditResult(A2, b2, inside, lab, idx, br, pl)


def path_coverage(polys, verts, tol: float = 1e-9) -> np.ndarray:
    """Sec. VI-B: segment k of the seed path is covered when both of its
    endpoints lie in one of the polytopes (A x <= b + tol), hence the whole
    segment, by convexity. ``polys`` is a list of (A, b). Returns [K] bool."""
    verts = np.atleast_2d(np.asarray(verts, dtype=np.float64))
    K = verts.shape[0] - 1
    out = np.zeros(K, dtype=bool)
    for k in range(K):
        out[k] = any(segment_contained(A, b, verts[k], verts[k + 1], tol) for A, b in polys)
    return out
