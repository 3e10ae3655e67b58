"""Write tests/golden/workloads.json: the seeded synthetic scenes whose
collision-freeness needs a collision checker, checked by the FP64 oracle only.

* planar3 scene: one seed segment L between two collision-free configurations
  and 16 obstacle disks (centres uniform in [-2.5, 2.5]^2, r in [0.1, 0.3])
  drawn one by one and rejected when they come within ``margin`` of the arm
  anywhere along L.
* dh7 scene: 64 obstacle spheres in the 1 m cube 0.5 m ahead of the base and
  a 10-segment seed path from a random walk of 0.5 rad steps inside 0.8x the
  joint limits that starts near the obstacles and, of 24 collision-free
  candidate steps, keeps the one closest to them; every segment is checked at
  <= 0.005 rad spacing and kept only when the oracle's signed distance is
  >= ``margin`` at every check point (the margin bounds how far the arm moves
  between check points, so the whole segment is collision-free).
* dh7 batched scenes: 8 obstacle sets of 128-1024 spheres in the same cube
  and 256 seed paths of 1-40 segments built the same way (written only when
  ``--batched`` is given; slower).
* forest scene: the point robot among 15 disks (Sec. V) and a seed path from
  the bottom left to the top right corner (``--only-forest`` rewrites it).
* boxes scene: the 11-box arm over a table-top scene with boxes and voxel
  spheres and an 8-segment seed path (``--only-boxes``).
* table_cloud scene: 1024 spheres of r = 0.02 from a synthetic table point
  cloud and a 64-segment seed path that runs close to them (of 12
  collision-free candidate steps the one with the least clearance)
  (``--stress``).

Run from the repository root:  python tests/golden/make_workloads.py
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import ezo_oracle as orc  # noqa: E402
from paper_2504_10783_gb300 import workloads as wl  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "workloads.json")


def segment_clearance(robot, env, v1, v2, spacing=0.005):
    n = max(2, int(math.ceil(np.linalg.norm(v2 - v1) / spacing)) + 1)
    t = np.linspace(0.0, 1.0, n)[:, None]
    q = (1.0 - t) * v1 + t * v2
    return float(orc.signed_distance(robot, env, q).min())


def planar_scene(seed=7, n_obs=16, margin=0.03):
    robot = wl.planar3_robot()
    rng = np.random.default_rng(seed)
    empty = wl.Env("none", np.zeros((0, 4)))
    while True:
        v1 = rng.uniform(0.8 * robot.q_lo, 0.8 * robot.q_hi)
        step = rng.standard_normal(3)
        v2 = np.clip(v1 + 1.2 * step / np.linalg.norm(step), 0.8 * robot.q_lo, 0.8 * robot.q_hi)
        if segment_clearance(robot, empty, v1, v2) >= margin:
            break
    t = np.linspace(0.0, 1.0, 400)[:, None]
    swept = orc.sphere_centres(robot, (1.0 - t) * v1 + t * v2).reshape(-1, 3)
    obs = []
    cand_seed = seed * 1000
    while len(obs) < n_obs:
        cand = wl.planar_disks_candidates(cand_seed, 64)
        cand_seed += 1
        for o in cand:
            d = np.linalg.norm(swept[:, :2] - o[None, :2], axis=1) - 0.1 - o[3]
            if d.min() >= margin:
                obs.append(o)
                if len(obs) == n_obs:
                    break
    env = wl.Env("planar_disks", np.asarray(obs))
    assert segment_clearance(robot, env, v1, v2) >= margin
    return {"robot": "planar3", "v1": v1.tolist(), "v2": v2.tolist(), "obstacles": env.spheres.tolist(),
            "seed": seed, "margin": margin}


def random_path(robot, env, rng, n_seg, step=0.5, margin=0.02, tries=400, hug=0):
    """Random walk of `step` rad inside 0.8x the limits. With hug > 0 the walk
    starts near the obstacles (clearance in [2 margin, 4 margin]) and each step
    keeps, of `hug` collision-free candidates, the one with the least
    clearance, so the path runs close to the obstacles."""
    while True:
        v = rng.uniform(0.8 * robot.q_lo, 0.8 * robot.q_hi)
        sd0 = orc.signed_distance(robot, env, v[None])[0]
        if sd0 >= 2 * margin and (not hug or sd0 <= 4 * margin):
            break
    verts = [v]
    while len(verts) < n_seg + 1:
        best, best_c, found = None, np.inf, 0
        for _ in range(tries):
            nxt = wl.random_walk_waypoints(rng, robot, verts[-1], step)
            c = segment_clearance(robot, env, verts[-1], nxt)
            if c < margin:
                continue
            if not hug:
                best = nxt
                break
            found += 1
            if c < best_c:
                best, best_c = nxt, c
            if found >= hug:
                break
        if best is None:
            return None
        verts.append(best)
    return np.asarray(verts)


def dh7_scene(seed=11, n_obs=64, n_seg=10):
    robot = wl.dh7_robot()
    env = wl.box_obstacles(seed, n_obs)
    rng = np.random.default_rng(seed + 1)
    path = None
    while path is None:
        path = random_path(robot, env, rng, n_seg, hug=24)
    return {"robot": "dh7", "env_seed": seed, "n_obs": n_obs, "path": path.tolist()}


def batched_scenes(seed=21, n_env=8, n_paths=256):
    robot = wl.dh7_robot()
    rng = np.random.default_rng(seed)
    envs = []
    for e in range(n_env):
        cnt = int(rng.integers(128, 1025))
        envs.append({"env_seed": seed * 100 + e, "n_obs": cnt})
    paths = []
    for p in range(n_paths):
        e = int(rng.integers(0, n_env))
        env = wl.box_obstacles(envs[e]["env_seed"], envs[e]["n_obs"])
        nseg = int(rng.integers(1, 41))
        path = None
        while path is None:
            path = random_path(robot, env, rng, nseg)
        paths.append({"env": e, "path": path.tolist()})
        print(f"batched path {p}: env {e}, {nseg} segments", flush=True)
    return {"robot": "dh7", "envs": envs, "paths": paths}


def stress_scene(seed=31, n_seg=64):
    robot = wl.dh7_robot()
    env = wl.table_cloud_obstacles(seed)
    rng = np.random.default_rng(seed + 1)
    path = None
    while path is None:
        path = random_path(robot, env, rng, n_seg, hug=12)
    return {"robot": "dh7", "cloud_seed": seed, "path": path.tolist()}


def forest_scene(seed=41, step=1.0, margin=0.02, max_steps=80):
    """Forest of Sec. V (15 disks of r = 0.35 in the central 7 x 7 square of
    the 10 x 10 domain, point robot): a seed path from (0.5, 0.5) toward
    (9.5, 9.5) in steps of ``step`` whose heading is the goal direction plus
    N(0, 0.6) rad noise, each segment kept when its clearance (checked every
    0.005) is at least ``margin``; the goal is appended once it is in reach
    by a collision-free segment."""
    robot = wl.point2_robot()
    env = wl.forest_obstacles(seed)
    rng = np.random.default_rng(seed + 1)
    goal = np.array([9.5, 9.5])
    verts = [np.array([0.5, 0.5])]
    for _ in range(max_steps):
        cur = verts[-1]
        if np.linalg.norm(goal - cur) <= 1.5 and segment_clearance(robot, env, cur, goal) >= margin:
            verts.append(goal)
            break
        for _ in range(200):
            phi = math.atan2(*(goal - cur)[::-1]) + rng.normal(0.0, 0.6)
            nxt = np.clip(cur + step * np.array([math.cos(phi), math.sin(phi)]), 0.2, 9.8)
            if segment_clearance(robot, env, cur, nxt) >= margin:
                verts.append(nxt)
                break
    assert np.allclose(verts[-1], goal)
    return {"robot": "point2", "forest_seed": seed, "path": np.asarray(verts).tolist()}


def box_scene(seed=51, n_seg=8):
    """Box geometries (Sec. IV-D, VII): the 11-box arm over a table-top scene
    (table, two boxes, voxel spheres) and an 8-segment seed path that keeps,
    of 8 collision-free candidate steps, the one with the least clearance."""
    robot = wl.box_arm_robot()
    env = wl.tabletop_box_env(seed)
    rng = np.random.default_rng(seed + 1)
    path = None
    while path is None:
        path = random_path(robot, env, rng, n_seg, hug=8)
    return {"robot": "box_arm", "env_seed": seed, "path": path.tolist()}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--batched", action="store_true")
    ap.add_argument("--stress", action="store_true")
    ap.add_argument("--only-stress", action="store_true", help="rewrite only the table_cloud scene")
    ap.add_argument("--only-forest", action="store_true", help="rewrite only the forest scene")
    ap.add_argument("--only-boxes", action="store_true", help="rewrite only the box scene")
    args = ap.parse_args()
    data = {}
    if os.path.exists(OUT):
        with open(OUT) as f:
            data = json.load(f)
    only = args.only_stress or args.only_forest or args.only_boxes
    if not only:
        data["planar3"] = planar_scene()
        data["dh7"] = dh7_scene()
    if not only or args.only_forest:
        data["forest"] = forest_scene()
    if not only or args.only_boxes:
        data["boxes"] = box_scene()
    if args.batched:
        data["dh7_batched"] = batched_scenes()
    if args.stress or args.only_stress:
        data["table_cloud"] = stress_scene()
    with open(OUT, "w") as f:
        json.dump(data, f, indent=1)
    print("wrote", OUT)


if __name__ == "__main__":
    main()
