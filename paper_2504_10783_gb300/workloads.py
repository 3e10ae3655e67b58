"""Seeded synthetic inputs: robot models, obstacle sets and candidate waypoints.

This module only builds input data (kinematic parameters, sphere placements,
obstacle spheres, random waypoints). It contains none of the edge-inflation
arithmetic: no forward kinematics, no collision test, no sampling, no
hyperplane placement. Both the CUDA path and the FP64 oracle consume what it
returns, so it must stay free of either side's computation.

The paper assumes a robot description with kinematics and collision geometry
(Sec. II) and obstacles given as spheres around perceived voxels (Sec. V-B).
Its own robot models (FR3, iiwa) are not published, so the workloads here are
synthetic stand-ins with the same structure:

* ``planar3`` - planar 3-link revolute arm, links of 1.0 m, 4 spheres of
  r = 0.1 m per link, self pairs between links 1 and 3 only.
* ``dh7`` - 7-DOF serial arm in standard DH form, 40 spheres along the four
  links with non-zero offset d, radii tapering from 0.08 m to 0.04 m, self
  pairs between all non-adjacent sphere-carrying links.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "Robot",
    "Env",
    "planar3_robot",
    "dh7_robot",
    "planar_disks_candidates",
    "box_obstacles",
    "table_cloud_obstacles",
    "uniform_configs",
    "random_walk_waypoints",
    "point2_robot",
    "forest_obstacles",
    "rot_zyx",
    "box_row",
    "box_arm_robot",
    "tabletop_box_env",
]


@dataclasses.dataclass
class Robot:
    """Serial chain in standard DH form with spheres fixed to its frames.

    Frame 0 is the base (identity). Frame i (1..n) is
    T_i = T_{i-1} Rz(q_i + theta_off_i) Tz(d_i) Tx(a_i) Rx(alpha_i)
    for a revolute joint (``joint_type[i-1] == 0``, the default) and
    T_i = T_{i-1} Rz(theta_off_i) Tz(d_i + q_i) Tx(a_i) Rx(alpha_i)
    for a prismatic one (``joint_type[i-1] == 1``).
    Sphere s sits at ``sphere_xyz[s]`` in frame ``sphere_frame[s]`` with radius
    ``sphere_r[s]``; ``sphere_link`` is a link id used only to build self pairs.
    Box k (optional) sits in frame ``box_frame[k]`` with centre ``box_xyz[k]``,
    axes the columns of ``box_rot[k]`` and half extents ``box_half[k]``.
    """

    name: str
    a: np.ndarray
    alpha: np.ndarray
    d: np.ndarray
    theta_off: np.ndarray
    q_lo: np.ndarray
    q_hi: np.ndarray
    sphere_frame: np.ndarray  # int32 [N_s]
    sphere_xyz: np.ndarray  # float64 [N_s, 3]
    sphere_r: np.ndarray  # float64 [N_s]
    sphere_link: np.ndarray  # int32 [N_s]
    self_pairs: np.ndarray  # int32 [P, 2]
    joint_type: np.ndarray | None = None  # int32 [n]: 0 revolute, 1 prismatic; None = all revolute
    # oriented boxes fixed to frames: centre in the frame, rotation (columns =
    # box axes in the frame), half extents; self pairs sphere x box, box x box
    box_frame: np.ndarray | None = None  # int32 [B]
    box_xyz: np.ndarray | None = None  # float64 [B, 3]
    box_rot: np.ndarray | None = None  # float64 [B, 3, 3]
    box_half: np.ndarray | None = None  # float64 [B, 3]
    self_sb: np.ndarray | None = None  # int32 [P, 2] (sphere, box)
    self_bb: np.ndarray | None = None  # int32 [P, 2] (box, box)

    @property
    def n_boxes(self) -> int:
        return 0 if self.box_frame is None else int(len(self.box_frame))

    @property
    def prismatic(self) -> np.ndarray:
        if self.joint_type is None:
            return np.zeros(self.n, dtype=bool)
        return np.asarray(self.joint_type) == 1

    @property
    def n(self) -> int:
        return int(self.a.shape[0])

    @property
    def n_spheres(self) -> int:
        return int(self.sphere_r.shape[0])

    def to_json(self) -> dict:
        return {k: (v.tolist() if isinstance(v, np.ndarray) else v)
                for k, v in dataclasses.asdict(self).items()}

    @staticmethod
    def from_json(d: dict) -> "Robot":
        ints = {"sphere_frame", "sphere_link", "self_pairs"}
        kw = {}
        for f in dataclasses.fields(Robot):
            v = d.get(f.name)
            if v is None:
                continue
            if f.name == "name":
                kw[f.name] = v
            elif f.name in ints or f.name == "joint_type":
                kw[f.name] = np.asarray(v, dtype=np.int32).reshape(-1, 2) if f.name == "self_pairs" \
                    else np.asarray(v, dtype=np.int32)
            else:
                kw[f.name] = np.asarray(v, dtype=np.float64)
        kw["sphere_xyz"] = kw["sphere_xyz"].reshape(-1, 3)
        for k in ("box_frame",):
            if k in kw:
                kw[k] = kw[k].astype(np.int32)
        for k in ("self_sb", "self_bb"):
            if k in kw:
                kw[k] = kw[k].astype(np.int32).reshape(-1, 2)
        if "box_xyz" in kw:
            kw["box_xyz"] = kw["box_xyz"].reshape(-1, 3)
            kw["box_rot"] = kw["box_rot"].reshape(-1, 3, 3)
            kw["box_half"] = kw["box_half"].reshape(-1, 3)
        return Robot(**kw)


@dataclasses.dataclass
class Env:
    """Obstacle spheres, one row (x, y, z, radius) each, and optional oriented
    boxes, one row (centre x, y, z, half extents hx, hy, hz, rotation R row
    major, 9 entries; the columns of R are the box axes in the world)."""

    name: str
    spheres: np.ndarray  # float64 [N_obs, 4]
    boxes: np.ndarray | None = None  # float64 [N_box, 15]

    @property
    def n_boxes(self) -> int:
        return 0 if self.boxes is None else int(self.boxes.shape[0])

    @property
    def n_obs(self) -> int:
        return int(self.spheres.shape[0])


def _pairs_between_links(link: np.ndarray, link_pairs) -> np.ndarray:
    out = []
    for la, lb in link_pairs:
        ia = np.nonzero(link == la)[0]
        ib = np.nonzero(link == lb)[0]
        for i in ia:
            for j in ib:
                out.append((int(i), int(j)))
    return np.asarray(out, dtype=np.int32).reshape(-1, 2)


def planar3_robot(link_len: float = 1.0, spheres_per_link: int = 4, r: float = 0.1) -> Robot:
    """Planar 3R arm: DH a_i = link_len, alpha = d = 0, limits [-pi, pi]^3.

    With standard DH, frame i sits at the distal end of link i and its x axis
    runs along the link, so a sphere a fraction f along link i (from the
    proximal joint) is the point ((f - 1) * link_len, 0, 0) of frame i.
    Spheres sit at f = (j + 0.5) / spheres_per_link.
    """
    n = 3
    frames, xyz, rad, link = [], [], [], []
    for i in range(1, n + 1):
        for j in range(spheres_per_link):
            f = (j + 0.5) / spheres_per_link
            frames.append(i)
            xyz.append(((f - 1.0) * link_len, 0.0, 0.0))
            rad.append(r)
            link.append(i)
    link = np.asarray(link, dtype=np.int32)
    return Robot(
        name="planar3",
        a=np.full(n, link_len), alpha=np.zeros(n), d=np.zeros(n), theta_off=np.zeros(n),
        q_lo=np.full(n, -math.pi), q_hi=np.full(n, math.pi),
        sphere_frame=np.asarray(frames, dtype=np.int32),
        sphere_xyz=np.asarray(xyz, dtype=np.float64),
        sphere_r=np.asarray(rad, dtype=np.float64),
        sphere_link=link,
        self_pairs=_pairs_between_links(link, [(1, 3)]),
    )


DH7_D = (0.34, 0.0, 0.40, 0.0, 0.40, 0.0, 0.126)
DH7_ALPHA = (-math.pi / 2, math.pi / 2, math.pi / 2, -math.pi / 2, -math.pi / 2, math.pi / 2, 0.0)
DH7_LIMITS = (2.9, 2.0, 2.9, 2.0, 2.9, 2.0, 3.0)
DH7_SPHERES_PER_LINK = (11, 13, 12, 4)


def dh7_robot(r_base: float = 0.08, r_tip: float = 0.04) -> Robot:
    """7-DOF arm, standard DH with a = 0.

    Joint i with d_i != 0 (i = 1, 3, 5, 7) carries a link from the origin of
    frame i-1 to the origin of frame i along the z axis of frame i-1, i.e. the
    points (0, 0, f d_i) of frame i-1. The four links get 11, 13, 12 and 4
    spheres at f = (j + 0.5) / count; the radius tapers linearly with arc
    length along the chain from r_base at the base to r_tip at the tip.
    Self pairs: every sphere of link A against every sphere of link B for the
    non-adjacent link pairs (1, 3), (1, 4), (2, 4).
    """
    d = np.asarray(DH7_D)
    total = float(d.sum())
    frames, xyz, rad, link = [], [], [], []
    arc0 = 0.0
    lid = 0
    for i in range(7):
        if d[i] == 0.0:
            continue
        cnt = DH7_SPHERES_PER_LINK[lid]
        lid += 1
        for j in range(cnt):
            f = (j + 0.5) / cnt
            arc = arc0 + f * d[i]
            frames.append(i)  # frame i-1 in 1-based joint numbering
            xyz.append((0.0, 0.0, f * d[i]))
            rad.append(r_base + (r_tip - r_base) * arc / total)
            link.append(lid)
        arc0 += d[i]
    link = np.asarray(link, dtype=np.int32)
    lim = np.asarray(DH7_LIMITS)
    return Robot(
        name="dh7",
        a=np.zeros(7), alpha=np.asarray(DH7_ALPHA), d=d, theta_off=np.zeros(7),
        q_lo=-lim, q_hi=lim,
        sphere_frame=np.asarray(frames, dtype=np.int32),
        sphere_xyz=np.asarray(xyz, dtype=np.float64),
        sphere_r=np.asarray(rad, dtype=np.float64),
        sphere_link=link,
        self_pairs=_pairs_between_links(link, [(1, 3), (1, 4), (2, 4)]),
    )


def chain_robot(n: int = 10, a: float = 0.15, r: float = 0.04, per_link: int = 2) -> Robot:
    """An n-joint DH chain for chains longer than the 7-DOF arm: link length a,
    twists alternating +-pi/2, a base offset d_1 = 0.2 m, joint limits +-2.5
    rad, per_link spheres of radius r per link on its distal frame k at
    o_k - (1 - f) a x_k, f = (i + 1/2) / per_link (along the a part of the
    link; 1/4 and 3/4 for two), and self pairs between links at least three
    apart."""
    a_ = np.full(n, a)
    alpha = np.array([np.pi / 2 if i % 2 == 0 else -np.pi / 2 for i in range(n)])
    d = np.zeros(n)
    d[0] = 0.2
    frames, xyz, rad, link = [], [], [], []
    for k in range(1, n + 1):
        for f in ((i + 0.5) / per_link for i in range(per_link)):
            frames.append(k)
            xyz.append((-(1 - f) * a, 0.0, 0.0))
            rad.append(r)
            link.append(k)
    link = np.asarray(link, dtype=np.int32)
    pairs = [(i, j) for i in range(1, n + 1) for j in range(i + 3, n + 1)]
    return Robot(name=f"chain{n}", a=a_, alpha=alpha, d=d, theta_off=np.zeros(n), q_lo=np.full(n, -2.5),
                 q_hi=np.full(n, 2.5), sphere_frame=np.asarray(frames, dtype=np.int32),
                 sphere_xyz=np.asarray(xyz, dtype=np.float64), sphere_r=np.asarray(rad, dtype=np.float64),
                 sphere_link=link, self_pairs=_pairs_between_links(link, pairs))


def point2_robot(side: float = 10.0) -> Robot:
    """A point moving in a square of side ``side`` (the Forest benchmark of
    Sec. V): two prismatic joints, the first along the base z axis
    (alpha = -pi/2 turns the next joint axis onto the base y axis), the second
    along y, so the point sits at (0, q_1, q_0). One sphere of radius 0 at
    frame 2; obstacles of the plane (x, y) are spheres at (0, y, x)."""
    n = 2
    return Robot(
        name="point2",
        a=np.zeros(n), alpha=np.array([-math.pi / 2, 0.0]), d=np.zeros(n), theta_off=np.zeros(n),
        q_lo=np.zeros(n), q_hi=np.full(n, side),
        sphere_frame=np.array([2], dtype=np.int32), sphere_xyz=np.zeros((1, 3)), sphere_r=np.zeros(1),
        sphere_link=np.array([2], dtype=np.int32), self_pairs=np.zeros((0, 2), dtype=np.int32),
        joint_type=np.ones(n, dtype=np.int32),
    )


def forest_obstacles(seed: int, count: int = 15, r: float = 0.35, side: float = 10.0,
                     centre: float = 7.0) -> Env:
    """Forest of Sec. V: ``count`` disks of radius ``r`` with centres uniform
    in the central square of side ``centre`` of the ``side`` x ``side``
    domain, as spheres (0, y, x, r) for point2_robot."""
    rng = np.random.default_rng(seed)
    lo = 0.5 * (side - centre)
    xy = rng.uniform(lo, lo + centre, size=(count, 2))
    sph = np.column_stack([np.zeros(count), xy[:, 1], xy[:, 0], np.full(count, r)])
    return Env("forest", sph)


def rot_zyx(yaw: float, pitch: float, roll: float) -> np.ndarray:
    """Rz(yaw) Ry(pitch) Rx(roll)."""
    cz, sz, cy, sy, cx, sx = (math.cos(yaw), math.sin(yaw), math.cos(pitch), math.sin(pitch), math.cos(roll),
                              math.sin(roll))
    Rz = np.array([[cz, -sz, 0.0], [sz, cz, 0.0], [0.0, 0.0, 1.0]])
    Ry = np.array([[cy, 0.0, sy], [0.0, 1.0, 0.0], [-sy, 0.0, cy]])
    Rx = np.array([[1.0, 0.0, 0.0], [0.0, cx, -sx], [0.0, sx, cx]])
    return Rz @ Ry @ Rx


def box_row(centre, half, R) -> np.ndarray:
    """One Env.boxes row."""
    return np.concatenate([np.asarray(centre, dtype=np.float64), np.asarray(half, dtype=np.float64),
                           np.asarray(R, dtype=np.float64).reshape(9)])


def box_arm_robot(w: float = 0.06) -> Robot:
    """The 7-DOF chain of dh7_robot described by 11 boxes and no spheres, as
    the hardware arm of Sec. VII: one box of half width ``w`` along each of the
    four link segments with d != 0 (fixed to the frame whose z axis carries the
    segment, from its origin to d along z) and a cube of half side ``w + 0.01``
    at each joint origin 1..7. Self pairs: every box pair whose frames differ by
    at least 3."""
    r = dh7_robot()
    n = r.n
    frames, xyz, half = [], [], []
    for i in range(n):
        if r.d[i] != 0.0:
            frames.append(i)
            xyz.append((0.0, 0.0, 0.5 * r.d[i]))
            half.append((w, w, 0.5 * abs(r.d[i])))
    for f in range(1, n + 1):
        frames.append(f)
        xyz.append((0.0, 0.0, 0.0))
        half.append((w + 0.01,) * 3)
    B = len(frames)
    fr = np.asarray(frames, dtype=np.int32)
    bb = [(i, j) for i in range(B) for j in range(i + 1, B) if abs(int(fr[i]) - int(fr[j])) >= 3]
    return Robot(
        name="box_arm", a=r.a, alpha=r.alpha, d=r.d, theta_off=r.theta_off, q_lo=r.q_lo, q_hi=r.q_hi,
        sphere_frame=np.zeros(0, dtype=np.int32), sphere_xyz=np.zeros((0, 3)), sphere_r=np.zeros(0),
        sphere_link=np.zeros(0, dtype=np.int32), self_pairs=np.zeros((0, 2), dtype=np.int32),
        box_frame=fr, box_xyz=np.asarray(xyz), box_rot=np.repeat(np.eye(3)[None], B, axis=0),
        box_half=np.asarray(half), self_sb=np.zeros((0, 2), dtype=np.int32),
        self_bb=np.asarray(bb, dtype=np.int32).reshape(-1, 2),
    )


def tabletop_box_env(seed: int, n_vox: int = 160, voxel: float = 0.08) -> Env:
    """Table-top scene of Sec. VII: a table box, a rotated box and a shelf-like
    box on it, and voxel spheres circumscribing ``voxel``-sized cubes (r =
    voxel sqrt(3) / 2) from a few seeded clusters above the table."""
    rng = np.random.default_rng(seed)
    boxes = [box_row((0.65, 0.0, -0.02), (0.45, 0.7, 0.02), np.eye(3)),
             box_row((0.6, -0.35, 0.12), (0.08, 0.05, 0.12), rot_zyx(rng.uniform(-1, 1), 0.0, 0.0)),
             box_row((0.75, 0.3, 0.2), (0.05, 0.2, 0.2), rot_zyx(rng.uniform(-0.5, 0.5), rng.uniform(-0.2, 0.2),
                                                            rng.uniform(-0.2, 0.2)))]
    centres = rng.uniform((0.4, -0.5, 0.05), (1.0, 0.5, 0.5), size=(5, 3))
    pts = centres[rng.integers(0, 5, size=n_vox)] + rng.normal(0.0, 0.06, size=(n_vox, 3))
    vox = np.unique(np.floor(pts / voxel).astype(np.int64), axis=0)
    c = (vox + 0.5) * voxel
    sph = np.column_stack([c, np.full(c.shape[0], voxel * math.sqrt(3.0) / 2.0)])
    return Env("tabletop_boxes", sph, np.asarray(boxes))


def planar_disks_candidates(seed: int, count: int, lo: float = -2.5, hi: float = 2.5,
                            r_lo: float = 0.1, r_hi: float = 0.3) -> np.ndarray:
    """Candidate obstacle disks in the plane z = 0: centres uniform in
    [lo, hi]^2, radii uniform in [r_lo, r_hi]. Rows are (x, y, 0, r)."""
    rng = np.random.default_rng(seed)
    xy = rng.uniform(lo, hi, size=(count, 2))
    r = rng.uniform(r_lo, r_hi, size=count)
    return np.column_stack([xy, np.zeros(count), r])


def box_obstacles(seed: int, count: int, box_lo=(0.5, -0.5, 0.0), box_hi=(1.5, 0.5, 1.0),
                  r_lo: float = 0.02, r_hi: float = 0.10, name: str = "box") -> Env:
    """Obstacle spheres with centres uniform in an axis-aligned box and radii
    uniform in [r_lo, r_hi] (default: the 1 m cube 0.5 m ahead of the base)."""
    rng = np.random.default_rng(seed)
    c = rng.uniform(np.asarray(box_lo), np.asarray(box_hi), size=(count, 3))
    r = rng.uniform(r_lo, r_hi, size=count)
    return Env(name=name, spheres=np.column_stack([c, r]))


def table_cloud_obstacles(seed: int, count: int = 1024, r: float = 0.02, voxel: float = 0.02,
                          table_lo=(0.3, -0.4), table_hi=(1.3, 0.4), table_z: float = 0.0,
                          n_clusters: int = 6, cluster_pts: int = 80, sigma: float = 0.05,
                          cluster_z: float = 0.1) -> Env:
    """Perception-like obstacle set: a planar table sampled on a ``voxel`` grid
    plus Gaussian clusters of object points on it, voxelised at ``voxel`` and
    reduced to ``count`` spheres of radius ``r`` at distinct voxel centres by a
    seeded random subset."""
    rng = np.random.default_rng(seed)
    nx = int(round((table_hi[0] - table_lo[0]) / voxel)) + 1
    ny = int(round((table_hi[1] - table_lo[1]) / voxel)) + 1
    gx, gy = np.meshgrid(table_lo[0] + voxel * np.arange(nx), table_lo[1] + voxel * np.arange(ny),
                         indexing="ij")
    table = np.column_stack([gx.ravel(), gy.ravel(), np.full(gx.size, table_z)])
    centres = np.column_stack([rng.uniform(table_lo[0], table_hi[0], n_clusters),
                               rng.uniform(table_lo[1], table_hi[1], n_clusters),
                               np.full(n_clusters, cluster_z)])
    pts = [table]
    for c in centres:
        p = c + sigma * rng.standard_normal((cluster_pts, 3))
        pts.append(p[p[:, 2] >= table_z])
    pts = np.concatenate(pts)
    vox = np.unique(np.floor(pts / voxel + 0.5).astype(np.int64), axis=0)
    if vox.shape[0] > count:
        vox = vox[np.sort(rng.choice(vox.shape[0], size=count, replace=False))]
    cen = vox.astype(np.float64) * voxel
    return Env(name="table_cloud", spheres=np.column_stack([cen, np.full(cen.shape[0], r)]))


def uniform_configs(seed: int, robot: Robot, count: int) -> np.ndarray:
    """Configurations uniform in the joint-limit box, shape [count, n]."""
    rng = np.random.default_rng(seed)
    return rng.uniform(robot.q_lo, robot.q_hi, size=(count, robot.n))


def random_walk_waypoints(rng: np.random.Generator, robot: Robot, start: np.ndarray,
                          step: float, shrink: float = 0.8) -> np.ndarray:
    """One candidate next waypoint: a random direction of length ``step`` from
    ``start``, clipped to ``shrink`` times the joint limits."""
    d = rng.standard_normal(robot.n)
    d *= step / np.linalg.norm(d)
    return np.clip(start + d, shrink * robot.q_lo, shrink * robot.q_hi)
