"""Thin ctypes binding of libezo.so (include/ezo.h). Argument marshalling only:
every step of the inflation runs in the library's CUDA kernels. Device
buffers are torch tensors; host inputs are numpy arrays. There is no CPU
fallback: importing this module on a machine without the built library, or
calling it without a CUDA device, raises."""
from __future__ import annotations

import ctypes as C
import dataclasses
import os

import numpy as np

from . import workloads

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libezo.so")

EZO_OK = 0
STATUS_NAMES = {0: "ok", 1: "invalid argument", 2: "segment in collision", 3: "capacity", 4: "timeout",
                5: "cuda error", 6: "max iterations"}
SEG_ACTIVE, SEG_ACCEPTED, SEG_IN_COLLISION, SEG_CAPACITY, SEG_MAX_ITER, SEG_IDLE, SEG_SKIPPED = 0, 1, 2, 3, 6, 7, 8
RUN_HOST_LOOP, RUN_GRAPH = 0, 1
STEP_NAMES = ("round_size", "sample", "check", "certify", "bisect", "place", "round_end")


class EzoError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"ezo status {status} ({STATUS_NAMES.get(status, '?')}): {msg}")
        self.status = status


class Params(C.Structure):
    _fields_ = [("eps", C.c_double), ("delta", C.c_double), ("tau", C.c_double), ("step_back_max", C.c_double),
                ("t_col", C.c_double), ("n_p", C.c_int32), ("n_f", C.c_int32), ("n_b", C.c_int32),
                ("n_mix", C.c_int32), ("n_it_max", C.c_int32), ("reserved0", C.c_int32), ("seed", C.c_uint64)]

    @staticmethod
    def make(**kw) -> "Params":
        p = Params()
        lib().ezo_params_default(C.byref(p))
        for k, v in kw.items():
            if not hasattr(p, k):
                raise KeyError(k)
            setattr(p, k, v)
        return p


class Shape(C.Structure):
    """Launch shapes of a batch's round kernels (ezo_shape)."""
    _fields_ = [("sample_fill_tiles", C.c_int32), ("check_lanes", C.c_int32), ("bisect_lanes", C.c_int32)]

    def as_dict(self) -> dict:
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


_lib = None
_P = C.c_void_p
_I32 = C.c_int32
_I64 = C.c_int64
_DP = C.POINTER(C.c_double)


def _sig(lib):
    f = lib
    f.ezo_last_error.restype = C.c_char_p
    f.ezo_params_default.argtypes = [C.POINTER(Params)]
    f.ezo_robot_create.argtypes = [_I32, _DP, _DP, _DP, _DP, _DP, _DP, _I32, C.POINTER(_I32), _DP, _DP, _I32,
                                   C.POINTER(_I32), C.POINTER(_I32), C.POINTER(_P)]
    f.ezo_robot_free.argtypes = [_P]
    f.ezo_robot_dof.argtypes = [_P]
    f.ezo_env_create.argtypes = [_I32, _DP, C.POINTER(_P)]
    f.ezo_env_free.argtypes = [_P]
    f.ezo_check_collision.argtypes = [_P, _P, _P, _I64, _I64, _P, _I32, _P]
    f.ezo_signed_distance.argtypes = [_P, _P, _P, _I64, _I64, _P, _P]
    f.ezo_hit_and_run.argtypes = [_P, _P, _I32, _I32, _I32, _DP, _DP, _I64, _I32, C.c_uint64, C.c_uint32, _I32, _P,
                                  _I64, _P]
    f.ezo_batch_create.argtypes = [_P, _I32, C.POINTER(_P), _I32, _DP, _DP, C.POINTER(_I32), C.POINTER(_I32),
                                   C.POINTER(C.c_uint32), C.POINTER(_I32), _DP, _DP, _I32, C.POINTER(Params),
                                   C.POINTER(_P)]
    f.ezo_batch_free.argtypes = [_P]
    f.ezo_batch_run.argtypes = [_P, _I32, _P]
    f.ezo_batch_reset.argtypes = [_P, _DP, _DP, _P]
    f.ezo_batch_run_path.argtypes = [_P, _I32, _I32, _P]
    f.ezo_batch_get_segment.argtypes = [_P, _I32, C.POINTER(_I32), C.POINTER(_I32), C.POINTER(_I32),
                                        C.POINTER(_I32), C.POINTER(_I64)]
    f.ezo_batch_get_polytope.argtypes = [_P, _I32, C.POINTER(_I32), _DP, _DP]
    f.ezo_batch_capacity.argtypes = [_P, C.POINTER(_I32), C.POINTER(_I32)]
    f.ezo_batch_step.argtypes = [_P, _I32, _P]
    f.ezo_batch_sync.argtypes = [_P, _P]
    f.ezo_batch_read.argtypes = [_P, _I32, _I32, _P, _I64]
    f.ezo_batch_write_samples.argtypes = [_P, _I32, C.POINTER(C.c_float), _I32]
    f.ezo_profile_enable.argtypes = [_I32]
    f.ezo_profile_read.argtypes = [_DP, C.POINTER(_I64), _I32]
    f.ezo_surrogate_num_params.restype = _I64
    f.ezo_surrogate_create.argtypes = [_P, C.c_uint64, C.POINTER(_P)]
    f.ezo_surrogate_free.argtypes = [_P]
    f.ezo_surrogate_get_params.argtypes = [_P, C.POINTER(C.c_float)]
    f.ezo_surrogate_set_params.argtypes = [_P, C.POINTER(C.c_float)]
    f.ezo_surrogate_train.argtypes = [_P, _P, _I64, _I32, _I32, C.c_float, C.c_uint64, C.c_float, C.c_float,
                                      C.POINTER(C.c_float), _P]
    f.ezo_surrogate_grad.argtypes = [_P, _P, _I64, _P, _I32, C.POINTER(C.c_float), C.POINTER(C.c_float), _P]
    f.ezo_surrogate_predict.argtypes = [_P, _P, _I64, _I64, _P, _P]
    f.ezo_surrogate_status.argtypes = [_P, C.POINTER(_I32), _I32, _P]
    f.ezo_batch_attach_surrogate.argtypes = [_P, _P, C.c_float]
    f.ezo_batch_set_sample_lanes.argtypes = [_P, _I32]
    f.ezo_batch_get_polytopes.argtypes = [_P, C.POINTER(_I32), C.POINTER(_I32), _DP, _DP, _I32, C.POINTER(_I32), _P]
    f.ezo_host_alloc.argtypes = [C.c_size_t, C.POINTER(C.c_void_p)]
    f.ezo_host_free.argtypes = [C.c_void_p]
    f.ezo_host_free.restype = None
    f.ezo_robot_add_boxes.argtypes = [_P, _I32, C.POINTER(_I32), _DP, _DP, _DP, _I32, C.POINTER(_I32), _I32,
                                      C.POINTER(_I32)]
    f.ezo_env_add_boxes.argtypes = [_P, _I32, _DP]
    f.ezo_path_points.argtypes = [_DP, _I32, _I32, C.c_double, C.POINTER(_I64), C.POINTER(_I64)]
    f.ezo_check_path.argtypes = [_P, _P, _DP, _I32, C.c_double, C.POINTER(C.c_uint8), _P, _I64,
                                 C.POINTER(_I64), _P]
    f.ezo_batch_set_polytope.argtypes = [_P, _I32, _I32, _DP, _DP, _P]
    f.ezo_batch_edit.argtypes = [_P, _I64, _DP, _P]
    f.ezo_batch_coverage.argtypes = [_P, C.POINTER(C.c_uint8), _P]
    f.ezo_batch_reinflate.argtypes = [_P, C.POINTER(C.c_uint8), _I32, _P]
    f.ezo_tune_lanes.argtypes = [_P, _P, _I64, C.POINTER(_I32), _P]
    f.ezo_set_autotune.argtypes = [_I32]
    f.ezo_probe_fp32_fma.argtypes = [_DP, _P]
    f.ezo_check_flops.argtypes = [_P, _P]
    f.ezo_check_flops.restype = C.c_double
    f.ezo_check_static_spheres.argtypes = [_P, _P]
    f.ezo_check_static_spheres.restype = _I32
    f.ezo_batch_get_shape.argtypes = [_P, C.POINTER(Shape)]
    f.ezo_batch_set_shape.argtypes = [_P, C.POINTER(Shape)]
    f.ezo_batch_tune.argtypes = [_P, _I32, C.POINTER(Shape), _P]
    f.ezo_inflate_segment.argtypes = [_P, _P, _DP, _DP, _DP, _DP, _I32, C.POINTER(Params), C.c_uint32,
                                      C.POINTER(_P), _P, _P]
    f.ezo_inflate_path.argtypes = [_P, _P, _DP, _I32, _DP, _DP, _I32, C.POINTER(Params), _I32, C.c_uint32,
                                   C.POINTER(_P), _P]
    f.ezo_inflate_batch.argtypes = [_P, _I32, C.POINTER(_P), _I32, C.POINTER(_I32), _DP, C.POINTER(_I32),
                                    C.POINTER(_I32), _DP, _DP, _I32, C.POINTER(Params), _I32, C.c_uint32,
                                    C.POINTER(_P), _P]
    f.ezo_polytope_get.argtypes = [_P, C.POINTER(_I32), C.POINTER(_I32), _DP, _DP]
    f.ezo_polytope_stats.argtypes = [_P, C.POINTER(_I32), _P]
    f.ezo_polytope_free.argtypes = [_P]
    f.ezo_scs_size.argtypes = [_P]
    f.ezo_scs_size.restype = _I32
    f.ezo_scs_get.argtypes = [_P, _I32]
    f.ezo_scs_get.restype = _P
    f.ezo_scs_free.argtypes = [_P]
    f.ezo_sphere_centres.argtypes = [_P, _P, _I64, _I64, _I32, _P, _P]
    f.ezo_fk_error.argtypes = [_P, _P, _I64, _I64, _P, _P]
    return lib


def lib():
    """The loaded library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run __graft_entry__.build() or "
                               "python -m paper_2504_10783_gb300.build")
        _lib = _sig(C.CDLL(LIB_PATH))
    return _lib


def _check(status: int):
    if status != EZO_OK:
        raise EzoError(status, lib().ezo_last_error().decode())


def _dp(a: np.ndarray):
    return a.ctypes.data_as(_DP)


def _ip(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(_I32))


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _ld(t) -> int:
    """Leading dimension of an [n, N] tensor (any value >= N when n == 1)."""
    return max(int(t.stride(0)), int(t.shape[1])) if t.shape[0] == 1 else int(t.stride(0))


def _need_cuda(t, dtype, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must have dtype {dtype}")


class Robot:
    """ezo_robot handle built from a workloads.Robot."""

    def __init__(self, r: workloads.Robot):
        self.desc = r
        f64 = lambda x: np.ascontiguousarray(x, dtype=np.float64)
        i32 = lambda x: np.ascontiguousarray(x, dtype=np.int32)
        self._keep = [f64(r.a), f64(r.alpha), f64(r.d), f64(r.theta_off), f64(r.q_lo), f64(r.q_hi),
                      i32(r.sphere_frame), f64(r.sphere_xyz.reshape(-1)), f64(r.sphere_r),
                      i32(r.self_pairs.reshape(-1)),
                      i32(r.joint_type) if getattr(r, "joint_type", None) is not None else None]
        k = self._keep
        h = _P()
        _check(lib().ezo_robot_create(r.n, _dp(k[0]), _dp(k[1]), _dp(k[2]), _dp(k[3]), _dp(k[4]), _dp(k[5]),
                                      r.n_spheres, _ip(k[6]), _dp(k[7]), _dp(k[8]), r.self_pairs.shape[0],
                                      _ip(k[9]), _ip(k[10]) if k[10] is not None else None, C.byref(h)))
        self.h = h
        self.n = r.n
        self.n_spheres = r.n_spheres
        # ezo_sphere_centres orders spheres by frame, stably
        self.sphere_order = np.argsort(np.asarray(r.sphere_frame), kind="stable")
        if getattr(r, "n_boxes", 0):
            i32 = lambda x: np.ascontiguousarray(x, dtype=np.int32)
            sb = i32(r.self_sb if r.self_sb is not None else np.zeros((0, 2))).reshape(-1)
            bb = i32(r.self_bb if r.self_bb is not None else np.zeros((0, 2))).reshape(-1)
            self._keep_boxes = [i32(r.box_frame), f64(r.box_xyz.reshape(-1)), f64(r.box_rot.reshape(-1)),
                                f64(r.box_half.reshape(-1)), sb, bb]
            kb = self._keep_boxes
            _check(lib().ezo_robot_add_boxes(self.h, r.n_boxes, _ip(kb[0]), _dp(kb[1]), _dp(kb[2]), _dp(kb[3]),
                                             sb.size // 2, _ip(sb) if sb.size else None, bb.size // 2,
                                             _ip(bb) if bb.size else None))

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.ezo_robot_free(self.h)
            self.h = None


class Env:
    """ezo_env handle built from an (N_obs, 4) array or a workloads.Env
    (spheres and, when present, oriented boxes)."""

    def __init__(self, spheres, boxes=None):
        if isinstance(spheres, workloads.Env):
            boxes = spheres.boxes if boxes is None else boxes
            spheres = spheres.spheres
        a = np.ascontiguousarray(spheres, dtype=np.float64).reshape(-1, 4)
        self.spheres = a
        h = _P()
        _check(lib().ezo_env_create(a.shape[0], _dp(a.reshape(-1)), C.byref(h)))
        self.h = h
        if boxes is not None and len(boxes):
            self.boxes = np.ascontiguousarray(boxes, dtype=np.float64).reshape(-1, 15)
            _check(lib().ezo_env_add_boxes(self.h, self.boxes.shape[0], _dp(self.boxes.reshape(-1))))

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.ezo_env_free(self.h)
            self.h = None


def check_collision(robot: Robot, env: Env, q_dev, flags_dev, lanes: int = 0, stream=None):
    """flags_dev[i] = 1 iff configuration q_dev[:, i] collides (q_dev: float32
    CUDA tensor [n, N] with unit stride along N)."""
    import torch
    _need_cuda(q_dev, torch.float32, "q_dev")
    _need_cuda(flags_dev, torch.uint8, "flags_dev")
    n, N = q_dev.shape
    if n != robot.n or (N > 1 and q_dev.stride(1) != 1) or flags_dev.numel() < N:
        raise ValueError("q_dev must be [n, N] with stride(1) == 1 and flags_dev must hold N entries")
    _check(lib().ezo_check_collision(robot.h, env.h, C.c_void_p(q_dev.data_ptr()), N, _ld(q_dev),
                                     C.c_void_p(flags_dev.data_ptr()), lanes, _stream(stream)))


def path_points(verts, step: float, n: int | None = None):
    """Point count of each edge of a piecewise-linear path checked at `step`
    (Sec. VI-B) and the total: (int64 [K], total)."""
    v = np.ascontiguousarray(np.atleast_2d(verts), dtype=np.float64)
    K = max(0, v.shape[0] - 1)
    cnt = np.zeros(max(K, 1), dtype=np.int64)
    tot = _I64()
    _check(lib().ezo_path_points(_dp(v), v.shape[0], n or v.shape[1], step, cnt.ctypes.data_as(C.POINTER(_I64)),
                                 C.byref(tot)))
    return cnt[:K], int(tot.value)


def check_path(robot: Robot, env: Env, verts, step: float, point_flags_dev=None, stream=None):
    """Collision check of a piecewise-linear path at `step` (Sec. VI-B):
    returns (edge flags bool [K], point count); point_flags_dev (uint8 CUDA
    tensor, optional) receives one flag per point in edge order."""
    import torch
    v = np.ascontiguousarray(np.atleast_2d(verts), dtype=np.float64)
    if v.shape[1] != robot.n:
        raise ValueError("verts must be [n_verts, n]")
    K = max(0, v.shape[0] - 1)
    edge = np.zeros(max(K, 1), dtype=np.uint8)
    cap, ptr = 0, None
    if point_flags_dev is not None:
        _need_cuda(point_flags_dev, torch.uint8, "point_flags_dev")
        cap, ptr = point_flags_dev.numel(), C.c_void_p(point_flags_dev.data_ptr())
    npts = _I64()
    _check(lib().ezo_check_path(robot.h, env.h, _dp(v), v.shape[0], step,
                                edge.ctypes.data_as(C.POINTER(C.c_uint8)), ptr, cap, C.byref(npts), _stream(stream)))
    return edge[:K].astype(bool), int(npts.value)


def signed_distance(robot: Robot, env: Env, q_dev, sd_dev, stream=None):
    import torch
    _need_cuda(q_dev, torch.float32, "q_dev")
    _need_cuda(sd_dev, torch.float32, "sd_dev")
    n, N = q_dev.shape
    if n != robot.n or (N > 1 and q_dev.stride(1) != 1) or sd_dev.numel() < N:
        raise ValueError("q_dev must be [n, N] with stride(1) == 1 and sd_dev must hold N entries")
    _check(lib().ezo_signed_distance(robot.h, env.h, C.c_void_p(q_dev.data_ptr()), N, _ld(q_dev),
                                     C.c_void_p(sd_dev.data_ptr()), _stream(stream)))


def sphere_centres(robot: Robot, q_dev, out_dev, fp64: bool = False, stream=None):
    """Sphere centres of the configurations q_dev (float32 [n, N]) into
    out_dev (float64 CUDA tensor [n_spheres, 3, N]): the collision checker's
    FP32 kinematics, or FP64 kinematics with fp64=True."""
    import torch
    _need_cuda(q_dev, torch.float32, "q_dev")
    _need_cuda(out_dev, torch.float64, "out_dev")
    n, N = q_dev.shape
    if n != robot.n or (N > 1 and q_dev.stride(1) != 1) or out_dev.numel() < 3 * robot.n_spheres * N or \
            not out_dev.is_contiguous():
        raise ValueError("q_dev must be [n, N] with stride(1) == 1 and out_dev contiguous [n_spheres, 3, N]")
    _check(lib().ezo_sphere_centres(robot.h, C.c_void_p(q_dev.data_ptr()), N, _ld(q_dev), 1 if fp64 else 0,
                                    C.c_void_p(out_dev.data_ptr()), _stream(stream)))


def fk_error(robot: Robot, q_dev, err_dev, stream=None):
    """err_dev[i] (float32 CUDA tensor) = largest distance in metres between a
    sphere centre of the checker's FP32 kinematics and of FP64 kinematics."""
    import torch
    _need_cuda(q_dev, torch.float32, "q_dev")
    _need_cuda(err_dev, torch.float32, "err_dev")
    n, N = q_dev.shape
    if n != robot.n or (N > 1 and q_dev.stride(1) != 1) or err_dev.numel() < N:
        raise ValueError("q_dev must be [n, N] with stride(1) == 1 and err_dev must hold N entries")
    _check(lib().ezo_fk_error(robot.h, C.c_void_p(q_dev.data_ptr()), N, _ld(q_dev), C.c_void_p(err_dev.data_ptr()),
                              _stream(stream)))


def hit_and_run(A_dev, b_dev, v1, v2, N: int, n_mix: int, seed: int, stream_id: int, round_k: int, out_dev,
                stream=None):
    """N hit-and-run walks inside {A x <= b} (A_dev float64 [m, n] CUDA,
    b_dev float64 [m]); writes out_dev float32 [n, N]."""
    import torch
    _need_cuda(A_dev, torch.float64, "A_dev")
    _need_cuda(b_dev, torch.float64, "b_dev")
    _need_cuda(out_dev, torch.float32, "out_dev")
    m, n = A_dev.shape
    v1 = np.ascontiguousarray(v1, dtype=np.float64)
    v2 = np.ascontiguousarray(v2, dtype=np.float64)
    if out_dev.shape[0] != n or out_dev.stride(1) != 1 or out_dev.shape[1] < N or A_dev.stride(1) != 1:
        raise ValueError("bad shapes")
    _check(lib().ezo_hit_and_run(C.c_void_p(A_dev.data_ptr()), C.c_void_p(b_dev.data_ptr()), m, n, A_dev.stride(0),
                                 _dp(v1), _dp(v2), N, n_mix, seed, stream_id, round_k,
                                 C.c_void_p(out_dev.data_ptr()), out_dev.stride(0), _stream(stream)))


@dataclasses.dataclass
class SegmentResult:
    status: int
    rounds: int
    m: int
    planes: int
    checks: int
    A: np.ndarray
    b: np.ndarray


class Batch:
    """ezo_batch: many segments inflated together (Algorithm 1 per segment)."""

    def __init__(self, robot: Robot, envs, v1, v2, params: Params, seg_env=None, seg_np=None, seg_stream=None,
                 path_first=None, A0=None, b0=None):
        envs = list(envs) if isinstance(envs, (list, tuple)) else [envs]
        self.robot = robot
        self.envs = envs
        self.n = robot.n
        v1 = np.ascontiguousarray(np.atleast_2d(v1), dtype=np.float64)
        v2 = np.ascontiguousarray(np.atleast_2d(v2), dtype=np.float64)
        self.B = v1.shape[0]
        self.v1, self.v2 = v1, v2
        arr = (_P * len(envs))(*[e.h for e in envs])
        keep = []

        def opt_i32(x):
            if x is None:
                return None
            a = np.ascontiguousarray(x, dtype=np.int32)
            keep.append(a)
            return _ip(a)

        def opt_u32(x):
            if x is None:
                return None
            a = np.ascontiguousarray(x, dtype=np.uint32)
            keep.append(a)
            return a.ctypes.data_as(C.POINTER(C.c_uint32))

        m0 = 0
        Ap = bp = None
        if A0 is not None:
            A0 = np.ascontiguousarray(A0, dtype=np.float64)
            b0 = np.ascontiguousarray(b0, dtype=np.float64)
            keep += [A0, b0]
            m0 = A0.shape[0]
            Ap, bp = _dp(A0), _dp(b0)
        self.params = params
        h = _P()
        _check(lib().ezo_batch_create(robot.h, len(envs), arr, self.B, _dp(v1), _dp(v2), opt_i32(seg_env),
                                      opt_i32(seg_np), opt_u32(seg_stream), opt_i32(path_first), Ap, bp, m0,
                                      C.byref(params), C.byref(h)))
        self.h = h
        mc, sc = _I32(), _I32()
        _check(lib().ezo_batch_capacity(h, C.byref(mc), C.byref(sc)))
        self.m_cap, self.s_cap = mc.value, sc.value

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.ezo_batch_free(self.h)
            self.h = None
        if getattr(self, "_pin", None) is not None and _lib is not None:
            self._pin = None
            for p in self._pin_ptrs:
                _lib.ezo_host_free(p)

    def reset(self, v1=None, v2=None, stream=None):
        a1 = a2 = None
        if v1 is not None:
            self._v1h = np.ascontiguousarray(v1, dtype=np.float64)
            a1 = _dp(self._v1h)
        if v2 is not None:
            self._v2h = np.ascontiguousarray(v2, dtype=np.float64)
            a2 = _dp(self._v2h)
        _check(lib().ezo_batch_reset(self.h, a1, a2, _stream(stream)))

    def run(self, mode: int = RUN_HOST_LOOP, stream=None):
        _check(lib().ezo_batch_run(self.h, mode, _stream(stream)))

    def run_path(self, sequential=True, mode: int = RUN_HOST_LOOP, stream=None):
        """sequential: True/1 one segment at a time, 2 wavefront over paths,
        False/0 speculative (all segments, skip rule applied afterwards)."""
        seq = 2 if sequential == 2 else (1 if sequential else 0)
        _check(lib().ezo_batch_run_path(self.h, seq, mode, _stream(stream)))

    def step(self, step: int, stream=None):
        _check(lib().ezo_batch_step(self.h, step, _stream(stream)))

    def sync(self, stream=None):
        _check(lib().ezo_batch_sync(self.h, _stream(stream)))

    def segment(self, g: int) -> SegmentResult:
        st, rd, m, pl = _I32(), _I32(), _I32(), _I32()
        ch = _I64()
        _check(lib().ezo_batch_get_segment(self.h, g, C.byref(st), C.byref(rd), C.byref(m), C.byref(pl),
                                           C.byref(ch)))
        A = np.zeros((self.m_cap, self.n))
        b = np.zeros(self.m_cap)
        mm = _I32()
        _check(lib().ezo_batch_get_polytope(self.h, g, C.byref(mm), _dp(A), _dp(b)))
        return SegmentResult(st.value, rd.value, m.value, pl.value, ch.value, A[: mm.value].copy(),
                             b[: mm.value].copy())

    def _pinned_io(self):
        """Page-locked host buffers for polytopes(), made once per batch."""
        if getattr(self, "_pin", None) is None:
            B, mc, n = self.B, self.m_cap, self.n
            sizes = ((B,), (B,), (B, mc, n), (B, mc))
            dts = (np.int32, np.int32, np.float64, np.float64)
            arrs, ptrs = [], []
            for shape, dt in zip(sizes, dts):
                nbytes = int(np.prod(shape)) * np.dtype(dt).itemsize
                p = C.c_void_p()
                _check(lib().ezo_host_alloc(nbytes, C.byref(p)))
                ptrs.append(p.value)
                buf = (C.c_char * nbytes).from_address(p.value)
                arrs.append(np.frombuffer(buf, dtype=dt).reshape(shape))
            self._pin, self._pin_ptrs = arrs, ptrs
        return self._pin

    def polytopes(self, stream=None):
        """Every segment's (status, A, b) with three device-to-host copies
        into page-locked buffers: returns (status int32 [B], list of A
        [m_g, n], list of b [m_g]) as copies; rows_read is then the rows
        copied per segment."""
        st, m, A, b = self._pinned_io()
        mr = _I32()
        _check(lib().ezo_batch_get_polytopes(self.h, st.ctypes.data_as(C.POINTER(_I32)), m.ctypes.data_as(C.POINTER(_I32)),
                                             _dp(A), _dp(b), self.m_cap, C.byref(mr), _stream(stream)))
        self.rows_read = int(mr.value)  # rows copied per segment (>= max m)
        return st.copy(), [A[g, : m[g]].copy() for g in range(self.B)], [b[g, : m[g]].copy() for g in range(self.B)]

    def state(self, g: int) -> dict:
        o = np.zeros(13, dtype=np.int32)
        _check(lib().ezo_batch_read(self.h, g, 6, C.c_void_p(o.ctypes.data), o.nbytes))
        keys = ("k", "status", "m", "n_samples", "m_test", "count", "n_cand", "planes", "rounds", "n_placed",
                "n_p", "env", "s_cap")
        return dict(zip(keys, (int(x) for x in o)))

    def read(self, g: int, what: str) -> np.ndarray:
        """A per-segment buffer of the current round; samples are [n, s_cap_g]
        with the segment's own capacity s_cap_g (its stride on the device)."""
        st = self.state(g)
        n, npp = self.n, st["n_p"]
        if what == "samples":
            o = np.zeros((n, st["s_cap"]), dtype=np.float32)
            code = 0
        elif what == "labels":
            o = np.zeros(st["s_cap"], dtype=np.uint8)
            code = 1
        elif what == "cand_idx":
            o = np.zeros(npp, dtype=np.int32)
            code = 2
        elif what == "c_star":
            o = np.zeros((n, npp), dtype=np.float64)
            code = 3
        elif what == "dist":
            o = np.zeros(npp, dtype=np.float64)
            code = 4
        elif what == "bits":
            o = np.zeros(npp, dtype=np.uint32)
            code = 5
        elif what == "placed_idx":
            o = np.zeros(self.params.n_f, dtype=np.int32)
            code = 7
        elif what == "placed_delta":
            o = np.zeros(self.params.n_f, dtype=np.float64)
            code = 8
        else:
            raise KeyError(what)
        _check(lib().ezo_batch_read(self.h, g, code, C.c_void_p(o.ctypes.data), o.nbytes))
        return o

    def check_split(self, g: int):
        """(exact checks at samples, exact checks at bisection midpoints)."""
        o = np.zeros(3, dtype=np.int64)
        _check(lib().ezo_batch_read(self.h, g, 9, C.c_void_p(o.ctypes.data), o.nbytes))
        return int(o[0]), int(o[1])

    def sample_flops(self, g: int) -> int:
        """Algorithmic FP32 flops of the hit-and-run walks of segment g."""
        o = np.zeros(3, dtype=np.int64)
        _check(lib().ezo_batch_read(self.h, g, 9, C.c_void_p(o.ctypes.data), o.nbytes))
        return int(o[2])

    def attach_surrogate(self, sur, margin: float = 0.0):
        """Surrogate-guided bisection (None detaches)."""
        self._sur = sur
        _check(lib().ezo_batch_attach_surrogate(self.h, sur.h if sur is not None else None, margin))

    def set_polytope(self, g: int, A, b, stream=None):
        """Replace segment g's current polytope with A x <= b (host FP64)."""
        A = np.ascontiguousarray(np.atleast_2d(A), dtype=np.float64)
        b = np.ascontiguousarray(b, dtype=np.float64)
        if A.shape[0] and A.shape[1] != self.n or b.shape[0] != A.shape[0]:
            raise ValueError("A must be [m, n] and b [m]")
        _check(lib().ezo_batch_set_polytope(self.h, g, A.shape[0], _dp(A), _dp(b), _stream(stream)))

    def edit(self, cfg, stream=None):
        """Sec. VI-B set editing with the given configurations [N, n]."""
        c = np.ascontiguousarray(np.atleast_2d(cfg), dtype=np.float64)
        if c.size and c.shape[1] != self.n:
            raise ValueError("cfg must be [N, n]")
        _check(lib().ezo_batch_edit(self.h, c.shape[0] if c.size else 0, _dp(c), _stream(stream)))

    def coverage(self, stream=None) -> np.ndarray:
        """Per segment: covered by some final polytope of its path (bool)."""
        out = np.zeros(self.B, dtype=np.uint8)
        _check(lib().ezo_batch_coverage(self.h, out.ctypes.data_as(C.POINTER(C.c_uint8)), _stream(stream)))
        return out.astype(bool)

    def reinflate(self, which, mode: int = RUN_HOST_LOOP, stream=None):
        """Inflate the segments with which[g] again from the domain."""
        w = np.ascontiguousarray(np.asarray(which, dtype=bool).astype(np.uint8))
        if w.shape[0] != self.B:
            raise ValueError("which must have one entry per segment")
        _check(lib().ezo_batch_reinflate(self.h, w.ctypes.data_as(C.POINTER(C.c_uint8)), mode, _stream(stream)))

    def shape(self) -> dict:
        sh = Shape()
        _check(lib().ezo_batch_get_shape(self.h, C.byref(sh)))
        return sh.as_dict()

    def set_shape(self, sample_fill_tiles: int, check_lanes: int, bisect_lanes: int):
        sh = Shape(sample_fill_tiles, check_lanes, bisect_lanes)
        _check(lib().ezo_batch_set_shape(self.h, C.byref(sh)))

    def tune(self, reps: int = 2, stream=None) -> dict:
        """Autotune the round kernels' launch shapes on this batch (cached per
        problem class); leaves the batch reset."""
        sh = Shape()
        _check(lib().ezo_batch_tune(self.h, reps, C.byref(sh), _stream(stream)))
        return sh.as_dict()

    def set_sample_lanes(self, lanes: int):
        """Lanes per hit-and-run walk (0 = chosen per round, else 1, 2, 4, 8)."""
        _check(lib().ezo_batch_set_sample_lanes(self.h, int(lanes)))

    def surrogate_evals(self, g: int) -> int:
        o = np.zeros(1, dtype=np.int64)
        _check(lib().ezo_batch_read(self.h, g, 11, C.c_void_p(o.ctypes.data), o.nbytes))
        return int(o[0])

    def summary(self) -> dict:
        o = np.zeros(4, dtype=np.int32)
        _check(lib().ezo_batch_read(self.h, 0, 10, C.c_void_p(o.ctypes.data), o.nbytes))
        return dict(zip(("active", "rounds", "sample_tiles", "bisect_tiles"), (int(x) for x in o)))

    def write_samples(self, g: int, samples: np.ndarray):
        s = np.ascontiguousarray(samples, dtype=np.float32)  # [n, count]
        _check(lib().ezo_batch_write_samples(self.h, g, s.ctypes.data_as(C.POINTER(C.c_float)), s.shape[1]))


def profile_enable(on: bool = True):
    _check(lib().ezo_profile_enable(1 if on else 0))


def profile_reset():
    _check(lib().ezo_profile_reset())


def profile_read() -> dict:
    ms = np.zeros(7)
    cnt = np.zeros(7, dtype=np.int64)
    _check(lib().ezo_profile_read(_dp(ms), cnt.ctypes.data_as(C.POINTER(_I64)), 7))
    return {STEP_NAMES[i]: (float(ms[i]), int(cnt[i])) for i in range(7)}


def tune_lanes(robot: Robot, env: Env, N: int, stream=None) -> int:
    """Autotuned lanes per configuration for a batch of N configurations."""
    out = _I32()
    _check(lib().ezo_tune_lanes(robot.h, env.h, N, C.byref(out), _stream(stream)))
    return out.value


def set_autotune(on: bool = True):
    _check(lib().ezo_set_autotune(1 if on else 0))


def probe_fp32_fma(stream=None) -> float:
    """Measured FP32 FMA rate of the current device in TFLOP/s."""
    out = C.c_double()
    _check(lib().ezo_probe_fp32_fma(C.byref(out), _stream(stream)))
    return out.value


def check_flops(robot: Robot, env: Env) -> float:
    return float(lib().ezo_check_flops(robot.h, env.h))


def check_static_spheres(robot: Robot, env: Env) -> int:
    """Robot spheres whose obstacle pairs the checker decides once for this
    obstacle set instead of per configuration (ezo_check_static_spheres)."""
    return int(lib().ezo_check_static_spheres(robot.h, env.h))


class Stats(C.Structure):
    _fields_ = [("status", C.c_int32), ("rounds", C.c_int32), ("m", C.c_int32), ("planes", C.c_int32),
                ("checks", C.c_int64), ("checks_bisect", C.c_int64), ("surrogate_evals", C.c_int64)]


# outcomes for which the one-call entry points still return their polytopes
_OUTCOMES = (EZO_OK, 2, 3, 6)


def _polytope_result(p) -> SegmentResult:
    m, n = _I32(), _I32()
    _check(lib().ezo_polytope_get(p, C.byref(m), C.byref(n), None, None))
    A = np.zeros((m.value, n.value))
    b = np.zeros(m.value)
    _check(lib().ezo_polytope_get(p, None, None, _dp(A), _dp(b)))
    st = Stats()
    _check(lib().ezo_polytope_stats(p, None, C.byref(st)))
    return SegmentResult(st.status, st.rounds, st.m, st.planes, st.checks, A, b)


def _domain(A0, b0):
    if A0 is None:
        return None, None, 0, []
    A0 = np.ascontiguousarray(A0, dtype=np.float64)
    b0 = np.ascontiguousarray(b0, dtype=np.float64)
    return _dp(A0), _dp(b0), A0.shape[0], [A0, b0]


def inflate_segment(robot: Robot, env: Env, v1, v2, params: Params, A0=None, b0=None, stream_id: int = 0,
                    stream=None) -> SegmentResult:
    """Algorithm 1 on one segment through ezo_inflate_segment; the domain is
    {A0 x <= b0}, or the joint-limit box when A0 is None."""
    v1 = np.ascontiguousarray(v1, dtype=np.float64)
    v2 = np.ascontiguousarray(v2, dtype=np.float64)
    Ap, bp, m0, keep = _domain(A0, b0)
    out = _P()
    st = lib().ezo_inflate_segment(robot.h, env.h, _dp(v1), _dp(v2), Ap, bp, m0, C.byref(params), stream_id,
                                   C.byref(out), None, _stream(stream))
    if st not in _OUTCOMES or not out.value:
        _check(st)
    try:
        return _polytope_result(out)
    finally:
        lib().ezo_polytope_free(out)


def _path_mode(sequential) -> int:
    """sequential True/1: the paper's order (0), 2: wavefront (1), False/0:
    speculative (2)."""
    return 1 if sequential == 2 else (0 if sequential else 2)


def _scs_results(scs):
    out = []
    for i in range(lib().ezo_scs_size(scs)):
        p = lib().ezo_scs_get(scs, i)
        seg = _I32()
        _check(lib().ezo_polytope_stats(p, C.byref(seg), None))
        out.append((seg.value, _polytope_result(p)))
    return out


def inflate_path(robot: Robot, env: Env, verts, params: Params, sequential=True, stream_base: int = 0, A0=None,
                 b0=None, stream=None):
    """Sec. VI-A path inflation through ezo_inflate_path; returns [(segment
    index, SegmentResult)] for the segments that were inflated (not skipped),
    in path order."""
    verts = np.ascontiguousarray(verts, dtype=np.float64)
    Ap, bp, m0, keep = _domain(A0, b0)
    out = _P()
    st = lib().ezo_inflate_path(robot.h, env.h, _dp(verts), verts.shape[0], Ap, bp, m0, C.byref(params),
                                _path_mode(sequential), stream_base, C.byref(out), _stream(stream))
    if st not in _OUTCOMES or not out.value:
        _check(st)
    try:
        return _scs_results(out)
    finally:
        lib().ezo_scs_free(out)


def inflate_batch(robot: Robot, envs, paths, params: Params, path_env=None, seg_np=None, sequential=2,
                  stream_base: int = 0, A0=None, b0=None, stream=None):
    """Many paths over several obstacle sets through ezo_inflate_batch:
    paths is a list of vertex arrays [n_verts_i, n]; returns one list of
    (segment index, SegmentResult) per path."""
    envs = list(envs)
    arr = (_P * len(envs))(*[e.h for e in envs])
    verts = np.ascontiguousarray(np.concatenate([np.asarray(p, dtype=np.float64) for p in paths]), dtype=np.float64)
    lens = np.ascontiguousarray([np.asarray(p).shape[0] - 1 for p in paths], dtype=np.int32)
    pe = None if path_env is None else np.ascontiguousarray(path_env, dtype=np.int32)
    sn = None if seg_np is None else np.ascontiguousarray(seg_np, dtype=np.int32)
    Ap, bp, m0, keep = _domain(A0, b0)
    out = (_P * len(paths))()
    st = lib().ezo_inflate_batch(robot.h, len(envs), arr, len(paths), _ip(lens), _dp(verts),
                                 _ip(pe) if pe is not None else None, _ip(sn) if sn is not None else None, Ap, bp,
                                 m0, C.byref(params), _path_mode(sequential), stream_base, out, _stream(stream))
    if st not in _OUTCOMES or not out[0]:
        _check(st)
    try:
        return [_scs_results(out[i]) for i in range(len(paths))]
    finally:
        for i in range(len(paths)):
            lib().ezo_scs_free(out[i])


class Surrogate:
    """ezo_surrogate: the BF16 MLP signed-distance estimate (not in the paper)."""

    def __init__(self, robot: Robot, seed: int = 1):
        h = _P()
        _check(lib().ezo_surrogate_create(robot.h, seed, C.byref(h)))
        self.h = h
        self.robot = robot
        self.n_params = int(lib().ezo_surrogate_num_params())

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.ezo_surrogate_free(self.h)
            self.h = None

    def params(self) -> np.ndarray:
        o = np.zeros(self.n_params, dtype=np.float32)
        _check(lib().ezo_surrogate_get_params(self.h, o.ctypes.data_as(C.POINTER(C.c_float))))
        return o

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        _check(lib().ezo_surrogate_set_params(self.h, p.ctypes.data_as(C.POINTER(C.c_float))))

    def train(self, env: Env, n_samples: int, epochs: int, batch: int = 4096, lr: float = 1e-3, data_seed: int = 7,
              label_lo: float = -0.1, label_hi: float = 0.3, stream=None) -> np.ndarray:
        losses = np.zeros(epochs, dtype=np.float32)
        _check(lib().ezo_surrogate_train(self.h, env.h, n_samples, epochs, batch, lr, data_seed, label_lo, label_hi,
                                         losses.ctypes.data_as(C.POINTER(C.c_float)), _stream(stream)))
        return losses

    def grad(self, q_dev, t_dev, stream=None):
        n, N = q_dev.shape
        g = np.zeros(self.n_params, dtype=np.float32)
        loss = C.c_float()
        _check(lib().ezo_surrogate_grad(self.h, C.c_void_p(q_dev.data_ptr()), _ld(q_dev), C.c_void_p(t_dev.data_ptr()),
                                        N, g.ctypes.data_as(C.POINTER(C.c_float)), C.byref(loss), _stream(stream)))
        return float(loss.value), g

    def predict(self, q_dev, out_dev, stream=None):
        n, N = q_dev.shape
        _check(lib().ezo_surrogate_predict(self.h, C.c_void_p(q_dev.data_ptr()), _ld(q_dev), N,
                                           C.c_void_p(out_dev.data_ptr()), _stream(stream)))

    def timed_out(self, reset: bool = False, stream=None) -> bool:
        """Whether a bounded wait of the tensor-core forward pass gave up."""
        out = _I32()
        _check(lib().ezo_surrogate_status(self.h, C.byref(out), 1 if reset else 0, _stream(stream)))
        return bool(out.value)
