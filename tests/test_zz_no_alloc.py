"""ezo_inflate_segment_noalloc, called through the C ABI, against the
allocating entry point (a one-segment batch) on the same inputs.

The no-allocation entry point serves callers that cannot allocate device
memory when they need a region (a real-time loop that must not block in
cudaMalloc, or an application that fixes device memory at start-up). Its
working memory is one shared file-scope device array, so two calls in a row
must each start from clean state: the second call inflates a different
segment, and a third repeats the first."""
import ctypes as C
import json
import os

import numpy as np
import pytest

from paper_2504_10783_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _scene():
    with open(os.path.join(GOLDEN, "workloads.json")) as f:
        s = json.load(f)["dh7"]
    return wl.dh7_robot(), wl.box_obstacles(s["env_seed"], s["n_obs"]), np.asarray(s["path"])


def _noalloc(ezo, robot, env, v1, v2, prm, stream_id):
    lib = ezo.lib()
    f = lib.ezo_inflate_segment_noalloc
    f.argtypes = [C.c_void_p, C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(ezo.Params),
                  C.c_uint32, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_int32),
                  C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int64), C.c_void_p]
    n = robot.n
    rows = 2 * n + prm.n_f * prm.n_it_max
    A = np.zeros((rows, n))
    b = np.zeros(rows)
    m, st, rd = C.c_int32(), C.c_int32(), C.c_int32()
    ch = C.c_int64()
    v1 = np.ascontiguousarray(v1, dtype=np.float64)
    v2 = np.ascontiguousarray(v2, dtype=np.float64)
    dp = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))
    status = f(robot.h, env.h, dp(v1), dp(v2), C.byref(prm), stream_id, dp(A), dp(b), C.byref(m), C.byref(st),
               C.byref(rd), C.byref(ch), C.c_void_p(torch.cuda.current_stream().cuda_stream))
    return status, A[: m.value], b[: m.value], st.value, rd.value, ch.value


def test_noalloc_matches_allocating_entry_point_on_consecutive_calls():
    from paper_2504_10783_gb300 import build, ezo
    build.build()
    rd, env_np, path = _scene()
    robot, env = ezo.Robot(rd), ezo.Env(env_np)
    prm = ezo.Params.make(n_p=4000, seed=11)
    # the references first (the allocating path), then a warm-up call: the
    # first call on a device loads the device code and the array
    refs = {seg: ezo.inflate_segment(robot, env, path[seg], path[seg + 1], prm, stream_id=seg) for seg in (0, 3)}
    assert _noalloc(ezo, robot, env, path[5], path[6], prm, 5)[0] == ezo.EZO_OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for seg in (0, 3, 0):
        st, A, b, status, rounds, checks = _noalloc(ezo, robot, env, path[seg], path[seg + 1], prm, seg)
        assert st == ezo.EZO_OK, ezo.lib().ezo_last_error()
        ref = refs[seg]
        assert (status, rounds, checks, A.shape[0]) == (ref.status, ref.rounds, ref.checks, ref.m)
        np.testing.assert_array_equal(A, ref.A)
        np.testing.assert_array_equal(b, ref.b)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, "device memory changed across calls that must not allocate"


def test_noalloc_rejects_oversized_work():
    from paper_2504_10783_gb300 import build, ezo
    build.build()
    rd, env_np, path = _scene()
    robot, env = ezo.Robot(rd), ezo.Env(env_np)
    prm = ezo.Params.make(n_p=1_000_000)
    st, *_ = _noalloc(ezo, robot, env, path[0], path[1], prm, 0)
    assert st == 3  # EZO_ERR_CAPACITY
    assert b"working memory" in ezo.lib().ezo_last_error()
