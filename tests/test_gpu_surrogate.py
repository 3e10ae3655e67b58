"""The BF16 tensor-core MLP surrogate against its FP64 oracle: gradients of
one batch per parameter tensor (relative L2 error <= 1e-2, the BF16 bound),
predictions, and training progress on exact signed-distance labels."""
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


def test_surrogate_gradient_matches_oracle(ezo):
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
    o = 0
    for name, shp in so.SHAPES:
        c = int(np.prod(shp))
        a, b = g[o:o + c].astype(np.float64), g_ref[o:o + c]
        rel = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)
        assert rel <= 1e-2, (name, rel)
        o += c


def test_surrogate_predict_matches_oracle(ezo):
    rd, _ = _scene()
    robot = ezo.Robot(rd)
    sur = ezo.Surrogate(robot, seed=4)
    rng = np.random.default_rng(2)
    N = 1000  # not a multiple of the 64-row tile
    q = rng.uniform(rd.q_lo, rd.q_hi, size=(N, 7)).astype(np.float32)
    out = torch.empty(N, device="cuda")
    sur.predict(torch.from_numpy(q.T.copy()).cuda(), out)
    torch.cuda.synchronize()
    y_ref, _ = so.forward(gpu_weights_as_used(sur.params()), bf16_round(so.features(q.astype(np.float64))))
    y = out.cpu().numpy()
    assert np.abs(y - y_ref).max() <= 1e-2 * max(1.0, np.abs(y_ref).max())


def test_surrogate_training_learns_signed_distance(ezo):
    rd, env_np = _scene()
    robot, env = ezo.Robot(rd), ezo.Env(env_np)
    sur = ezo.Surrogate(robot, seed=5)
    losses = sur.train(env, n_samples=1 << 18, epochs=4, batch=4096, lr=1e-3, data_seed=11)
    assert np.all(np.isfinite(losses)) and losses[-1] < 0.5 * losses[0]
    # held-out configurations: compare with exact labels
    q = wl.uniform_configs(9, rd, 4096).astype(np.float32)
    out = torch.empty(q.shape[0], device="cuda")
    sur.predict(torch.from_numpy(q.T.copy()).cuda(), out)
    torch.cuda.synchronize()
    sd = np.clip(orc.signed_distance(rd, env_np, q.astype(np.float64)), -0.1, 0.3)
    rmse = float(np.sqrt(np.mean((out.cpu().numpy() - sd) ** 2)))
    assert rmse < 0.5 * float(np.std(sd)), (rmse, float(np.std(sd)))
