"""Benchmark of the EI-ZO hot path on GB300.

One step = inflating the 10-segment seed path of the 7-DOF arm (40 spheres,
64 obstacle spheres) at eps = delta = 0.05 (N_p = 10^4, N_f = 10, N_ms = 60,
N_b = 10, N_it = 50): every round of Algorithm 1 for every segment (all
segments speculatively in one batched run, then the containment skip of
Sec. VI-A). Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--mode graph|host]
  python bench.py --impl reference ...   (the FP64 CPU oracle, bounded samples)
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "configs collision-checked/s; ms per 10-segment SCS inflation at ε=δ=0.05"
WORKLOAD = ("7-DOF DH arm (d=[0.34,0,0.40,0,0.40,0,0.126], 40 spheres r 0.04-0.08, 228 self pairs), "
            "64 obstacle spheres in the 1 m cube 0.5 m ahead, 10-segment collision-free seed path, "
            "eps=delta=0.05, tau=0.5, N_p=1e4, N_f=10, N_ms=60, N_b=10, Delta_max=0.01, N_it=50")
PARAMS = dict(eps=0.05, delta=0.05, tau=0.5, step_back_max=0.01, t_col=1e-3, n_p=10000, n_f=10, n_b=10, n_mix=60,
              n_it_max=50, seed=1)
N_SEEDS = 20
SEGSTATE_BYTES = 112  # sizeof(SegState): per-segment device state read back with the polytopes
# DRAM bytes of one round step (dram__bytes_read.sum + dram__bytes_write.sum,
# ncu, the second round of this workload's 10 segments), summed over the
# step's kernels: sampling = the one-lane and the shared-walk kernels,
# bisection = projection, halvings and end points; None where not captured
# for the current kernels
TRAFFIC = {"sample": 60416 + 46080, "check": 2866688, "bisect": 1279488 + 248064 + 1303296}
# DRAM bytes of one 2e6-configuration checker launch (same ncu capture recipe);
# None until captured for the current kernel
CHECKER_TRAFFIC_2E6 = 56046848 + 139008
KIND_NAMES = ("round_size", "sample", "check", "certify", "bisect", "place", "round_end")


def load_scene():
    from paper_2504_10783_gb300 import workloads as wl
    with open(os.path.join(ROOT, "tests", "golden", "workloads.json")) as f:
        s = json.load(f)["dh7"]
    return wl.dh7_robot(), wl.box_obstacles(s["env_seed"], s["n_obs"]), np.asarray(s["path"])


# ------------------------------------------------------------------ clocks --
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "100", "-i", str(self.index)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 8:
                continue
            try:
                sm.append(float(p[0]))
                smax.append(float(p[1]))
            except ValueError:
                continue
            for nm, v in zip(names, p[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------- multi-rank --
def aggregate_ranks(ms: float, units: float, dist=None):
    """Whole-job timing over replicas: every rank inflates its own path, the
    job time is the slowest rank's and the units add up (weak scaling). With
    no process group the inputs are returned unchanged."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return ms, units
    import torch
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    u = torch.tensor([units], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


# --------------------------------------------------------------- oracle legs --
def oracle_sample(seconds: float, seg_list=None):
    """Runs the FP64 oracle on segments of the bench path until `seconds`
    have passed; returns (checks, elapsed, segments inflated, rounds)."""
    from oracle import ezo_oracle as orc
    rd, env, path = load_scene()
    prm = orc.Params(**PARAMS)
    A0, b0 = orc.joint_box(rd)
    checks = rounds = segs = 0
    t0 = time.perf_counter()
    for k in (seg_list if seg_list is not None else range(path.shape[0] - 1)):
        res = orc.eizo(rd, env, path[k], path[k + 1], A0, b0, prm, stream=k)
        checks += res.checks
        rounds += res.rounds
        segs += 1
        if time.perf_counter() - t0 >= seconds:
            break
    return checks, time.perf_counter() - t0, segs, rounds


def oracle_worker(args):
    """One host core: segments w, w + P, .. of the bench path (cycling, with
    a fresh Philox stream per pass) until `seconds` have passed."""
    w, P, seconds = args
    from oracle import ezo_oracle as orc
    rd, env, path = load_scene()
    K = path.shape[0] - 1
    prm = orc.Params(**PARAMS)
    A0, b0 = orc.joint_box(rd)
    checks = segs = 0
    t0 = time.perf_counter()
    i = w
    while time.perf_counter() - t0 < seconds:
        k = i % K
        res = orc.eizo(rd, env, path[k], path[k + 1], A0, b0, prm, stream=k + 1000 * (i // K))
        checks += res.checks
        segs += 1
        i += P
    return checks, time.perf_counter() - t0, segs


def cpu_leg(seconds: float, workers: int = 1):
    if workers <= 1:
        checks, el, segs, rounds = oracle_sample(seconds)
        print(json.dumps({"checks": checks, "seconds": el, "segments": segs, "rounds": rounds}))
        return
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(workers) as pool:
        res = pool.map(oracle_worker, [(w, workers, seconds) for w in range(workers)])
    print(json.dumps({"checks": sum(r[0] for r in res), "seconds": max(r[1] for r in res),
                      "segments": sum(r[2] for r in res), "workers": workers}))


def run_cpu_baseline(seconds: float = 15.0) -> dict:
    """The FP64 oracle on the host: all cores (one process per core, each on
    its own segments) as the baseline, and one core beside it."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    me = os.path.abspath(__file__)
    out1 = subprocess.run([sys.executable, me, "--cpu-leg", "--seconds", str(seconds)],
                          capture_output=True, text=True, env=env, timeout=600)
    d1 = json.loads(out1.stdout.strip().splitlines()[-1])
    P = max(1, min(os.cpu_count() or 1, 64))
    outp = subprocess.run([sys.executable, me, "--cpu-leg", "--seconds", str(seconds), "--cpu-workers", str(P)],
                          capture_output=True, text=True, env=env, timeout=900)
    dp = json.loads(outp.stdout.strip().splitlines()[-1])
    one = {"value": d1["checks"] / d1["seconds"], "cores": 1, "ms_per_segment": 1e3 * d1["seconds"] / d1["segments"],
           "sample": f"Algorithm 1 on the first {d1['segments']} segment(s) of the bench path ({d1['rounds']} rounds, "
                     f"{d1['checks']} exact checks) in {d1['seconds']:.1f} s on 1 host thread"}
    return {"value": dp["checks"] / dp["seconds"], "unit": "configs/s", "cores": P, "kind": "oracle",
            "sample": f"FP64 numpy oracle, Algorithm 1 on segments of the bench path, {P} processes (one per host "
                      f"core, one numpy thread each): {dp['segments']} segment inflations, {dp['checks']} exact "
                      f"checks in {dp['seconds']:.1f} s",
            "one_core": one}


def oracle_round(seg: int):
    """One round (k = 1) of Algorithm 1 on segment `seg` of the bench path with
    the oracle: sampling, labels, test, bisection, placement."""
    from oracle import ezo_oracle as orc
    rd, env, path = load_scene()
    prm = orc.Params(**PARAMS)
    A0, b0 = orc.joint_box(rd)
    t0 = time.perf_counter()
    ns = orc.batch_size(1, prm.eps, prm.delta, prm.tau, prm.n_p)
    S = orc.hit_and_run(A0, b0, path[seg], path[seg + 1], ns, prm.n_mix, prm.seed, seg, 1)
    rr = orc.eizo_round(rd, env, A0, b0, path[seg], path[seg + 1], 1, prm, S)
    return ns + rr.cand_index.shape[0] * prm.n_b, time.perf_counter() - t0


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    _, _, path = load_scene()
    K = path.shape[0] - 1
    for w in range(args.warmup):
        oracle_round(w % K)
    tot_c = 0
    tot_t = 0.0
    segs = 0
    for s in range(args.steps):
        c, t = oracle_round(s % K)
        tot_c += c
        tot_t += t
        segs += 1
    v = tot_c / tot_t
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "configs/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD + "; one step = round 1 of Algorithm 1 on one segment of the path",
                       "l2": "host oracle"},
            "cpu_baseline": {"value": v, "unit": "configs/s", "cores": 1, "kind": "oracle",
                             "sample": f"round 1 of {segs} segment inflations of the bench path, FP64 numpy oracle"},
            "e2e": {"value": v, "unit": "configs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# --------------------------------------------------- batched and stress workloads --
def _event_ms(torch, stream, fn, label=""):
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    fn()
    b.record(stream)
    b.synchronize()
    ms = a.elapsed_time(b)
    if label:
        print(f"[bench] {label}: {ms:.1f} ms", file=sys.stderr, flush=True)
    return ms


def measure_batched(ezo, torch, stream, scenes, rd, robot, paths=256, speculative=True):
    """Batched form (Sec. VI-A per path, many paths): 8 obstacle sets of
    128-1024 spheres, seed paths of 1-40 segments, per-segment N_p
    log-uniform in [1e3, 1e5]. The wavefront mode (each path in order, the
    current segments of all paths in one batched run per wave; every wave,
    its skip rule and its rounds in one graph launch) and, with
    `speculative`, all segments at once in one graph, against the per-segment
    launch loop of the plain method. Configs/s count the exact checks of the
    segments each mode keeps."""
    from paper_2504_10783_gb300 import workloads as wl
    sc = scenes["dh7_batched"]
    envs_np = [wl.box_obstacles(e["env_seed"], e["n_obs"]) for e in sc["envs"]]
    envs = [ezo.Env(e) for e in envs_np]
    use = sc["paths"][:paths]
    v1, v2, seg_env, path_first = [], [], [], []
    for pth in use:
        verts = np.asarray(pth["path"])
        first = len(v1)
        for k in range(verts.shape[0] - 1):
            v1.append(verts[k])
            v2.append(verts[k + 1])
            seg_env.append(pth["env"])
            path_first.append(first)
    B = len(v1)
    rng = np.random.default_rng(5)
    seg_np = np.round(10 ** rng.uniform(3, 5, B)).astype(np.int32)
    prm = ezo.Params.make(eps=0.05, delta=0.05, n_p=10000, n_f=10, n_b=10, n_mix=60, n_it_max=50, seed=1)
    bt = ezo.Batch(robot, envs, np.asarray(v1), np.asarray(v2), prm, seg_env=seg_env, seg_np=seg_np,
                   seg_stream=np.arange(B), path_first=path_first)

    def kept_checks():
        c = k = 0
        for g in range(B):
            if bt.segment(g).status not in (ezo.SEG_SKIPPED, ezo.SEG_IDLE):
                k += 1
                c += sum(bt.check_split(g))
        return c, k

    out = {"paths": len(use), "segments": B, "samples_per_round": int(seg_np.sum()),
           "obstacles": [e["n_obs"] for e in sc["envs"]]}
    t_wave = [_event_ms(torch, stream, lambda: (bt.reset(), bt.run_path(sequential=2, mode=ezo.RUN_GRAPH)),
                        "wavefront graph") for _ in range(2)]
    c_wave, k_wave = kept_checks()
    polys_wave = bt.polytopes()
    t_loop = _event_ms(torch, stream, lambda: (bt.reset(), bt.run_path(sequential=True)), "per-segment loop")
    c_loop, k_loop = kept_checks()
    polys_loop = bt.polytopes()
    same = bool(np.array_equal(polys_wave[0], polys_loop[0]) and
                all(np.array_equal(a, b) for a, b in zip(polys_wave[1], polys_loop[1])))
    out.update({"wavefront_graph_ms": float(min(t_wave)), "wavefront_kept_segments": int(k_wave),
                "wavefront_configs_per_s": c_wave / (min(t_wave) / 1e3),
                "per_segment_loop_ms": float(t_loop), "loop_kept_segments": int(k_loop),
                "loop_configs_per_s": c_loop / (t_loop / 1e3),
                "speedup_wavefront_vs_loop": float(t_loop / min(t_wave)),
                "same_polytopes_wavefront_and_loop": same})
    if speculative:
        t_graph = [_event_ms(torch, stream, lambda: (bt.reset(), bt.run_path(sequential=False, mode=ezo.RUN_GRAPH)),
                             "batched graph") for _ in range(2)]
        c_all = sum(sum(bt.check_split(g)) for g in range(B))
        c_spec, k_spec = kept_checks()
        out.update({"speculative_graph_ms": float(min(t_graph)), "speculative_kept_segments": int(k_spec),
                    "speculative_checks_all_segments": int(c_all),
                    "speculative_configs_per_s_kept": c_spec / (min(t_graph) / 1e3),
                    "speedup_speculative_vs_loop": float(t_loop / min(t_graph))})
    return out


def measure_stress(ezo, torch, stream, scenes, rd, robot, np_stress, sur_samples=1 << 23, graph_speculative=True):
    """Perception-like stress scene: the 7-DOF arm among the 1024-sphere table
    cloud, 64-segment path, np_stress samples per round: the plain method (one
    segment at a time), the same order with every round in one graph, the
    speculative batch, and the in-order run with surrogate-guided
    bisection."""
    from paper_2504_10783_gb300 import workloads as wl
    sc = scenes["table_cloud"]
    env_np = wl.table_cloud_obstacles(sc["cloud_seed"])
    env = ezo.Env(env_np)
    verts = np.asarray(sc["path"])
    K = verts.shape[0] - 1
    prm = ezo.Params.make(eps=0.05, delta=0.05, n_p=np_stress, n_f=10, n_b=10, n_mix=60, n_it_max=50, seed=1)
    bt = ezo.Batch(robot, [env], verts[:-1], verts[1:], prm, seg_stream=np.arange(K),
                   path_first=np.zeros(K, np.int32))

    def counts():
        c = k = 0
        for g in range(K):
            if bt.segment(g).status not in (ezo.SEG_SKIPPED, ezo.SEG_IDLE):
                k += 1
                c += sum(bt.check_split(g))
        return int(c), int(k)

    t_plain = _event_ms(torch, stream, lambda: (bt.reset(), bt.run_path(sequential=True)), "plain")
    c_plain, k_plain = counts()
    t_wave = _event_ms(torch, stream, lambda: (bt.reset(), bt.run_path(sequential=2, mode=ezo.RUN_GRAPH)),
                       "in order, rounds in one graph")
    c_wave, k_wave = counts()
    out = {"segments": K, "obstacles": int(env_np.n_obs), "n_p": np_stress,
           "plain_ms": t_plain, "plain_kept_checks": c_plain, "plain_kept": k_plain,
           "in_order_graph_ms": t_wave, "in_order_graph_kept_checks": c_wave}
    if graph_speculative:
        t_batch = _event_ms(torch, stream, lambda: (bt.reset(), bt.run_path(sequential=False, mode=ezo.RUN_GRAPH)),
                            "batched")
        c_batch, k_batch = counts()
        out.update({"batched_ms": t_batch, "batched_kept_checks": c_batch, "batched_kept": k_batch})
    sur = ezo.Surrogate(robot, seed=7)
    t_train = _event_ms(torch, stream, lambda: sur.train(env, n_samples=sur_samples, epochs=4, batch=4096,
                                                         lr=1e-3, data_seed=13), "surrogate training")
    bt.attach_surrogate(sur, 0.0)
    t_wave_sur = _event_ms(torch, stream, lambda: (bt.reset(), bt.run_path(sequential=2, mode=ezo.RUN_GRAPH)),
                           "in order + surrogate")
    c_wave_sur, _ = counts()
    evals = sum(bt.surrogate_evals(g) for g in range(K))
    out.update({"surrogate_train_ms": t_train, "surrogate_train_samples": sur_samples,
                "in_order_surrogate_ms": t_wave_sur, "in_order_surrogate_kept_checks": c_wave_sur,
                "surrogate_evals": int(evals)})
    return out


def run_workload(args):
    """--workload batched: the batched form (measure_batched, all three
    modes). --workload stress: the stress scene at --np-stress samples per
    round (measure_stress). --workload surrogate: the MLP's forward pass alone
    on 2^rows_log2 configurations."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2504_10783_gb300 import ezo, workloads as wl
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    with open(os.path.join(ROOT, "tests", "golden", "workloads.json")) as f:
        scenes = json.load(f)
    rd = wl.dh7_robot()
    robot = ezo.Robot(rd)
    out = {"workload": args.workload}
    if args.workload == "batched":
        out.update(measure_batched(ezo, torch, stream, scenes, rd, robot, paths=args.paths))
    elif args.workload == "surrogate":
        # inference of the BF16 MLP alone (tensor-core forward pass with the
        # features computed in the kernel) on 2^rows_log2 configurations; the
        # weights are the seeded initialisation (the time does not depend on them)
        nb = 1 << args.rows_log2
        sur = ezo.Surrogate(robot, seed=6)
        q = torch.from_numpy(wl.uniform_configs(11, rd, nb).astype(np.float32).T.copy()).cuda()
        y = torch.empty(nb, device="cuda")
        for _ in range(args.warmup):
            sur.predict(q, y)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            sur.predict(q, y)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        gemm_flops = 2.0 * nb * (64 * 256 + 2 * 256 * 256)
        peak, src = bf16_peak()
        tf = gemm_flops / (ms / 1e3) / 1e12
        out.update({"rows": nb, "ms": ms, "rows_per_s": nb / (ms / 1e3), "gemm_tflops": tf, "peak": peak,
                    "peak_source": src, "frac": tf / peak, "nan_outputs": int(torch.isnan(y).sum()),
                    "wait_timed_out": sur.timed_out()})
    elif args.workload == "train":
        # surrogate training on exact labels of the benchmark scene: 2^rows_log2
        # uniform configurations labelled by the exact signed-distance kernel,
        # `steps` epochs of mini-batches of 3200 (every hidden-layer GEMM of the
        # forward and backward passes on tcgen05), Adam; CUDA events around
        # the whole call (labels, features, GEMMs, Adam)
        nb = 1 << args.rows_log2
        s7 = scenes["dh7"]
        env = ezo.Env(wl.box_obstacles(s7["env_seed"], s7["n_obs"]))
        sur = ezo.Surrogate(robot, seed=6)
        for _ in range(args.warmup):
            sur.train(env, n_samples=4 * 3200, epochs=1, batch=3200, lr=1e-3, data_seed=3)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        losses = sur.train(env, n_samples=nb, epochs=args.steps, batch=3200, lr=1e-3, data_seed=12)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        # GEMM flops per sample and epoch: forward 2 (64 + 256 + 256) 256,
        # backward (dW3, dZ2, dW2, dZ1, dW1) 2 (4 x 256 + 64) 256
        gemm_per_sample = 2.0 * 256 * (64 + 256 + 256) + 2.0 * 256 * (4 * 256 + 64)
        peak, src = bf16_peak()
        tf = gemm_per_sample * nb * args.steps / (ms / 1e3) / 1e12
        out.update({"samples": nb, "epochs": args.steps, "batch": 3200, "ms": ms,
                    "samples_per_s": nb * args.steps / (ms / 1e3), "gemm_flops_per_sample": gemm_per_sample,
                    "gemm_tflops_whole_call": tf, "peak": peak, "peak_source": src, "frac_whole_call": tf / peak,
                    "what": "GEMM flops over the whole training call (labels, features, Adam included): "
                            "a lower bound on the GEMM kernels' rate",
                    "loss_per_epoch": [float(x) for x in losses]})
    else:
        out.update(measure_stress(ezo, torch, stream, scenes, rd, robot, args.np_stress))
    print(json.dumps(out))


# ------------------------------------------------------------------- GPU leg --
def bf16_peak():
    """Dense BF16 peak in TFLOP/s for a kernel timed alone: the measured burst
    figure of this GPU pool when the peaks file is present, else 1900."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"]), "measured (cuBLAS bf16 burst)"
    except (OSError, KeyError, ValueError):
        return 1900.0, "fallback"


def measure_surrogate(ezo, torch, robot, env, rd, env_np, batches, mode, stream, flush, K, args):
    """Trains the BF16 MLP on 10^7 exact labels (4 epochs, mini-batches of
    3200), reports its false-negative / false-positive rates on 2^20 fresh
    uniform configurations and on the exact bisection midpoints of the
    path's last rounds, and times the path with surrogate-guided bisection on
    the same Philox seeds as the timed exact steps (mean over the seeds, like
    ms_per_step)."""
    from paper_2504_10783_gb300 import workloads as wl
    sur = ezo.Surrogate(robot, seed=6)
    n_train = 10_000_000
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sur.train(env, n_samples=n_train, epochs=4, batch=3200, lr=1e-3, data_seed=12)
    e1.record(stream)
    e1.synchronize()
    train_ms = e0.elapsed_time(e1)
    q = torch.from_numpy(wl.uniform_configs(10, rd, 1 << 20).astype(np.float32).T.copy()).cuda()  # held out
    y = torch.empty(q.shape[1], device="cuda")
    flags = torch.empty(q.shape[1], dtype=torch.uint8, device="cuda")
    sur.predict(q, y)
    ezo.check_collision(robot, env, q, flags)
    torch.cuda.synchronize()
    yv, col = y.cpu().numpy(), flags.cpu().numpy().astype(bool)
    fn0 = float(np.mean(yv[col] >= 0.0)) if col.any() else 0.0
    fp0 = float(np.mean(yv[~col] < 0.0))
    # the exact bisection midpoints of round 1 of every segment (seed 1, run
    # step by step up to the bisection): midpoint s of a candidate is
    # c_proj + f_s (c - c_proj) with f_s from the decisions before it, and its
    # exact label is decision s
    bt0 = batches[0]
    bt0.reset()
    for step in range(5):
        bt0.step(step)
    bt0.sync()
    n_b = PARAMS["n_b"]
    mids, labs = [], []
    for g in range(K):
        st = bt0.state(g)
        nc = st["n_cand"]
        if nc == 0:
            continue
        S = bt0.read(g, "samples")[:, : st["n_samples"]].T.astype(np.float64)
        c = S[bt0.read(g, "cand_idx")[:nc]]
        v1, v2 = bt0.v1[g], bt0.v2[g]
        e = v2 - v1
        al = np.clip(((c - v1) @ e) / max(float(e @ e), 1e-300), 0.0, 1.0)
        pp = v1[None, :] + al[:, None] * e[None, :]
        bits = bt0.read(g, "bits")[:nc]
        lo, hi = np.zeros(nc), np.ones(nc)
        for s_ in range(n_b):
            f = 0.5 * (lo + hi)
            d = ((bits >> s_) & 1).astype(bool)
            mids.append((pp + f[:, None] * (c - pp)).astype(np.float32))
            labs.append(d)
            hi = np.where(d, f, hi)
            lo = np.where(d, lo, f)
    fn_mid = fp_mid = None
    n_mid = 0
    if mids:
        qm = torch.from_numpy(np.ascontiguousarray(np.concatenate(mids).T)).cuda()
        ym = torch.empty(qm.shape[1], device="cuda")
        sur.predict(qm, ym)
        torch.cuda.synchronize()
        ymv, lm = ym.cpu().numpy(), np.concatenate(labs)
        n_mid = int(lm.size)
        fn_mid = float(np.mean(ymv[lm] >= 0.0)) if lm.any() else 0.0
        fp_mid = float(np.mean(ymv[~lm] < 0.0)) if (~lm).any() else 0.0
    times = []
    samp = bisc = evals = 0
    for bt in batches:
        bt.attach_surrogate(sur, 0.0)
        bt.reset()
        bt.run_path(sequential=False, mode=mode)  # builds this batch's graph with the surrogate step
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        bt.reset()
        bt.run_path(sequential=False, mode=mode)
        b.record(stream)
        b.synchronize()
        times.append(a.elapsed_time(b))
        for g in range(K):
            x, y2 = bt.check_split(g)
            samp += x
            bisc += y2
            evals += bt.surrogate_evals(g)
        bt.attach_surrogate(None)
    ns = len(batches)
    # each candidate takes n_b surrogate steps, then one exact check of its end
    # point, and n_b exact steps when that end point is free
    n_b = PARAMS["n_b"]
    n_cand = evals / n_b
    n_fail = max(0.0, (bisc - n_cand) / n_b)
    # inference throughput of the MLP alone (features, three BF16 GEMMs with
    # fused bias + SiLU, output layer) on 2^20 configurations, timed alone
    # against the burst BF16 peak
    nb = 1 << 20
    qb = torch.from_numpy(wl.uniform_configs(11, rd, nb).astype(np.float32).T.copy()).cuda()
    yb = torch.empty(nb, device="cuda")
    for _ in range(3):
        sur.predict(qb, yb)
    e0.record(stream)
    for _ in range(10):
        sur.predict(qb, yb)
    e1.record(stream)
    e1.synchronize()
    inf_ms = e0.elapsed_time(e1) / 10
    gemm_flops = 2.0 * nb * (64 * 256 + 2 * 256 * 256)  # the three hidden-layer GEMMs (features padded to 64)
    peak_bf16, peak_src = bf16_peak()
    inf_tf = gemm_flops / (inf_ms / 1e3) / 1e12
    return {"ms_per_path": float(np.mean(times)), "ms_per_path_seed1": float(times[0]), "seeds": ns,
            "train_ms": train_ms, "train_samples": n_train, "epochs": 4,
            "fn_rate_margin0": fn0, "fp_rate_margin0": fp0,
            "bisection_midpoints": {"count": n_mid, "fn_rate_margin0": fn_mid, "fp_rate_margin0": fp_mid,
                                    "what": "exact midpoints of round 1's bisections (exact run, seed 1, all "
                                            "segments), labelled by the exact decisions"},
            "sample_checks_per_path": samp / ns,
            "bisection_checks_per_path": bisc / ns, "surrogate_evals_per_path": evals / ns,
            "held_out_configs": 1 << 20,
            "end_points_verified_in_collision": (1.0 - n_fail / n_cand) if n_cand else None,
            "inference": {"batch": nb, "ms": inf_ms, "gemm_tflops": inf_tf, "peak": peak_bf16, "peak_source": peak_src,
                          "frac": inf_tf / peak_bf16,
                          "what": "GEMM flops of the three hidden layers / time of the whole forward pass"},
            "what": "same path, bisection steps on the BF16 MLP, end points verified exactly, exact fallback"}


def measure_checker(ezo, torch, robot, env, rd, stream, flush, props, sm_max, flops_cfg, N=2_000_000, reps=10,
                    traffic=None):
    """ezo_check_collision on N uniform configurations (configurations and
    flags resident in HBM, L2 flushed between launches), CUDA events."""
    g = torch.Generator(device="cuda").manual_seed(1)
    lo = torch.tensor(rd.q_lo, dtype=torch.float32, device="cuda")[:, None]
    hi = torch.tensor(rd.q_hi, dtype=torch.float32, device="cuda")[:, None]
    q = lo + (hi - lo) * torch.rand((rd.n, N), generator=g, device="cuda")
    flags = torch.empty(N, dtype=torch.uint8, device="cuda")
    for _ in range(3):
        ezo.check_collision(robot, env, q, flags)
    ms = 0.0
    for _ in range(reps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ezo.check_collision(robot, env, q, flags)
        e1.record(stream)
        e1.synchronize()
        ms += e0.elapsed_time(e1)
    per = ms / reps
    tf = N * flops_cfg / (per / 1e3) / 1e12
    peak = props.multi_processor_count * 128 * 2 * sm_max * 1e6 / 1e12
    # the pair tests run per configuration: the count of every pair less the
    # obstacle pairs of the base-frame spheres decided once per obstacle set
    static = ezo.check_static_spheres(robot, env)
    tested = flops_cfg - 8.0 * static * env.spheres.shape[0]
    tf_tested = N * tested / (per / 1e3) / 1e12
    return {"batch": N, "configs_per_s": N / (per / 1e3), "ms_per_launch": per,
            "roofline": {"bound": "alu", "achieved": tf, "peak": peak, "unit": "TFLOP/s", "frac": tf / peak,
                         "flops_per_config": flops_cfg,
                         "static_spheres": static, "flops_per_config_tested": tested,
                         "achieved_tested": tf_tested, "frac_tested": tf_tested / peak,
                         "flops_note": "flops_per_config counts every pair (8 flops per robot-obstacle and "
                                       "self pair, plus the kinematics); the obstacle pairs of the first "
                                       "static_spheres robot spheres, "
                                       "on the fixed base frame and clear of every obstacle, are decided once "
                                       "per obstacle set, so the pair tests run per configuration come to "
                                       "flops_per_config_tested",
                         "traffic": traffic},
            "paper_context": "paper: ~8.6 M configs/s, Franka (1187 pairs), RTX 3090, same batch size",
            "launches": reps + 3}



def measure_fk_error(ezo, torch, robot, bt, K):
    """FP32 forward kinematics of the collision checker against FP64 (the same
    chain from the FP64 constants) on the samples of the last round of every
    segment of a bench batch: per configuration, the largest distance between
    a sphere's FP32 and FP64 centre, in metres (ezo_fk_error)."""
    qs = []
    for g in range(K):
        ns = bt.state(g)["n_samples"]
        qs.append(bt.read(g, "samples")[:, :ns])
    q = torch.from_numpy(np.ascontiguousarray(np.concatenate(qs, axis=1))).cuda()
    err = torch.empty(q.shape[1], dtype=torch.float32, device="cuda")
    ezo.fk_error(robot, q, err)
    e = err.cpu().numpy().astype(np.float64)
    return {"configs": int(e.size), "max_m": float(e.max()), "p99_m": float(np.quantile(e, 0.99)),
            "median_m": float(np.median(e)), "label_band_m": 1e-5,
            "what": "per configuration: max over the 40 spheres of |c_FP32 - c_FP64| (FP32 = the checker's "
                    "kinematics), over the last round's samples of every segment of the seed-1 path"}


def measure_forest(ezo, torch, stream, flush, props, sm_max, N=2_000_000, reps=10):
    """Forest benchmark of Sec. V: the point robot among 15 disks of r = 0.35.
    The collision checker on N uniform configurations (the paper's batch and
    its 19.9 M configs/s on an RTX 3090), and the seed path inflated with the
    paper's Forest parameters (eps = 0.01, delta = 0.05, N_p = 1000,
    N_f = 10, N_ms = 30, Delta_max = 0.01), Philox seeds 1..5."""
    from paper_2504_10783_gb300 import workloads as wl
    with open(os.path.join(ROOT, "tests", "golden", "workloads.json")) as f:
        s = json.load(f)["forest"]
    rd, env_np, path = wl.point2_robot(), wl.forest_obstacles(s["forest_seed"]), np.asarray(s["path"])
    robot, env = ezo.Robot(rd), ezo.Env(env_np)
    g = torch.Generator(device="cuda").manual_seed(1)
    q = 10.0 * torch.rand((2, N), generator=g, device="cuda")
    flags = torch.empty(N, dtype=torch.uint8, device="cuda")
    for _ in range(3):
        ezo.check_collision(robot, env, q, flags)
    ms = 0.0
    for _ in range(reps):
        flush.zero_()
        ms += _event_ms(torch, stream, lambda: ezo.check_collision(robot, env, q, flags))
    per = ms / reps
    flops_cfg = ezo.check_flops(robot, env)
    peak = props.multi_processor_count * 128 * 2 * sm_max * 1e6 / 1e12
    K = path.shape[0] - 1
    times, kept = [], []
    for sd in range(1, 6):
        prm = ezo.Params.make(eps=0.01, delta=0.05, n_p=1000, n_f=10, n_b=10, n_mix=30, step_back_max=0.01,
                              n_it_max=50, seed=sd)
        bt = ezo.Batch(robot, [env], path[:-1], path[1:], prm, seg_stream=np.arange(K, dtype=np.uint32),
                       path_first=np.zeros(K, np.int32))
        for _ in range(2):
            bt.reset()
            bt.run_path(sequential=False, mode=ezo.RUN_GRAPH)
        for _ in range(3):
            flush.zero_()
            times.append(_event_ms(torch, stream, lambda: (bt.reset(),
                                                           bt.run_path(sequential=False, mode=ezo.RUN_GRAPH))))
        kept.append(int(sum(bt.segment(k).status != ezo.SEG_SKIPPED for k in range(K))))
    return {"checker": {"batch": N, "configs_per_s": N / (per / 1e3), "ms_per_launch": per,
                        "roofline": {"bound": "alu", "achieved": N * flops_cfg / (per / 1e3) / 1e12, "peak": peak,
                                     "unit": "TFLOP/s", "frac": N * flops_cfg / (per / 1e3) / 1e12 / peak},
                        "paper_context": "paper: ~19.9 M configs/s in the Forest, RTX 3090, same batch size"},
            "path": {"segments": K, "ms_median": float(np.median(times)), "ms_p90": float(np.percentile(times, 90)),
                     "kept_segments": kept, "seeds": "1..5"},
            "launches": 3 + reps}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--mode", default="graph", choices=["graph", "host"])
    ap.add_argument("--cpu-leg", action="store_true")
    ap.add_argument("--seconds", type=float, default=15.0)
    ap.add_argument("--cpu-workers", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-surrogate", action="store_true")
    ap.add_argument("--only-checker", action="store_true",
                    help="only the collision checker on 2e6 configurations (for profiling)")
    ap.add_argument("--no-extras", action="store_true",
                    help="only the timed path steps and the kernel pass (no plain, surrogate or checker legs)")
    ap.add_argument("--no-tune", action="store_true",
                    help="keep the default launch shapes of the round kernels (for profiling runs)")
    ap.add_argument("--workload", default="path", choices=["path", "batched", "stress", "surrogate", "train"])
    ap.add_argument("--rows-log2", type=int, default=20,
                    help="surrogate: log2 of the configurations per call; train: log2 of the labelled samples")
    ap.add_argument("--paths", type=int, default=256, help="batched: number of seed paths")
    ap.add_argument("--np-stress", type=int, default=1_000_000, help="stress: samples per round and segment")
    args = ap.parse_args()
    if args.cpu_leg:
        cpu_leg(args.seconds, args.cpu_workers)
        return
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload != "path":
        run_workload(args)
        return

    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    import __graft_entry__
    __graft_entry__.build()
    from paper_2504_10783_gb300 import ezo

    rd, env_np, path = load_scene()
    robot, env = ezo.Robot(rd), ezo.Env(env_np)
    if args.only_checker:
        # autotuner (4 lane counts x 4 launches), 3 warm-up and 10 timed launches
        flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
        props = torch.cuda.get_device_properties(local)
        print(json.dumps(measure_checker(ezo, torch, robot, env, rd, torch.cuda.current_stream(), flush, props,
                                         2070.0, ezo.check_flops(robot, env))))
        return
    K = path.shape[0] - 1
    mode = ezo.RUN_GRAPH if args.mode == "graph" else ezo.RUN_HOST_LOOP
    streams = np.arange(K, dtype=np.uint32) + 1000 * rank  # each rank inflates its own random draw
    # one batch per Philox seed 1..N_SEEDS; step i inflates the path with seed 1 + i % N_SEEDS
    batches = [ezo.Batch(robot, [env], path[:-1], path[1:], ezo.Params.make(**dict(PARAMS, seed=sd)),
                         seg_stream=streams, path_first=np.zeros(K, np.int32)) for sd in range(1, N_SEEDS + 1)]
    bt = batches[0]
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")  # > 129 MB L2

    def step(i, run_mode=mode):
        b = batches[i % N_SEEDS]
        b.reset()
        b.run_path(sequential=False, mode=run_mode)

    # launch shapes of the round kernels from the autotuner (timed on the
    # seed-1 batch; the other batches are of the same class and take the
    # cached shape), then every batch once (graph instantiation)
    shape = batches[0].shape()
    if not args.no_tune:
        shape = batches[0].tune(reps=2)
        for b in batches[1:]:
            b.tune(reps=2)
    for i in range(N_SEEDS):
        step(i)
    for i in range(max(3, args.warmup)):
        step(i)
    torch.cuda.synchronize()

    # per-seed work: exact checks (sample labels, bisection midpoints), FP32
    # FLOPs of the walks, kept segments and rounds (the same on every run)
    flops_cfg = ezo.check_flops(robot, env)
    pairs_cfg = rd.n_spheres * env_np.n_obs + rd.self_pairs.shape[0]
    work = []
    for b in batches:
        samp = bisc = sflops = kept = kept_checks = 0
        for g in range(K):
            x, y2 = b.check_split(g)
            samp += x
            bisc += y2
            sflops += b.sample_flops(g)
            if b.segment(g).status != ezo.SEG_SKIPPED:
                kept += 1
                kept_checks += x + y2
        work.append({"sample_checks": samp, "bisection_checks": bisc, "sample_flops": sflops, "kept": kept,
                     "kept_checks": kept_checks, "rounds": b.summary()["rounds"]})

    # ---- timed region: device-resident inputs, L2 flushed between steps ----
    clk = ClockSampler(local)
    clk.start()
    barrier()
    torch.cuda.synchronize()
    times = []
    launches = 0
    units = 0
    units_all_segments = 0
    for i in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step(i)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        w = work[i % N_SEEDS]
        # useful work: the exact checks of the segments the skip rule keeps
        units += w["kept_checks"]
        units_all_segments += w["sample_checks"] + w["bisection_checks"]
        # the reset and the first sizing, 8 kernels per round (the one-lane
        # and the shared-walk sampler, one of which returns at once; labels;
        # certification; the bisection's projection, halvings and end
        # points; the placement that closes the round), containment and the
        # skip rule
        launches += 8 * w["rounds"] + 4
    torch.cuda.synchronize()
    barrier()
    clocks = clk.stop()
    ms = float(np.sum(times))
    ms, units_all = aggregate_ranks(ms, units, dist)
    value = units_all / (ms / 1e3)

    # ---- roofline of the dominant kernel (FP32 ALU bound): the same steps
    #      in host-loop mode with CUDA events around every kernel launch on
    #      the launching stream (a graph launch cannot be split by events) ----
    props = torch.cuda.get_device_properties(local)
    sm_max = clocks.get("sm_max_mhz") or 2070.0
    peak = props.multi_processor_count * 128 * 2 * sm_max * 1e6 / 1e12  # TFLOP/s, FP32 FMA
    ezo.profile_enable(True)
    ezo.profile_reset()
    for i in range(args.steps):
        flush.zero_()
        step(i, ezo.RUN_HOST_LOOP)
    torch.cuda.synchronize()
    prof = ezo.profile_read()
    ezo.profile_enable(False)
    other_launches = int(sum(v[1] for v in prof.values()))
    tot = {"check": 0.0, "bisect": 0.0, "sample": 0.0}
    for i in range(args.steps):
        w = work[i % N_SEEDS]
        tot["check"] += w["sample_checks"] * flops_cfg
        tot["bisect"] += w["bisection_checks"] * flops_cfg
        tot["sample"] += w["sample_flops"]
    dom = max(tot, key=lambda k: prof[k][0])
    ach = tot[dom] / (prof[dom][0] / 1e3) / 1e12
    path_tf = sum(tot.values()) / (float(np.sum(times)) / 1e3) / 1e12
    per_kernel = {}
    for k in tot:
        a_k = tot[k] / (prof[k][0] / 1e3) / 1e12
        per_kernel[k] = {"achieved": a_k, "frac": a_k / peak, "ms_per_step": prof[k][0] / args.steps,
                         "launches_per_step": prof[k][1] / args.steps, "flops_per_step": tot[k] / args.steps,
                         "traffic": TRAFFIC.get(k)}
    per_kernel["sample"]["flops"] = "(2mn + 5m + 6n) x N_ms per walk (m rows, n joints)"
    per_kernel["check"]["flops"] = (f"{flops_cfg:.0f} per configuration (8 per pair x {pairs_cfg} pairs + FK; the "
                                    f"obstacle pairs of {ezo.check_static_spheres(robot, env)} base-frame spheres "
                                    "are decided once per obstacle set)")
    per_kernel["bisect"]["flops"] = f"{flops_cfg:.0f} per midpoint check (FP64 projection and planes not counted)"
    roofline = {"kernel": dom, "bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                "frac": ach / peak, "traffic": TRAFFIC.get(dom),
                "per_launch_ms": prof[dom][0] / prof[dom][1],
                "peak_note": f"FP32 FMA peak = {props.multi_processor_count} SMs x 128 lanes x 2 x {sm_max:.0f} MHz",
                "measured_in": "host-loop pass over the same steps, CUDA events around each launch",
                "kernels": per_kernel,
                "kernel_ms_per_step": {k: round(v[0] / args.steps, 4) for k, v in prof.items()},
                "whole_path": {"achieved": path_tf, "frac": path_tf / peak,
                               "what": "all algorithmic FP32 FLOPs of the path (walks + exact checks) / step time"}}
    # calibration beside the nominal peak: the achieved rate of independent
    # FMA chains on every SM (outside the timed region)
    ffma = ezo.probe_fp32_fma(stream)
    roofline["fma_probe"] = {"measured": ffma, "unit": "TFLOP/s", "frac_of_nominal": ffma / peak,
                             "kernel_frac_of_measured": ach / ffma}
    w0 = work[0]
    samp, bisc, kept = w0["sample_checks"], w0["bisection_checks"], w0["kept"]
    checks_per_step = units / args.steps

    # ---- the plain method for comparison: one segment at a time in path order
    #      (host launch loop, containment skip before each segment) ----
    plain_ms = []
    for b_ in ([] if args.no_extras else batches):  # the same seeds as the timed steps
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b_.reset()
        b_.run_path(sequential=True, mode=ezo.RUN_HOST_LOOP)
        e1.record(stream)
        e1.synchronize()
        plain_ms.append(e0.elapsed_time(e1))
    plain = None
    if plain_ms:
        kept_plain = sum(bt.segment(g).status != ezo.SEG_SKIPPED for g in range(K))
        plain = {"ms_per_path": float(np.mean(plain_ms)), "ms_per_path_seed1": float(plain_ms[0]),
                 "seeds": len(plain_ms), "kept_segments_seed1": int(kept_plain),
                 "what": "sequential per-segment inflation (paper's order), host-driven launch loop, mean over seeds"}

    # ---- batched + learned surrogate: train on exact
    #      labels, then the same path with surrogate-guided bisection ----
    sur_info = None
    if not args.no_surrogate and not args.no_extras:
        sur_info = measure_surrogate(ezo, torch, robot, env, rd, env_np, batches, mode, stream, flush, K, args)
        exact_mean = float(np.mean([w["sample_checks"] + w["bisection_checks"] for w in work]))
        sur_info["exact_checks_per_path_without_surrogate"] = exact_mean
        sur_info["exact_checks_saved_per_path"] = exact_mean - (sur_info["sample_checks_per_path"] +
                                                                sur_info["bisection_checks_per_path"])
        sur_info["exact_only_ms_per_path"] = float(np.mean(times))

    # ---- the collision checker alone on the paper's batch size (2e6 configs) ----
    checker = checker_1e8 = forest = {"launches": 0}
    envs_more = {}
    if not args.no_extras:
        forest = measure_forest(ezo, torch, stream, flush, props, sm_max)
        checker = measure_checker(ezo, torch, robot, env, rd, stream, flush, props, sm_max, flops_cfg,
                                  traffic=CHECKER_TRAFFIC_2E6)
        checker_1e8 = measure_checker(ezo, torch, robot, env, rd, stream, flush, props, sm_max, flops_cfg,
                                      N=100_000_000, reps=3)
        # the checker on two more obstacle sets:
        # the planar arm among 16 disks and the arm among a 1024-sphere cloud
        from paper_2504_10783_gb300 import workloads as wl
        with open(os.path.join(ROOT, "tests", "golden", "workloads.json")) as f:
            pl = json.load(f)["planar3"]
        envs_more = {}
        for name, rdx, envx in (("planar3_16_disks", wl.planar3_robot(), wl.Env("planar", np.asarray(pl["obstacles"]))),
                                ("dh7_table_cloud_1024", rd, wl.table_cloud_obstacles(31))):
            rx, ex = ezo.Robot(rdx), ezo.Env(envx)
            envs_more[name] = measure_checker(ezo, torch, rx, ex, rdx, stream, flush, props, sm_max,
                                              ezo.check_flops(rx, ex))

    # ---- forward-kinematics error of the checker against FP64 ----
    fk_err = measure_fk_error(ezo, torch, robot, batches[0], K)

    # ---- batched form (8 obstacle sets, 256 paths, uneven N_p) and the
    #      perception-like stress scene (1024 spheres, 64 segments) ----
    batched = stress = None
    if not args.no_extras:
        with open(os.path.join(ROOT, "tests", "golden", "workloads.json")) as f:
            scenes = json.load(f)
        batched = measure_batched(ezo, torch, stream, scenes, rd, robot, paths=256, speculative=False)
        stress = measure_stress(ezo, torch, stream, scenes, rd, robot, np_stress=100_000, sur_samples=1 << 22)

    # ---- end to end through the public API with host buffers ----
    # the step's inputs in pinned host memory
    v1h = torch.from_numpy(np.ascontiguousarray(path[:-1])).pin_memory().numpy()
    v2h = torch.from_numpy(np.ascontiguousarray(path[1:])).pin_memory().numpy()
    e2e_times = []
    d2h = 0
    e2e_units = 0
    for b in batches:
        b.polytopes()  # the page-locked readback buffers, made once per batch
    for i in range(args.steps):
        b = batches[i % N_SEEDS]
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        b.reset(v1h, v2h)
        b.run_path(sequential=False, mode=mode)
        status, As, bs = b.polytopes()  # every segment's polytope in three copies
        d2h = int(K * (b.rows_read * (rd.n + 1) * 8 + SEGSTATE_BYTES))
        e2e_times.append(time.perf_counter() - t0)
        w = work[i % N_SEEDS]
        e2e_units += w["kept_checks"]
    e2e_s = float(np.sum(e2e_times))
    e2e = {"value": world * e2e_units / e2e_s, "unit": "configs/s",
           "h2d_bytes_per_step": int(v1h.nbytes + v2h.nbytes), "d2h_bytes_per_step": int(d2h),
           "ms_per_step": 1e3 * e2e_s / args.steps}

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    line = {"metric": METRIC, "value": value, "unit": "configs/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "mode": args.mode, "segments": K, "seeds": f"1..{N_SEEDS}, step i: seed 1 + i % {N_SEEDS}",
                       "checks_per_step": checks_per_step,
                       "value_counts": "exact checks of the segments the skip rule keeps (Sec. VI-A); the "
                                       "speculative run also inflates the segments it then drops",
                       "checks_per_step_all_segments": units_all_segments / args.steps,
                       "seed1": {"kept_segments": kept, "sample_checks": samp,
                                                                      "bisection_checks": bisc},
                       "ms_per_10_segment_path": ms / args.steps,
                       "ms_p50": float(np.percentile(times, 50)), "ms_p90": float(np.percentile(times, 90)),
                       "l2": "flushed between steps (256 MiB write)", "parallelism": f"replicas x{world}",
                       "round_kernel_shape": shape},
            "roofline": roofline, "plain_sequential": plain, "surrogate": sur_info, "checker_2e6": checker, "checker_1e8": checker_1e8, "checker_other_envs_2e6": envs_more,
            "forest": forest, "fk_error": fk_err, "batched": batched, "stress": stress, "e2e": e2e,
            "gpu_launches": launches,
            "gpu_launches_outside_timed_region": other_launches + checker["launches"] + checker_1e8["launches"] +
            forest["launches"] + sum(c["launches"] for c in envs_more.values()) + 4,  # + the FMA probe
            "clocks": clocks}
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = run_cpu_baseline(args.seconds)
    print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
