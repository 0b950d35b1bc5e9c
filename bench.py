"""Benchmark: env-steps/s of a full PPO training iteration (rollout + update) at 4096 robots.

One step = one training iteration of the paper's loop (Sec. 2): 24 policy steps for 4096 robots
(batched actor/critic inference, env-side math with 187 height samples, reward, termination,
curriculum) on the seeded physics stand-in, the critic's last value, GAE with advantage
normalisation, and 5 epochs x 4 minibatches of the clipped PPO update with Algorithm 1 and Adam,
replayed as one CUDA graph.  value = whole-job env-steps/s (robots x steps x iterations / device
time), inputs resident in HBM, L2 flushed between timed iterations.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun (N > 1) every rank trains an independent replica (the method needs no exchange
between learners on different GPUs); time is the max over ranks.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "env-steps/sec (rollout+PPO update) at 4096 envs, BF16 vs FP32 GPU, same accuracy"
WORKLOAD = dict(num_envs=4096, num_steps=24, grid=(17, 11), hidden=(512, 256, 128), epochs=5, minibatches=4)
WORKLOAD_NAME = ("rough-terrain PPO iteration: 4096 robots x 24 steps (B=98304), obs 235 = 48 + 17x11 heights "
                 "(bilinear from an 800x1600 fp32 heightfield, 10 levels x 20 columns of 8 m tiles), actor/critic "
                 "512-256-128 ELU, 5 epochs x 4 minibatches of 24576, Algorithm 1 + Adam; seeded physics stand-in")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--fp32-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the grouped-learner and 16384-robot lines")
    ap.add_argument("--sweep", action="store_true", help="HBM size sweep of the env-step and GAE kernels (one JSON line per size)")
    ap.add_argument("--robots-sweep", action="store_true",
                    help="throughput against the number of parallel robots at three batch sizes (one JSON line per point)")
    ap.add_argument("--tiles-out", default=None, help="write the full autotune report (every trial) to this JSON file")
    ap.add_argument("--profile-run", type=int, default=0, metavar="K",
                    help="for profiler captures: build the BF16 learner (tile shapes from --tiles), run K iterations "
                         "without the graph and without timing, exit")
    ap.add_argument("--tiles", default=None,
                    help="apply the GEMM tile shapes of a saved autotune report instead of autotuning (for profiler runs, "
                         "where serialised launches would distort the autotuner's timings)")
    return ap.parse_args()


def dist_info():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


def reduce_max_time(total_ms, device="cpu"):
    """Max over ranks of the timed region (replicas finish when the slowest does)."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(total_ms)
    t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, num_envs, num_steps, steps, total_ms):
    """env-steps/s of all replicas together: every rank processed num_envs x num_steps x steps."""
    return world * num_envs * num_steps * steps / (total_ms / 1000.0)


def read_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    except Exception:
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0}, "fallback"


# dram__bytes_read.sum + dram__bytes_write.sum summed over the GEMM launches of one iteration of
# the rough-terrain workload (ncu, one pass per launch), with the SHA-1 of the GEMM source (the
# kernel file followed by its device-primitive header) it was captured on: the figure is reported
# only while that source is unchanged (null otherwise, until captured again).
GEMM_DRAM = {"gemm_tc_sha1": "06a3d82111684bc5e050a9fa7d4affebbdb94143", "bytes_per_iteration": 7983.27e6 + 298.74e6}
GEMM_SOURCES = ("gemm_tc.cu", "tc_prims.cuh")


def gemm_traffic():
    import hashlib
    h = hashlib.sha1()
    for name in GEMM_SOURCES:
        with open(os.path.join(ROOT, "paper_2109_11978_b300", "csrc", name), "rb") as f:
            h.update(f.read())
    sha = h.hexdigest()
    ok = GEMM_DRAM["gemm_tc_sha1"] == sha and GEMM_DRAM["bytes_per_iteration"] is not None
    return (GEMM_DRAM["bytes_per_iteration"] if ok else None), sha


def gemm_flops_per_iteration(w, O):
    """Algorithmic FLOPs of the MLP GEMM launches of one iteration (logical, unpadded sizes)."""
    N, T, E, MB = w["num_envs"], w["num_steps"], w["epochs"], w["minibatches"]
    Mb = N * T // MB
    dims = [O] + list(w["hidden"])
    layers = list(zip(dims[:-1], dims[1:]))
    fwd_row = sum(2 * i * o for i, o in layers)                 # one net, one row, hidden layers
    dx_row = sum(2 * i * o for i, o in layers[1:])
    rollout = T * N * 2 * fwd_row + N * fwd_row                   # act (actor + critic) + last value
    update = E * MB * Mb * 2 * (fwd_row + dx_row + fwd_row)      # forward, input grads, weight grads
    return rollout + update


def gemm_bytes_per_iteration(w, O, splits):
    """Algorithmic HBM bytes of the MLP GEMM launches of one iteration: every operand read once and
    every result written once per launch (bf16 activations, gradients and weights, fp32 split-K
    partials of the weight gradients, `splits` per hidden layer), nothing kept between launches.
    The layer-0 input is the padded observation row (both networks read the same rows)."""
    N, T, E, MB = w["num_envs"], w["num_steps"], w["epochs"], w["minibatches"]
    Mb = N * T // MB
    Op = (O + 63) // 64 * 64
    dims = [Op] + list(w["hidden"])
    layers = list(zip(dims[:-1], dims[1:]))

    def fwd(rows, nets):
        b = 0
        for l, (i, o) in enumerate(layers):
            a_in = rows * i * 2 * (1 if l == 0 else nets)
            b += a_in + nets * (o * i * 2 + rows * o * 2)
        return b

    dx = sum(2 * (Mb * o * 2 + o * i * 2 + Mb * i * 2 + Mb * i * 2) for (i, o) in layers[1:])
    dw = 0
    for l, (i, o) in enumerate(layers):
        x_in = Mb * i * 2 * (1 if l == 0 else 2)
        dw += 2 * Mb * o * 2 + x_in + 2 * splits[l] * o * i * 4
    rollout = T * fwd(N, 2) + fwd(N, 1)
    update = E * MB * (fwd(Mb, 2) + dx + dw)
    return rollout + update


class ClockSampler:
    """nvidia-smi SM clock / throttle-reason samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        out_dir = os.environ.get("BENCH_OUT_DIR") or __import__("tempfile").gettempdir()
        self.path = os.path.join(out_dir, f"bench_clocks_gpu{gpu_index}.csv")

    def start(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "25"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            return
        # nvidia-smi takes a moment to start: the timed region begins once its first sample is out,
        # so that the samples fall inside it (every 25 ms over a region of ~0.1 s)
        import time
        t0 = time.time()
        while time.time() - t0 < 5.0 and self.proc.poll() is None:
            if os.path.getsize(self.path) > 0:
                break
            time.sleep(0.005)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(power) if power else None}


def make_learner(api, synth, precision, seed, w=WORKLOAD):
    O = 48 + w["grid"][0] * w["grid"][1]
    cfg = api.default_config(num_envs=w["num_envs"], num_steps=w["num_steps"], grid_x=w["grid"][0],
                             grid_y=w["grid"][1], obs_dim=O, obs_pad=(O + 63) // 64 * 64, hidden=list(w["hidden"]),
                             epochs=w["epochs"], minibatches=w["minibatches"], precision=precision, seed=seed)
    params = synth.xavier_params(seed + 1, O, w["hidden"], 12)
    hf = synth.heightfield(seed + 2)
    return api.Learner(cfg, hf, params), O


def time_iterations(torch, L, steps, warmup, flush):
    """Per-iteration CUDA-event time (ms) of `steps` graph replays after `warmup`, with an L2
    flush (a 256 MB write) between iterations outside the timed events."""
    s = torch.cuda.current_stream()
    for _ in range(warmup):
        L.train_iteration(use_graph=True)
    torch.cuda.synchronize()
    e0 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    e1 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    for i in range(steps):
        flush.zero_()
        e0[i].record(s)
        L.train_iteration(use_graph=True)
        e1[i].record(s)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in zip(e0, e1)]


def profile_iterations(torch, api, L, steps, flush):
    """In-graph CUDA-event time per kernel class (ms per iteration, launches per iteration) over
    `steps` replays of the graph rebuilt with event nodes around every launch; a separate run from
    the timed one, since the events themselves cost time."""
    api.rl_profile_enable(L.ctx, api.RL_PROF_ALL, True)
    L.train_iteration(use_graph=True)          # capture the graph with the event nodes
    torch.cuda.synchronize()
    acc = {name: [0.0, 0] for name in api.RL_PROF_NAMES}
    for _ in range(steps):
        flush.zero_()
        L.train_iteration(use_graph=True)
        torch.cuda.synchronize()
        for cls, name in enumerate(api.RL_PROF_NAMES):
            ms, n = api.rl_profile_read_class(L.ctx, cls)
            acc[name][0] += ms
            acc[name][1] += n
    api.rl_profile_enable(L.ctx, api.RL_PROF_ALL, False)
    return {name: {"ms_per_iteration": v[0] / steps, "launches_per_iteration": v[1] / steps} for name, v in acc.items()}


GROUP_SIZES = (512, 1024, 1536, 2048, 3072, 4096, 6144, 8192)


def grouped_learners(torch, api, synth, steps=5, warmup=2):
    """8 independent BF16 learners of uneven robot counts in one grouped CUDA graph."""
    cfgs, hfs, params = [], [], []
    for i, n in enumerate(GROUP_SIZES):
        cfgs.append(api.default_config(num_envs=n, seed=30 + i, precision=api.RL_BF16))
        hfs.append(synth.heightfield(32 + i))
        params.append(synth.xavier_params(31 + i, 235, WORKLOAD["hidden"], 12))
    g = api.rl_group_create(cfgs, hfs, params)
    for i in range(len(GROUP_SIZES)):          # each learner's GEMM tile shapes for its own sizes
        api.rl_autotune(api.rl_group_learner(g, i))
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    for _ in range(warmup):
        api.rl_group_train_iteration(g, use_graph=True)
    torch.cuda.synchronize()
    s = torch.cuda.current_stream()
    times = []
    for _ in range(steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s)
        api.rl_group_train_iteration(g, use_graph=True)
        b.record(s)
        b.synchronize()
        times.append(a.elapsed_time(b))
    status = max(abs(api.rl_last_device_status(api.rl_group_learner(g, i))) for i in range(len(GROUP_SIZES)))
    api.rl_group_destroy(g)
    total = sum(GROUP_SIZES) * 24
    return {"learners": list(GROUP_SIZES), "env_steps_per_iteration": total, "ms_per_step": sum(times) / len(times),
            "env_steps_per_s": total * len(times) / (sum(times) / 1000.0), "device_status": -status,
            "what": "8 independent BF16 learners (own weights, Adam, alpha, curriculum), obs 235, 512-256-128, "
                    "24 steps, 5x4 update each, tile shapes autotuned per learner, replayed as one CUDA graph with "
                    "one branch per learner"}


def large_config(torch, api, synth, steps=3, warmup=2):
    """The full captured iteration at 16384 robots (B = 393216, minibatch 98304)."""
    w = dict(WORKLOAD)
    w["num_envs"] = 16384
    L, O = make_learner(api, synth, api.RL_BF16, seed=40, w=w)
    api.rl_autotune(L.ctx)                     # tile shapes for this learner's own sizes, as the main line
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    L.train_iteration(use_graph=True)
    times = time_iterations(torch, L, steps, warmup, flush)
    status = api.rl_last_device_status(L.ctx)
    L.close()
    return {"num_envs": 16384, "ms_per_step": sum(times) / len(times),
            "env_steps_per_s": 16384 * 24 * len(times) / (sum(times) / 1000.0), "device_status": status,
            "tiles": "autotuned"}


def actuator_lstm(torch, api, reps=5):
    """Throughput of the batched LSTM actuator cell (Sec. 3.3) at the workload's 4096 robots x 12
    joints: 96 chained substeps (24 policy steps x 4) per replay, random weights, CUDA events.
    Bytes per joint-substep: h and c read and written (4 x 128 B), inputs 8 B, torque 4 B."""
    n = WORKLOAD["num_envs"] * 12
    g = torch.Generator(device="cuda").manual_seed(3)
    w = (torch.rand(api.N.RL_ACT_WEIGHTS, device="cuda", generator=g) - 0.5) * 0.6
    x = torch.randn((n, 2), device="cuda", generator=g)
    h = torch.zeros((n, 32), device="cuda")
    c = torch.zeros((n, 32), device="cuda")
    tau = torch.empty(n, device="cuda")
    steps = WORKLOAD["num_steps"] * 4
    for _ in range(steps):
        api.rl_actuator_lstm_step(w, x, h, c, tau)
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(reps * steps):
        api.rl_actuator_lstm_step(w, x, h, c, tau)
    e1.record(s)
    torch.cuda.synchronize()
    us = e0.elapsed_time(e1) * 1000.0 / (reps * steps)
    return {"joints": n, "us_per_substep": round(us, 3), "ms_per_iteration_96_substeps": round(us * steps / 1000.0, 4),
            "joint_substeps_per_s": n / (us * 1e-6), "hbm_gbs": n * 524 / (us * 1e-6) / 1e9}


def robots_sweep(torch, api, synth, steps=3, warmup=2, quiet=False):
    """Throughput against the number of parallel robots (Sec. 4.1, Fig. 3): batch sizes B = 49152,
    98304 and 196608 samples per iteration with N = 128 ... 16384 robots (T = B / N steps), and the
    20000 robots x 50 steps = 1 M configuration; the full iteration (rollout, GAE, 5 x 4 PPO update
    with minibatch B / 4; 5 minibatches of 200000 for the 1 M point, whose quarter is not a whole
    number of 64-row blocks) on the rough-terrain network, BF16, default tile shapes, one CUDA
    graph per configuration."""
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    points = [(n, b // n, 4) for b in (49152, 98304, 196608) for n in (128, 256, 512, 1024, 2048, 4096, 8192, 16384)]
    points.append((20000, 50, 5))
    rows = []
    for n, t, mbs in points:
        w = dict(WORKLOAD)
        w["num_envs"], w["num_steps"], w["minibatches"] = n, t, mbs
        L, _ = make_learner(api, synth, api.RL_BF16, seed=50, w=w)
        L.train_iteration(use_graph=True)
        times = time_iterations(torch, L, steps, warmup, flush)
        status = api.rl_last_device_status(L.ctx)
        L.close()
        ms = sum(times) / len(times)
        row = {"num_envs": n, "num_steps": t, "batch": n * t, "minibatch": n * t // mbs, "ms_per_iteration": round(ms, 4),
               "env_steps_per_s": n * t / (ms / 1000.0), "device_status": status}
        if not quiet:
            print(json.dumps({"robots_sweep": row}), flush=True)
        rows.append(row)
    return rows


# Algorithmic bytes per robot-step of rl_env_step: fp32 state 57 x 4 + int state 3 x 4 read and
# written, actions 48 + value 4 read, observation row (256 x 2 bf16 or x 4 fp32), reward 4,
# done 1, time-out 1, level 4 written.
ENV_BYTES = {"bf16": 2 * 240 + 52 + 256 * 2 + 10, "fp32": 2 * 240 + 52 + 256 * 4 + 10}
GAE_BYTES_PER_SAMPLE = 17 + 8        # r, V, d read, A, R written + normalisation pass (read + write A)


ADAM_BYTES_PER_PARAM = 30     # p, m, v read + written (24), gradient read (4), bf16 copy written (2)


def sweep(torch, api, synth, reps=10):
    """Achieved HBM bandwidth of the memory-bound kernels at sizes past the L2 (126 MB)."""
    peaks, src = read_peaks()
    hbm = peaks.get("hbm_gbs", 6400.0)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    s = torch.cuda.current_stream()

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        tot = 0.0
        for _ in range(reps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(s)
            fn()
            b.record(s)
            b.synchronize()
            tot += a.elapsed_time(b)
        return tot / reps

    lines = []
    for n in (4096, 65536, 262144, 1048576):
        for form in ("bf16", "fp32"):
            cfg = api.default_config(num_envs=n, num_steps=1, minibatches=1, hidden=[64, 64],
                                     precision=api.RL_BF16 if form == "bf16" else api.RL_FP32)
            L = api.Learner(cfg, synth.heightfield(2), synth.xavier_params(1, 235, (64, 64), 12))
            sf, si = synth.random_env_state(3, n)
            L.set_state(torch.from_numpy(sf).cuda(), torch.from_numpy(si).cuda())
            act = torch.randn(n, 12, device="cuda")
            val = torch.randn(n, device="cuda")
            obs = torch.empty((n, 256), dtype=torch.bfloat16 if form == "bf16" else torch.float32, device="cuda")
            rew = torch.empty(n, device="cuda")
            dn = torch.empty(n, dtype=torch.uint8, device="cuda")
            to = torch.empty(n, dtype=torch.uint8, device="cuda")
            lv = torch.empty(n, dtype=torch.int32, device="cuda")
            ms = timed(lambda: api.rl_env_step(L.ctx, 0, act, val, obs, rew, dn, to, lv))
            gbs = ENV_BYTES[form] * n / (ms / 1000.0) / 1e9
            lines.append({"kernel": "env_step_kernel", "obs": form, "robots": n, "ms": ms, "bytes_per_robot": ENV_BYTES[form],
                          "achieved_gbs": gbs, "peak_gbs": hbm, "frac": gbs / hbm, "peak_source": src})
            L.close()
    for n in (4096, 65536, 262144, 1048576):
        T = 24
        r, v = torch.randn(T, n, device="cuda"), torch.randn(T, n, device="cuda")
        lv, d = torch.randn(n, device="cuda"), (torch.rand(T, n, device="cuda") < 0.05).to(torch.uint8)
        adv, ret = torch.empty(T, n, device="cuda"), torch.empty(T, n, device="cuda")
        ws = torch.empty(api.rl_gae_workspace_bytes(T, n) // 4 + 4, device="cuda")
        ms = timed(lambda: api.rl_gae(0.99, 0.95, r, v, lv, d, adv, ret, normalize=True, workspace=ws))
        byt = GAE_BYTES_PER_SAMPLE * T * n + 4 * n
        gbs = byt / (ms / 1000.0) / 1e9
        lines.append({"kernel": "gae_scan_kernel+gae_normalize_kernel", "T": T, "robots": n, "ms": ms,
                      "bytes_per_sample": GAE_BYTES_PER_SAMPLE, "achieved_gbs": gbs, "peak_gbs": hbm, "frac": gbs / hbm,
                      "peak_source": src})
        del r, v, lv, d, adv, ret, ws
    # Adam (rl_adam_step: the update's Adam kernel on one gradient): p, m, v read and written, g read,
    # the bf16 copy written = 30 B per parameter; the learner's 571,801 parameters, then past the L2
    for n in (571801, 4 * 2 ** 20, 16 * 2 ** 20, 64 * 2 ** 20):
        p_ = torch.randn(n, device="cuda") * 1e-3
        g_ = torch.randn(n, device="cuda") * 1e-2
        m_, v_ = torch.zeros(n, device="cuda"), torch.zeros(n, device="cuda")
        wb_ = torch.empty(n, dtype=torch.bfloat16, device="cuda")
        ms = timed(lambda: api.rl_adam_step(p_, g_, m_, v_, 1e-3, 1, 1, wb_))
        gbs = ADAM_BYTES_PER_PARAM * n / (ms / 1000.0) / 1e9
        lines.append({"kernel": "adam_kernel", "params": n, "ms": ms, "bytes_per_param": ADAM_BYTES_PER_PARAM,
                      "achieved_gbs": gbs, "peak_gbs": hbm, "frac": gbs / hbm, "peak_source": src})
        del p_, g_, m_, v_, wb_
    return lines


def cpu_baseline(seconds_budget=20.0, n_envs=256):
    """The FP64 oracle, as it stands, on a bounded sample of the same workload."""
    from oracle import config as OC
    from oracle.train import Learner
    from paper_2109_11978_b300 import synth
    w = dict(WORKLOAD)
    w["num_envs"] = n_envs
    O = 48 + 17 * 11
    ecfg = OC.EnvConfig(num_envs=n_envs)
    pcfg = OC.PPOConfig(epochs=w["epochs"], minibatches=w["minibatches"])
    L = Learner(ecfg, pcfg, w["hidden"], synth.heightfield(2), synth.xavier_params(1, O, w["hidden"], 12))
    t0 = time.perf_counter()
    iters = 0
    while True:
        L.iterate(w["num_steps"])
        iters += 1
        if time.perf_counter() - t0 > seconds_budget * 0.5 or iters >= 4:
            break
    dt = time.perf_counter() - t0
    cores = len(os.sched_getaffinity(0))
    try:
        from threadpoolctl import threadpool_info
        threads = max([d.get("num_threads", 1) for d in threadpool_info()] or [1])
    except ImportError:          # numpy's BLAS defaults to one thread per available core
        threads = int(os.environ.get("OMP_NUM_THREADS", cores))
    return {"value": n_envs * w["num_steps"] * iters / dt, "unit": "env-steps/s", "cores": min(cores, threads),
            "host_cores": cores, "blas_threads": threads, "kind": "oracle",
            "sample": f"{iters} full iteration(s) of the same workload at {n_envs} robots x 24 steps "
                      f"(1/{4096 // n_envs} of the robots; same obs, MLP sizes, 5x4 update at minibatch "
                      f"{n_envs * 24 // 4}), FP64 numpy, {dt:.1f} s"}


# The two small configurations beside the headline: C1 tiny (64 robots x 24 steps, obs 48, actor /
# critic 48-64-64, 1 epoch x 2 minibatches) and C2 flat terrain (4096 x 24, obs 48, 512-256-128,
# 5 x 4), both in the plain FP32 form, with no height samples.
SMALL_CONFIGS = {
    "C1 tiny": dict(num_envs=64, num_steps=24, grid=(0, 0), hidden=(64, 64), epochs=1, minibatches=2),
    "C2 flat": dict(num_envs=4096, num_steps=24, grid=(0, 0), hidden=(512, 256, 128), epochs=5, minibatches=4),
}


def small_configs(torch, api, synth, steps=10, warmup=3, oracle_budget=6.0):
    """GPU env-steps/s of C1 and C2 (plain FP32 GPU form, graph replay, median) next to the FP64
    oracle on the host cores (C1 whole iterations, C2 a bounded sample at 256 robots)."""
    from oracle import config as OC
    from oracle.train import Learner as OLearner
    out = {}
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    for name, w in SMALL_CONFIGS.items():
        O = 48
        cfg = api.default_config(num_envs=w["num_envs"], num_steps=w["num_steps"], grid_x=0, grid_y=0, obs_dim=O,
                                 obs_pad=64, hidden=list(w["hidden"]), epochs=w["epochs"], minibatches=w["minibatches"],
                                 precision=api.RL_FP32, seed=10)
        L = api.Learner(cfg, None, synth.xavier_params(11, O, w["hidden"], 12))
        times = time_iterations(torch, L, steps, warmup, flush)
        status = api.rl_last_device_status(L.ctx)
        L.close()
        ms = statistics.median(times)
        gpu = w["num_envs"] * w["num_steps"] / (ms / 1000.0)
        n_or = min(w["num_envs"], 256)
        ol = OLearner(OC.EnvConfig(num_envs=n_or, grid_x=0, grid_y=0, seed=10),
                      OC.PPOConfig(epochs=w["epochs"], minibatches=w["minibatches"], seed=10), list(w["hidden"]), None,
                      synth.xavier_params(11, O, w["hidden"], 12))
        t0 = time.perf_counter()
        iters = 0
        while iters < 1 or (time.perf_counter() - t0 < oracle_budget and iters < 4):
            ol.iterate(w["num_steps"])
            iters += 1
        dt = time.perf_counter() - t0
        out[name] = {"gpu_fp32_env_steps_per_s": gpu, "gpu_ms_per_iteration": ms, "device_status": status,
                     "oracle_env_steps_per_s": n_or * w["num_steps"] * iters / dt, "oracle_cores": len(os.sched_getaffinity(0)),
                     "oracle_sample": f"{iters} iteration(s) at {n_or} robots x {w['num_steps']} steps, {dt:.1f} s",
                     "config": {k: (list(v) if isinstance(v, tuple) else v) for k, v in w.items()}}
    return out


def run_reference(args):
    rank, world, _ = dist_info()
    if rank != 0:
        return 0
    n_envs = 128
    from oracle import config as OC
    from oracle.train import Learner
    from paper_2109_11978_b300 import synth
    O = 48 + 17 * 11
    ecfg = OC.EnvConfig(num_envs=n_envs)
    pcfg = OC.PPOConfig(epochs=5, minibatches=4)
    L = Learner(ecfg, pcfg, WORKLOAD["hidden"], synth.heightfield(2), synth.xavier_params(1, O, WORKLOAD["hidden"], 12))
    for _ in range(args.warmup):
        L.iterate(24)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        L.iterate(24)
    dt = time.perf_counter() - t0
    v = n_envs * 24 * args.steps / dt
    cores = len(os.sched_getaffinity(0))
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "env-steps/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1000 / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded physics stand-in)",
           "config": {"workload": WORKLOAD_NAME, "sample": f"{n_envs} robots x 24 steps per step"},
           "cpu_baseline": {"value": v, "unit": "env-steps/s", "cores": cores, "kind": "oracle",
                            "sample": f"each step: one full iteration at {n_envs} robots x 24 steps (FP64 oracle)"},
           "e2e": {"value": v, "unit": "env-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


def select_tiles(api, L, args):
    """Autotune the update's GEMM sites (default) or apply the shapes of a saved report."""
    site_id = {"forward": 0, "input_grad": 1, "weight_grad": 2, "act_forward": 3}
    if args.tiles:
        with open(args.tiles) as f:
            rep = json.load(f)
        rep = rep.get("autotune", rep)
        fused_id = {"forward_fused": 0, "act_forward_fused": 3}     # cluster: 1 when the fused form was kept
        for s in rep["sites"]:
            if s["site"] in fused_id:
                api.rl_set_forward_fused(L.ctx, fused_id[s["site"]], s.get("cluster", 0))
            else:
                api.rl_set_gemm_tiles(L.ctx, site_id[s["site"]], s["layer"], s["bn"], s.get("cluster", 1), s["splits"])
        return {"sites": rep["sites"], "source": f"applied from {os.path.basename(args.tiles)}"}
    rep = api.rl_autotune(L.ctx)
    rep["source"] = "autotuned in this run"
    if args.tiles_out:
        with open(args.tiles_out, "w") as f:
            json.dump(rep, f, indent=1)
    return rep


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.sweep:
        import torch
        from paper_2109_11978_b300 import api, synth
        for line in sweep(torch, api, synth):
            print(json.dumps(line), flush=True)
        return 0
    if args.robots_sweep:
        import torch
        from paper_2109_11978_b300 import api, synth
        robots_sweep(torch, api, synth)
        return 0
    if args.profile_run:
        import torch
        from paper_2109_11978_b300 import api, synth
        L, _ = make_learner(api, synth, api.RL_BF16, seed=0)
        if args.tiles:
            select_tiles(api, L, args)
        for _ in range(args.profile_run):
            L.train_iteration(use_graph=False)
        torch.cuda.synchronize()
        status = api.rl_last_device_status(L.ctx)
        L.close()
        print(json.dumps({"profile_run": args.profile_run, "device_status": status}))
        return 0 if status == 0 else 1
    rank, world, local = dist_info()
    import torch
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2109_11978_b300 import api, synth
    w = WORKLOAD
    N, T = w["num_envs"], w["num_steps"]
    peaks, peak_src = read_peaks()

    # --- BF16 form: the headline --------------------------------------------------------
    L, O = make_learner(api, synth, api.RL_BF16, seed=1000 * rank)
    tuned = select_tiles(api, L, args)      # tile widths / clusters / split counts of every update GEMM site
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    # untimed: build the graph once and count the launches of one iteration
    L.train_iteration(use_graph=True)
    torch.cuda.synchronize()
    launches = api.rl_launches_per_iteration(L.ctx)
    clocks = ClockSampler(local)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    times = time_iterations(torch, L, args.steps, args.warmup, flush)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    # the median iteration (every rank's times are per-iteration CUDA-event times); the max over
    # ranks of the median, times the step count, is the job's timed region
    med_ms = reduce_max_time(statistics.median(times), device="cuda")
    total_ms = med_ms * args.steps
    mean_ms = reduce_max_time(sum(times) / len(times), device="cuda")
    status = api.rl_last_device_status(L.ctx)
    value = whole_job_rate(world, N, T, args.steps, total_ms)

    # per-class in-graph kernel times (separate, profiled run); dominant kernel: the tcgen05 GEMMs
    breakdown = profile_iterations(torch, api, L, min(args.steps, 5), flush)
    gemm_ms = breakdown["gemm"]["ms_per_iteration"]
    gemm_n = breakdown["gemm"]["launches_per_iteration"]
    flops_iter = gemm_flops_per_iteration(w, O)
    splits = {s_["layer"]: s_["splits"] for s_ in tuned["sites"] if s_["site"] == "weight_grad"}
    bytes_iter = gemm_bytes_per_iteration(w, O, [splits.get(l, 1) for l in range(len(w["hidden"]))])
    gemm_s = gemm_ms / 1000.0 if gemm_ms > 0 else None
    # the GEMM launches last 5-30 us each: the burst peaks are the fair denominators (the sustained
    # BF16 figure, for seconds-long loops under the power cap, is reported beside it)
    peak = peaks.get("bf16_tflops", 1800.0)
    peak_sus = peaks.get("bf16_tflops_sustained", 1400.0)
    hbm = peaks.get("hbm_gbs", 6400.0)
    t_flop = flops_iter / (peak * 1e12)          # s per iteration at the tensor peak
    t_byte = bytes_iter / (hbm * 1e9)            # s per iteration at the HBM peak
    tflops = flops_iter / gemm_s / 1e12 if gemm_s else None
    gbs = bytes_iter / gemm_s / 1e9 if gemm_s else None
    traffic, gemm_sha = gemm_traffic()
    # the roofline binds at the lower ceiling: with the iteration's arithmetic intensity below the
    # ridge point (every MLP GEMM here: K <= 512, outputs as wide as their inputs) that is HBM
    hbm_bound = t_byte >= t_flop
    roof = {"bound": "hbm" if hbm_bound else "tensor",
            "kernel": "tc_gemm_kernel (all MLP GEMM launches of the iteration)",
            "achieved": gbs if hbm_bound else tflops, "peak": hbm if hbm_bound else peak,
            "unit": "GB/s" if hbm_bound else "TFLOP/s",
            "frac": ((gbs / hbm) if hbm_bound else (tflops / peak)) if gemm_s else None,
            "traffic": traffic,
            "traffic_note": "DRAM bytes (read + write) of the iteration's GEMM launches from one ncu capture on this "
                            "GEMM source (sha1 " + gemm_sha[:12] + "), per iteration like achieved; null when the "
                            "source has changed since the capture",
            "peak_source": f"hbm_gbs copy bandwidth / bf16_tflops burst ({peak_src})",
            "algorithmic_bytes_per_iteration": bytes_iter, "algorithmic_flops_per_iteration": flops_iter,
            "arithmetic_intensity_flop_per_byte": flops_iter / bytes_iter,
            "ridge_flop_per_byte": peak * 1e12 / (hbm * 1e9),
            "roofline_time_ms": max(t_flop, t_byte) * 1e3,
            "tensor": {"achieved": tflops, "peak": peak, "unit": "TFLOP/s", "frac": (tflops / peak) if tflops else None,
                       "frac_of_sustained": (tflops / peak_sus) if tflops else None},
            "gemm_ms_per_iteration": gemm_ms, "gemm_launches_per_iteration": gemm_n,
            "gemm_share_of_step": gemm_ms / (total_ms / args.steps) if total_ms else None,
            "achieved_note": "algorithmic bytes (every operand read once, every result written once per launch) and "
                             "FLOPs of the iteration's GEMM launches / their summed in-graph CUDA-event time "
                             "(profiled run)"}

    # --- end to end through the public API with host buffers: the caller keeps the simulator state
    # in pinned host memory between iterations; each step passes it in (rl_env_set_state), trains
    # one iteration (rl_train_iteration, statistics to pinned host memory) and takes the state back
    # (rl_env_get_state), host-timed with the stream synchronised every step
    sf_h = torch.empty((api.RL_NF, N), dtype=torch.float32).pin_memory()
    si_h = torch.empty((api.RL_NI, N), dtype=torch.int32).pin_memory()
    stats_host = torch.empty(api.RL_NSTATS, dtype=torch.float32).pin_memory()
    api.rl_env_get_state(L.ctx, sf_h, si_h)
    torch.cuda.synchronize()

    def e2e_step():
        api.rl_env_set_state(L.ctx, sf_h, si_h)
        L.train_iteration(use_graph=True, stats_host=stats_host)
        api.rl_env_get_state(L.ctx, sf_h, si_h)
        torch.cuda.synchronize()

    # untimed warm-up: the profiled run above left a graph with event nodes, re-captured here
    for _ in range(args.warmup):
        e2e_step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_step()
    e2e_s = time.perf_counter() - t0
    state_bytes = sf_h.numel() * sf_h.element_size() + si_h.numel() * si_h.element_size()
    e2e = {"value": world * N * T * args.steps / e2e_s, "unit": "env-steps/s", "h2d_bytes_per_step": state_bytes,
           "d2h_bytes_per_step": state_bytes + stats_host.numel() * stats_host.element_size(),
           "note": "host-timed through the C ABI with pinned host buffers: per iteration the env state in "
                   "(rl_env_set_state), rl_train_iteration with its statistics copied out, the env state out "
                   "(rl_env_get_state), stream synchronised; after the same warm-up iterations as the device-timed "
                   "run"}
    L.close()
    del flush

    # --- FP32 form on the same workload (comparison) --------------------------------------
    compare = None
    if args.fp32_steps > 0:
        Lf, _ = make_learner(api, synth, api.RL_FP32, seed=1000 * rank)
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
        Lf.train_iteration(use_graph=True)
        ft = time_iterations(torch, Lf, args.fp32_steps, 1, flush)
        fv = N * T * len(ft) / (sum(ft) / 1000.0)
        compare = {"fp32_env_steps_per_s": fv, "fp32_ms_per_step": sum(ft) / len(ft), "bf16_over_fp32": value / world / fv,
                   "note": "same workload, FP32 CUDA-core GEMMs; both forms pass their oracle tolerances "
                           "(1e-5 FP32, 2e-2 BF16 gradients) in tests/"}
        Lf.close()
        del flush

    extra = {}
    if not args.no_extra:
        extra["grouped_learners"] = grouped_learners(torch, api, synth)
        extra["robots_16384"] = large_config(torch, api, synth)
        extra["actuator_lstm"] = actuator_lstm(torch, api)
        extra["hbm_sweep"] = sweep(torch, api, synth, reps=5)
        extra["small_configs"] = small_configs(torch, api, synth)
        extra["robots_sweep"] = robots_sweep(torch, api, synth, quiet=True)
    if rank != 0:
        return 0
    out = {"metric": METRIC, "value": value, "unit": "env-steps/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "ms_per_step_mean": mean_ms,
           "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "bf16", "data": "synthetic (seeded physics stand-in replaces PhysX)",
           "config": {"workload": WORKLOAD_NAME, "num_envs": N, "num_steps": T, "batch": N * T,
                      "minibatch": N * T // w["minibatches"], "parallelism": f"replicas x{world}",
                      "l2": "flushed (256 MB write) between timed iterations", "graph": "one CUDA graph per iteration",
                      "statistic": "median of the timed iterations (value and ms_per_step)",
                      "per_step_ms": [round(t, 4) for t in times]},
           "roofline": roof, "kernel_breakdown_in_graph": breakdown,
           "gpu_launches": launches * args.steps, "launches_per_step": launches,
           "autotune": {k: tuned[k] for k in ("sites", "pairs_resident", "source") if k in tuned},
           "e2e": e2e, "clocks": clk, "device_status": status}
    if compare:
        out["compare"] = compare
    out.update(extra)
    if not args.no_cpu_baseline and world == 1:
        out["cpu_baseline"] = cpu_baseline()
    elif not args.no_cpu_baseline:
        out["cpu_baseline"] = None
    print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
