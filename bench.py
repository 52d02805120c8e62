#!/usr/bin/env python
"""Planning-step benchmark of the VOiLA hot path on B300.

One step = one SIR belief update (N particles: propose with g_T, weight with
the likelihood MLP, normalise, resample) followed by the Monte-Carlo rollout
of the updated belief over K action sequences x H steps with the generator
and reward MLPs, the per-sequence return reduction and the argmax, and the
PORPP log-sum-exp backup of the returns (value and policy).

Default workload ("mid_bf16"): state 8, action 2, observation 6, latent 8;
3x256 SiLU MLPs with BF16 weights; N=4096, K=1024, H=20, gamma=0.98; all
inputs seeded and synthetic (random-init weights shaped like the paper's
models). Metric: rollout transition-steps/s = N*K*H per step.

Prints one JSON line. Under torchrun each rank runs an independent replica
on its own GPU (weak scaling, no data-path collective).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "rollout transition-steps/s"
UNIT = "transition-steps/s"


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["mid_bf16", "mid_fp32", "small_fp32", "batched", "sweep", "distill", "infonce", "pw"], default="mid_bf16")
    ap.add_argument("--cpu-seqs", type=int, default=8, help="action sequences in the oracle CPU sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fp32-seqs", type=int, default=16, help="sequences for the FP32-form comparison (0: skip)")
    ap.add_argument("--no-forms", action="store_true", help="skip the FP32/FP8 form comparison")
    ap.add_argument("--prec", choices=["bf16", "fp8"], default="bf16",
                    help="mid_bf16 workload: the precision form of the timed step's MLPs (fp8: E4M3 hidden "
                         "layers with per-channel scales)")
    ap.add_argument("--batched-schedules", action="store_true",
                    help="batched workload: also time every candidate schedule of the autotuner")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the compact records of the other configurations in the default run")
    ap.add_argument("--sweep-err-seqs", type=int, default=64, help="sequences of the sweep's FP64 error subset")
    ap.add_argument("--sweep-err-N", type=int, default=256, help="particles of the sweep's FP64 error subset")
    ap.add_argument("--distill-cpu-rows", type=int, default=12288, help="rows of the distillation oracle sample")
    ap.add_argument("--B", type=int, default=None, help="override the distillation batch (profiling runs)")
    ap.add_argument("--N", type=int, default=None, help="override particles (profiling runs)")
    ap.add_argument("--K", type=int, default=None, help="override action sequences (profiling runs)")
    ap.add_argument("--H", type=int, default=None, help="override horizon (profiling runs)")
    return ap.parse_args()


def warm_until(fn, seconds: float) -> None:
    """Repeats fn (at least once) until `seconds` of wall time have passed, so a
    short timed region starts with the GPU at its working clock (a sub-ms call
    timed right after an idle GPU otherwise reads up to 2x slow)."""
    import torch
    t0 = time.perf_counter()
    while True:
        fn()
        torch.cuda.synchronize()
        if time.perf_counter() - t0 >= seconds:
            return


def max_over_ranks(value: float, world: int, device) -> float:
    """The slowest rank's time (the whole-job clock) across `world` replicas."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(units_per_rank: int, world: int, slowest_s: float) -> float:
    """Whole-job throughput of `world` independent replicas (weak scaling)."""
    return units_per_rank * world / slowest_s


def make_workload(name, args=None):
    from paper_2606_19729_b300 import workloads as WL
    kw = {}
    for key in ("N", "K", "H"):
        v = getattr(args, key, None) if args is not None else None
        if v is not None:
            kw[key] = v
    if name == "mid_bf16":
        prec = {"bf16": WL.PREC_BF16, "fp8": WL.PREC_FP8}[getattr(args, "prec", None) or "bf16"]
        return WL.mid_bf16(prec=prec, **kw)
    if name == "mid_fp32":
        return WL.mid_bf16(prec=WL.PREC_FP32, **kw)
    return WL.small_fp32(**kw)


def flops_per_transition(wl) -> int:
    """Algorithmic FLOPs of one transition: 2 * sum(in * out) over the generator
    and (if it is an MLP) the reward head."""
    f = sum(2 * w.shape[0] * w.shape[1] for w in wl.g_T.W)
    if wl.reward_mlp is not None and wl.goal is None:
        f += sum(2 * w.shape[0] * w.shape[1] for w in wl.reward_mlp.W)
    return f


def workload_config(wl, args):
    return {
        "workload": f"{wl.name}: N={wl.N} particles x K={wl.K} sequences x H={wl.H}, "
                    f"d_s={wl.d_s} d_a={wl.d_a} d_o={wl.d_o} d_omega={wl.d_omega}, "
                    f"MLPs {'x'.join(str(d) for d in wl.g_T.dims)} "
                    f"{ {0: 'FP32', 1: 'BF16', 2: 'FP8 e4m3 (hidden layers, per-channel scales)'}[wl.prec] }; "
                    "belief update + rollout per step",
        "N": wl.N, "K": wl.K, "H": wl.H,
        "l2": "flushed (256 MB write) before every timed step",
        "inputs": "synthetic, seeded; random-init weights",
    }


class Clocks:
    """Samples nvidia-smi clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu_index = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.gpu_index)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        if not getattr(self, "out", ""):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def blas_threads() -> int:
    """Threads numpy's BLAS runs with (the oracle's parallelism), else the host's cores."""
    try:
        import threadpoolctl
        info = threadpoolctl.threadpool_info()
        n = max([i.get("num_threads", 1) for i in info if i.get("user_api") == "blas"] + [0])
        if n:
            return n
    except ImportError:
        pass
    for var in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        if os.environ.get(var, "").isdigit():
            return int(os.environ[var])
    return len(os.sched_getaffinity(0))


def cpu_baseline(wl, seqs, particles=None):
    """The FP64 oracle, as it stands, on a bounded sample: one belief update of all
    N particles plus the rollout of `seqs` sequences x all N particles x H.
    With `particles` (the device's resampled belief) the rollout starts from
    them, so its returns are the FP64 reference for the device's J[:seqs]."""
    from oracle import voila_oracle as O

    def om(spec):
        return O.MLP(spec.W, spec.b, spec.act)

    obs = np.zeros(wl.d_o)
    ks = list(range(seqs))
    t0 = time.perf_counter()
    res = O.belief_update(om(wl.g_T), O.Likelihood(O.LIK_MLP, mlp=om(wl.ell)), wl.particles, wl.actions[0, 0],
                          obs, wl.d_omega, wl.lam, wl.seed, 1)
    start = res.particles_out if particles is None else particles
    R = O.Reward(O.REWARD_MLP, mlp=om(wl.reward_mlp)) if wl.goal is None else O.Reward(O.REWARD_GOAL, wl.goal)
    J, _ = O.rollout(om(wl.g_T), R, start, wl.actions, wl.d_omega, wl.gamma, wl.seed, k_index=ks)
    dt = time.perf_counter() - t0
    cores = blas_threads()
    trans = seqs * wl.N * wl.H
    return {"value": trans / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"FP64 numpy oracle: 1 belief update of {wl.N} particles + rollout of {seqs} of {wl.K} "
                      f"sequences x {wl.N} particles x H={wl.H} ({trans} transitions) in {dt:.2f} s"}, J, res


_ONE_CORE_CHILD = """
import json, sys, time
import numpy as np
sys.path.insert(0, sys.argv[1])
from paper_2606_19729_b300 import workloads as WL
from oracle import voila_oracle as O
kind, prec, N, K, H, seqs = sys.argv[3], int(sys.argv[4]), *map(int, sys.argv[5:9])
wl = WL.mid_bf16(prec=prec, N=N, K=K, H=H) if kind == "mid" else WL.small_fp32(N=N, K=K, H=H)
om = lambda spec: O.MLP(spec.W, spec.b, spec.act)
R = O.Reward(O.REWARD_MLP, mlp=om(wl.reward_mlp)) if wl.goal is None else O.Reward(O.REWARD_GOAL, wl.goal)
p = np.load(sys.argv[2])
t0 = time.perf_counter()
O.rollout(om(wl.g_T), R, p, wl.actions, wl.d_omega, wl.gamma, wl.seed, k_index=list(range(seqs)))
print(json.dumps({"dt": time.perf_counter() - t0}))
"""


def one_core_oracle(wl, particles, seqs: int = 1):
    """The oracle's rollout of `seqs` sequences x all particles in a fresh
    interpreter whose BLAS runs one thread: the single-core figure beside the
    all-core one."""
    import tempfile
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    kind = "mid" if wl.name.startswith("mid") else "small"
    with tempfile.TemporaryDirectory() as tmp:
        path = os.path.join(tmp, "particles.npy")
        np.save(path, np.asarray(particles, dtype=np.float64))
        r = subprocess.run([sys.executable, "-c", _ONE_CORE_CHILD, os.path.dirname(os.path.abspath(__file__)), path,
                            kind, str(wl.prec), str(wl.N), str(wl.K), str(wl.H), str(seqs)],
                           env=env, capture_output=True, text=True, timeout=300)
    if r.returncode != 0:
        return {"value": None, "unit": UNIT, "cores": 1, "error": (r.stderr.strip().splitlines() or ["?"])[-1]}
    dt = json.loads(r.stdout.strip().splitlines()[-1])["dt"]
    trans = seqs * wl.N * wl.H
    return {"value": trans / dt, "unit": UNIT, "cores": 1,
            "sample": f"rollout of {seqs} of {wl.K} sequences x {wl.N} particles x H={wl.H} ({trans} transitions) "
                      f"in {dt:.2f} s, one BLAS thread (a fresh interpreter)"}


def oracle_belief(wl, lam):
    """The FP64 oracle's belief update on the error leg's inputs (prior particles,
    a = actions[0, 0], o = 0, step 1, planner 0) at temperature `lam`."""
    from oracle import voila_oracle as O
    om = lambda spec: O.MLP(spec.W, spec.b, spec.act)  # noqa: E731
    return O.belief_update(om(wl.g_T), O.Likelihood(O.LIK_MLP, mlp=om(wl.ell)), wl.particles, wl.actions[0, 0],
                           np.zeros(wl.d_o), wl.d_omega, lam, wl.seed, 1)


def device_belief_weights(V, g, ell_mlp, wl, lam=None):
    """The device belief update on the oracle leg's inputs (prior particles,
    a = actions[0, 0], o = 0, step 1, planner 0): its normalised weights and the
    median time of one call (ms)."""
    import torch
    lik = V.mlp_likelihood(ell_mlp)
    N = wl.N
    parts = torch.from_numpy(wl.particles).float().cuda()
    a0 = torch.from_numpy(np.ascontiguousarray(wl.actions[0, 0])).float().cuda()
    obs = torch.zeros(wl.d_o, dtype=torch.float32, device="cuda")
    out = torch.empty_like(parts)
    w = torch.empty(N, dtype=torch.float64, device="cuda")
    ws = V.alloc_workspace(V.voila_belief_update_workspace_size(g, lik, N))

    lam = wl.lam if lam is None else lam

    def call():
        V.voila_belief_update(g, lik, parts, None, a0, obs, wl.d_omega, lam, wl.seed, 1, 0, out, None, w, None,
                              None, ws)

    warm_until(call, 0.3)
    ts = []
    for _ in range(20):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        call()
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    assert V.workspace_status(ws) == V.OK
    return w.cpu().numpy(), statistics.median(ts)


def logw_err(w, w_ref):
    """max |log w - log w_ref| over the weights the reference gives more than 1e-9."""
    big = w_ref > 1e-9
    return float(np.max(np.abs(np.log(np.maximum(w[big], 1e-300)) - np.log(w_ref[big]))))


def load_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


# Fallback denominators (no MEASURED_PEAKS.json): one earlier B300 measurement.
FALLBACK_BF16_BURST, FALLBACK_BF16_SUSTAINED = 1800.0, 1400.0


def measure_fp8_peak(n: int = 8192, reps: int = 10):
    """Dense E4M3 GEMM rate of this GPU: torch._scaled_mm (cuBLASLt) on n^3,
    2 n^3 FLOP, best of `reps` by CUDA events. None if the call is unavailable."""
    import torch
    try:
        a = torch.randn(n, n, device="cuda").to(torch.float8_e4m3fn)
        b = torch.randn(n, n, device="cuda").to(torch.float8_e4m3fn)
        one = torch.ones((), device="cuda")
        f = lambda: torch._scaled_mm(a, b.t(), scale_a=one, scale_b=one, out_dtype=torch.bfloat16)  # noqa: E731
        for _ in range(3):
            f()
        torch.cuda.synchronize()
        best = float("inf")
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            f()
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1) / 1e3)
        del a, b
        return 2.0 * n ** 3 / best / 1e12
    except (RuntimeError, AttributeError, TypeError):
        return None


def fp32_roofline(achieved: float, peaks: dict, clocks, nsm: int) -> dict:
    """FP32 CUDA-core roofline: SMs x 128 FMA lanes x 2 FLOP x SM clock (the
    kernel's sampled median clock when known, else the maximum)."""
    mhz = (clocks or {}).get("sm_mhz") or peaks.get("sm_max_mhz", 2032.0)
    peak = nsm * 128 * 2 * mhz * 1e6 / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": None, "peak_source": f"FP32 FMA: {nsm} SMs x 128 lanes x 2 FLOP x {mhz:.0f} MHz (derived)"}


def tensor_roofline(achieved: float, peaks: dict, clocks: dict, kind: str = "bf16", fp8_peak=None) -> dict:
    """Roofline block of a tensor-core kernel. The denominator is the measured
    burst rate of the kernel's operand type (BF16: cuBLAS from MEASURED_PEAKS.json;
    FP8: the torch._scaled_mm probe of this run, else twice the BF16 burst, the
    nominal ratio), taken as it stands when the kernel's sampled median SM clock
    is within 5 % of the maximum and scaled to that median clock otherwise. The
    ratio to the power-capped sustained BF16 figure is kept as a side field."""
    burst = peaks.get("bf16_tflops", FALLBACK_BF16_BURST)
    sustained = peaks.get("bf16_tflops_sustained", FALLBACK_BF16_SUSTAINED)
    src = "measured (MEASURED_PEAKS.json)" if peaks else "fallback"
    if kind == "fp8":
        if fp8_peak:
            base, basis = fp8_peak, "measured e4m3 burst (torch._scaled_mm 8192^3, best of 10, this run)"
        else:
            base, basis = 2.0 * burst, f"bf16 burst x 2 (nominal e4m3/bf16 ratio), bf16 {src}"
    else:
        base, basis = burst, f"bf16 burst (cuBLAS 8192^3), {src}"
    smax = peaks.get("sm_max_mhz", 2032.0)
    med = (clocks or {}).get("sm_mhz")
    if med and med < 0.95 * smax:
        peak = base * med / smax
        basis += f", scaled to the kernel's median SM clock {med:.0f} of {smax:.0f} MHz"
    else:
        peak = base
        basis += " (the kernel ran within 5% of the maximum SM clock)" if med else " (clock unsampled)"
    out = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
           "peak_source": basis}
    if kind == "bf16":
        out["frac_vs_sustained_bf16"] = achieved / sustained
    return out


def profiled_traffic(form: str, wl):
    """(DRAM bytes per launch, ncu tensor-pipe %) of the mid-size rollout kernel in
    `form` ("bf16" or "fp8") from profiles/, or (None, None) when the capture was
    taken on another kernel source or the workload is not the full mid-size one."""
    try:
        import hashlib
        with open(os.path.join(ROOT, "profiles", f"rollout_tc_mid_{form}_traffic.json")) as f:
            prof = json.load(f)
        src = b"".join(open(os.path.join(ROOT, "paper_2606_19729_b300", "csrc", n), "rb").read()
                       for n in ("tc.cu", "tc_ptx.cuh"))
        if (hashlib.sha256(src).hexdigest()[:16] == prof["source_sha16"] and wl.name == "mid_bf16"
                and (wl.N, wl.K, wl.H) == (4096, 1024, 20)):
            return prof["dram_read_bytes"] + prof["dram_write_bytes"], prof.get("tensor_pipe_pct")
    except (OSError, KeyError, ValueError):
        pass
    return None, None


def fp32_form(V, wl, seqs, planner, particles, stream):
    """The plain FP32 CUDA-core form on the same workload, timed on a slice of
    `seqs` action sequences (throughput per transition does not depend on K)."""
    import torch
    from paper_2606_19729_b300 import workloads as WL
    g32 = V.DeviceMLP([torch.from_numpy(w) for w in wl.g_T.W], [torch.from_numpy(b) for b in wl.g_T.b],
                      wl.g_T.act, V.FP32)
    r32 = V.DeviceMLP([torch.from_numpy(w) for w in wl.reward_mlp.W], [torch.from_numpy(b) for b in wl.reward_mlp.b],
                      wl.reward_mlp.act, V.FP32)
    R32 = V.mlp_reward(r32)
    acts = torch.from_numpy(np.ascontiguousarray(wl.actions[:seqs])).float().cuda()
    J = torch.empty(seqs, dtype=torch.float64, device="cuda")
    ws = V.alloc_workspace(V.voila_rollout_workspace_size(g32, R32, wl.N, seqs, wl.H))
    V.voila_rollout(g32, R32, particles, None, acts, wl.d_omega, wl.gamma, wl.seed, planner, J, None, None, ws)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    reps = 2
    for _ in range(reps):
        V.voila_rollout(g32, R32, particles, None, acts, wl.d_omega, wl.gamma, wl.seed, planner, J, None, None, ws)
    e1.record(stream)
    torch.cuda.synchronize()
    sec = e0.elapsed_time(e1) / 1e3 / reps
    return {"value": seqs * wl.N * wl.H / sec, "unit": UNIT, "dtype": "f32",
            "sample": f"{seqs} of {wl.K} sequences x {wl.N} particles x H={wl.H}, same weights in FP32"}


def fp8_form(V, wl, planner, particles, stream, peaks=None, fp8_peak=None):
    """The FP8 e4m3 form (hidden layers E4M3 with per-channel scales) on the full
    workload, same particles and weights; returns its throughput, its roofline
    against the E4M3 tensor rate, and J."""
    import torch
    g8 = V.DeviceMLP([torch.from_numpy(w) for w in wl.g_T.W], [torch.from_numpy(b) for b in wl.g_T.b],
                     wl.g_T.act, V.FP8E4M3)
    r8 = V.DeviceMLP([torch.from_numpy(w) for w in wl.reward_mlp.W], [torch.from_numpy(b) for b in wl.reward_mlp.b],
                     wl.reward_mlp.act, V.FP8E4M3)
    R8 = V.mlp_reward(r8)
    acts = torch.from_numpy(wl.actions).float().cuda()
    J = torch.empty(wl.K, dtype=torch.float64, device="cuda")
    ws = V.alloc_workspace(V.voila_rollout_workspace_size(g8, R8, wl.N, wl.K, wl.H))
    V.voila_rollout(g8, R8, particles, None, acts, wl.d_omega, wl.gamma, wl.seed, planner, J, None, None, ws)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 12
    with Clocks(torch.cuda.current_device()) as clk:
        e0.record(stream)
        for _ in range(reps):
            V.voila_rollout(g8, R8, particles, None, acts, wl.d_omega, wl.gamma, wl.seed, planner, J, None, None, ws)
        e1.record(stream)
        torch.cuda.synchronize()
    assert V.workspace_status(ws) == V.OK
    sec = e0.elapsed_time(e1) / 1e3 / reps
    achieved = flops_per_transition(wl) * wl.N * wl.K * wl.H / sec / 1e12
    clocks = clk.summary()
    return {"value": wl.N * wl.K * wl.H / sec, "unit": UNIT, "dtype": "e4m3 hidden layers, bf16 first/last",
            "rollout_ms": 1e3 * sec, "sample": "full workload, same particles and weights",
            "roofline": dict(tensor_roofline(achieved, peaks or {}, clocks, "fp8", fp8_peak),
                             traffic=profiled_traffic("fp8", wl)[0], tensor_pipe_pct_ncu=profiled_traffic("fp8", wl)[1],
                             kernel="rollout_tc_kernel FP8 instantiation (voila_rollout call)",
                             flops="algorithmic, as the BF16 line (543,232 per transition)"),
            "clocks": clocks}, J.cpu().numpy()


def run_reference(args, rank):
    """The oracle as the reference arm: bounded samples of the same workload, timed on the host."""
    if rank != 0:
        return
    wl = make_workload(args.workload, args)
    seqs = 2
    for _ in range(args.warmup):
        cpu_baseline(wl, seqs)
    t0 = time.perf_counter()
    last = None
    for _ in range(args.steps):
        last, _, _ = cpu_baseline(wl, seqs)
    dt = time.perf_counter() - t0
    value = args.steps * seqs * wl.N * wl.H / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(wl, args),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": last["cores"], "kind": "oracle",
                             "sample": f"each step: {last['sample']}"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def small_planners_record(V, WL, g, R, wl, rank, stream, reps=20):
    """64 small planners (N log-uniform in [64, 1024], K in {8..64}, H in {5..30},
    seed 5): the regime the batched launch is for, where one planner's rollout
    is a fraction of a wave of CTA pairs. One autotuned batched launch captured in
    a CUDA graph against 64 sequential voila_rollout calls, eager and captured in
    a graph, each the median of `reps`; J must be identical."""
    import torch
    Ns, Ks, Hs = WL.batched_planners(seed=5, N_range=(64, 1024), K_range=(8, 64), H_range=(5, 30))
    items = []
    for i, (N, K, H) in enumerate(zip(Ns, Ks, Hs)):
        parts, acts = WL.planner_inputs(2000 + i, int(N), int(K), int(H))
        items.append({"particles": torch.from_numpy(parts).float().cuda(),
                      "actions": torch.from_numpy(acts).float().cuda(), "planner_id": 64 * rank + i,
                      "J": torch.empty(int(K), dtype=torch.float64, device="cuda"),
                      "best_k": torch.empty(1, dtype=torch.int32, device="cuda")})
    E = int(np.sum(Ns.astype(np.int64) * Ks * Hs))
    pl = V.make_planners(items)
    ws = V.alloc_workspace(V.voila_rollout_batched_workspace_size(g, R, pl))
    big = max(V.voila_rollout_workspace_size(g, R, int(N), int(K), int(H)) for N, K, H in zip(Ns, Ks, Hs))
    ws1 = V.alloc_workspace(big)

    def timed(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts), statistics.pstdev(ts)

    with torch.cuda.stream(stream):
        best, _ = V.voila_rollout_batched_autotune(g, R, pl, wl.d_s, wl.d_a, wl.d_omega, wl.gamma, wl.seed, ws,
                                                   stream=stream)
        gb = torch.cuda.CUDAGraph()
        with torch.cuda.graph(gb, stream=stream):
            V.voila_rollout_batched(g, R, pl, wl.d_s, wl.d_a, wl.d_omega, wl.gamma, wl.seed, best, ws, stream=stream)
        b_ms, b_sd = timed(gb.replay)
        J_b = [it["J"].clone() for it in items]

        def sequential():
            for it in items:
                V.voila_rollout(g, R, it["particles"], None, it["actions"], wl.d_omega, wl.gamma, wl.seed,
                                it["planner_id"], it["J"], None, it["best_k"], ws1, stream=stream)
        s_ms, s_sd = timed(sequential)
        same = all(torch.equal(a, it["J"]) for a, it in zip(J_b, items))
        gs = torch.cuda.CUDAGraph()
        with torch.cuda.graph(gs, stream=stream):
            sequential()
        sg_ms, sg_sd = timed(gs.replay)
    return {"workload": f"64 planners, N log-uniform [64, 1024], K in [8, 64], H in [5, 30] (seed 5); {E} transitions",
            "schedule": best, "batched_graph_ms": b_ms, "batched_stdev_ms": b_sd,
            "sequential_eager_ms": s_ms, "sequential_eager_stdev_ms": s_sd,
            "sequential_graph_ms": sg_ms, "sequential_graph_stdev_ms": sg_sd,
            "value_batched": E / (b_ms / 1e3), "value_sequential_graph": E / (sg_ms / 1e3),
            "repeats": reps, "batched_equals_sequential": same}


def batched_record(args, rank, world, local):
    """64 independent planners (uneven N, K, H from seed 4) sharing the mid-size BF16
    MLPs: one autotuned, graph-captured batched launch per step, against the same
    work as 64 sequential voila_rollout calls."""
    import torch
    from paper_2606_19729_b300 import voila as V
    from paper_2606_19729_b300 import workloads as WL

    torch.cuda.set_device(local)
    wl = WL.mid_bf16(N=8, K=1, H=1)
    g = V.DeviceMLP.from_spec(wl.g_T)
    rm = V.DeviceMLP.from_spec(wl.reward_mlp)
    R = V.mlp_reward(rm)
    Ns, Ks, Hs = WL.batched_planners(seed=4)
    items = []
    for i, (N, K, H) in enumerate(zip(Ns, Ks, Hs)):
        parts, acts = WL.planner_inputs(1000 + i, int(N), int(K), int(H))
        items.append({"particles": torch.from_numpy(parts).float().cuda(),
                      "actions": torch.from_numpy(acts).float().cuda(), "planner_id": 64 * rank + i,
                      "J": torch.empty(int(K), dtype=torch.float64, device="cuda"),
                      "best_k": torch.empty(1, dtype=torch.int32, device="cuda")})
    E = int(np.sum(Ns.astype(np.int64) * Ks * Hs))
    pl = V.make_planners(items)
    ws = V.alloc_workspace(V.voila_rollout_batched_workspace_size(g, R, pl))
    stream = torch.cuda.Stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    with torch.cuda.stream(stream):
        best, tune_ms = V.voila_rollout_batched_autotune(g, R, pl, wl.d_s, wl.d_a, wl.d_omega, wl.gamma, wl.seed,
                                                         ws, stream=stream)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            V.voila_rollout_batched(g, R, pl, wl.d_s, wl.d_a, wl.d_omega, wl.gamma, wl.seed, best, ws,
                                    stream=stream)
        for _ in range(args.warmup):
            graph.replay()
        torch.cuda.synchronize()
        assert V.workspace_status(ws, stream) == V.OK
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        with Clocks(local) as clk:
            for i in range(args.steps):
                flush.fill_(i & 0xFF)
                ev[i][0].record(stream)
                graph.replay()
                ev[i][1].record(stream)
            torch.cuda.synchronize()
        batched_s = sum(a.elapsed_time(b) for a, b in ev) / 1e3
        J_batched = [it["J"].clone() for it in items]
        # the same work as 64 sequential single-problem launches
        big = max(V.voila_rollout_workspace_size(g, R, int(N), int(K), int(H)) for N, K, H in zip(Ns, Ks, Hs))
        ws1 = V.alloc_workspace(big)

        def sequential():
            for it in items:
                V.voila_rollout(g, R, it["particles"], None, it["actions"], wl.d_omega, wl.gamma, wl.seed,
                                it["planner_id"], it["J"], None, it["best_k"], ws1, stream=stream)
        sequential()
        torch.cuda.synchronize()
        seq_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(max(1, args.steps))]
        for a, b in seq_ev:
            flush.fill_(1)
            a.record(stream)
            sequential()
            b.record(stream)
        torch.cuda.synchronize()
        seq_s = sum(a.elapsed_time(b) for a, b in seq_ev) / 1e3
        same = all(torch.equal(a, it["J"]) for a, it in zip(J_batched, items))
        # paired: the two forms alternate, so slow drifts of the clock affect both alike
        pairs = []
        for i in range(max(1, args.steps)):
            e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            flush.fill_(3)
            e[0].record(stream)
            graph.replay()
            e[1].record(stream)
            flush.fill_(4)
            e[2].record(stream)
            sequential()
            e[3].record(stream)
            pairs.append(e)
        torch.cuda.synchronize()
        paired = [(e[0].elapsed_time(e[1]), e[2].elapsed_time(e[3])) for e in pairs]
        # every candidate schedule of the autotuner, timed alone on the same work
        sched_ms = {}
        if getattr(args, "batched_schedules", False):
            full = torch.cuda.get_device_properties(local).multi_processor_count // 2
            names = {"two-tile static LPT": 1, "two-tile static table order": 0, "two-tile queue LPT": 3,
                     "two-tile queue table order": 2, f"two-tile queue LPT {full - 2} pairs": 3 | ((full - 2) << 8),
                     f"two-tile static LPT {full * 7 // 8} pairs": 1 | ((full * 7 // 8) << 8),
                     "one-tile queue LPT": 7, "one-tile static LPT": 5}
            for nm, sc in names.items():
                ts = []
                for _ in range(3):
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    flush.fill_(2)
                    e0.record(stream)
                    V.voila_rollout_batched(g, R, pl, wl.d_s, wl.d_a, wl.d_omega, wl.gamma, wl.seed, sc, ws,
                                            stream=stream)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    ts.append(e0.elapsed_time(e1))
                sched_ms[nm] = {"schedule": sc, "ms_median_of_3": statistics.median(ts)}
    b_ms = [a.elapsed_time(b) for a, b in ev]
    s_ms = [a.elapsed_time(b) for a, b in seq_ev]
    peaks = load_peaks()
    clocks = clk.summary()
    fpt = flops_per_transition(wl)
    achieved = fpt * E * args.steps / batched_s / 1e12
    line = {"metric": METRIC, "value": E * args.steps / batched_s, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * batched_s / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
            "data": "synthetic (seeded inputs, random-init weights)",
            "config": {"workload": f"batched: 64 planners, N log-uniform [512, 16384], K in [128, 1024], "
                                   f"H in [5, 30] (seed 4), 3x256 SiLU BF16 MLPs shared; {E} transitions per step",
                       "l2": "flushed (256 MB write) before every timed step",
                       "launch": "one autotuned batched launch captured in a CUDA graph"},
            "schedule": best, "autotune_ms": tune_ms,
            "batched_ms": {"repeats": len(b_ms), "min": min(b_ms), "median": statistics.median(b_ms),
                           "max": max(b_ms), "stdev": statistics.pstdev(b_ms)},
            "sequential_64_launches": {"value": E * len(seq_ev) / seq_s, "ms_per_step": 1e3 * seq_s / len(seq_ev),
                                       "repeats": len(s_ms), "min": min(s_ms), "median": statistics.median(s_ms),
                                       "max": max(s_ms), "stdev": statistics.pstdev(s_ms)},
            "batched_equals_sequential": same,
            "paired": {"pairs": len(paired), "batched_ms": [round(b, 3) for b, _ in paired],
                       "sequential_ms": [round(q, 3) for _, q in paired],
                       "sequential_minus_batched_ms_median": statistics.median(q - b for b, q in paired),
                       "sequential_minus_batched_ms_min": min(q - b for b, q in paired),
                       "batched_faster_in": sum(1 for b, q in paired if q > b)},
            "roofline": dict(tensor_roofline(achieved, peaks, clocks, "bf16"), traffic=None,
                             kernel="rollout_tc_kernel (batched)"),
            "gpu_launches": 4 * args.steps, "clocks": clocks}
    if sched_ms:
        line["schedules"] = sched_ms
    line["small_planners"] = small_planners_record(V, WL, g, R, wl, rank, stream)
    return line


def run_batched(args, rank, world, local):
    line = batched_record(args, rank, world, local)
    if rank == 0:
        print(json.dumps(line), flush=True)


def sweep_record(args, rank, world, local, fp8_peak=None):
    """Precision sweep (state 12, action 3, latent 16, 4x512 SiLU generator, GOAL
    reward, 16384 x 2048 x 25): FP32 (CUDA cores, on a slice of sequences), BF16 and
    FP8 (tensor cores, full workload), each form's return error against the FP64
    oracle on a subset: the first `--sweep-err-seqs` sequences and `--sweep-err-N`
    particles, run by every form and by the oracle as the same smaller problem."""
    import torch
    from paper_2606_19729_b300 import voila as V
    from paper_2606_19729_b300 import workloads as WL

    torch.cuda.set_device(local)
    wl = WL.sweep()
    stream = torch.cuda.current_stream()
    peaks = load_peaks()
    if fp8_peak is None:
        fp8_peak = measure_fp8_peak()
    parts = torch.from_numpy(wl.particles).float().cuda()
    acts = torch.from_numpy(wl.actions).float().cuda()
    R = V.goal_reward(list(wl.goal))
    forms = {}
    Js = {}
    for name, prec in (("bf16", V.BF16), ("fp8_e4m3", V.FP8E4M3), ("fp32_cuda_cores", V.FP32)):
        g = V.DeviceMLP([torch.from_numpy(w) for w in wl.g_T.W], [torch.from_numpy(b) for b in wl.g_T.b],
                        wl.g_T.act, prec)
        K = wl.K if prec != V.FP32 else args.fp32_seqs
        a = acts if prec != V.FP32 else acts[:K].contiguous()
        J = torch.empty(K, dtype=torch.float64, device="cuda")
        ws = V.alloc_workspace(V.voila_rollout_workspace_size(g, R, wl.N, K, wl.H))
        V.voila_rollout(g, R, parts, None, a, wl.d_omega, wl.gamma, wl.seed, 0, J, None, None, ws)
        torch.cuda.synchronize()
        reps = max(1, args.steps) if prec != V.FP32 else 1
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        with Clocks(local) as clk:
            for e0, e1 in ev:
                e0.record(stream)
                V.voila_rollout(g, R, parts, None, a, wl.d_omega, wl.gamma, wl.seed, 0, J, None, None, ws)
                e1.record(stream)
            torch.cuda.synchronize()
        assert V.workspace_status(ws) == V.OK
        sec = sum(e0.elapsed_time(e1) for e0, e1 in ev) / 1e3 / reps
        fpt = sum(2 * w.shape[0] * w.shape[1] for w in wl.g_T.W)
        achieved = fpt * wl.N * K * wl.H / sec / 1e12
        clocks = clk.summary()
        forms[name] = {"value": wl.N * K * wl.H / sec, "unit": UNIT, "rollout_ms": 1e3 * sec,
                       "achieved_tflops": achieved,
                       "sample": f"{K} of {wl.K} sequences x {wl.N} particles x H={wl.H}", "clocks": clocks}
        if prec == V.FP32:
            forms[name]["roofline"] = dict(fp32_roofline(achieved, peaks, clocks,
                                                         torch.cuda.get_device_properties(0).multi_processor_count),
                                           kernel="rollout_simt_kernel")
        else:
            forms[name]["roofline"] = dict(
                tensor_roofline(achieved, peaks, clocks, "fp8" if prec == V.FP8E4M3 else "bf16", fp8_peak),
                kernel="rollout_tc_kernel (wide)")
        # the error subset, as its own smaller problem (same counters as the oracle's)
        Ns, Ks = min(args.sweep_err_N, wl.N), min(args.sweep_err_seqs, wl.K)
        Jsub = torch.empty(Ks, dtype=torch.float64, device="cuda")
        wss = V.alloc_workspace(V.voila_rollout_workspace_size(g, R, Ns, Ks, wl.H))
        V.voila_rollout(g, R, parts[:Ns].contiguous(), None, acts[:Ks].contiguous(), wl.d_omega, wl.gamma, wl.seed, 0,
                        Jsub, None, None, wss)
        torch.cuda.synchronize()
        assert V.workspace_status(wss) == V.OK
        Js[name] = Jsub.cpu().numpy()
    if rank == 0 and not args.no_cpu_baseline:
        from oracle import voila_oracle as O
        Ns, Ks = min(args.sweep_err_N, wl.N), min(args.sweep_err_seqs, wl.K)
        t0 = time.perf_counter()
        Jo, _ = O.rollout(O.MLP(wl.g_T.W, wl.g_T.b, wl.g_T.act), O.Reward(O.REWARD_GOAL, wl.goal),
                          wl.particles[:Ns], wl.actions[:Ks], wl.d_omega, wl.gamma, wl.seed)
        dt = time.perf_counter() - t0
        for name in forms:
            forms[name]["err_vs_fp64"] = float(np.max(np.abs(Js[name] - Jo)) / np.max(np.abs(Jo)))
            forms[name]["err_sample"] = f"J of {Ks} sequences x {Ns} particles x H={wl.H}, max abs error / max |J|"
        cpu = {"value": Ks * Ns * wl.H / dt, "unit": UNIT, "cores": blas_threads(), "kind": "oracle",
               "sample": f"FP64 oracle rollout of {Ks} sequences x {Ns} particles x H={wl.H} in {dt:.1f} s"}
    else:
        cpu = None
    b = forms["bf16"]
    line = {"metric": METRIC, "value": b["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": 1, "ms_per_step": b["rollout_ms"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16", "data": "synthetic (seeded inputs, random-init weights)",
            "config": {"workload": "sweep: N=16384 x K=2048 x H=25, d_s=12 d_a=3 d_omega=16, generator 31x512x512x512x512x12 "
                                   "SiLU, GOAL reward; forms FP32 / BF16 / FP8 e4m3 (per-channel scales)"},
            "forms": forms, "peaks_this_run": {"e4m3_tflops_burst": fp8_peak},
            "roofline": dict(b["roofline"], traffic=None),
            "gpu_launches": 3 * args.steps, "clocks": b["clocks"]}
    if cpu:
        line["cpu_baseline"] = cpu
    return line


def run_sweep(args, rank, world, local):
    line = sweep_record(args, rank, world, local)
    if rank == 0:
        print(json.dumps(line), flush=True)


# FP32 FMA peak of the CUDA cores: 148 SMs x 128 FP32 lanes x 2 FLOP x 2032 MHz.
FP32_ALU_TFLOPS = 148 * 128 * 2 * 2032e6 / 1e12


def distill_flops(wl):
    """Algorithmic FLOPs per sample: T teacher calls, student forward, backward (2x forward)."""
    teacher = sum(2 * w.shape[0] * w.shape[1] for w in wl.teacher.W) * wl.T
    student = sum(2 * w.shape[0] * w.shape[1] for w in wl.student.W)
    return teacher, student * 3


def distill_record(args, rank, world, local):
    """Distillation training step (Eq. 3), B=65536: teacher DDIM targets (32 steps of
    the 82-512-512-512-8 SiLU denoiser), student 18-256-256-256-8 forward with BF16
    weights, MSE, hand-written backward, Adam on FP32 master weights."""
    import torch
    from paper_2606_19729_b300 import voila as V
    from paper_2606_19729_b300 import workloads as WL
    from paper_2606_19729_b300.distill import Distiller

    torch.cuda.set_device(local)
    if world > 1 and not torch.distributed.is_initialized():
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    wl = WL.distill(B=args.B or 65536, teacher_prec=WL.PREC_BF16)
    B = wl.B
    stream = torch.cuda.current_stream()
    teacher = V.DeviceMLP.from_spec(wl.teacher)
    d = Distiller(teacher, [torch.from_numpy(w) for w in wl.student.W], [torch.from_numpy(b) for b in wl.student.b],
                  wl.student.act, V.BF16, B, wl.T, wl.beta0, wl.beta1, wl.emb_dim, lr=wl.lr)
    S, A, om = (torch.from_numpy(x).float().cuda() for x in (wl.S, wl.A, wl.omega))
    # each step trains on the batch and samples the teacher targets of the next
    # batch (here the same synthetic batch) on a second stream meanwhile
    # (Distiller.step_overlapped; the same results as the plain step)
    losses = torch.empty(args.warmup + args.steps, dtype=torch.float64, device="cuda")
    for i in range(args.warmup):
        d.step_overlapped(S, A, om, S, A, om, loss_out=losses[i:i + 1])
    d.join()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    with Clocks(local) as clk:
        t_all0 = torch.cuda.Event(enable_timing=True)
        t_all1 = torch.cuda.Event(enable_timing=True)
        t_all0.record(stream)
        for i in range(args.steps):
            d.step_overlapped(S, A, om, S, A, om, loss_out=losses[args.warmup + i:args.warmup + i + 1])
        d.join()  # the last step's sampler is inside the timed region
        t_all1.record(stream)
        torch.cuda.synchronize()
    sec = max_over_ranks(t_all0.elapsed_time(t_all1) / 1e3, world, torch.device("cuda", local))
    value = aggregate_rate(B * args.steps, world, sec)
    lo = losses.cpu().numpy()
    # the plain step (sampler, then the student's step, on one stream) beside it
    pl0 = torch.cuda.Event(enable_timing=True)
    pl1 = torch.cuda.Event(enable_timing=True)
    for _ in range(2):
        d.step(S, A, om)
    pl0.record(stream)
    for _ in range(args.steps):
        d.step(S, A, om)
    pl1.record(stream)
    torch.cuda.synchronize()
    plain_ms = pl0.elapsed_time(pl1) / args.steps
    # the dominant kernel alone: the teacher sampler, same inputs, CUDA events on its
    # stream, back to back for long enough to run under the power cap
    Y = torch.empty(B, wl.d_x, device="cuda")
    tws = V.alloc_workspace(V.voila_ddim_sample_workspace_size(teacher, wl.T))
    reps = max(100, args.steps)
    tev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    for e0, e1 in tev:
        e0.record(stream)
        V.voila_ddim_sample(teacher, S, A, om, wl.T, wl.beta0, wl.beta1, wl.emb_dim, Y, tws, stream)
        e1.record(stream)
    torch.cuda.synchronize()
    ddim_s = sum(e0.elapsed_time(e1) for e0, e1 in tev) / 1e3 / reps
    assert V.workspace_status(tws) == V.OK and V.workspace_status(d.ws) == V.OK
    f_teacher, f_student = distill_flops(wl)
    achieved = f_teacher * B / ddim_s / 1e12
    peaks = load_peaks()
    clocks = clk.summary()
    # end to end: each step copies the next batch's inputs from pinned host memory
    # into one of two device buffers and reads the loss back (the training
    # stream synchronised; the sampler of the next batch keeps running)
    hS, hA, hO = (x.cpu().pin_memory() for x in (S, A, om))
    hl = torch.empty(1, dtype=torch.float64).pin_memory()
    bufs = [tuple(torch.empty_like(x) for x in (S, A, om)) for _ in range(2)]
    d.join()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    # the first step also samples its own batch's targets: 30 steps or more keep that one extra
    # sampler pass a small share of the loop
    e2e_steps = max(30, args.steps)
    for x, h in zip(bufs[0], (hS, hA, hO)):
        x.copy_(h, non_blocking=True)
    for i in range(e2e_steps):
        cur_b, nxt_b = bufs[i % 2], bufs[(i + 1) % 2]
        for x, h in zip(nxt_b, (hS, hA, hO)):
            x.copy_(h, non_blocking=True)
        l = d.step_overlapped(*cur_b, *nxt_b)
        hl.copy_(l, non_blocking=True)
        torch.cuda.current_stream().synchronize()
    d.join()
    torch.cuda.synchronize()
    e2e_sec = max_over_ranks((time.perf_counter() - t0), world, torch.device("cuda", local))
    line = {"metric": "distillation samples/s", "value": value, "unit": "samples/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sec / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
            "data": "synthetic (seeded inputs, random-init teacher and student)",
            "config": {"workload": f"distill: B={B}, teacher 82x512x512x512x8 SiLU + 64-d step embedding "
                                   f"(BF16, tensor cores), {wl.T} DDIM steps, linear beta 1e-4..0.02; student "
                                   "18x256x256x256x8 SiLU, BF16 forward copy (FP32 arithmetic), FP32 master, Adam",
                       "l2": "inputs resident; the step's working set (teacher activations, saved "
                             "pre-activations, gradients) exceeds L2",
                       "launch": "the teacher sampler of the next batch on a second, high-priority stream "
                                 "while the student trains (its GEMMs one CTA per tile); every step is one "
                                 "sampler pass and one student step"},
            "loss": {"first": float(lo[0]), "last": float(lo[-1])},
            "plain_step": {"ms_per_step": plain_ms, "value": aggregate_rate(B, world, plain_ms / 1e3),
                           "note": "sampler, then the student's step, on one stream"},
            "teacher_ms": 1e3 * ddim_s,
            "roofline": dict(tensor_roofline(achieved, peaks, clocks, "bf16"), traffic=None,
                             kernel="rollout_tc_kernel (DDIM sampler mode)",
                             flops="algorithmic: 2 x (82x512 + 512x512 x 2 + 512x8) x 32 steps per sample"),
            "e2e": {"value": B * e2e_steps * world / e2e_sec, "unit": "samples/s",
                    "h2d_bytes_per_step": int(sum(x.numel() * 4 for x in (hS, hA, hO))), "d2h_bytes_per_step": 8},
            "gpu_launches": None, "clocks": clocks}
    n_layers = len(wl.student.W)
    # per step (BF16 student, tensor cores): sampler 3 (pack, embeddings, kernel),
    # concat 1, forward (input prep, 2 padded weights, L-1 transposed weights,
    # L GEMMs), loss 2, backward (delta prep, bias sum of the output, L-1 delta
    # GEMMs, L weight GEMMs, L partial sums, L-1 bias sums), adam 1, publish 1
    L_ = n_layers
    line["gpu_launches"] = args.steps * (3 + 1 + (1 + 2 + (L_ - 1) + L_) + 2 + (2 + (L_ - 1) + 3 * L_ + (L_ - 1)) + 2)
    if rank == 0 and not args.no_cpu_baseline:
        from oracle import voila_oracle as O
        rows = args.distill_cpu_rows
        t0 = time.perf_counter()
        tm = O.MLP(wl.teacher.W, wl.teacher.b, wl.teacher.act)  # the BF16-rounded teacher
        fwd = O.MLP([WL.round_bf16(w) for w in wl.student.W], wl.student.b, wl.student.act)
        s_hat = O.distill_targets(tm, wl.S[:rows], wl.A[:rows], wl.omega[:rows], wl.T, wl.beta0, wl.beta1,
                                  wl.emb_dim)
        L, gW, gb = O.distill_loss_and_grad(fwd, wl.S[:rows], wl.A[:rows], wl.omega[:rows], s_hat)
        p0 = O.flat_params(O.MLP(wl.student.W, wl.student.b, wl.student.act))
        g = np.concatenate([x for l in range(len(gW)) for x in (gW[l].ravel(), gb[l].ravel())])
        O.adam_step([p0], [g], O.adam_init([p0]), lr=wl.lr)
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": rows / dt, "unit": "samples/s", "cores": blas_threads(), "kind": "oracle",
                                "sample": f"FP64 oracle distillation step on {rows} of {B} rows "
                                          f"(DDIM targets, loss, gradient, Adam) in {dt:.1f} s"}
    return line


def run_distill(args, rank, world, local):
    line = distill_record(args, rank, world, local)
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_infonce(args, rank, world, local):
    """InfoNCE objective of the likelihood model (Eq. 6) on B=1024 tuples: the
    16-256-256-256-1 SiLU likelihood (BF16) on all B^2 = 1,048,576 pairs on the
    tensor cores, row log-sum-exp, loss and dloss/dL; then the likelihood's
    training step (FP32 arithmetic, hand-written backward, Adam) timed beside it."""
    import torch
    from paper_2606_19729_b300 import voila as V
    from paper_2606_19729_b300 import workloads as WL

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    wl = WL.infonce(B=args.B or 1024)
    B = wl.B
    stream = torch.cuda.current_stream()
    ell = V.DeviceMLP.from_spec(wl.ell)
    S, A, Ob = (torch.from_numpy(x).float().cuda() for x in (wl.S, wl.A, wl.O))
    L = torch.empty(B, B, device="cuda")
    G = torch.empty(B, B, device="cuda")
    lse = torch.empty(B, dtype=torch.float64, device="cuda")
    loss = torch.empty(1, dtype=torch.float64, device="cuda")
    ws = V.alloc_workspace(V.voila_infonce_workspace_size(ell, B))

    def fwd():
        V.voila_infonce_forward(ell, S, A, Ob, L, lse, loss, G, ws)

    for _ in range(args.warmup):
        fwd()
    warm_until(fwd, 0.3)
    reps = max(args.steps, 50)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    with Clocks(local) as clk:
        for e0, e1 in ev:
            e0.record(stream)
            fwd()
            e1.record(stream)
        torch.cuda.synchronize()
    assert V.workspace_status(ws) == V.OK
    fwd_s = sum(a.elapsed_time(b) for a, b in ev) / 1e3 / reps
    sec = max_over_ranks(fwd_s * reps, world, torch.device("cuda", local))
    pairs = B * B
    value = aggregate_rate(pairs * reps, world, sec)
    fpp = sum(2 * w.shape[0] * w.shape[1] for w in wl.ell.W)
    achieved = fpp * pairs / fwd_s / 1e12
    peaks = load_peaks()
    clocks = clk.summary()
    # training step of the likelihood (tensor cores for the BF16 planning shapes), a few steps
    master = torch.cat([torch.cat([w.float().reshape(-1), b.reshape(-1)]) for w, b in zip(ell.W, ell.b)])
    m, v = torch.zeros_like(master), torch.zeros_like(master)
    sws = V.alloc_workspace(V.voila_infonce_step_workspace_size(ell, B))
    step_losses = torch.empty(3, dtype=torch.float64, device="cuda")
    sev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(3)]
    for i, (e0, e1) in enumerate(sev):
        e0.record(stream)
        V.voila_infonce_step(ell, master, m, v, V.voila_adam(wl.lr, 0.9, 0.999, 1e-8, i + 1), S, A, Ob,
                             step_losses[i:i + 1], None, sws)
        e1.record(stream)
    torch.cuda.synchronize()
    step_ms = [a.elapsed_time(b) for a, b in sev]
    line = {"metric": "InfoNCE pair evaluations/s", "value": value, "unit": "pairs/s", "n_gpus": world,
            "steps": reps, "warmup": args.warmup, "ms_per_step": 1e3 * fwd_s, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
            "data": "synthetic (seeded tuples, random-init likelihood)",
            "config": {"workload": f"infonce: B={B} tuples (B^2={pairs} pairs), likelihood 16x256x256x256x1 SiLU "
                                   "BF16 on the tensor cores; row log-sum-exp, loss, dloss/dL"},
            "loss": loss.item(),
            "roofline": dict(tensor_roofline(achieved, peaks, clocks, "bf16"), traffic=None,
                             kernel="voila_infonce_forward (weight pack + pair kernel + row LSE + loss)"),
            "train_step": {"ms": statistics.median(step_ms), "loss_first": float(step_losses[0].item()),
                           "loss_last": float(step_losses[-1].item()),
                           "note": "BF16 likelihood: tensor-core training forward and backward over all B^2 pair rows"},
            "gpu_launches": 4 * reps, "clocks": clocks}
    if rank == 0 and not args.no_cpu_baseline:
        from oracle import voila_oracle as O
        rows = 256  # tuples i of the sample: their B-pair rows of logits and log-sum-exp
        t0 = time.perf_counter()
        X = O.infonce_pairs(wl.S, wl.A, wl.O).reshape(B, B, -1)[:rows].reshape(-1, wl.ell.dims[0])
        Lo = O.mlp_forward(O.MLP(wl.ell.W, wl.ell.b, wl.ell.act), X)[:, 0].reshape(rows, B)
        mo = Lo.max(axis=1, keepdims=True)
        _ = mo[:, 0] + np.log(np.exp(Lo - mo).sum(axis=1))
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": rows * B / dt, "unit": "pairs/s", "cores": blas_threads(), "kind": "oracle",
                                "sample": f"FP64 oracle logits and row log-sum-exp of {rows} of {B} rows "
                                          f"({rows * B} pairs) in {dt:.1f} s"}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_pw(args, rank, world, local):
    """Progressive widening (Sec. 4.3) of 65536 simulations over 4096 action nodes:
    grouping, widening decisions, f_Z observations of the new branches, branch
    likelihoods (16-256-256-256-1, BF16 weights, FP32 arithmetic), per-branch SIR
    resampling. The tree is restored before every call so each call does the same work."""
    import torch
    from paper_2606_19729_b300 import voila as V
    from paper_2606_19729_b300 import workloads as WL

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    wl = WL.pw(M=args.B or 65536)
    M = wl.M
    stream = torch.cuda.current_stream()
    tree = V.PWTree(torch.from_numpy(wl.act), torch.from_numpy(wl.N0), torch.from_numpy(wl.C0),
                    torch.from_numpy(wl.obs0))
    N0, C0, obs0 = tree.N.clone(), tree.C.clone(), tree.obs.clone()
    g_Z = V.DeviceMLP.from_spec(wl.g_Z)
    ell = V.DeviceMLP.from_spec(wl.ell)
    lik = V.mlp_likelihood(ell)
    node = torch.from_numpy(wl.node).to(device="cuda", dtype=torch.int32)
    s_next = torch.from_numpy(wl.s_next).float().cuda()
    branch = torch.empty(M, dtype=torch.int32, device="cuda")
    s_out = torch.empty_like(s_next)
    ws = V.alloc_workspace(V.voila_progressive_widening_workspace_size(tree, g_Z, lik, M))

    def call():
        V.voila_progressive_widening(tree, node, s_next, g_Z, lik, wl.d_omega, wl.k_o, wl.alpha_o, wl.lam, wl.seed,
                                     0, rank, branch, s_out, ws)

    def restore():
        tree.N.copy_(N0)
        tree.C.copy_(C0)
        tree.obs.copy_(obs0)

    for _ in range(args.warmup):
        restore()
        call()
    warm_until(lambda: (restore(), call()), 0.3)
    assert V.workspace_status(ws) == V.OK
    reps = max(args.steps, 100)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    with Clocks(local) as clk:
        for e0, e1 in ev:
            restore()
            e0.record(stream)
            call()
            e1.record(stream)
        torch.cuda.synchronize()
    assert V.workspace_status(ws) == V.OK
    call_s = sum(a.elapsed_time(b) for a, b in ev) / 1e3 / reps
    sec = max_over_ranks(call_s * reps, world, torch.device("cuda", local))
    widened = int((tree.C - C0).sum().item())
    fz = sum(2 * w.shape[0] * w.shape[1] for w in wl.g_Z.W)
    fl = sum(2 * w.shape[0] * w.shape[1] for w in wl.ell.W)
    flops = fl * M + fz * widened
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    peak = nsm * 128 * 2 * 2032e6 / 1e12
    line = {"metric": "progressive-widening simulations/s", "value": aggregate_rate(M * reps, world, sec),
            "unit": "simulations/s", "n_gpus": world, "steps": reps, "warmup": args.warmup,
            "ms_per_step": 1e3 * call_s, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16", "data": "synthetic (seeded tree and simulations, random-init f_Z and likelihood)",
            "config": {"workload": f"pw: M={M} simulations over {wl.n_nodes} action nodes (skewed), C_max={wl.C_max}, "
                                   f"k_o={wl.k_o}, alpha_o={wl.alpha_o}; f_Z 18x256x256x256x6 and likelihood "
                                   "16x256x256x256x1 SiLU (BF16, tensor cores)"},
            "widened_per_call": widened,
            "roofline": {"bound": "alu", "achieved": flops / call_s / 1e12, "peak": peak, "unit": "TFLOP/s",
                         "frac": flops / call_s / 1e12 / peak, "traffic": None,
                         "kernel": "voila_progressive_widening (whole call; likelihood MLP dominates the FLOPs)",
                         "peak_kind": "FP32 FMA lanes x max SM clock (derived)"},
            "gpu_launches": None, "clocks": clk.summary()}
    def radix_passes(vmax):
        n = 0
        while vmax >> (8 * n):
            n += 1
        return n
    tiles = (M + 2047) // 2048
    per_pass = 2 + (1 if tiles > 64 else 0)  # counts, (scan,) scatter
    passes = radix_passes(wl.n_nodes) + radix_passes(wl.n_nodes * wl.C_max)
    # keys, 2 sorts, thresholds, group bounds, widen, assign, observation sampler (pack,
    # kernel), likelihood (pack, fused-output pack, kernel), keys, small- and large-group
    # resampling
    line["gpu_launches"] = reps * (13 + per_pass * passes)
    if rank == 0 and not args.no_cpu_baseline:
        from oracle import voila_oracle as O
        sel = np.ones(M, bool)
        tree_o = O.PWTree(wl.act.copy(), wl.N0.copy(), wl.C0.copy(), wl.obs0.copy())
        t0 = time.perf_counter()
        O.progressive_widening(tree_o, wl.node[sel], wl.s_next[sel], O.MLP(wl.g_Z.W, wl.g_Z.b, wl.g_Z.act),
                               O.Likelihood(O.LIK_MLP, mlp=O.MLP(wl.ell.W, wl.ell.b, wl.ell.act)), wl.d_omega,
                               wl.k_o, wl.alpha_o, wl.lam, wl.seed, 0, sim_index=np.nonzero(sel)[0])
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": int(sel.sum()) / dt, "unit": "simulations/s", "cores": blas_threads(),
                                "kind": "oracle", "sample": f"FP64 oracle widening of all {int(sel.sum())} simulations "
                                                            f"(one call) in {dt:.1f} s"}
    if rank == 0:
        print(json.dumps(line), flush=True)


def small_fp32_record(args, local):
    """The plain FP32 configuration in full (N=256, K=64, H=10, 2x64 tanh MLPs,
    GOAL reward): one planning step (belief update with the MLP likelihood, then
    the rollout of the updated belief, reduction and argmax) on the CUDA cores,
    timed by CUDA events over many steps; J against the FP64 oracle from the same
    resampled particles."""
    import torch
    from paper_2606_19729_b300 import voila as V
    from paper_2606_19729_b300 import workloads as WL
    from oracle import voila_oracle as O

    wl = WL.small_fp32()
    dev = torch.device("cuda", local)
    g = V.DeviceMLP.from_spec(wl.g_T)
    lik = V.mlp_likelihood(V.DeviceMLP.from_spec(wl.ell))
    R = V.goal_reward(list(wl.goal))
    P = torch.from_numpy(wl.particles).float().to(dev)
    A = torch.from_numpy(wl.actions).float().to(dev)
    a0 = A[0, 0].contiguous()
    # one observation drawn from the samplers: s' = g_T(s_true, a, w), o = g_Z(s', a, w_Z)
    gz = V.DeviceMLP.from_spec(wl.g_Z)
    s_true = torch.from_numpy(WL.true_state(wl.seed, wl.d_s, 0.5)).float().to(dev).reshape(1, -1)
    s_next = torch.empty((1, wl.d_s), device=dev)
    V.voila_generator_fwd_seeded(g, s_true, a0.reshape(1, -1), 0, wl.d_omega, wl.seed, 5, 0, 0, s_next)
    obs2 = torch.empty((1, wl.d_o), device=dev)
    V.voila_generator_fwd_seeded(gz, s_next, a0.reshape(1, -1), 0, wl.d_omega, wl.seed, V.STREAM_OBS_OMEGA, 0, 0,
                                 obs2)
    obs = obs2.reshape(-1).contiguous()
    p_new = torch.empty_like(P)
    J = torch.empty(wl.K, dtype=torch.float64, device=dev)
    best = torch.empty(1, dtype=torch.int32, device=dev)
    ws_b = V.alloc_workspace(V.voila_belief_update_workspace_size(g, lik, wl.N))
    ws_r = V.alloc_workspace(V.voila_rollout_workspace_size(g, R, wl.N, wl.K, wl.H))
    stream = torch.cuda.current_stream()

    def step():
        V.voila_belief_update(g, lik, P, None, a0, obs, wl.d_omega, wl.lam, wl.seed, 1, 0, p_new, None, None,
                              None, None, ws_b)
        V.voila_rollout(g, R, p_new, None, A, wl.d_omega, wl.gamma, wl.seed, 0, J, None, best, ws_r)

    warm_until(step, 0.3)
    # enough steps for ~1.5 s of timed region, so that the clock sampler (one
    # nvidia-smi sample per 200 ms) sees it
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(20):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    reps = int(min(20000, max(200, 1500.0 / (e0.elapsed_time(e1) / 20))))
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(reps)]
    with Clocks(local) as clk:
        for e in ev:
            e[0].record(stream)
            V.voila_belief_update(g, lik, P, None, a0, obs, wl.d_omega, wl.lam, wl.seed, 1, 0, p_new, None, None,
                                  None, None, ws_b)
            e[1].record(stream)
            V.voila_rollout(g, R, p_new, None, A, wl.d_omega, wl.gamma, wl.seed, 0, J, None, best, ws_r)
            e[2].record(stream)
        torch.cuda.synchronize()
    assert V.workspace_status(ws_b) == V.OK and V.workspace_status(ws_r) == V.OK
    step_ms = statistics.median(e[0].elapsed_time(e[2]) for e in ev)
    roll_ms = statistics.median(e[1].elapsed_time(e[2]) for e in ev)
    trans = wl.N * wl.K * wl.H
    clocks = clk.summary()
    achieved = flops_per_transition(wl) * trans / (roll_ms / 1e3) / 1e12
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    Jo, _ = O.rollout(O.MLP(wl.g_T.W, wl.g_T.b, wl.g_T.act), O.Reward(O.REWARD_GOAL, wl.goal),
                      p_new.cpu().double().numpy(), wl.actions, wl.d_omega, wl.gamma, wl.seed)
    Jd = J.cpu().numpy()
    # the same step captured once in a CUDA graph and replayed: the calls issue
    # no host synchronisation, so the graph holds the same launches without the
    # gaps between them
    gs = torch.cuda.Stream()
    gs.wait_stream(stream)
    with torch.cuda.stream(gs):
        step()
        gs.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=gs):
            step()
        for _ in range(20):
            graph.replay()
        gev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        for e0, e1 in gev:
            e0.record(gs)
            graph.replay()
            e1.record(gs)
        gs.synchronize()
    assert V.workspace_status(ws_b) == V.OK and V.workspace_status(ws_r) == V.OK
    graph_ms = statistics.median(e0.elapsed_time(e1) for e0, e1 in gev)
    return {"workload": "small_fp32: N=256 x K=64 x H=10, d_s=4 d_a=2 d_o=4 d_omega=4, 2x64 tanh FP32, GOAL "
                        "reward; belief update + rollout per step",
            "value": trans / (step_ms / 1e3), "unit": UNIT, "ms_per_step": step_ms, "rollout_ms": roll_ms,
            "graph_step": {"ms_per_step": graph_ms, "value": trans / (graph_ms / 1e3),
                           "note": "the same calls captured once in a CUDA graph and replayed"},
            "belief_update_ms": statistics.median(e[0].elapsed_time(e[1]) for e in ev), "dtype": "f32",
            "roofline": dict(fp32_roofline(achieved, load_peaks(), clocks, nsm),
                             kernel="rollout_rows_kernel (8 threads per row)",
                             note="latency bound: 16,384 rows, 163,840 transitions per launch"),
            "err_vs_fp64": {"J_normwise": float(np.max(np.abs(Jd - Jo)) / np.max(np.abs(Jo))), "tolerance": 1e-5,
                            "sample": "all 64 sequences, from the device's resampled particles"},
            "steps_timed": reps, "clocks": clocks}


def config_records(args, rank, world, local, fp8_peak):
    """Compact records of the other configurations, for the default run's line:
    the plain FP32 configuration, the precision sweep at full size, the
    distillation step and the batched planners."""
    import copy
    out = {}
    out["c1_small_fp32"] = small_fp32_record(args, local)
    a = copy.copy(args)
    a.steps, a.warmup = 2, 1
    sw = sweep_record(a, rank, world, local, fp8_peak)
    out["c3_sweep"] = {"workload": sw["config"]["workload"],
                       "forms": {k: {kk: v.get(kk) for kk in ("value", "rollout_ms", "roofline", "err_vs_fp64",
                                                              "err_sample", "sample", "clocks")}
                                 for k, v in sw["forms"].items()},
                       "cpu_baseline": sw.get("cpu_baseline")}
    a = copy.copy(args)
    a.steps, a.warmup = 10, 3
    d = distill_record(a, rank, world, local)
    out["c4_distill"] = {k: d.get(k) for k in ("metric", "value", "unit", "ms_per_step", "teacher_ms", "roofline",
                                               "loss", "e2e", "cpu_baseline", "clocks", "plain_step")}
    out["c4_distill"]["workload"] = d["config"]["workload"]
    out["c4_distill"]["launch"] = d["config"]["launch"]
    a = copy.copy(args)
    a.steps, a.warmup = 10, 1  # 10 repeats and 10 alternating pairs: the forms differ by a fraction of a percent
    b = batched_record(a, rank, world, local)
    out["c5_batched"] = {k: b.get(k) for k in ("value", "unit", "ms_per_step", "schedule", "autotune_ms",
                                               "batched_ms", "sequential_64_launches", "batched_equals_sequential",
                                               "paired",
                                               "roofline", "clocks", "small_planners")}
    out["c5_batched"]["workload"] = b["config"]["workload"]
    return out


def main():
    args = parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if args.workload == "batched":
        run_batched(args, rank, world, local)
        return
    if args.workload == "sweep":
        run_sweep(args, rank, world, local)
        return
    if args.workload == "distill":
        run_distill(args, rank, world, local)
        return
    if args.workload == "infonce":
        run_infonce(args, rank, world, local)
        return
    if args.workload == "pw":
        run_pw(args, rank, world, local)
        return

    import torch
    import torch.distributed as dist

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_2606_19729_b300 import voila as V

    wl = make_workload(args.workload, args)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    planner = rank  # independent noise per replica

    g = V.DeviceMLP.from_spec(wl.g_T)
    gz = V.DeviceMLP.from_spec(wl.g_Z)
    ell = V.DeviceMLP.from_spec(wl.ell)
    lik = V.mlp_likelihood(ell)
    if wl.goal is None:
        rm = V.DeviceMLP.from_spec(wl.reward_mlp)
        R = V.mlp_reward(rm)
    else:
        R = V.goal_reward(list(wl.goal))
    N, K, H = wl.N, wl.K, wl.H

    particles = torch.from_numpy(wl.particles).float().to(dev)
    actions = torch.from_numpy(wl.actions).float().to(dev)
    action = actions[0, 0].contiguous()
    # the observation is drawn from the samplers: s' = g_T(s_true, a, w), o = g_Z(s', a, w_Z)
    from paper_2606_19729_b300 import workloads as WL
    s_true = torch.from_numpy(WL.true_state(wl.seed, wl.d_s, 1.0)).float().to(dev).reshape(1, -1)
    s_next = torch.empty((1, wl.d_s), device=dev)
    # (the FP8 form draws the observation with the same weights in BF16: the seeded
    # sampler forward runs FP32 and BF16 MLPs)
    as_bf16 = lambda spec: V.DeviceMLP([torch.from_numpy(x) for x in spec.W],  # noqa: E731
                                       [torch.from_numpy(x) for x in spec.b], spec.act, V.BF16)
    g_draw, gz_draw = (g, gz) if wl.prec != 2 else (as_bf16(wl.g_T), as_bf16(wl.g_Z))
    V.voila_generator_fwd_seeded(g_draw, s_true, action.reshape(1, -1), 0, wl.d_omega, wl.seed, 5, 0, planner,
                                 s_next)
    obs2 = torch.empty((1, wl.d_o), device=dev)
    V.voila_generator_fwd_seeded(gz_draw, s_next, action.reshape(1, -1), 0, wl.d_omega, wl.seed, V.STREAM_OBS_OMEGA,
                                 0, planner, obs2)
    obs = obs2.reshape(-1).contiguous()

    p_new = torch.empty_like(particles)
    J = torch.empty(K, dtype=torch.float64, device=dev)
    best = torch.empty(1, dtype=torch.int32, device=dev)
    Vb = torch.empty(1, dtype=torch.float64, device=dev)
    pi = torch.empty(K, dtype=torch.float64, device=dev)
    eta = 1.0
    ws_b = V.alloc_workspace(V.voila_belief_update_workspace_size(g, lik, N))
    ws_r = V.alloc_workspace(V.voila_rollout_workspace_size(g, R, N, K, H))
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def step(p_in, obs_t, act_seq, a0):
        V.voila_belief_update(g, lik, p_in, None, a0, obs_t, wl.d_omega, wl.lam, wl.seed, 1, planner, p_new, None,
                              None, None, None, ws_b)
        V.voila_rollout(g, R, p_new, None, act_seq, wl.d_omega, wl.gamma, wl.seed, planner, J, None, best, ws_r)
        V.voila_preference_backup(J, None, eta, Vb, pi)

    for _ in range(args.warmup):
        step(particles, obs, actions, action)
    torch.cuda.synchronize()
    assert V.workspace_status(ws_b) == V.OK and V.workspace_status(ws_r) == V.OK

    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        for i in range(args.steps):
            flush.fill_(i & 0xFF)
            ev[i][0].record(stream)
            V.voila_belief_update(g, lik, particles, None, action, obs, wl.d_omega, wl.lam, wl.seed, 1, planner,
                                  p_new, None, None, None, None, ws_b)
            ev[i][1].record(stream)
            V.voila_rollout(g, R, p_new, None, actions, wl.d_omega, wl.gamma, wl.seed, planner, J, None, best,
                            ws_r)
            ev[i][2].record(stream)
            V.voila_preference_backup(J, None, eta, Vb, pi)
            ev[i][3].record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    step_ms = [e[0].elapsed_time(e[3]) for e in ev]
    roll_ms = [e[1].elapsed_time(e[2]) for e in ev]
    total_s = max_over_ranks(sum(step_ms) / 1e3, world, dev)
    assert V.workspace_status(ws_b) == V.OK and V.workspace_status(ws_r) == V.OK
    trans_per_step = N * K * H
    value = aggregate_rate(trans_per_step * args.steps, world, total_s)

    # end to end through the public API with host buffers (pinned), copies inside the timed region
    h_particles = torch.from_numpy(wl.particles).float().pin_memory()
    h_actions = torch.from_numpy(wl.actions).float().pin_memory()
    h_obs = obs.cpu().pin_memory()
    h_J = torch.empty(K, dtype=torch.float64).pin_memory()
    h_best = torch.empty(1, dtype=torch.int32).pin_memory()
    h_V = torch.empty(1, dtype=torch.float64).pin_memory()
    d_particles = torch.empty_like(particles)
    d_actions = torch.empty_like(actions)
    d_obs = torch.empty_like(obs)
    h2d = h_particles.numel() * 4 + h_actions.numel() * 4 + h_obs.numel() * 4
    d2h = K * 8 + 4 + 8
    e2e_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
    for i in range(args.steps + 1):
        flush.fill_(i & 0xFF)
        if i > 0:
            e2e_ev[i - 1][0].record(stream)
        d_particles.copy_(h_particles, non_blocking=True)
        d_actions.copy_(h_actions, non_blocking=True)
        d_obs.copy_(h_obs, non_blocking=True)
        step(d_particles, d_obs, d_actions, d_actions[0, 0])
        h_J.copy_(J, non_blocking=True)
        h_best.copy_(best, non_blocking=True)
        h_V.copy_(Vb, non_blocking=True)
        if i > 0:
            e2e_ev[i - 1][1].record(stream)
        torch.cuda.synchronize()
    e2e_s = max_over_ranks(sum(a.elapsed_time(b) for a, b in e2e_ev) / 1e3, world, dev)
    e2e_value = aggregate_rate(trans_per_step * args.steps, world, e2e_s)

    peaks = load_peaks()
    clocks = clk.summary()
    fpt = flops_per_transition(wl)
    roll_avg_s = sum(roll_ms) / len(roll_ms) / 1e3
    traffic, tensor_pipe = profiled_traffic("fp8" if wl.prec == 2 else "bf16", wl)
    if wl.prec == 1:
        achieved = fpt * trans_per_step / roll_avg_s / 1e12
        roof = dict(tensor_roofline(achieved, peaks, clocks, "bf16"), traffic=traffic,
                    kernel="rollout_tc_kernel (voila_rollout call: weight pack + rollout + return reduction)",
                    tensor_pipe_pct_ncu=tensor_pipe)
    elif wl.prec == 2:
        achieved = fpt * trans_per_step / roll_avg_s / 1e12
        roof = dict(tensor_roofline(achieved, peaks, clocks, "fp8", measure_fp8_peak()), traffic=traffic,
                    kernel="rollout_tc_kernel FP8 instantiation (voila_rollout call: scale + weight pack + rollout "
                           "+ return reduction)", tensor_pipe_pct_ncu=tensor_pipe)
    else:
        achieved = fpt * trans_per_step / roll_avg_s / 1e12
        roof = fp32_roofline(achieved, peaks, clocks, torch.cuda.get_device_properties(dev).multi_processor_count)
        # MLPs of at most two 64-unit hidden layers run on the row kernel, wider ones tiled
        small = max(max(w.shape) for w in wl.g_T.W) <= 64 and len(wl.g_T.W) == 3
        roof["kernel"] = "rollout_rows_kernel" if small else "rollout_simt_kernel"

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {0: "f32", 1: "bf16", 2: "e4m3 hidden layers, bf16 first/last"}[wl.prec],
            "data": "synthetic (seeded inputs, random-init weights)",
            "config": dict(workload_config(wl, args), parallelism=f"replicas x{world}"),
            "rollout_ms": statistics.median(roll_ms), "belief_update_ms": statistics.median(
                [e[0].elapsed_time(e[1]) for e in ev]),
            "roofline": roof,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            # BF16: weight pack, fused-output pack, tensor-core proposal, resampling (belief update); weight
            # pack, fused-output pack, rollout, reduce + argmax (rollout); backup. FP32: proposal, resampling,
            # rollout, reduce + argmax, backup. Resampling: one launch up to 2048 particles, four above.
            # FP8: one channel-scale launch more in each of the two packs
            "gpu_launches": ({0: 5, 1: 9, 2: 11}[wl.prec] + (1 if N <= 2048 else 4)) * args.steps,
            "clocks": clocks}
    J8 = None
    if wl.prec == 1 and rank == 0 and not args.no_forms:
        line["forms"] = {}
        if args.fp32_seqs > 0:
            f32 = fp32_form(V, wl, args.fp32_seqs, planner, p_new, stream)
            nsm = torch.cuda.get_device_properties(dev).multi_processor_count
            f32["roofline"] = fp32_roofline(fpt * f32["value"] / 1e12, peaks, None, nsm)
            line["forms"]["fp32_cuda_cores"] = f32
        fp8_peak = measure_fp8_peak()
        line["peaks_this_run"] = {"e4m3_tflops_burst": fp8_peak,
                                  "how": "torch._scaled_mm e4m3 x e4m3 -> bf16, 8192^3, best of 10 (CUDA events)"}
        line["forms"]["fp8_e4m3"], J8 = fp8_form(V, wl, planner, p_new, stream, peaks, fp8_peak)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the device's resampled particles and J of this exact step, against FP64
        V.voila_belief_update(g, lik, particles, None, action, obs, wl.d_omega, wl.lam, wl.seed, 1, planner, p_new,
                              None, None, None, None, ws_b)
        V.voila_rollout(g, R, p_new, None, actions, wl.d_omega, wl.gamma, wl.seed, planner, J, None, best, ws_r)
        torch.cuda.synchronize()
        cb, Jo, bres = cpu_baseline(wl, args.cpu_seqs, p_new.cpu().double().numpy())
        cb["one_core"] = one_core_oracle(wl, p_new.cpu().double().numpy())
        line["cpu_baseline"] = cb
        Jd = J[: args.cpu_seqs].cpu().numpy()
        if J8 is not None:
            line["forms"]["fp8_e4m3"]["err_vs_fp64"] = float(
                np.max(np.abs(J8[: args.cpu_seqs] - Jo)) / np.max(np.abs(Jo)))
        line["err_vs_fp64"] = {"J_normwise": float(np.max(np.abs(Jd - Jo)) / np.max(np.abs(Jo))),
                               "sample": f"J of {args.cpu_seqs} of {wl.K} sequences (all particles) vs the FP64 oracle "
                                         "from the same resampled particles",
                               "tolerance": {0: 1e-5, 1: 2e-2, 2: 6e-2}[wl.prec]}
        # belief-update weights of the device forms against the FP64 oracle's (same inputs)
        ell_lam = wl.lam / max(float(np.max(np.abs(bres.ell))), 1e-300)
        w_dev, ms_dev = device_belief_weights(V, g, V.DeviceMLP.from_spec(wl.ell), wl)
        line["err_vs_fp64"]["belief_logw_maxabs"] = logw_err(w_dev, bres.w)
        line["err_vs_fp64"]["belief_sample"] = (f"max |log w - log w*| over the {wl.N} particles' weights "
                                                f"(lambda / max|l*| = {ell_lam:.3g})")
        # and at a low temperature, where the weights are far from flat: lambda = the
        # spread of the oracle's likelihoods over the particles, so that the tempered
        # log-weights spread by about one (ESS well below N)
        lam_low = max(float(np.std(bres.ell)), 1e-6)
        bres_low = oracle_belief(wl, lam_low)
        w_low, _ = device_belief_weights(V, g, V.DeviceMLP.from_spec(wl.ell), wl, lam=lam_low)
        line["err_vs_fp64"]["belief_low_temperature"] = {
            "lambda": lam_low, "logw_maxabs": logw_err(w_low, bres_low.w), "ess_over_N": bres_low.ess / wl.N,
            "sample": "max |log w - log w*| over the weights above 1e-9, same inputs as belief_logw_maxabs"}
        if wl.prec == 1 and "forms" in line and "fp8_e4m3" in line["forms"]:
            mk8 = lambda spec: V.DeviceMLP([torch.from_numpy(x) for x in spec.W],  # noqa: E731
                                           [torch.from_numpy(x) for x in spec.b], spec.act, V.FP8E4M3)
            w8, ms8 = device_belief_weights(V, mk8(wl.g_T), mk8(wl.ell), wl)
            line["forms"]["fp8_e4m3"]["belief_update_ms"] = ms8
            line["forms"]["fp8_e4m3"]["belief_logw_err_vs_fp64"] = logw_err(w8, bres.w)
    if rank == 0 and world == 1 and wl.prec == 1 and not args.no_configs:
        line["configs"] = config_records(args, rank, world, local,
                                         (line.get("peaks_this_run") or {}).get("e4m3_tflops_burst"))
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
