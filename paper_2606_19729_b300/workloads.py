"""Seeded synthetic inputs for the rollout and belief-update workloads.

This module only draws inputs (weights, particles, action sequences) from
numpy's PCG64 generator and rounds them to the storage precision of a form.
It holds none of the method's arithmetic, so both the CUDA path and the CPU
oracle can be fed from it.

The paper's robot tasks (FloorPositioning, LeggedNavigation, TargetFinding,
Sec. 5.1) need simulators, datasets and trained weights that are not
available; these workloads stand in for them with random-init MLPs shaped
like the paper's models (Sec. 5.2 architecture paragraph) and the sizes of
the five workload configurations:

* ``small_fp32``  d_s=4, d_a=2, d_o=4, d_omega=4, MLPs 2x64 tanh, N=256, K=64, H=10
* ``mid_bf16``    d_s=8, d_a=2, d_o=6, d_omega=8, MLPs 3x256 SiLU, N=4096, K=1024, H=20
* ``sweep``       d_s=12, d_a=3, d_omega=16, generator 4x512 SiLU, N=16384, K=2048, H=25
* ``distill``     teacher 3x512 + 64-d step embedding, student 3x256, B=65536
* ``batched``     64 planners sharing the mid-size MLPs, uneven N, K, H
* ``infonce``     likelihood 16->256x3->1 on B=1024 tuples (B^2 pairs)
* ``pw``          progressive widening: 65536 simulations over 4096 action nodes
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Dict, List, Optional

import numpy as np

ACT_IDENTITY, ACT_TANH, ACT_SILU = 0, 1, 2
PREC_FP32, PREC_BF16, PREC_FP8 = 0, 1, 2


def round_bf16(x: np.ndarray) -> np.ndarray:
    """Round FP64 values to the nearest bfloat16 (ties to even), returned as FP64."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    u = x.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    u = (u + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def round_to(x: np.ndarray, prec: int) -> np.ndarray:
    """Storage rounding of a weight tensor for precision form `prec` (the FP8 form
    is handed BF16 weights and quantises them itself)."""
    if prec in (PREC_BF16, PREC_FP8):
        return round_bf16(x)
    return np.asarray(x, np.float32).astype(np.float64)


@dataclass
class MLPSpec:
    """Weights W[l] [out, in] and biases b[l] [out] as FP64 arrays, already rounded
    to what the device stores (FP32 or BF16 weights; FP32 biases)."""
    W: List[np.ndarray]
    b: List[np.ndarray]
    act: int
    prec: int = PREC_FP32

    @property
    def dims(self) -> List[int]:
        return [self.W[0].shape[1]] + [w.shape[0] for w in self.W]


def xavier_mlp(rng: np.random.Generator, dims: List[int], act: int, prec: int,
               bias_scale: float = 0.1) -> MLPSpec:
    """Xavier-uniform weights U(+-sqrt(6/(fan_in+fan_out))) (Glorot and Bengio, 2010).

    Biases are drawn U(+-bias_scale) rather than left at zero so that every
    bias path is exercised.
    """
    W, b = [], []
    for din, dout in zip(dims[:-1], dims[1:]):
        a = math.sqrt(6.0 / (din + dout))
        W.append(round_to(rng.uniform(-a, a, size=(dout, din)), prec))
        b.append(round_to(rng.uniform(-bias_scale, bias_scale, size=(dout,)), PREC_FP32))
    return MLPSpec(W, b, act, prec)


@dataclass
class Workload:
    name: str
    d_s: int
    d_a: int
    d_o: int
    d_omega: int
    N: int
    K: int
    H: int
    gamma: float
    seed: int
    prec: int
    g_T: MLPSpec
    g_Z: Optional[MLPSpec]
    ell: Optional[MLPSpec]
    reward_mlp: Optional[MLPSpec]
    goal: Optional[np.ndarray]
    particles: np.ndarray          # [N, d_s]
    actions: np.ndarray            # [K, H, d_a]
    lam: float = 1.0
    extra: Dict = field(default_factory=dict)


def small_fp32(seed: int = 0, N: int = 256, K: int = 64, H: int = 10) -> Workload:
    """Plain FP32 workload: 2x64 tanh MLPs, particles ~N(0, 0.5^2 I), actions U[-1,1]^2."""
    rng = np.random.default_rng(seed)
    d_s, d_a, d_o, d_w = 4, 2, 4, 4
    g_T = xavier_mlp(rng, [d_s + d_a + d_w, 64, 64, d_s], ACT_TANH, PREC_FP32)
    g_Z = xavier_mlp(rng, [d_s + d_a + d_w, 64, 64, d_o], ACT_TANH, PREC_FP32)
    ell = xavier_mlp(rng, [d_s + d_a + d_o, 64, 64, 1], ACT_TANH, PREC_FP32)
    rew = xavier_mlp(rng, [d_s + d_a, 64, 64, 1], ACT_TANH, PREC_FP32)
    particles = round_to(rng.normal(0.0, 0.5, size=(N, d_s)), PREC_FP32)
    actions = round_to(rng.uniform(-1.0, 1.0, size=(K, H, d_a)), PREC_FP32)
    return Workload("small_fp32", d_s, d_a, d_o, d_w, N, K, H, 0.95, seed, PREC_FP32,
                    g_T, g_Z, ell, rew, np.array([1.0, 1.0]), particles, actions)


def mid_bf16(seed: int = 1, N: int = 4096, K: int = 1024, H: int = 20,
             prec: int = PREC_BF16) -> Workload:
    """Mid-size planning step: 3x256 SiLU MLPs, particles ~N(0, I), actions U[-1,1]^2."""
    rng = np.random.default_rng(seed)
    d_s, d_a, d_o, d_w = 8, 2, 6, 8
    g_T = xavier_mlp(rng, [d_s + d_a + d_w, 256, 256, 256, d_s], ACT_SILU, prec)
    g_Z = xavier_mlp(rng, [d_s + d_a + d_w, 256, 256, 256, d_o], ACT_SILU, prec)
    ell = xavier_mlp(rng, [d_s + d_a + d_o, 256, 256, 256, 1], ACT_SILU, prec)
    rew = xavier_mlp(rng, [d_s + d_a, 256, 256, 256, 1], ACT_SILU, prec)
    particles = round_to(rng.normal(0.0, 1.0, size=(N, d_s)), PREC_FP32)
    actions = round_to(rng.uniform(-1.0, 1.0, size=(K, H, d_a)), PREC_FP32)
    return Workload("mid_bf16", d_s, d_a, d_o, d_w, N, K, H, 0.98, seed, prec,
                    g_T, g_Z, ell, rew, None, particles, actions)


def sweep(seed: int = 2, N: int = 16384, K: int = 2048, H: int = 25,
          prec: int = PREC_BF16) -> Workload:
    """Precision-sweep rollout: 4x512 SiLU generator, GOAL reward at (1, 1)."""
    rng = np.random.default_rng(seed)
    d_s, d_a, d_w = 12, 3, 16
    g_T = xavier_mlp(rng, [d_s + d_a + d_w, 512, 512, 512, 512, d_s], ACT_SILU, prec)
    particles = round_to(rng.normal(0.0, 1.0, size=(N, d_s)), PREC_FP32)
    actions = round_to(rng.uniform(-1.0, 1.0, size=(K, H, d_a)), PREC_FP32)
    return Workload("sweep", d_s, d_a, 0, d_w, N, K, H, 0.98, seed, prec,
                    g_T, None, None, None, np.array([1.0, 1.0]), particles, actions)


def true_state(rng_seed: int, d_s: int, scale: float) -> np.ndarray:
    """The synthetic episode's true state, drawn from the particle prior."""
    rng = np.random.default_rng(rng_seed + 1000)
    return round_to(rng.normal(0.0, scale, size=(d_s,)), PREC_FP32)



@dataclass
class DistillWorkload:
    """Distillation step (Eq. 3): teacher denoiser, student generator, one batch."""
    name: str
    d_s: int
    d_a: int
    d_x: int
    B: int
    T: int
    beta0: float
    beta1: float
    emb_dim: int
    seed: int
    teacher: MLPSpec
    student: MLPSpec               # FP32 master values (the forward copy rounds them)
    S: np.ndarray                  # [B, d_s] ~ N(0, I)
    A: np.ndarray                  # [B, d_a] ~ U[-1, 1]
    omega: np.ndarray              # [B, d_x] ~ N(0, I)
    lr: float = 1e-3
    adam_betas: tuple = (0.9, 0.999)
    adam_eps: float = 1e-8


def distill(seed: int = 3, B: int = 65536, teacher_prec: int = PREC_FP32) -> DistillWorkload:
    """Teacher 82->512x3->8 SiLU (input [s; a; x_t; 64-d step embedding]), 32 DDIM
    steps with linear beta 1e-4..0.02; student 18->256x3->8 SiLU with FP32
    master weights; s ~ N(0, I_8), a ~ U[-1, 1]^2, omega ~ N(0, I_8)."""
    rng = np.random.default_rng(seed)
    d_s, d_a, d_x, emb = 8, 2, 8, 64
    teacher = xavier_mlp(rng, [d_s + d_a + d_x + emb, 512, 512, 512, d_x], ACT_SILU, teacher_prec)
    student = xavier_mlp(rng, [d_s + d_a + d_x, 256, 256, 256, d_x], ACT_SILU, PREC_FP32)
    S = round_to(rng.normal(0.0, 1.0, size=(B, d_s)), PREC_FP32)
    A = round_to(rng.uniform(-1.0, 1.0, size=(B, d_a)), PREC_FP32)
    omega = round_to(rng.normal(0.0, 1.0, size=(B, d_x)), PREC_FP32)
    return DistillWorkload("distill", d_s, d_a, d_x, B, 32, 1e-4, 0.02, emb, seed, teacher, student, S, A, omega)



@dataclass
class InfoNCEWorkload:
    """Likelihood-model objective (Eq. 6) on B synthetic tuples (s'_i, a_i, o_i)."""
    name: str
    d_s: int
    d_a: int
    d_o: int
    B: int
    seed: int
    ell: MLPSpec
    S: np.ndarray                  # [B, d_s] ~ N(0, I)
    A: np.ndarray                  # [B, d_a] ~ U[-1, 1]
    O: np.ndarray                  # [B, d_o] = s'[:d_o] + 0.1 N(0, I)
    lr: float = 1e-3


def infonce(seed: int = 5, B: int = 1024, prec: int = PREC_BF16) -> InfoNCEWorkload:
    """Likelihood 16->256x3->1 SiLU (the planning shapes: s' 8, a 2, o 6); the
    observation of tuple i is the first 6 state coordinates plus N(0, 0.1^2)."""
    rng = np.random.default_rng(seed)
    d_s, d_a, d_o = 8, 2, 6
    ell = xavier_mlp(rng, [d_s + d_a + d_o, 256, 256, 256, 1], ACT_SILU, prec)
    S = round_to(rng.normal(0.0, 1.0, size=(B, d_s)), PREC_FP32)
    A = round_to(rng.uniform(-1.0, 1.0, size=(B, d_a)), PREC_FP32)
    O = round_to(S[:, :d_o] + rng.normal(0.0, 0.1, size=(B, d_o)), PREC_FP32)
    return InfoNCEWorkload("infonce", d_s, d_a, d_o, B, seed, ell, S, A, O)



@dataclass
class PWWorkload:
    """A batch of simulations at the action nodes of a belief tree (Sec. 4.3)."""
    name: str
    d_s: int
    d_a: int
    d_o: int
    d_omega: int
    M: int
    n_nodes: int
    C_max: int
    k_o: float
    alpha_o: float
    lam: float
    seed: int
    g_Z: MLPSpec
    ell: MLPSpec
    act: np.ndarray       # [n_nodes, d_a] ~ U[-1, 1]
    N0: np.ndarray        # [n_nodes] prior visit counts
    C0: np.ndarray        # [n_nodes] = min(C_max, ceil(k_o N0^alpha_o))
    obs0: np.ndarray      # [n_nodes, C_max, d_o]: existing branches ~ N(0, I), the rest 0
    node: np.ndarray      # [M] action node of each simulation
    s_next: np.ndarray    # [M, d_s] ~ N(0, I)


def pw(seed: int = 6, M: int = 65536, n_nodes: int = 4096, C_max: int = 32, prec: int = PREC_BF16,
       k_o: float = 2.1, alpha_o: float = 0.3) -> PWWorkload:
    """Planning shapes (s' 8, a 2, o 6, omega_Z 8; f_Z 18->256x3->6 and l 16->256x3->1
    SiLU). Node visits are skewed: node = floor(n_nodes u^2), so a few nodes hold
    many simulations; prior visit counts are uniform on 0..200."""
    rng = np.random.default_rng(seed)
    d_s, d_a, d_o, d_w = 8, 2, 6, 8
    g_Z = xavier_mlp(rng, [d_s + d_a + d_w, 256, 256, 256, d_o], ACT_SILU, prec)
    ell = xavier_mlp(rng, [d_s + d_a + d_o, 256, 256, 256, 1], ACT_SILU, prec)
    act = round_to(rng.uniform(-1.0, 1.0, size=(n_nodes, d_a)), PREC_FP32)
    N0 = rng.integers(0, 201, size=n_nodes).astype(np.int64)
    C0 = np.minimum(C_max, np.ceil(k_o * np.power(N0.astype(np.float64), alpha_o))).astype(np.int64)
    obs0 = np.zeros((n_nodes, C_max, d_o))
    for a in range(n_nodes):
        obs0[a, :C0[a]] = round_to(rng.normal(0.0, 1.0, size=(C0[a], d_o)), PREC_FP32)
    node = np.minimum(n_nodes - 1, np.floor(n_nodes * rng.uniform(0.0, 1.0, size=M) ** 2)).astype(np.int64)
    s_next = round_to(rng.normal(0.0, 1.0, size=(M, d_s)), PREC_FP32)
    return PWWorkload("pw", d_s, d_a, d_o, d_w, M, n_nodes, C_max, k_o, alpha_o, 1.0, seed, g_Z, ell, act, N0, C0,
                      obs0, node, s_next)


def batched_planners(seed: int = 4, P: int = 64, N_range=(512, 16384), K_range=(128, 1024), H_range=(5, 30)):
    """Per-planner (N_p, K_p, H_p): N log-uniform in N_range (default [512, 16384]),
    K uniform in K_range (default {128..1024}), H uniform in H_range (default {5..30})."""
    rng = np.random.default_rng(seed)
    N = np.rint(np.exp(rng.uniform(math.log(N_range[0]), math.log(N_range[1]), size=P))).astype(int)
    K = rng.integers(K_range[0], K_range[1] + 1, size=P)
    H = rng.integers(H_range[0], H_range[1] + 1, size=P)
    return N, K, H


def planner_inputs(seed: int, N: int, K: int, H: int, d_s: int = 8, d_a: int = 2):
    """Particles ~N(0, I) and actions U[-1,1]^d_a of one planner of the batched workload."""
    rng = np.random.default_rng(seed)
    particles = round_to(rng.normal(0.0, 1.0, size=(N, d_s)), PREC_FP32)
    actions = round_to(rng.uniform(-1.0, 1.0, size=(K, H, d_a)), PREC_FP32)
    return particles, actions
