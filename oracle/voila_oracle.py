"""Plain FP64 CPU oracle for the VOiLA planning-loop hot path.

TEST INFRASTRUCTURE ONLY. This module is the checker that the CUDA path is
compared against. Only the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it;
the product library never does, and it shares no code with the CUDA sources.

What it computes (paper sections cited per function):

* Philox4x32-10 counter-based random numbers (Salmon, Moraes, Dror and Shaw,
  "Parallel Random Numbers: As Easy as 1, 2, 3", SC'11), uniforms and
  Box-Muller normals: the latent noise omega_T ~ N(0, I) of Eq. 2 and
  omega_Z of Eq. 5.
* The distilled feed-forward generator s' = f_T(s, a, omega_T) (Eq. 2), here
  an MLP y = act(x W^T + b) with a linear last layer (Sec. 4.2.1, Sec. 5.2
  architecture paragraph).
* The Monte-Carlo rollout: discounted return sum_t gamma^t R(., a_t)
  (Sec. 2.1 value definition) reduced per action sequence into the
  Monte-Carlo estimate of R(b, a) (Sec. 2.2, preference equation Eq. 1).
* The SIR particle-filter belief update (Sec. 3 last paragraph; belief
  operator of Sec. 2.1): proposals from f_T, weights exp(l(s', a, o)/lambda)
  (Sec. 4.2.3, last paragraph), normalisation, systematic resampling.

Readings taken where the paper is silent:
* the reward scores the post-transition state s_{t+1};
* resampling happens at every update (no ESS threshold) and is systematic;
* weights are quantised to multiples of 2^-52 before the prefix sum, so the
  prefix sum is exact in FP64 whatever the summation order;
* the counter layout of the random streams below.

Every floating-point step here is FP64; no blocking or fusion beyond a
library matmul per layer.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import numpy as np

# ---------------------------------------------------------------------------
# Philox4x32-10 (Salmon et al., SC'11, Sec. 4.2 / Table 2).
# ---------------------------------------------------------------------------
MASK32 = np.uint64(0xFFFFFFFF)
PHILOX_M0 = np.uint64(0xD2511F53)  # multiplier applied to counter word 0
PHILOX_M1 = np.uint64(0xCD9E8D57)  # multiplier applied to counter word 2
PHILOX_W0 = np.uint64(0x9E3779B9)  # Weyl increment of key word 0 (golden ratio)
PHILOX_W1 = np.uint64(0xBB67AE85)  # Weyl increment of key word 1 (sqrt(3)-1)
PHILOX_ROUNDS = 10

# Stream ids carried in the top four bits of counter word 3.
STREAM_ROLLOUT_OMEGA = 0   # omega_T(n, k, t) of a rollout
STREAM_BELIEF_OMEGA = 1    # omega_T(i, 0, step) of the belief-update proposal
STREAM_RESAMPLE = 2        # the single uniform u0 of systematic resampling
STREAM_OBS_OMEGA = 3       # omega_Z(n, k, t) of the observation sampler
STREAM_TRUE_STATE = 5      # the simulated true state of a synthetic episode


def philox4x32_10(c0, c1, c2, c3, k0: int, k1: int):
    """Philox4x32 with 10 rounds, vectorised over counter arrays.

    One round maps (c0, c1, c2, c3) with key (k0, k1) to
    (hi(M1*c2) ^ c1 ^ k0, lo(M1*c2), hi(M0*c0) ^ c3 ^ k1, lo(M0*c0)) and then
    bumps the key by the Weyl constants (SC'11, Sec. 4.2). Returns four
    uint32 arrays.
    """
    c0 = np.asarray(c0, dtype=np.uint64) & MASK32
    c1 = np.asarray(c1, dtype=np.uint64) & MASK32
    c2 = np.asarray(c2, dtype=np.uint64) & MASK32
    c3 = np.asarray(c3, dtype=np.uint64) & MASK32
    c0, c1, c2, c3 = np.broadcast_arrays(c0, c1, c2, c3)
    k0 = np.uint64(k0) & MASK32
    k1 = np.uint64(k1) & MASK32
    for _ in range(PHILOX_ROUNDS):
        p0 = PHILOX_M0 * c0          # < 2^64: exact in uint64
        p1 = PHILOX_M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK32
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
        k0 = (k0 + PHILOX_W0) & MASK32
        k1 = (k1 + PHILOX_W1) & MASK32
    return (c0.astype(np.uint32), c1.astype(np.uint32),
            c2.astype(np.uint32), c3.astype(np.uint32))


def counter_word3(stream: int, planner: int, block: int) -> int:
    """Counter word 3 = stream << 28 | planner << 12 | block."""
    if not (0 <= stream < 16 and 0 <= planner < 65536 and 0 <= block < 4096):
        raise ValueError("stream/planner/block out of range")
    return (stream << 28) | (planner << 12) | block


def seed_key(seed: int):
    """Philox key = (low 32 bits, high 32 bits) of the 64-bit seed."""
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return seed & 0xFFFFFFFF, seed >> 32


def uniform24(x):
    """uint32 -> uniform in (0, 1): (2 * (x >> 9) + 1) * 2^-24.

    The top 23 bits pick one of 2^23 cell midpoints; the value has at most 24
    significant bits, so it is exact in FP32 and FP64.
    """
    x = np.asarray(x, dtype=np.uint64)
    return ((x >> np.uint64(9)).astype(np.float64) * 2.0 + 1.0) * 2.0 ** -24


def uniform53(x0, x1):
    """Two uint32 words -> uniform in [0, 1) with 53 random bits."""
    x0 = np.asarray(x0, dtype=np.uint64)
    x1 = np.asarray(x1, dtype=np.uint64)
    m = (x0 << np.uint64(21)) | (x1 >> np.uint64(11))
    return m.astype(np.float64) * 2.0 ** -53


def box_muller(u_a, u_b):
    """Box-Muller (1958): (r cos 2 pi u_b, r sin 2 pi u_b), r = sqrt(-2 ln u_a)."""
    r = np.sqrt(-2.0 * np.log(u_a))
    th = 2.0 * math.pi * u_b
    return r * np.cos(th), r * np.sin(th)


def normals(seed: int, c0, c1, c2, stream: int, planner: int, dim: int):
    """dim standard normals per counter triple (c0, c1, c2).

    Block b (counter word 3 low bits) yields four uniforms u0..u3 and the
    normals (z0, z1) = BM(u0, u1), (z2, z3) = BM(u2, u3); blocks are
    concatenated and cut to dim. Output shape = broadcast(c0, c1, c2) + (dim,).
    """
    k0, k1 = seed_key(seed)
    c0, c1, c2 = np.broadcast_arrays(np.asarray(c0, dtype=np.uint64),
                                     np.asarray(c1, dtype=np.uint64),
                                     np.asarray(c2, dtype=np.uint64))
    cols = []
    for b in range((dim + 3) // 4):
        w0, w1, w2, w3 = philox4x32_10(c0, c1, c2, counter_word3(stream, planner, b), k0, k1)
        z0, z1 = box_muller(uniform24(w0), uniform24(w1))
        z2, z3 = box_muller(uniform24(w2), uniform24(w3))
        cols += [z0, z1, z2, z3]
    return np.stack(cols[:dim], axis=-1)


def resample_uniform(seed: int, step: int, planner: int) -> float:
    """The systematic-resampling offset u0 in [0, 1) of belief update `step`."""
    k0, k1 = seed_key(seed)
    w0, w1, _, _ = philox4x32_10(0, 0, step, counter_word3(STREAM_RESAMPLE, planner, 0), k0, k1)
    return float(uniform53(w0, w1))


# ---------------------------------------------------------------------------
# MLP forward (Eq. 2 generator form; Sec. 5.2 architectures).
# ---------------------------------------------------------------------------
ACT_IDENTITY, ACT_TANH, ACT_SILU = 0, 1, 2


@dataclass
class MLP:
    """Weights W[l] of shape [out, in], biases b[l] of shape [out], all FP64."""
    W: List[np.ndarray]
    b: List[np.ndarray]
    act: int = ACT_TANH

    @property
    def dims(self) -> List[int]:
        return [self.W[0].shape[1]] + [w.shape[0] for w in self.W]


def activation(h: np.ndarray, act: int) -> np.ndarray:
    if act == ACT_IDENTITY:
        return h
    if act == ACT_TANH:
        return np.tanh(h)
    if act == ACT_SILU:
        with np.errstate(over="ignore"):
            return h / (1.0 + np.exp(-h))
    raise ValueError(f"unknown activation {act}")


def mlp_forward(mlp: MLP, x: np.ndarray) -> np.ndarray:
    """y = L_last(act(... act(L_1 x))), L_l(h) = h W_l^T + b_l; last layer linear."""
    h = np.asarray(x, dtype=np.float64)
    n = len(mlp.W)
    for l in range(n):
        h = h @ np.asarray(mlp.W[l], np.float64).T + np.asarray(mlp.b[l], np.float64)
        if l < n - 1:
            h = activation(h, mlp.act)
    return h


def mlp_forward_saved(mlp: MLP, x: np.ndarray):
    """Forward that also returns the pre-activations z_l of every layer."""
    h = np.asarray(x, dtype=np.float64)
    zs = []
    n = len(mlp.W)
    for l in range(n):
        z = h @ mlp.W[l].T + mlp.b[l]
        zs.append(z)
        h = activation(z, mlp.act) if l < n - 1 else z
    return h, zs


def activation_grad(z: np.ndarray, act: int) -> np.ndarray:
    """d act(z) / dz."""
    if act == ACT_IDENTITY:
        return np.ones_like(z)
    if act == ACT_TANH:
        return 1.0 - np.tanh(z) ** 2
    if act == ACT_SILU:
        with np.errstate(over="ignore"):
            sg = 1.0 / (1.0 + np.exp(-z))
        return sg * (1.0 + z * (1.0 - sg))
    raise ValueError(act)


def mlp_backward(mlp: MLP, x: np.ndarray, dY: np.ndarray):
    """Chain rule through the MLP: returns dX, [dW_l], [db_l] for loss L with dL/dY = dY."""
    x = np.asarray(x, np.float64)
    _, zs = mlp_forward_saved(mlp, x)
    n = len(mlp.W)
    inputs = [x] + [activation(z, mlp.act) for z in zs[:-1]]
    dW = [None] * n
    db = [None] * n
    g = np.asarray(dY, np.float64)
    for l in reversed(range(n)):
        if l < n - 1:
            g = g * activation_grad(zs[l], mlp.act)
        dW[l] = g.T @ inputs[l]
        db[l] = g.sum(axis=0)
        g = g @ mlp.W[l]
    return g, dW, db


# ---------------------------------------------------------------------------
# Reward and likelihood heads.
# ---------------------------------------------------------------------------
REWARD_GOAL, REWARD_MLP = 0, 1
LIK_MLP, LIK_GAUSSIAN = 0, 1


@dataclass
class Reward:
    """GOAL: r = -||s[:len(goal)] - goal||^2.  MLP: r = R([s; a]) (scalar output)."""
    kind: int = REWARD_GOAL
    goal: Optional[np.ndarray] = None
    mlp: Optional[MLP] = None


def reward(R: Reward, s_next: np.ndarray, a: np.ndarray) -> np.ndarray:
    """R(s_{t+1}, a_t) per row (reading: the post-transition state is scored)."""
    if R.kind == REWARD_GOAL:
        g = np.asarray(R.goal, np.float64)
        d = s_next[..., : g.shape[0]] - g
        return -np.sum(d * d, axis=-1)
    if R.kind == REWARD_MLP:
        a = np.broadcast_to(a, s_next.shape[:-1] + (a.shape[-1],))
        return mlp_forward(R.mlp, np.concatenate([s_next, a], axis=-1))[..., 0]
    raise ValueError(R.kind)


@dataclass
class Likelihood:
    """MLP: l = ell([s'; a; o]) (Sec. 4.2.3).  GAUSSIAN (test kind): l = -||o - s'[:d_o]||^2 / (2 sigma^2)."""
    kind: int = LIK_MLP
    mlp: Optional[MLP] = None
    sigma: float = 1.0


def likelihood(L: Likelihood, s_next: np.ndarray, a: np.ndarray, o: np.ndarray) -> np.ndarray:
    if L.kind == LIK_MLP:
        B = s_next.shape[0]
        x = np.concatenate([s_next, np.broadcast_to(a, (B, a.shape[-1])),
                            np.broadcast_to(o, (B, o.shape[-1]))], axis=-1)
        return mlp_forward(L.mlp, x)[:, 0]
    if L.kind == LIK_GAUSSIAN:
        d = o[None, :] - s_next[:, : o.shape[0]]
        return -np.sum(d * d, axis=-1) / (2.0 * L.sigma ** 2)
    raise ValueError(L.kind)


# ---------------------------------------------------------------------------
# Rollout: G_{n,k} = sum_{t<H} gamma^t R(s_{t+1}, a_{k,t}),  J_k = sum_n w_n G_{n,k}.
# ---------------------------------------------------------------------------
def rollout(g_T: MLP, R: Reward, particles: np.ndarray, actions: np.ndarray,
            d_omega: int, gamma: float, seed: int, planner: int = 0,
            w: Optional[np.ndarray] = None, k_index: Optional[Sequence[int]] = None,
            return_states: bool = False, n_offset: int = 0):
    """Monte-Carlo rollout of every particle under every action sequence.

    particles [N, d_s]; actions [K, H, d_a]. omega_T(n, k, t) comes from
    stream STREAM_ROLLOUT_OMEGA at counter (n, k, t). `k_index` restricts the
    evaluation to a subset of sequences (their global indices keep the noise
    counters of the full problem); `n_offset` is the global index of the first
    particle when `particles` is a block of a larger belief (particle n draws
    at counter n + n_offset). Returns J [K'] and G [K', N].
    """
    particles = np.asarray(particles, np.float64)
    actions = np.asarray(actions, np.float64)
    N, d_s = particles.shape
    K, H, d_a = actions.shape
    ks = np.arange(K) if k_index is None else np.asarray(k_index)
    Kp = ks.shape[0]
    s = np.broadcast_to(particles[None, :, :], (Kp, N, d_s)).copy()
    G = np.zeros((Kp, N))
    nn = np.arange(N)[None, :] + n_offset
    kk = ks[:, None]
    states = [s.copy()] if return_states else None
    for t in range(H):
        a_t = np.broadcast_to(actions[ks, t, :][:, None, :], (Kp, N, d_a))
        parts = [s, a_t]
        if d_omega > 0:
            parts.append(normals(seed, nn, kk, t, STREAM_ROLLOUT_OMEGA, planner, d_omega))
        x = np.concatenate(parts, axis=-1).reshape(Kp * N, -1)
        s = mlp_forward(g_T, x).reshape(Kp, N, d_s)
        r = reward(R, s, a_t)
        G += gamma ** t * r
        if return_states:
            states.append(s.copy())
    wv = np.full(N, 1.0 / N) if w is None else np.asarray(w, np.float64)
    J = G @ wv
    if return_states:
        return J, G, states
    return J, G


def best_sequence(J: np.ndarray) -> int:
    """argmax_k J_k, lowest index on ties."""
    return int(np.flatnonzero(J == np.max(J))[0])


# ---------------------------------------------------------------------------
# Belief update (SIR): propagate, weight, normalise, resample.
# ---------------------------------------------------------------------------
class DegenerateWeights(ValueError):
    """Every log-weight is -inf: the observation has zero likelihood under all particles."""


class NonFiniteWeights(ValueError):
    """A log-weight is NaN or +inf."""


def log_normalise(lw: np.ndarray):
    """Normalised weights by log-sum-exp: w_i = exp(lw_i - m) / sum_j exp(lw_j - m).

    Returns (w, logZ) with logZ = log sum_i exp(lw_i).
    """
    lw = np.asarray(lw, np.float64)
    if np.any(np.isnan(lw)) or np.any(lw == np.inf):
        raise NonFiniteWeights("log-weight is NaN or +inf")
    m = np.max(lw)
    if m == -np.inf:
        raise DegenerateWeights("all log-weights are -inf")
    e = np.exp(lw - m)
    Z = np.sum(e)
    return e / Z, m + math.log(Z)


def quantise_weights(w: np.ndarray) -> np.ndarray:
    """q_i = rn(w_i * 2^52) * 2^-52 (round half to even)."""
    return np.rint(np.asarray(w, np.float64) * 2.0 ** 52) * 2.0 ** -52


def systematic_resample(q: np.ndarray, u0: float) -> np.ndarray:
    """Systematic resampling (Kitagawa 1996; Arulampalam et al. 2002, Alg. 2).

    C = inclusive prefix sum of q; p_j = ((u0 + j) * C_{N-1}) / N;
    idx_j = min{i : C_i > p_j}, or N-1 when no such i exists.
    """
    q = np.asarray(q, np.float64)
    N = q.shape[0]
    C = np.cumsum(q)
    j = np.arange(N, dtype=np.float64)
    p = ((u0 + j) * C[-1]) / N
    idx = np.searchsorted(C, p, side="right")
    return np.minimum(idx, N - 1).astype(np.int32)


@dataclass
class BeliefResult:
    particles_out: np.ndarray
    idx: np.ndarray
    w: np.ndarray          # quantised normalised weights (pre-resample)
    logZ: float
    ess: float
    s_prop: np.ndarray     # propagated particles s'_i
    ell: np.ndarray        # likelihood values l_i
    u0: float


def belief_update(g_T: MLP, L: Likelihood, particles: np.ndarray, action: np.ndarray,
                  obs: np.ndarray, d_omega: int, lam: float, seed: int, step: int,
                  planner: int = 0, logw: Optional[np.ndarray] = None) -> BeliefResult:
    """One SIR step (Sec. 3): s'_i = f_T(s_i, a, omega_i); lw_i = logw_i + l_i / lambda;
    normalise by log-sum-exp; quantise; systematic resampling; gather."""
    particles = np.asarray(particles, np.float64)
    action = np.asarray(action, np.float64)
    obs = np.asarray(obs, np.float64)
    N = particles.shape[0]
    parts = [particles, np.broadcast_to(action, (N, action.shape[0]))]
    if d_omega > 0:
        parts.append(normals(seed, np.arange(N), 0, step, STREAM_BELIEF_OMEGA, planner, d_omega))
    s_prop = mlp_forward(g_T, np.concatenate(parts, axis=-1))
    ell = likelihood(L, s_prop, action, obs)
    lw = ell / lam + (0.0 if logw is None else np.asarray(logw, np.float64))
    w, logZ = log_normalise(lw)
    q = quantise_weights(w)
    ess = 1.0 / np.sum(q * q)
    u0 = resample_uniform(seed, step, planner)
    idx = systematic_resample(q, u0)
    return BeliefResult(s_prop[idx], idx, q, logZ, ess, s_prop, ell, u0)


# ---------------------------------------------------------------------------
# Observation drawn from the observation sampler (Eq. 5).
# ---------------------------------------------------------------------------
def sample_observation(g_Z: MLP, s_next: np.ndarray, action: np.ndarray, d_omega: int,
                       seed: int, n: int = 0, k: int = 0, t: int = 0, planner: int = 0):
    """z = f_Z(s', a, omega_Z), omega_Z from stream STREAM_OBS_OMEGA at counter (n, k, t)."""
    parts = [np.asarray(s_next, np.float64), np.asarray(action, np.float64)]
    if d_omega > 0:
        parts.append(normals(seed, n, k, t, STREAM_OBS_OMEGA, planner, d_omega))
    return mlp_forward(g_Z, np.concatenate(parts, axis=-1))


def generator_forward_seeded(g_T: MLP, s: np.ndarray, a: np.ndarray, d_omega: int, seed: int,
                             stream: int, step: int, planner: int = 0):
    """f_T(s_i, a_i, omega(i, 0, step)) for a batch: the seeded form of Eq. 2."""
    B = s.shape[0]
    parts = [np.asarray(s, np.float64), np.asarray(a, np.float64)]
    if d_omega > 0:
        parts.append(normals(seed, np.arange(B), 0, step, stream, planner, d_omega))
    return mlp_forward(g_T, np.concatenate(parts, axis=-1))


# ---------------------------------------------------------------------------
# Distillation (Sec. 4.2.1, Eq. 3): the teacher's deterministic ODE sampler
# (DDIM, eta = 0) on a v-prediction denoiser, and the student's MSE loss.
# Readings (the paper names a cosine schedule and v-prediction without the
# step count; the workload fixes 32 steps and a linear beta from 1e-4 to 0.02):
#   abar_t = prod_{s <= t} (1 - beta_s), t = 0 .. T-1, abar_{-1} = 1;
#   x_{T-1} = omega (the student's latent noise, so s_hat is a function of
#   (s, a, omega) as Eq. 3 needs); for t = T-1 .. 0, with v = v_T(s, a, x_t, t):
#     x0 = sqrt(abar_t) x_t - sqrt(1 - abar_t) v,
#     eps = sqrt(1 - abar_t) x_t + sqrt(abar_t) v,
#     x_{t-1} = sqrt(abar_{t-1}) x0 + sqrt(1 - abar_{t-1}) eps;
#   s_hat = x_{-1}. The step embedding is [sin(t f_i), cos(t f_i)],
#   f_i = 10000^(-i/(dim/2)), i < dim/2, appended to [s; a; x_t].
# ---------------------------------------------------------------------------
def step_embedding(t: float, dim: int = 64) -> np.ndarray:
    half = dim // 2
    f = 10000.0 ** (-np.arange(half, dtype=np.float64) / half)
    return np.concatenate([np.sin(t * f), np.cos(t * f)])


def ddim_schedule(T: int = 32, beta0: float = 1e-4, beta1: float = 0.02) -> np.ndarray:
    """abar_t for t = 0 .. T-1 (linear beta)."""
    beta = np.linspace(beta0, beta1, T)
    return np.cumprod(1.0 - beta)


def ddim_sample(v_pred, s: np.ndarray, a: np.ndarray, omega: np.ndarray, abar: np.ndarray) -> np.ndarray:
    """Deterministic DDIM from x = omega; v_pred(s, a, x, t) -> v (batched)."""
    x = np.asarray(omega, np.float64).copy()
    T = abar.shape[0]
    for t in range(T - 1, -1, -1):
        v = v_pred(s, a, x, t)
        ab = abar[t]
        ab_prev = abar[t - 1] if t > 0 else 1.0
        x0 = math.sqrt(ab) * x - math.sqrt(1.0 - ab) * v
        eps = math.sqrt(1.0 - ab) * x + math.sqrt(ab) * v
        x = math.sqrt(ab_prev) * x0 + math.sqrt(1.0 - ab_prev) * eps
    return x


def teacher_v(teacher: MLP, emb_dim: int = 64):
    """The denoising MLP v_T([s; a; x_t; emb(t)]) as a v-predictor."""
    def f(s, a, x, t):
        B = x.shape[0]
        e = np.broadcast_to(step_embedding(t, emb_dim), (B, emb_dim))
        return mlp_forward(teacher, np.concatenate([s, a, x, e], axis=-1))
    return f


def distill_loss_and_grad(student: MLP, s, a, omega, s_hat):
    """L = mean_i ||s_hat_i - f_T(s_i, a_i, omega_i)||^2 (Eq. 3) and its gradient."""
    x = np.concatenate([s, a, omega], axis=-1)
    y = mlp_forward(student, x)
    B = x.shape[0]
    r = y - s_hat
    L = float(np.sum(r * r) / B)
    dX, dW, db = mlp_backward(student, x, 2.0 * r / B)
    return L, dW, db


# ---------------------------------------------------------------------------
# Optimiser of the distillation step. The paper does not name one (reading:
# Adam, Kingma and Ba, ICLR 2015, Algorithm 1, on FP32-kept master weights).
# ---------------------------------------------------------------------------
@dataclass
class AdamState:
    m: List[np.ndarray]
    v: List[np.ndarray]
    t: int = 0


def adam_init(params: Sequence[np.ndarray]) -> AdamState:
    return AdamState([np.zeros_like(p, dtype=np.float64) for p in params],
                     [np.zeros_like(p, dtype=np.float64) for p in params], 0)


def adam_step(params: Sequence[np.ndarray], grads: Sequence[np.ndarray], state: AdamState,
              lr: float = 1e-3, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8) -> List[np.ndarray]:
    """Biased moment estimates, their bias corrections, and the update."""
    state.t += 1
    out = []
    for i, (p, g) in enumerate(zip(params, grads)):
        g = np.asarray(g, np.float64)
        state.m[i] = beta1 * state.m[i] + (1.0 - beta1) * g
        state.v[i] = beta2 * state.v[i] + (1.0 - beta2) * g * g
        m_hat = state.m[i] / (1.0 - beta1 ** state.t)
        v_hat = state.v[i] / (1.0 - beta2 ** state.t)
        out.append(np.asarray(p, np.float64) - lr * m_hat / (np.sqrt(v_hat) + eps))
    return out


def flat_params(m: MLP) -> np.ndarray:
    """[W_0, b_0, W_1, b_1, ...] flattened row-major."""
    return np.concatenate([x for l in range(len(m.W)) for x in (m.W[l].ravel(), m.b[l].ravel())])


def distill_targets(teacher: MLP, s, a, omega, T: int = 32, beta0: float = 1e-4, beta1: float = 0.02,
                    emb_dim: int = 64) -> np.ndarray:
    """s_hat' of Eq. 3: the teacher's DDIM sample from omega."""
    return ddim_sample(teacher_v(teacher, emb_dim), s, a, omega, ddim_schedule(T, beta0, beta1))


# ---------------------------------------------------------------------------
# PORPP preference backup over the root's action sequences (Sec. 2.2): with
# one level of preferences Psi_k = (1/eta) log pi_0(a_k | b) + J_k, the value is
# the log-sum-exp operator V = (1/eta) log sum_k exp(eta Psi_k) and the
# induced policy is pi(a_k | b) = exp(eta Psi_k) / sum_j exp(eta Psi_j).
# Reading: the reference policy pi_0 is uniform (1/K) unless given.
# ---------------------------------------------------------------------------
def preference_backup(J: np.ndarray, eta: float, log_pi0: Optional[np.ndarray] = None):
    """Returns (V, pi) in FP64; the sum runs after subtracting the maximum."""
    J = np.asarray(J, np.float64)
    K = J.shape[0]
    lp = np.full(K, -math.log(K)) if log_pi0 is None else np.asarray(log_pi0, np.float64)
    x = eta * J + lp                       # eta * Psi_k
    m = float(np.max(x))
    e = np.exp(x - m)
    Z = float(np.sum(e))
    return (m + math.log(Z)) / eta, e / Z


# ---------------------------------------------------------------------------
# InfoNCE likelihood objective (Eq. 6, Sec. 4.2.3): the likelihood model on
# all B x B combinations (s'_i, a_i, o_j), row log-sum-exp, the loss and its
# gradient with respect to the B x B logits and to the model's weights.
# ---------------------------------------------------------------------------
def infonce_pairs(s_next: np.ndarray, a: np.ndarray, o: np.ndarray) -> np.ndarray:
    """Rows [s'_i; a_i; o_j] in the order i * B + j."""
    B = s_next.shape[0]
    return np.concatenate([np.repeat(np.asarray(s_next, np.float64), B, axis=0),
                           np.repeat(np.asarray(a, np.float64), B, axis=0),
                           np.tile(np.asarray(o, np.float64), (B, 1))], axis=-1)


def infonce_logits(ell: MLP, s_next, a, o) -> np.ndarray:
    """L[i, j] = ell(s'_i, a_i, o_j)."""
    B = s_next.shape[0]
    return mlp_forward(ell, infonce_pairs(s_next, a, o))[:, 0].reshape(B, B)


def infonce_loss(L: np.ndarray):
    """Eq. 6 on a logit matrix: loss = -(1/B) sum_i (L_ii - lse_i), lse_i =
    log sum_j exp(L_ij); dloss/dL = (softmax_j(L_i.) - [i == j]) / B."""
    L = np.asarray(L, np.float64)
    B = L.shape[0]
    m = L.max(axis=1, keepdims=True)
    lse = m[:, 0] + np.log(np.sum(np.exp(L - m), axis=1))
    loss = -float(np.mean(np.diag(L) - lse))
    G = (np.exp(L - lse[:, None]) - np.eye(B)) / B
    return loss, lse, G


def infonce_loss_and_grad(ell: MLP, s_next, a, o):
    """Loss of Eq. 6 and its gradient with respect to the likelihood model's weights."""
    X = infonce_pairs(s_next, a, o)
    B = s_next.shape[0]
    L = mlp_forward(ell, X)[:, 0].reshape(B, B)
    loss, lse, G = infonce_loss(L)
    _, dW, db = mlp_backward(ell, X, G.reshape(-1, 1))
    return loss, lse, dW, db


# ---------------------------------------------------------------------------
# Vectorised progressive widening of the observation branches (Sec. 4.3):
# simulations are grouped by their parent action node; an action node a gets
# a new observation branch, sampled by f_Z (Eq. 5), when
#     |C(a)| < k_o N(a)^alpha_o,
# otherwise the simulation joins an existing branch. The successor states of
# each (action node, branch) are then weighted by exp(l(s', a, o_branch)/lambda)
# and resampled.
# Readings (the paper leaves these open):
# * within a node, simulations are taken in batch order; the m-th one of the
#   node sees the visit count N(a) + m + 1 and the branch count left by the
#   earlier ones; a branch cap C_max bounds |C(a)|;
# * the threshold k_o n^alpha_o is evaluated in FP64 as k_o * pow(n, alpha_o);
# * a simulation that does not widen joins branch floor(u |C(a)|), u the
#   24-bit uniform of word 0 of Philox at counter (m, step, 0, stream 6);
# * omega_Z of simulation m is drawn at counter (m, 0, step) of stream 3;
# * each (node, branch) group is resampled as the SIR step does (log-sum-exp
#   normalisation, 2^-52 quantisation, systematic resampling), with u0 from
#   counter (node, branch, step, stream 2 block 1).
# ---------------------------------------------------------------------------
STREAM_PW_BRANCH = 6


@dataclass
class PWTree:
    """The action-node tensors the widening reads and updates."""
    act: np.ndarray    # [n_nodes, d_a] action of each action node
    N: np.ndarray      # [n_nodes] visit counts
    C: np.ndarray      # [n_nodes] observation-branch counts
    obs: np.ndarray    # [n_nodes, C_max, d_o] branch observations


@dataclass
class PWResult:
    branch: np.ndarray     # [M] branch of each simulation
    widened: np.ndarray    # [M] bool: the simulation created its branch
    ell: np.ndarray        # [M] l(s'_m, a, o_branch)
    w: np.ndarray          # [M] quantised weight within its (node, branch) group
    idx: np.ndarray        # [M] simulation whose successor state fills slot m
    s_out: np.ndarray      # [M, d_s] resampled successor states


def pw_branch_uniform(seed: int, m, step: int, planner: int):
    k0, k1 = seed_key(seed)
    m = np.asarray(m, dtype=np.uint64)
    w0, _, _, _ = philox4x32_10(m, step, 0, counter_word3(STREAM_PW_BRANCH, planner, 0), k0, k1)
    return uniform24(w0)


def pw_group_uniform(seed: int, node: int, branch: int, step: int, planner: int) -> float:
    k0, k1 = seed_key(seed)
    w0, w1, _, _ = philox4x32_10(node, branch, step, counter_word3(STREAM_RESAMPLE, planner, 1), k0, k1)
    return float(uniform53(w0, w1))


def progressive_widening(tree: PWTree, node: np.ndarray, s_next: np.ndarray, g_Z: MLP, L: Likelihood,
                         d_omega: int, k_o: float, alpha_o: float, lam: float, seed: int, step: int,
                         planner: int = 0, sim_index: Optional[np.ndarray] = None) -> PWResult:
    """Updates `tree` in place (N, C, obs) and returns the per-simulation results.

    sim_index: the batch index of each given simulation (default 0 .. M-1), so
    that the simulations of a subset of nodes can be replayed with their own
    random counters; idx holds batch indices too.
    """
    node = np.asarray(node, np.int64)
    s_next = np.asarray(s_next, np.float64)
    M = node.shape[0]
    gid = np.arange(M) if sim_index is None else np.asarray(sim_index, np.int64)
    C_max = tree.obs.shape[1]
    branch = np.zeros(M, np.int64)
    widened = np.zeros(M, bool)
    for a in np.unique(node):
        ms = np.nonzero(node == a)[0]          # ascending simulation index
        C = int(tree.C[a])
        n0 = int(tree.N[a])
        for r, m in enumerate(ms):
            n = n0 + r + 1
            if C < C_max and C < k_o * math.pow(n, alpha_o):
                branch[m] = C
                widened[m] = True
                x = [s_next[m], tree.act[a]]
                if d_omega > 0:
                    x.append(np.reshape(normals(seed, gid[m], 0, step, STREAM_OBS_OMEGA, planner, d_omega), -1))
                tree.obs[a, C] = mlp_forward(g_Z, np.concatenate(x)[None, :])[0]
                C += 1
            else:
                u = float(pw_branch_uniform(seed, gid[m], step, planner))
                branch[m] = min(C - 1, int(math.floor(u * C)))
        tree.N[a] = n0 + len(ms)
        tree.C[a] = C
    ell = np.empty(M)
    for m in range(M):
        ell[m] = likelihood(L, s_next[m:m + 1], np.asarray(tree.act[node[m]], np.float64),
                            np.asarray(tree.obs[node[m], branch[m]], np.float64))[0]
    w = np.zeros(M)
    idx = np.zeros(M, np.int64)
    for key in sorted(set(zip(node.tolist(), branch.tolist()))):
        ms = np.nonzero((node == key[0]) & (branch == key[1]))[0]
        wg, _ = log_normalise(ell[ms] / lam)
        q = quantise_weights(wg)
        u0 = pw_group_uniform(seed, key[0], key[1], step, planner)
        w[ms] = q
        idx[ms] = ms[systematic_resample(q, u0)]
    return PWResult(branch, widened, ell, w, gid[idx], s_next[idx])
