"""Pins of the FP64 oracle against things other than itself (CPU only).

Each test ties one oracle function to an independent source: another
implementation of the same published algorithm, a library routine, a closed
form, a mathematical invariant or brute force on tiny inputs.
"""
import json
import math
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest
import scipy.special
import scipy.stats
import torch

from oracle import voila_oracle as O
from paper_2606_19729_b300 import workloads as WL

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


# --------------------------------------------------------------------------
# Philox4x32-10 against Triton's independent Python implementation, run in
# Triton's CPU interpreter (a separate process so the interpreter switch
# cannot leak into other tests).
# --------------------------------------------------------------------------
_TRITON_SCRIPT = textwrap.dedent(
    """
    import os, sys, json
    os.environ["TRITON_INTERPRET"] = "1"
    import torch, triton, triton.language as tl

    @triton.jit
    def kern(out_ptr, c_ptr, seed, n, BLOCK: tl.constexpr):
        i = tl.arange(0, BLOCK)
        m = i < n
        c0 = tl.load(c_ptr + 4 * i + 0, mask=m).to(tl.uint32)
        c1 = tl.load(c_ptr + 4 * i + 1, mask=m).to(tl.uint32)
        c2 = tl.load(c_ptr + 4 * i + 2, mask=m).to(tl.uint32)
        c3 = tl.load(c_ptr + 4 * i + 3, mask=m).to(tl.uint32)
        a, b, c, d = tl.philox(seed, c0, c1, c2, c3)
        tl.store(out_ptr + 4 * i + 0, a.to(tl.int64), mask=m)
        tl.store(out_ptr + 4 * i + 1, b.to(tl.int64), mask=m)
        tl.store(out_ptr + 4 * i + 2, c.to(tl.int64), mask=m)
        tl.store(out_ptr + 4 * i + 3, d.to(tl.int64), mask=m)

    cases = json.loads(sys.stdin.read())
    res = []
    for seed, ctrs in cases:
        c = torch.tensor(ctrs, dtype=torch.int64).reshape(-1)
        out = torch.zeros_like(c)
        kern[(1,)](out, c, seed, len(ctrs), BLOCK=64)
        res.append([int(v) & 0xFFFFFFFF for v in out.tolist()])
    print(json.dumps(res))
    """
)


def test_philox_matches_independent_implementation():
    rng = np.random.default_rng(123)
    cases = []
    seeds = [0, 1, 0xFFFFFFFF, 0x123456789ABCDEF, 2 ** 64 - 1, int(rng.integers(0, 2 ** 63))]
    for seed in seeds:
        ctrs = rng.integers(0, 2 ** 32, size=(64, 4), dtype=np.uint64)
        ctrs[0] = [0, 0, 0, 0]
        ctrs[1] = [0xFFFFFFFF] * 4
        cases.append([seed, ctrs.tolist()])
    proc = subprocess.run([sys.executable, "-c", _TRITON_SCRIPT], input=json.dumps(cases),
                          capture_output=True, text=True, timeout=600)
    if proc.returncode != 0:
        pytest.skip("triton interpreter unavailable: " + proc.stderr[-300:])
    ref = json.loads(proc.stdout.strip().splitlines()[-1])
    for (seed, ctrs), want in zip(cases, ref):
        c = np.array(ctrs, dtype=np.uint64)
        k0, k1 = O.seed_key(seed)
        got = np.stack(O.philox4x32_10(c[:, 0], c[:, 1], c[:, 2], c[:, 3], k0, k1), axis=1)
        assert got.reshape(-1).tolist() == want


def test_philox_rounds_are_a_bijection_sample():
    # Distinct counters must give distinct outputs (Philox is a bijection of the counter space).
    n = np.arange(1 << 16, dtype=np.uint64)
    w = O.philox4x32_10(n, 0, 0, 0, 7, 9)
    packed = {(int(a), int(b), int(c), int(d)) for a, b, c, d in zip(*w)}
    assert len(packed) == n.size


def test_uniform24_range_and_exactness():
    x = np.array([0, 1, 511, 512, 0x7FFFFFFF, 0xFFFFFFFF], dtype=np.uint64)
    u = O.uniform24(x)
    assert u[0] == 2.0 ** -24 and u[1] == 2.0 ** -24 and u[2] == 2.0 ** -24
    assert u[3] == 3 * 2.0 ** -24
    assert u[-1] == 1.0 - 2.0 ** -24
    assert np.all(u.astype(np.float32).astype(np.float64) == u)   # exact in FP32
    assert np.all((u > 0) & (u < 1))


def test_uniform53_range():
    assert O.uniform53(0, 0) == 0.0
    assert O.uniform53(0xFFFFFFFF, 0xFFFFFFFF) == 1.0 - 2.0 ** -53
    assert O.uniform53(0, 1 << 11) == 2.0 ** -53


def test_box_muller_invariants():
    rng = np.random.default_rng(5)
    ua = rng.uniform(1e-9, 1.0, 1000)
    ub = rng.uniform(0.0, 1.0, 1000)
    z0, z1 = O.box_muller(ua, ub)
    np.testing.assert_allclose(z0 * z0 + z1 * z1, -2.0 * np.log(ua), rtol=1e-12, atol=1e-14)
    ang = np.mod(np.arctan2(z1, z0), 2 * math.pi)
    d = np.abs(ang - 2 * math.pi * ub)
    d = np.minimum(d, 2 * math.pi - d)
    assert np.max(d[np.abs(ua - 1) > 1e-6]) < 1e-9


def test_normals_are_standard_normal():
    z = O.normals(42, np.arange(1 << 14), 3, 5, O.STREAM_ROLLOUT_OMEGA, 0, 8)
    assert z.shape == (1 << 14, 8)
    flat = z.reshape(-1)
    assert abs(flat.mean()) < 0.01 and abs(flat.var() - 1.0) < 0.02
    assert scipy.stats.kstest(flat, "norm").pvalue > 1e-4
    # Columns from different Philox words and blocks are uncorrelated.
    c = np.corrcoef(z.T)
    assert np.max(np.abs(c - np.eye(8))) < 0.05
    # Different streams give different numbers for the same counter.
    z2 = O.normals(42, np.arange(16), 3, 5, O.STREAM_BELIEF_OMEGA, 0, 8)
    assert not np.allclose(z2, z[:16])


# --------------------------------------------------------------------------
# MLP forward/backward against torch (float64) and finite differences.
# --------------------------------------------------------------------------
def _torch_mlp(spec, x):
    h = torch.tensor(x, dtype=torch.float64)
    for l, (W, b) in enumerate(zip(spec.W, spec.b)):
        h = torch.nn.functional.linear(h, torch.tensor(W), torch.tensor(b))
        if l < len(spec.W) - 1:
            h = {O.ACT_TANH: torch.tanh, O.ACT_SILU: torch.nn.functional.silu,
                 O.ACT_IDENTITY: lambda v: v}[spec.act](h)
    return h


@pytest.mark.parametrize("act", [O.ACT_TANH, O.ACT_SILU, O.ACT_IDENTITY])
def test_mlp_forward_matches_torch(act):
    rng = np.random.default_rng(1)
    spec = WL.xavier_mlp(rng, [10, 64, 32, 4], act, WL.PREC_FP32)
    x = rng.normal(size=(37, 10)) * 3
    got = O.mlp_forward(O.MLP(spec.W, spec.b, act), x)
    want = _torch_mlp(spec, x).numpy()
    np.testing.assert_allclose(got, want, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("act", [O.ACT_TANH, O.ACT_SILU])
def test_mlp_backward_matches_autograd_and_fd(act):
    rng = np.random.default_rng(2)
    spec = WL.xavier_mlp(rng, [6, 16, 16, 3], act, WL.PREC_FP32)
    m = O.MLP(spec.W, spec.b, act)
    x = rng.normal(size=(16, 6))
    dY = rng.normal(size=(16, 3))
    dX, dW, db = O.mlp_backward(m, x, dY)
    # autograd
    xt = torch.tensor(x, requires_grad=True)
    Ws = [torch.tensor(W, requires_grad=True) for W in spec.W]
    bs = [torch.tensor(b, requires_grad=True) for b in spec.b]
    h = xt
    for l in range(3):
        h = torch.nn.functional.linear(h, Ws[l], bs[l])
        if l < 2:
            h = torch.tanh(h) if act == O.ACT_TANH else torch.nn.functional.silu(h)
    (h * torch.tensor(dY)).sum().backward()
    np.testing.assert_allclose(dX, xt.grad.numpy(), rtol=1e-12, atol=1e-12)
    for l in range(3):
        np.testing.assert_allclose(dW[l], Ws[l].grad.numpy(), rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(db[l], bs[l].grad.numpy(), rtol=1e-12, atol=1e-12)
    # central differences on a few weight entries, h = 1e-6
    def loss(mm):
        return float(np.sum(O.mlp_forward(mm, x) * dY))
    for l, (i, j) in [(0, (3, 2)), (1, (5, 7)), (2, (1, 9))]:
        Wp = [w.copy() for w in spec.W]
        Wm = [w.copy() for w in spec.W]
        Wp[l][i, j] += 1e-6
        Wm[l][i, j] -= 1e-6
        fd = (loss(O.MLP(Wp, spec.b, act)) - loss(O.MLP(Wm, spec.b, act))) / 2e-6
        assert abs(fd - dW[l][i, j]) < 1e-6 * max(1.0, abs(fd))


# --------------------------------------------------------------------------
# Rollout closed forms.
# --------------------------------------------------------------------------
def _linear_generator(d_s, d_a, d_w, sigma, two_layer=False):
    """s' = s + P a + sigma * omega, P = first d_a coordinates."""
    W = np.zeros((d_s, d_s + d_a + d_w))
    W[:, :d_s] = np.eye(d_s)
    for i in range(min(d_a, d_s)):
        W[i, d_s + i] = 1.0
    for i in range(min(d_w, d_s)):
        W[i, d_s + d_a + i] = sigma
    b = np.zeros(d_s)
    if two_layer:
        return O.MLP([W, np.eye(d_s)], [b, np.zeros(d_s)], O.ACT_IDENTITY)
    return O.MLP([W], [b], O.ACT_IDENTITY)


@pytest.mark.parametrize("sigma,two_layer", [(0.0, False), (0.0, True), (0.3, False), (0.3, True)])
def test_rollout_linear_closed_form(sigma, two_layer):
    rng = np.random.default_rng(3)
    N, K, H, d_s, d_a, d_w = 5, 3, 7, 4, 2, 4
    gamma, seed = 0.9, 11
    particles = rng.normal(size=(N, d_s))
    actions = rng.uniform(-1, 1, size=(K, H, d_a))
    goal = np.array([1.0, -0.5])
    g = _linear_generator(d_s, d_a, d_w, sigma, two_layer)
    J, G = O.rollout(g, O.Reward(O.REWARD_GOAL, goal), particles, actions, d_w, gamma, seed)
    # closed form: s_t = s_0 + P cumsum(a) + sigma cumsum(omega)
    G_ref = np.zeros((K, N))
    for k in range(K):
        for n in range(N):
            s = particles[n].copy()
            for t in range(H):
                s[:d_a] += actions[k, t]
                if sigma:
                    s[:d_w] += sigma * O.normals(seed, n, k, t, O.STREAM_ROLLOUT_OMEGA, 0, d_w)
                G_ref[k, n] += gamma ** t * -np.sum((s[:2] - goal) ** 2)
    np.testing.assert_allclose(G, G_ref, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(J, G_ref.mean(axis=1), rtol=1e-12, atol=1e-12)


def test_rollout_constant_reward_geometric_series():
    # Identity generator, zero actions: r_t is constant, G = r (1 - gamma^H) / (1 - gamma).
    N, K, H, d_s, d_a = 3, 2, 12, 2, 2
    g = _linear_generator(d_s, d_a, 0, 0.0)
    particles = np.array([[0.0, 0.0], [1.0, 1.0], [2.0, 0.0]])
    actions = np.zeros((K, H, d_a))
    goal = np.array([1.0, 1.0])
    gamma = 0.95
    J, G = O.rollout(g, O.Reward(O.REWARD_GOAL, goal), particles, actions, 0, gamma, 0)
    r = -np.array([2.0, 0.0, 2.0])
    np.testing.assert_allclose(G, np.tile(r * (1 - gamma ** H) / (1 - gamma), (K, 1)), rtol=1e-14)


def test_rollout_weights_and_subset():
    wl = WL.small_fp32(N=9, K=5, H=3)
    g = O.MLP(wl.g_T.W, wl.g_T.b, wl.g_T.act)
    R = O.Reward(O.REWARD_GOAL, wl.goal)
    w = np.random.default_rng(0).dirichlet(np.ones(9))
    J, G = O.rollout(g, R, wl.particles, wl.actions, wl.d_omega, wl.gamma, wl.seed, w=w)
    np.testing.assert_allclose(J, G @ w, rtol=1e-14)
    # evaluating a subset of sequences reproduces the same rows (noise keyed by global k)
    Js, Gs = O.rollout(g, R, wl.particles, wl.actions, wl.d_omega, wl.gamma, wl.seed, w=w, k_index=[4, 1])
    np.testing.assert_allclose(Gs, G[[4, 1]], rtol=1e-14)  # BLAS blocking may differ by an ulp


def test_best_sequence_lowest_index_on_ties():
    assert O.best_sequence(np.array([1.0, 3.0, 3.0, 2.0])) == 1
    assert O.best_sequence(np.array([-5.0])) == 0


# --------------------------------------------------------------------------
# Weights, log-sum-exp and systematic resampling.
# --------------------------------------------------------------------------
def test_log_normalise_matches_brute_force_and_scipy():
    rng = np.random.default_rng(4)
    for N in range(1, 9):
        lw = rng.normal(size=N) * 30
        w, logZ = O.log_normalise(lw)
        brute = math.log(math.fsum(math.exp(v) for v in lw))
        assert abs(logZ - brute) < 1e-12 * max(1, abs(brute))
        assert abs(logZ - scipy.special.logsumexp(lw)) < 1e-12 * max(1, abs(brute))
        np.testing.assert_allclose(w, [math.exp(v - brute) for v in lw], rtol=1e-12)
    with pytest.raises(O.DegenerateWeights):
        O.log_normalise(np.full(4, -np.inf))
    with pytest.raises(O.NonFiniteWeights):
        O.log_normalise(np.array([0.0, np.nan]))


def test_gaussian_likelihood_gives_analytic_weights():
    rng = np.random.default_rng(6)
    N, d_s, d_o, sigma = 200, 4, 3, 0.7
    s = rng.normal(size=(N, d_s))
    o = rng.normal(size=d_o)
    ell = O.likelihood(O.Likelihood(O.LIK_GAUSSIAN, sigma=sigma), s, np.zeros(2), o)
    w, _ = O.log_normalise(ell)
    dens = np.array([scipy.stats.multivariate_normal(mean=s[i, :d_o], cov=sigma ** 2 * np.eye(d_o)).pdf(o)
                     for i in range(N)])
    np.testing.assert_allclose(w, dens / dens.sum(), rtol=1e-10)


def test_quantised_weights_sum_to_one_and_prefix_is_order_free():
    rng = np.random.default_rng(7)
    for N in [1, 2, 7, 256, 4096, 16384]:
        w, _ = O.log_normalise(rng.normal(size=N) * 5)
        q = O.quantise_weights(w)
        assert abs(np.sum(q) - 1.0) <= N * 2.0 ** -52
        assert np.all(q * 2.0 ** 52 == np.rint(q * 2.0 ** 52))
        fwd = math.fsum(q)
        acc = 0.0
        for v in q[::-1]:
            acc += v
        pair = q.copy()
        while pair.size > 1:
            if pair.size % 2:
                pair = np.append(pair, 0.0)
            pair = pair[0::2] + pair[1::2]
        assert acc == fwd == pair[0] == np.cumsum(q)[-1]


def _brute_systematic(q, u0):
    N = len(q)
    C = []
    acc = 0.0
    for v in q:
        acc += v
        C.append(acc)
    out = []
    for j in range(N):
        p = ((u0 + j) * C[-1]) / N
        i = 0
        while i < N and not (C[i] > p):
            i += 1
        out.append(min(i, N - 1))
    return out


def test_systematic_resampling_brute_force_and_properties():
    rng = np.random.default_rng(8)
    for N in [1, 2, 3, 5, 8, 13]:
        for _ in range(20):
            w, _ = O.log_normalise(rng.normal(size=N) * 2)
            q = O.quantise_weights(w)
            u0 = float(rng.uniform())
            idx = O.systematic_resample(q, u0)
            assert idx.tolist() == _brute_systematic(q, u0)
            # each particle is drawn floor(N q_i) or ceil(N q_i) times
            counts = np.bincount(idx, minlength=N)
            assert np.all(counts >= np.floor(N * q - 1e-9)) and np.all(counts <= np.ceil(N * q + 1e-9))
            assert np.all(np.diff(idx) >= 0)
    # uniform weights -> identity; one-hot -> all equal
    for N in [4, 64, 1024]:
        q = O.quantise_weights(np.full(N, 1.0 / N))
        assert O.systematic_resample(q, 0.37).tolist() == list(range(N))
        oh = np.zeros(N)
        oh[N // 3] = 1.0
        assert set(O.systematic_resample(oh, 0.9).tolist()) == {N // 3}


def test_belief_update_identity_proposal_gaussian():
    # Identity proposal (no noise): weights are the analytic Gaussian posterior over particles.
    rng = np.random.default_rng(9)
    N, d_s, d_a, d_o = 64, 3, 2, 2
    g = _linear_generator(d_s, d_a, 0, 0.0)
    s = rng.normal(size=(N, d_s))
    a = np.zeros(d_a)
    o = np.array([0.2, -0.1])
    res = O.belief_update(g, O.Likelihood(O.LIK_GAUSSIAN, sigma=0.5), s, a, o, 0, 1.0, 5, 2)
    dens = np.exp(-np.sum((s[:, :d_o] - o) ** 2, axis=1) / (2 * 0.25))
    np.testing.assert_allclose(res.w, dens / dens.sum(), rtol=1e-9, atol=1e-15)
    np.testing.assert_array_equal(res.particles_out, s[res.idx])
    assert abs(res.ess - 1.0 / np.sum((dens / dens.sum()) ** 2)) < 1e-9 * res.ess
    # temperature lambda flattens: lambda -> large gives ESS -> N
    res2 = O.belief_update(g, O.Likelihood(O.LIK_GAUSSIAN, sigma=0.5), s, a, o, 0, 1e6, 5, 2)
    assert res2.ess > N * 0.999


# --------------------------------------------------------------------------
# Distillation pieces: schedule, embedding, DDIM sampler, loss gradient.
# --------------------------------------------------------------------------
def test_ddim_schedule_and_embedding():
    ab = O.ddim_schedule(32)
    assert ab.shape == (32,) and np.all(np.diff(ab) < 0) and 0 < ab[-1] < ab[0] < 1
    assert abs(ab[0] - (1 - 1e-4)) < 1e-15 and abs(ab[1] - (1 - 1e-4) * (1 - (1e-4 + (0.02 - 1e-4) / 31))) < 1e-15
    e = O.step_embedding(7.0, 64)
    np.testing.assert_allclose(e[:32] ** 2 + e[32:] ** 2, 1.0, rtol=1e-14)
    assert e[0] == math.sin(7.0) and e[32] == math.cos(7.0)
    z = O.step_embedding(0.0, 64)
    assert np.all(z[:32] == 0) and np.all(z[32:] == 1)


def test_ddim_exact_predictor_recovers_target():
    # A predictor that returns the exact v of a fixed clean sample x0*
    # (v = sqrt(ab) eps - sqrt(1-ab) x0*, eps implied by x_t) must land on x0*.
    rng = np.random.default_rng(11)
    ab = O.ddim_schedule(32)
    x_star = rng.normal(size=(5, 8))

    def v_exact(s, a, x, t):
        eps = (x - math.sqrt(ab[t]) * x_star) / math.sqrt(1 - ab[t])
        return math.sqrt(ab[t]) * eps - math.sqrt(1 - ab[t]) * x_star

    out = O.ddim_sample(v_exact, None, None, rng.normal(size=(5, 8)), ab)
    np.testing.assert_allclose(out, x_star, rtol=1e-9, atol=1e-9)


def test_ddim_zero_predictor_closed_form():
    ab = O.ddim_schedule(32)
    w = np.random.default_rng(12).normal(size=(4, 8))
    out = O.ddim_sample(lambda s, a, x, t: np.zeros_like(x), None, None, w, ab)
    f = 1.0
    for t in range(31, -1, -1):
        abp = ab[t - 1] if t > 0 else 1.0
        f *= math.sqrt(abp * ab[t]) + math.sqrt((1 - abp) * (1 - ab[t]))
    np.testing.assert_allclose(out, f * w, rtol=1e-12)


def test_distill_gradient_matches_finite_differences():
    rng = np.random.default_rng(13)
    spec = WL.xavier_mlp(rng, [18, 16, 16, 8], O.ACT_SILU, WL.PREC_FP32)
    m = O.MLP(spec.W, spec.b, O.ACT_SILU)
    s, a, w = rng.normal(size=(16, 8)), rng.uniform(-1, 1, size=(16, 2)), rng.normal(size=(16, 8))
    target = rng.normal(size=(16, 8))
    L, dW, db = O.distill_loss_and_grad(m, s, a, w, target)
    for l, (i, j) in [(0, (2, 5)), (2, (7, 3))]:
        Wp = [x.copy() for x in spec.W]
        Wm = [x.copy() for x in spec.W]
        Wp[l][i, j] += 1e-6
        Wm[l][i, j] -= 1e-6
        Lp, _, _ = O.distill_loss_and_grad(O.MLP(Wp, spec.b, O.ACT_SILU), s, a, w, target)
        Lm, _, _ = O.distill_loss_and_grad(O.MLP(Wm, spec.b, O.ACT_SILU), s, a, w, target)
        assert abs((Lp - Lm) / 2e-6 - dW[l][i, j]) < 1e-6 * max(1.0, abs(dW[l][i, j]))


# --------------------------------------------------------------------------
# Adam (Kingma and Ba, Algorithm 1): a closed form and an independent
# implementation (torch.optim.Adam in FP64).
# --------------------------------------------------------------------------
def test_adam_constant_gradient_closed_form():
    # with a constant gradient the bias-corrected moments are exactly g and g^2,
    # so every step moves p by -lr g / (|g| + eps)
    rng = np.random.default_rng(7)
    p0 = [rng.standard_normal((5, 3)), rng.standard_normal(5)]
    g = [rng.standard_normal((5, 3)), rng.standard_normal(5) * 1e-3]
    st = O.adam_init(p0)
    p = p0
    lr, eps = 1e-2, 1e-6
    for _ in range(7):
        p = O.adam_step(p, g, st, lr=lr, beta1=0.8, beta2=0.95, eps=eps)
    for pi, p0i, gi in zip(p, p0, g):
        np.testing.assert_allclose(pi, p0i - 7 * lr * gi / (np.abs(gi) + eps), rtol=0, atol=1e-12)


def test_adam_matches_torch_optim():
    rng = np.random.default_rng(8)
    shapes = [(4, 6), (4,), (2, 4), (2,)]
    p0 = [rng.standard_normal(s) for s in shapes]
    tp = [torch.tensor(x, dtype=torch.float64, requires_grad=True) for x in p0]
    opt = torch.optim.Adam(tp, lr=3e-3, betas=(0.9, 0.99), eps=1e-7)
    st = O.adam_init(p0)
    p = p0
    for _ in range(5):
        g = [rng.standard_normal(s) for s in shapes]
        for t, gi in zip(tp, g):
            t.grad = torch.tensor(gi)
        opt.step()
        p = O.adam_step(p, g, st, lr=3e-3, beta1=0.9, beta2=0.99, eps=1e-7)
    for pi, t in zip(p, tp):
        np.testing.assert_allclose(pi, t.detach().numpy(), rtol=1e-13, atol=1e-15)


def test_flat_params_layout():
    m = O.MLP([np.arange(6.0).reshape(3, 2), np.arange(3.0).reshape(1, 3)],
              [np.array([10.0, 11.0, 12.0]), np.array([20.0])], act=O.ACT_SILU)
    np.testing.assert_array_equal(O.flat_params(m), [0, 1, 2, 3, 4, 5, 10, 11, 12, 0, 1, 2, 20])


# --------------------------------------------------------------------------
# PORPP log-sum-exp backup: scipy's logsumexp, the eta -> infinity limit and a
# constant-preference closed form.
# --------------------------------------------------------------------------
def test_preference_backup_against_scipy_and_limits():
    rng = np.random.default_rng(13)
    J = rng.standard_normal(37) * 5.0
    lp = np.log(rng.dirichlet(np.ones(37)))
    for eta in (0.1, 1.0, 7.5):
        V, pi = O.preference_backup(J, eta, lp)
        assert math.isclose(V, scipy.special.logsumexp(eta * J + lp) / eta, rel_tol=1e-14)
        np.testing.assert_allclose(pi, scipy.special.softmax(eta * J + lp), rtol=1e-12)
        assert abs(pi.sum() - 1.0) < 1e-14
    # eta -> infinity: V -> max_k J_k and pi -> one-hot on the argmax
    V, pi = O.preference_backup(J, 1e6)
    assert abs(V - J.max()) < 1e-4 and pi[np.argmax(J)] > 0.999
    # equal preferences under the uniform reference policy: V = J, pi uniform
    V, pi = O.preference_backup(np.full(16, -3.25), 2.0)
    assert math.isclose(V, -3.25, rel_tol=1e-15) and np.allclose(pi, 1 / 16)
    # huge returns do not overflow (the maximum is subtracted first)
    V, _ = O.preference_backup(np.array([1e4, 1e4 - 1.0]), 1.0)
    assert math.isclose(V, 1e4 + math.log1p(math.exp(-1.0)) - math.log(2.0), rel_tol=1e-15)


# --------------------------------------------------------------------------
# InfoNCE (Eq. 6): brute-force pairs, scipy's logsumexp, the constant-logit
# closed form log B, and finite differences of the loss.
# --------------------------------------------------------------------------
def _tiny_ell(rng, d_in=7, h=5):
    return O.MLP([rng.standard_normal((h, d_in)) * 0.7, rng.standard_normal((1, h)) * 0.7],
                 [rng.standard_normal(h) * 0.1, rng.standard_normal(1) * 0.1], O.ACT_TANH)


def test_infonce_logits_brute_force():
    rng = np.random.default_rng(21)
    B, ds, da, do = 5, 3, 2, 2
    s, a, o = rng.standard_normal((B, ds)), rng.standard_normal((B, da)), rng.standard_normal((B, do))
    ell = _tiny_ell(rng)
    L = O.infonce_logits(ell, s, a, o)
    for i in range(B):
        for j in range(B):
            h = np.tanh(ell.W[0] @ np.concatenate([s[i], a[i], o[j]]) + ell.b[0])
            assert math.isclose(L[i, j], float((ell.W[1] @ h + ell.b[1])[0]), rel_tol=1e-13, abs_tol=1e-14)


def test_infonce_loss_scipy_and_constant_logits():
    rng = np.random.default_rng(22)
    L = rng.standard_normal((9, 9)) * 3
    loss, lse, G = O.infonce_loss(L)
    assert math.isclose(loss, -np.mean(np.diag(L) - scipy.special.logsumexp(L, axis=1)), rel_tol=1e-14)
    np.testing.assert_allclose(G, (scipy.special.softmax(L, axis=1) - np.eye(9)) / 9, atol=1e-15)
    np.testing.assert_allclose(G.sum(axis=1), 0.0, atol=1e-15)
    loss, _, _ = O.infonce_loss(np.full((12, 12), 4.5))
    assert math.isclose(loss, math.log(12.0), rel_tol=1e-15)


def test_infonce_weight_gradient_finite_differences():
    rng = np.random.default_rng(23)
    B, ds, da, do = 4, 3, 2, 2
    s, a, o = rng.standard_normal((B, ds)), rng.standard_normal((B, da)), rng.standard_normal((B, do))
    ell = _tiny_ell(rng)
    _, _, dW, db = O.infonce_loss_and_grad(ell, s, a, o)
    h = 1e-6
    for l in range(2):
        for idx in [(0, 0), (ell.W[l].shape[0] - 1, ell.W[l].shape[1] - 1)]:
            Wp = [w.copy() for w in ell.W]
            Wm = [w.copy() for w in ell.W]
            Wp[l][idx] += h
            Wm[l][idx] -= h
            fp = O.infonce_loss(O.infonce_logits(O.MLP(Wp, ell.b, ell.act), s, a, o))[0]
            fm = O.infonce_loss(O.infonce_logits(O.MLP(Wm, ell.b, ell.act), s, a, o))[0]
            assert math.isclose(dW[l][idx], (fp - fm) / (2 * h), rel_tol=1e-5, abs_tol=1e-9)
        bp = [v.copy() for v in ell.b]
        bm = [v.copy() for v in ell.b]
        bp[l][0] += h
        bm[l][0] -= h
        fp = O.infonce_loss(O.infonce_logits(O.MLP(ell.W, bp, ell.act), s, a, o))[0]
        fm = O.infonce_loss(O.infonce_logits(O.MLP(ell.W, bm, ell.act), s, a, o))[0]
        assert math.isclose(db[l][0], (fp - fm) / (2 * h), rel_tol=1e-5, abs_tol=1e-9)


# --------------------------------------------------------------------------
# Progressive widening (Sec. 4.3): branch counts against the closed form
# ceil(k n^alpha), batch-split invariance of the widening decisions, and the
# Gaussian-likelihood weights of a two-simulation group.
# --------------------------------------------------------------------------
def _pw_setup(n_nodes, C_max, d_s=4, d_a=2, d_o=3, seed=31):
    rng = np.random.default_rng(seed)
    tree = O.PWTree(rng.uniform(-1, 1, (n_nodes, d_a)), np.zeros(n_nodes, np.int64), np.zeros(n_nodes, np.int64),
                    np.zeros((n_nodes, C_max, d_o)))
    g_Z = O.MLP([rng.standard_normal((8, d_s + d_a + 2)) * 0.5, rng.standard_normal((d_o, 8)) * 0.5],
                [np.zeros(8), np.zeros(d_o)], O.ACT_TANH)
    return rng, tree, g_Z


def test_pw_branch_count_closed_form():
    # k = 1, alpha = 1/2: the threshold grows by at most 1 per visit, so after n
    # visits |C| = ceil(sqrt(n)) (capped), whatever the batching
    for C_max in (100, 7):
        rng, tree, g_Z = _pw_setup(1, C_max)
        M = 200
        s = rng.standard_normal((M, 4))
        res = O.progressive_widening(tree, np.zeros(M, np.int64), s, g_Z, O.Likelihood(O.LIK_GAUSSIAN, sigma=1.0),
                                     2, 1.0, 0.5, 1.0, seed=3, step=0)
        expect = [min(C_max, math.ceil(math.sqrt(n))) for n in range(1, M + 1)]
        assert tree.C[0] == expect[-1] and tree.N[0] == M
        grew = np.diff([0] + expect) > 0
        np.testing.assert_array_equal(res.widened, grew)
        assert np.all(res.branch < tree.C[0]) and np.all(res.branch >= 0)
    # alpha = 1, k = 1: every visit widens until the cap
    rng, tree, g_Z = _pw_setup(1, 5)
    res = O.progressive_widening(tree, np.zeros(9, np.int64), rng.standard_normal((9, 4)), g_Z,
                                 O.Likelihood(O.LIK_GAUSSIAN, sigma=1.0), 2, 1.0, 1.0, 1.0, seed=3, step=0)
    np.testing.assert_array_equal(res.widened, [True] * 5 + [False] * 4)
    np.testing.assert_array_equal(res.branch[:5], np.arange(5))


def test_pw_widening_is_batch_split_invariant():
    rng, tree_a, g_Z = _pw_setup(6, 16)
    _, tree_b, _ = _pw_setup(6, 16)
    M = 120
    node = rng.integers(0, 6, M)
    s = rng.standard_normal((M, 4))
    lik = O.Likelihood(O.LIK_GAUSSIAN, sigma=0.7)
    ra = O.progressive_widening(tree_a, node, s, g_Z, lik, 2, 1.3, 0.6, 1.0, seed=5, step=2)
    rb1 = O.progressive_widening(tree_b, node[:50], s[:50], g_Z, lik, 2, 1.3, 0.6, 1.0, seed=5, step=2)
    rb2 = O.progressive_widening(tree_b, node[50:], s[50:], g_Z, lik, 2, 1.3, 0.6, 1.0, seed=5, step=3)
    np.testing.assert_array_equal(ra.widened, np.concatenate([rb1.widened, rb2.widened]))
    np.testing.assert_array_equal(tree_a.N, tree_b.N)
    np.testing.assert_array_equal(tree_a.C, tree_b.C)
    np.testing.assert_array_equal(tree_a.N, np.bincount(node, minlength=6))


def test_pw_group_weights_gaussian_closed_form():
    # two simulations of one node, k = 0.9 and alpha small: the first widens
    # (0 < 0.9), the second joins branch 0 (1 >= 0.9 * 2^0.001); weights are the normalised Gaussian densities
    rng, tree, g_Z = _pw_setup(1, 4)
    s = np.array([[0.1, -0.2, 0.3, 0.0], [0.5, 0.4, -0.1, 0.2]])
    sigma, lam = 0.8, 1.25
    res = O.progressive_widening(tree, np.zeros(2, np.int64), s, g_Z, O.Likelihood(O.LIK_GAUSSIAN, sigma=sigma),
                                 2, 0.9, 1e-3, lam, seed=9, step=1)
    np.testing.assert_array_equal(res.widened, [True, False])
    np.testing.assert_array_equal(res.branch, [0, 0])
    o = tree.obs[0, 0]
    d2 = np.sum((o[None, :] - s[:, :3]) ** 2, axis=1)
    p = np.exp(-d2 / (2 * sigma ** 2 * lam))
    np.testing.assert_allclose(res.w, p / p.sum(), atol=2 ** -52)
    assert set(res.idx.tolist()) <= {0, 1}
    np.testing.assert_array_equal(res.s_out, s[res.idx])


def test_pw_join_choice_is_uniform():
    u = O.pw_branch_uniform(11, np.arange(40000), 0, 0)
    counts = np.bincount(np.floor(u * 5).astype(int), minlength=5)
    chi2 = np.sum((counts - 8000.0) ** 2 / 8000.0)
    assert chi2 < 20.5   # 4 degrees of freedom, p ~ 4e-4
