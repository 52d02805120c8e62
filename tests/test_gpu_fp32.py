"""Parity of the FP32 CUDA path with the FP64 oracle (FP32 tolerance 1e-5 relative)."""
import numpy as np
import pytest
import torch

from oracle import voila_oracle as O
from paper_2606_19729_b300 import workloads as WL
from tests.helpers import cuda, oracle_mlp, rel_err

pytestmark = pytest.mark.gpu
TOL_FP32 = 1e-5


@pytest.fixture(scope="module")
def V():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_19729_b300 import voila
    return voila


def test_philox_words_bit_exact(V):
    n = 1 << 20
    out = torch.empty(4 * n, dtype=torch.int32, device="cuda")
    seed, c1, c2, c3 = 0x0123456789ABCDEF, 7, 11, O.counter_word3(0, 3, 1)
    V.voila_philox_fill(seed, c1, c2, c3, out)
    got = out.cpu().numpy().view(np.uint32).reshape(n, 4)
    k0, k1 = O.seed_key(seed)
    want = np.stack(O.philox4x32_10(np.arange(n), c1, c2, c3, k0, k1), axis=1)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("dim", [1, 4, 8, 13, 16])
def test_normals_match(V, dim):
    n = 4096
    out = torch.empty((n, dim), dtype=torch.float32, device="cuda")
    V.voila_normal_fill(99, 5, 6, O.STREAM_ROLLOUT_OMEGA, 2, out)
    want = O.normals(99, np.arange(n), 5, 6, O.STREAM_ROLLOUT_OMEGA, 2, dim)
    got = out.cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(got, want, rtol=2e-6, atol=2e-6)


def _rollout_dev(V, wl, g_spec, reward, K=None, w=None, with_G=True, planner=0):
    g = V.DeviceMLP.from_spec(g_spec)
    acts = wl.actions if K is None else wl.actions[:K]
    N, Kk = wl.particles.shape[0], acts.shape[0]
    J = torch.empty(Kk, dtype=torch.float64, device="cuda")
    G = torch.empty((Kk, N), dtype=torch.float64, device="cuda") if with_G else None
    best = torch.empty(1, dtype=torch.int32, device="cuda")
    ws = V.alloc_workspace(V.voila_rollout_workspace_size(g, reward, N, Kk, acts.shape[1]))
    wt = None if w is None else cuda(w, torch.float64)
    V.voila_rollout(g, reward, cuda(wl.particles), wt, cuda(acts), wl.d_omega, wl.gamma, wl.seed, planner,
                    J, G, best, ws)
    torch.cuda.synchronize()
    return J.cpu().numpy(), (G.cpu().numpy() if with_G else None), int(best.item())


def test_rollout_small_fp32_goal(V):
    wl = WL.small_fp32()
    J, G, best = _rollout_dev(V, wl, wl.g_T, V.goal_reward(wl.goal))
    Jo, Go = O.rollout(oracle_mlp(wl.g_T), O.Reward(O.REWARD_GOAL, wl.goal), wl.particles, wl.actions,
                       wl.d_omega, wl.gamma, wl.seed)
    assert rel_err(G, Go) < TOL_FP32
    assert rel_err(J, Jo) < TOL_FP32
    np.testing.assert_allclose(J, Jo, rtol=TOL_FP32)   # GOAL returns are < 0: elementwise is defined
    assert best == O.best_sequence(J)


def test_rollout_small_fp32_mlp_reward_weighted(V):
    wl = WL.small_fp32(N=133, K=7, H=4)
    rew = V.DeviceMLP.from_spec(wl.reward_mlp)
    w = np.random.default_rng(3).dirichlet(np.ones(133))
    J, G, _ = _rollout_dev(V, wl, wl.g_T, V.mlp_reward(rew), w=w, planner=5)
    Jo, Go = O.rollout(oracle_mlp(wl.g_T), O.Reward(O.REWARD_MLP, mlp=oracle_mlp(wl.reward_mlp)),
                       wl.particles, wl.actions, wl.d_omega, wl.gamma, wl.seed, planner=5, w=w)
    assert rel_err(G, Go) < TOL_FP32
    assert rel_err(J, Jo) < TOL_FP32


@pytest.mark.parametrize("N,K,H", [(1, 1, 1), (31, 3, 2), (33, 2, 3), (127, 1, 5), (129, 2, 1), (5, 4, 0)])
def test_rollout_ragged_and_degenerate_sizes(V, N, K, H):
    wl = WL.small_fp32(N=N, K=K, H=H)
    J, G, _ = _rollout_dev(V, wl, wl.g_T, V.goal_reward(wl.goal))
    Jo, Go = O.rollout(oracle_mlp(wl.g_T), O.Reward(O.REWARD_GOAL, wl.goal), wl.particles, wl.actions,
                       wl.d_omega, wl.gamma, wl.seed)
    if H == 0:
        assert np.all(G == 0) and np.all(J == 0)
    else:
        assert rel_err(G, Go) < TOL_FP32


def test_rollout_without_G_output(V):
    wl = WL.small_fp32(N=64, K=8, H=3)
    J, _, _ = _rollout_dev(V, wl, wl.g_T, V.goal_reward(wl.goal), with_G=False)
    Jo, _ = O.rollout(oracle_mlp(wl.g_T), O.Reward(O.REWARD_GOAL, wl.goal), wl.particles, wl.actions,
                      wl.d_omega, wl.gamma, wl.seed)
    assert rel_err(J, Jo) < TOL_FP32


def test_rollout_empty_is_noop(V):
    wl = WL.small_fp32(N=4, K=2, H=2)
    g = V.DeviceMLP.from_spec(wl.g_T)
    J = torch.full((1,), 7.0, dtype=torch.float64, device="cuda")
    ws = V.alloc_workspace(1024)
    V.voila_rollout(g, V.goal_reward(wl.goal), cuda(wl.particles[:0]), None, cuda(wl.actions), wl.d_omega,
                    wl.gamma, 0, 0, J, None, None, ws)
    assert J.item() == 7.0


def _belief(V, wl, lik_dev, lik_or, N=None, logw=None, lam=1.0, step=3):
    g = V.DeviceMLP.from_spec(wl.g_T)
    parts = wl.particles if N is None else wl.particles[:N]
    N = parts.shape[0]
    a = wl.actions[0, 0]
    s_true = WL.true_state(wl.seed, wl.d_s, 0.5)
    s_next = O.generator_forward_seeded(oracle_mlp(wl.g_T), s_true[None], a[None], wl.d_omega, wl.seed,
                                        O.STREAM_TRUE_STATE, 0)
    o = O.sample_observation(oracle_mlp(wl.g_Z), s_next[0], a, wl.d_omega, wl.seed)
    out = torch.empty((N, wl.d_s), dtype=torch.float32, device="cuda")
    idx = torch.empty(N, dtype=torch.int32, device="cuda")
    w = torch.empty(N, dtype=torch.float64, device="cuda")
    lz = torch.empty(1, dtype=torch.float64, device="cuda")
    ess = torch.empty(1, dtype=torch.float64, device="cuda")
    ws = V.alloc_workspace(V.voila_belief_update_workspace_size(g, lik_dev, N))
    V.voila_belief_update(g, lik_dev, cuda(parts), None if logw is None else cuda(logw, torch.float64),
                          cuda(a), cuda(o.astype(np.float32)), wl.d_omega, lam, wl.seed, step, 0, out, idx, w, lz,
                          ess, ws)
    assert V.workspace_status(ws) == V.OK
    res = O.belief_update(oracle_mlp(wl.g_T), lik_or, parts, a, o.astype(np.float32).astype(np.float64),
                          wl.d_omega, lam, wl.seed, step, logw=logw)
    return (out.cpu().numpy(), idx.cpu().numpy(), w.cpu().numpy(), lz.item(), ess.item()), res


def _check_belief(got, res, tol):
    out, idx, w, lz, ess = got
    N = w.shape[0]
    assert abs(np.sum(w) - 1.0) <= N * 2.0 ** -52          # quantised weights sum to one
    assert np.all(w * 2.0 ** 52 == np.rint(w * 2.0 ** 52))
    big = res.w > 1e-6
    np.testing.assert_allclose(w[big], res.w[big], rtol=tol)
    assert np.max(np.abs(w - res.w)) < tol
    assert abs(lz - res.logZ) < tol * max(1.0, abs(res.logZ))
    assert abs(ess - res.ess) < tol * res.ess * 10
    # indices: bit-exact given the device's own weights and the same u0
    assert np.array_equal(idx, O.systematic_resample(w, res.u0))
    # gather: every output row is the proposal of its index (proposals match the oracle)
    np.testing.assert_allclose(out, res.s_prop[idx], rtol=tol, atol=tol)


def test_belief_update_small_fp32_mlp(V):
    wl = WL.small_fp32()
    ell = V.DeviceMLP.from_spec(wl.ell)
    got, res = _belief(V, wl, V.mlp_likelihood(ell), O.Likelihood(O.LIK_MLP, mlp=oracle_mlp(wl.ell)))
    _check_belief(got, res, TOL_FP32)


@pytest.mark.parametrize("N", [1, 2, 255, 257, 1000])
def test_belief_update_gaussian_ragged(V, N):
    wl = WL.small_fp32(N=1000)
    got, res = _belief(V, wl, V.gaussian_likelihood(0.3), O.Likelihood(O.LIK_GAUSSIAN, sigma=0.3), N=N,
                       lam=1.25)
    _check_belief(got, res, TOL_FP32)


def test_belief_update_with_prior_logw(V):
    wl = WL.small_fp32()
    logw = np.log(np.random.default_rng(1).dirichlet(np.ones(256)))
    got, res = _belief(V, wl, V.gaussian_likelihood(0.5), O.Likelihood(O.LIK_GAUSSIAN, sigma=0.5), logw=logw)
    _check_belief(got, res, TOL_FP32)


@pytest.mark.parametrize("N", [2048, 2049, 4096, 16385, 70001, 262144])
def test_belief_update_many_cta_resampling(V, N):
    # above 2048 particles the resampling runs in CTAs of 4096 particles
    # (segment partials combined in order, segment-local exact prefix sums)
    # and one search-and-gather thread per output; 262144 is the largest N
    # the call takes
    wl = WL.small_fp32(N=N)
    logw = np.random.default_rng(N).normal(0.0, 1.0, size=N)
    got, res = _belief(V, wl, V.gaussian_likelihood(0.3), O.Likelihood(O.LIK_GAUSSIAN, sigma=0.3), logw=logw,
                       step=5)
    _check_belief(got, res, TOL_FP32)


@pytest.mark.parametrize("N", [64, 20000])
def test_belief_update_degenerate_and_nonfinite_status(V, N):
    wl = WL.small_fp32(N=N)
    g = V.DeviceMLP.from_spec(wl.g_T)
    lik = V.gaussian_likelihood(0.5)
    out = torch.empty((N, wl.d_s), dtype=torch.float32, device="cuda")
    ws = V.alloc_workspace(V.voila_belief_update_workspace_size(g, lik, N))
    a = cuda(wl.actions[0, 0])
    o = cuda(np.zeros(wl.d_o))
    logw = torch.full((N,), -float("inf"), dtype=torch.float64, device="cuda")
    V.voila_belief_update(g, lik, cuda(wl.particles[:N]), logw, a, o, wl.d_omega, 1.0, 0, 0, 0, out, None, None,
                          None, None, ws)
    assert V.workspace_status(ws) == V.ERR_DEGENERATE
    logw[N - 3] = float("nan")
    V.voila_belief_update(g, lik, cuda(wl.particles[:N]), logw, a, o, wl.d_omega, 1.0, 0, 0, 0, out, None, None,
                          None, None, ws)
    assert V.workspace_status(ws) == V.ERR_NONFINITE
    logw.fill_(0.0)
    V.voila_belief_update(g, lik, cuda(wl.particles[:N]), logw, a, o, wl.d_omega, 1.0, 0, 0, 0, out, None, None,
                          None, None, ws)
    assert V.workspace_status(ws) == V.OK


def test_generator_fwd_plain_and_seeded(V):
    wl = WL.small_fp32()
    g = V.DeviceMLP.from_spec(wl.g_T)
    rng = np.random.default_rng(0)
    X = rng.normal(size=(301, g.dims[0])).astype(np.float32)
    Y = torch.empty((301, wl.d_s), dtype=torch.float32, device="cuda")
    V.voila_generator_fwd(g, cuda(X), Y)
    want = O.mlp_forward(oracle_mlp(wl.g_T), X.astype(np.float64))
    assert rel_err(Y.cpu().numpy(), want) < TOL_FP32
    S = wl.particles[:77]
    A = rng.uniform(-1, 1, size=(77, wl.d_a)).astype(np.float32)
    Y2 = torch.empty((77, wl.d_s), dtype=torch.float32, device="cuda")
    V.voila_generator_fwd_seeded(g, cuda(S), cuda(A), wl.d_a, wl.d_omega, 5, O.STREAM_OBS_OMEGA, 9, 1, Y2)
    want2 = O.generator_forward_seeded(oracle_mlp(wl.g_T), S, A, wl.d_omega, 5, O.STREAM_OBS_OMEGA, 9, 1)
    assert rel_err(Y2.cpu().numpy(), want2) < TOL_FP32


def test_argument_errors_raise(V):
    wl = WL.small_fp32(N=8, K=2, H=2)
    g = V.DeviceMLP.from_spec(wl.g_T)
    J = torch.empty(2, dtype=torch.float64, device="cuda")
    ws = V.alloc_workspace(64)
    with pytest.raises(V.VoilaError) as e:
        V.voila_rollout(g, V.goal_reward(wl.goal), cuda(wl.particles), None, cuda(wl.actions), wl.d_omega,
                        wl.gamma, 0, 0, J, None, None, ws)
    assert e.value.code == V.ERR_WORKSPACE
    with pytest.raises(V.VoilaError) as e:   # d_omega inconsistent with the generator's input width
        V.voila_rollout(g, V.goal_reward(wl.goal), cuda(wl.particles), None, cuda(wl.actions), 3,
                        wl.gamma, 0, 0, J, None, None, ws)
    assert e.value.code == V.ERR_SHAPE


@pytest.mark.parametrize("mlp_reward", [False, True])
def test_row_kernel_group_sizes_give_the_same_bits(V, mlp_reward):
    # the small-MLP FP32 kernel takes 8 threads per row when a launch's rows fit
    # in one wave (here the two 40-sequence shards, 10,240 rows each) and 4
    # threads per row above (the whole 80-sequence problem, 20,480 rows); both
    # accumulate every layer in input order, so the returns agree bit for bit,
    # and both match the FP64 oracle
    wl = WL.small_fp32(N=256, K=80, H=6)
    g = V.DeviceMLP.from_spec(wl.g_T)
    if mlp_reward:
        R, Ro = V.mlp_reward(V.DeviceMLP.from_spec(wl.reward_mlp)), O.Reward(O.REWARD_MLP, mlp=oracle_mlp(wl.reward_mlp))
    else:
        R, Ro = V.goal_reward(wl.goal), O.Reward(O.REWARD_GOAL, wl.goal)
    P, A = cuda(wl.particles), cuda(wl.actions)
    N, K, H = 256, 80, 6
    J = torch.empty(K, dtype=torch.float64, device="cuda")
    G = torch.empty((K, N), dtype=torch.float64, device="cuda")
    ws = V.alloc_workspace(V.voila_rollout_workspace_size(g, R, N, K, H))
    V.voila_rollout(g, R, P, None, A, wl.d_omega, wl.gamma, wl.seed, 0, J, G, None, ws)
    Gs = torch.empty((K, N), dtype=torch.float64, device="cuda")
    Js = torch.empty(K, dtype=torch.float64, device="cuda")
    wss = V.alloc_workspace(V.voila_rollout_workspace_size(g, R, N, K // 2, H))
    for k0 in (0, K // 2):
        V.voila_rollout_shard(g, R, P, None, 0, N, A[k0:k0 + K // 2].contiguous(), k0, wl.d_omega, wl.gamma,
                              wl.seed, 0, Js[k0:k0 + K // 2], Gs[k0:k0 + K // 2], None, wss)
        assert V.workspace_status(wss) == V.OK
    assert V.workspace_status(ws) == V.OK
    assert torch.equal(G, Gs) and torch.equal(J, Js)
    Jo, Go = O.rollout(oracle_mlp(wl.g_T), Ro, wl.particles, wl.actions, wl.d_omega, wl.gamma, wl.seed)
    assert rel_err(G.cpu().numpy(), Go) < TOL_FP32
    assert rel_err(J.cpu().numpy(), Jo) < TOL_FP32
