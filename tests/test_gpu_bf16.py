"""Parity of the BF16 tensor-core rollout with the FP64 oracle (BF16 tolerance on
returns: 2e-2 normwise relative, ||J - J*||_inf / ||J*||_inf)."""
import numpy as np
import pytest
import torch

from oracle import voila_oracle as O
from paper_2606_19729_b300 import workloads as WL
from tests.helpers import cuda, oracle_mlp, rel_err

pytestmark = pytest.mark.gpu
TOL_BF16 = 2e-2


@pytest.fixture(scope="module")
def V():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_19729_b300 import voila
    return voila


def _device_rollout(V, g_spec, reward, particles, actions, d_omega, gamma, seed, planner=0, with_G=True):
    g = V.DeviceMLP.from_spec(g_spec)
    N, K, H = particles.shape[0], actions.shape[0], actions.shape[1]
    J = torch.empty(K, dtype=torch.float64, device="cuda")
    G = torch.empty((K, N), dtype=torch.float64, device="cuda") if with_G else None
    best = torch.empty(1, dtype=torch.int32, device="cuda")
    ws = V.alloc_workspace(V.voila_rollout_workspace_size(g, reward, N, K, H))
    V.voila_rollout(g, reward, cuda(particles), None, cuda(actions), d_omega, gamma, seed, planner, J, G, best, ws)
    assert V.workspace_status(ws) == V.OK
    return J.cpu().numpy(), (G.cpu().numpy() if with_G else None), int(best.item())


def _mid_case(V, N, K, H, goal=False, planner=0):
    wl = WL.mid_bf16(N=N, K=K, H=H)
    if goal:
        rdev, ror = V.goal_reward([1.0, 1.0]), O.Reward(O.REWARD_GOAL, np.array([1.0, 1.0]))
    else:
        rm = V.DeviceMLP.from_spec(wl.reward_mlp)
        rdev, ror = V.mlp_reward(rm), O.Reward(O.REWARD_MLP, mlp=oracle_mlp(wl.reward_mlp))
    J, G, best = _device_rollout(V, wl.g_T, rdev, wl.particles, wl.actions, wl.d_omega, wl.gamma, wl.seed,
                                 planner)
    Jo, Go = O.rollout(oracle_mlp(wl.g_T), ror, wl.particles, wl.actions, wl.d_omega, wl.gamma, wl.seed,
                       planner=planner)
    return J, G, best, Jo, Go


def test_bf16_rollout_mid_mlp_reward(V):
    J, G, best, Jo, Go = _mid_case(V, 256, 4, 3)
    assert rel_err(J, Jo) < TOL_BF16
    assert rel_err(G, Go) < TOL_BF16
    assert best == int(np.argmax(J))


@pytest.mark.parametrize("N,K,H", [(300, 3, 2), (5, 3, 1), (128, 1, 4), (129, 2, 2), (1, 1, 1)])
def test_bf16_rollout_ragged(V, N, K, H):
    J, G, _, Jo, Go = _mid_case(V, N, K, H, planner=3)
    assert rel_err(G, Go) < TOL_BF16
    assert rel_err(J, Jo) < TOL_BF16


def test_bf16_rollout_goal_reward(V):
    J, G, _, Jo, Go = _mid_case(V, 384, 2, 5, goal=True)
    assert rel_err(G, Go) < TOL_BF16
    np.testing.assert_allclose(J, Jo, rtol=TOL_BF16)


def test_bf16_rollout_zero_horizon(V):
    wl = WL.mid_bf16(N=64, K=2, H=0)
    rm = V.DeviceMLP.from_spec(wl.reward_mlp)
    J, G, _ = _device_rollout(V, wl.g_T, V.mlp_reward(rm), wl.particles, wl.actions, wl.d_omega, wl.gamma, 0)
    assert np.all(G == 0) and np.all(J == 0)


def test_bf16_rollout_sweep_dims(V):
    # state 12, action 3, latent 16 (the precision-sweep dimensions) with a 3x256 generator
    rng = np.random.default_rng(2)
    g = WL.xavier_mlp(rng, [31, 256, 256, 256, 12], WL.ACT_SILU, WL.PREC_BF16)
    particles = WL.round_to(rng.normal(size=(200, 12)), WL.PREC_FP32)
    actions = WL.round_to(rng.uniform(-1, 1, size=(3, 4, 3)), WL.PREC_FP32)
    J, G, _ = _device_rollout(V, g, V.goal_reward([1.0, 1.0]), particles, actions, 16, 0.98, 2)
    Jo, Go = O.rollout(oracle_mlp(g), O.Reward(O.REWARD_GOAL, np.array([1.0, 1.0])), particles, actions, 16,
                       0.98, 2)
    assert rel_err(G, Go) < TOL_BF16


def test_bf16_rollout_full_mid_size_sampled(V):
    """Full mid-size problem (4096 x 1024 x 20) in the bench's launch shape; the
    oracle evaluates a sample of sequences (rows are independent)."""
    wl = WL.mid_bf16()
    rm = V.DeviceMLP.from_spec(wl.reward_mlp)
    J, G, best = _device_rollout(V, wl.g_T, V.mlp_reward(rm), wl.particles, wl.actions, wl.d_omega, wl.gamma,
                                 wl.seed)
    ks = [0, 1, 517, 1023]
    Jo, Go = O.rollout(oracle_mlp(wl.g_T), O.Reward(O.REWARD_MLP, mlp=oracle_mlp(wl.reward_mlp)), wl.particles,
                       wl.actions, wl.d_omega, wl.gamma, wl.seed, k_index=ks)
    assert rel_err(J[ks], Jo) < TOL_BF16
    assert rel_err(G[ks], Go) < TOL_BF16
    assert np.all(np.isfinite(J))
    assert best == int(np.flatnonzero(J == J.max())[0])
