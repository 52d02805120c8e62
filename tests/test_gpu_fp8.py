"""FP8 e4m3 form of the rollout (hidden layers E4M3 with per-channel scales,
first and last layers BF16) against the FP64 oracle: 6e-2 on returns."""
import numpy as np
import pytest
import torch

from oracle import voila_oracle as O
from paper_2606_19729_b300 import workloads as WL
from tests.helpers import cuda, oracle_mlp, rel_err

pytestmark = pytest.mark.gpu
TOL_FP8 = 6e-2


@pytest.fixture(scope="module")
def V():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_19729_b300 import voila
    return voila


def _run(V, wl, ks=None, goal=False):
    g = V.DeviceMLP.from_spec(wl.g_T)
    if goal:
        R, Ro = V.goal_reward([1.0, 1.0]), O.Reward(O.REWARD_GOAL, np.array([1.0, 1.0]))
    else:
        rm = V.DeviceMLP.from_spec(wl.reward_mlp)
        R, Ro = V.mlp_reward(rm), O.Reward(O.REWARD_MLP, mlp=oracle_mlp(wl.reward_mlp))
    N, K, H = wl.N, wl.K, wl.H
    J = torch.empty(K, dtype=torch.float64, device="cuda")
    G = torch.empty((K, N), dtype=torch.float64, device="cuda")
    ws = V.alloc_workspace(V.voila_rollout_workspace_size(g, R, N, K, H))
    V.voila_rollout(g, R, cuda(wl.particles), None, cuda(wl.actions), wl.d_omega, wl.gamma, wl.seed, 0, J, G, None, ws)
    assert V.workspace_status(ws) == V.OK
    Jo, Go = O.rollout(oracle_mlp(wl.g_T), Ro, wl.particles, wl.actions, wl.d_omega, wl.gamma, wl.seed, k_index=ks)
    J, G = J.cpu().numpy(), G.cpu().numpy()
    if ks is not None:
        J, G = J[ks], G[ks]
    return J, G, Jo, Go


@pytest.mark.parametrize("N,K,H", [(256, 4, 3), (300, 3, 2), (129, 2, 5)])
def test_fp8_rollout_small(V, N, K, H):
    wl = WL.mid_bf16(N=N, K=K, H=H, prec=WL.PREC_FP8)
    J, G, Jo, Go = _run(V, wl)
    assert rel_err(J, Jo) < TOL_FP8
    assert rel_err(G, Go) < TOL_FP8


def test_fp8_rollout_goal_reward(V):
    wl = WL.mid_bf16(N=256, K=2, H=4, prec=WL.PREC_FP8)
    J, G, Jo, Go = _run(V, wl, goal=True)
    assert rel_err(G, Go) < TOL_FP8


def test_fp8_rollout_full_mid_size_sampled(V):
    wl = WL.mid_bf16(prec=WL.PREC_FP8)
    ks = [0, 3, 700, 1023]
    J, G, Jo, Go = _run(V, wl, ks=ks)
    assert rel_err(J, Jo) < TOL_FP8
    assert rel_err(G, Go) < TOL_FP8


def test_fp8_form_takes_silu_mlps_only(V):
    # the E4M3 epilogues apply SiLU; an FP8 MLP with another activation is refused
    rng = np.random.default_rng(7)
    g = V.DeviceMLP.from_spec(WL.xavier_mlp(rng, [18, 256, 256, 256, 8], WL.ACT_TANH, WL.PREC_FP8))
    rm = V.DeviceMLP.from_spec(WL.xavier_mlp(rng, [10, 256, 256, 256, 1], WL.ACT_TANH, WL.PREC_FP8))
    R = V.mlp_reward(rm)
    parts = torch.zeros((16, 8), dtype=torch.float32, device="cuda")
    acts = torch.zeros((2, 3, 2), dtype=torch.float32, device="cuda")
    J = torch.empty(2, dtype=torch.float64, device="cuda")
    ws = V.alloc_workspace(V.voila_rollout_workspace_size(g, R, 16, 2, 3))
    with pytest.raises(V.VoilaError) as e:
        V.voila_rollout(g, R, parts, None, acts, 8, 0.98, 1, 0, J, None, None, ws)
    assert e.value.code == V.ERR_UNSUPPORTED
