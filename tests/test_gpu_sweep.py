"""Precision-sweep workload (state 12, action 3, latent 16, 4x512 SiLU generator,
GOAL reward): BF16 and FP8 forms on 512-wide layers against the FP64 oracle."""
import numpy as np
import pytest
import torch

from oracle import voila_oracle as O
from paper_2606_19729_b300 import workloads as WL
from tests.helpers import cuda, oracle_mlp, rel_err

pytestmark = pytest.mark.gpu
TOL = {WL.PREC_BF16: 2e-2, WL.PREC_FP8: 6e-2}


@pytest.fixture(scope="module")
def V():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_19729_b300 import voila
    return voila


def _run(V, wl, ks=None):
    g = V.DeviceMLP.from_spec(wl.g_T)
    R = V.goal_reward(list(wl.goal))
    N, K, H = wl.N, wl.K, wl.H
    J = torch.empty(K, dtype=torch.float64, device="cuda")
    G = torch.empty((K, N), dtype=torch.float64, device="cuda")
    ws = V.alloc_workspace(V.voila_rollout_workspace_size(g, R, N, K, H))
    V.voila_rollout(g, R, cuda(wl.particles), None, cuda(wl.actions), wl.d_omega, wl.gamma, wl.seed, 0, J, G, None, ws)
    assert V.workspace_status(ws) == V.OK
    Jo, Go = O.rollout(oracle_mlp(wl.g_T), O.Reward(O.REWARD_GOAL, wl.goal), wl.particles, wl.actions,
                       wl.d_omega, wl.gamma, wl.seed, k_index=ks)
    J, G = J.cpu().numpy(), G.cpu().numpy()
    if ks is not None:
        J, G = J[ks], G[ks]
    return J, G, Jo, Go


@pytest.mark.parametrize("prec", [WL.PREC_BF16, WL.PREC_FP8])
@pytest.mark.parametrize("N,K,H", [(256, 3, 3), (300, 2, 2), (129, 1, 4)])
def test_sweep_small(V, prec, N, K, H):
    wl = WL.sweep(N=N, K=K, H=H, prec=prec)
    J, G, Jo, Go = _run(V, wl)
    assert rel_err(G, Go) < TOL[prec]
    np.testing.assert_allclose(J, Jo, rtol=TOL[prec])   # GOAL returns are negative


@pytest.mark.parametrize("prec", [WL.PREC_BF16, WL.PREC_FP8])
def test_sweep_full_size_sampled(V, prec):
    """16384 particles x 2048 sequences x H=25 in one launch; oracle on two sequences."""
    wl = WL.sweep(prec=prec)
    ks = [5, 2047]
    J, G, Jo, Go = _run(V, wl, ks=ks)
    assert rel_err(J, Jo) < TOL[prec]
    assert rel_err(G, Go) < TOL[prec]


@pytest.mark.parametrize("prec", [WL.PREC_BF16, WL.PREC_FP8])
def test_mixed_width_wide_generator(V, prec):
    # 31 -> 512 -> 256 -> 512 -> 12: a 256-wide layer between 512-wide ones runs
    # the wide kernel's other half-layer cases (one column group reading K = 512,
    # and K = 256 feeding two groups) against the oracle
    import dataclasses
    wl = WL.sweep(N=300, K=2, H=3, prec=prec)
    rng = np.random.default_rng(21)
    wl = dataclasses.replace(wl, g_T=WL.xavier_mlp(rng, [31, 512, 256, 512, 12], WL.ACT_SILU, prec))
    J, G, Jo, Go = _run(V, wl)
    assert rel_err(G, Go) < TOL[prec]
    np.testing.assert_allclose(J, Jo, rtol=TOL[prec])
