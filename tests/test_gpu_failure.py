"""Device-side failure detection without a GPU fault: a bounded wait that
nothing completes gives up after its limit, records VOILA_ERR_TIMEOUT (and its
site) in the workspace status word and returns, and the context stays usable
(a tensor-core rollout right after matches the FP64 oracle)."""
import numpy as np
import pytest
import torch

from oracle import voila_oracle as O
from paper_2606_19729_b300 import workloads as WL
from tests.helpers import cuda, oracle_mlp, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def V():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_19729_b300 import voila
    return voila


@pytest.mark.parametrize("limit", [0, 2_000_000])
def test_bounded_wait_times_out_and_reports(V, limit):
    ws = V.alloc_workspace(256)
    V.voila_selftest_wait_timeout(ws, limit)  # 2e6 cycles: about 1 ms of SM clock
    assert V.workspace_status(ws) == V.ERR_TIMEOUT
    assert int(ws[4:8].view(torch.int32).item()) == 99  # the site the wait recorded


def test_context_usable_after_timeout(V):
    ws = V.alloc_workspace(256)
    V.voila_selftest_wait_timeout(ws, 1_000_000)
    assert V.workspace_status(ws) == V.ERR_TIMEOUT
    wl = WL.mid_bf16(N=256, K=3, H=2)
    g = V.DeviceMLP.from_spec(wl.g_T)
    rm = V.DeviceMLP.from_spec(wl.reward_mlp)
    R = V.mlp_reward(rm)
    J = torch.empty(3, dtype=torch.float64, device="cuda")
    wsr = V.alloc_workspace(V.voila_rollout_workspace_size(g, R, 256, 3, 2))
    V.voila_rollout(g, R, cuda(wl.particles), None, cuda(wl.actions), wl.d_omega, wl.gamma, wl.seed, 0, J, None,
                    None, wsr)
    assert V.workspace_status(wsr) == V.OK
    Jo, _ = O.rollout(oracle_mlp(wl.g_T), O.Reward(O.REWARD_MLP, mlp=oracle_mlp(wl.reward_mlp)), wl.particles,
                      wl.actions, wl.d_omega, wl.gamma, wl.seed)
    assert rel_err(J.cpu().numpy(), Jo) < 2e-2
