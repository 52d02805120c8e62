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


def _rollout_status(V, wl, g, R, parts, w, acts):
    N, K, H = parts.shape[0], acts.shape[0], acts.shape[1]
    J = torch.empty(K, dtype=torch.float64, device="cuda")
    G = torch.empty((K, N), dtype=torch.float64, device="cuda")
    ws = V.alloc_workspace(V.voila_rollout_workspace_size(g, R, N, K, H))
    V.voila_rollout(g, R, parts, w, acts, wl.d_omega, wl.gamma, wl.seed, 0, J, G, None, ws)
    return V.workspace_status(ws), J, G


@pytest.mark.parametrize("prec", [WL.PREC_BF16, WL.PREC_FP32])
def test_rollout_reports_nonfinite_values(V, prec):
    # a NaN or infinite particle weight, or a NaN particle, reaches J: the
    # reduction latches VOILA_ERR_NONFINITE; finite inputs in the same
    # workspace size give VOILA_OK (the status word is cleared by every call)
    wl = WL.mid_bf16(N=300, K=4, H=3, prec=prec)
    g = V.DeviceMLP.from_spec(wl.g_T)
    R = V.mlp_reward(V.DeviceMLP.from_spec(wl.reward_mlp))
    parts, acts = cuda(wl.particles), cuda(wl.actions)
    w = torch.full((300,), 1.0 / 300, dtype=torch.float64, device="cuda")
    st, J, _ = _rollout_status(V, wl, g, R, parts, w, acts)
    assert st == V.OK and bool(torch.isfinite(J).all())
    for bad in (float("nan"), float("inf")):
        wb = w.clone()
        wb[137] = bad
        st, J, G = _rollout_status(V, wl, g, R, parts, wb, acts)
        assert st == V.ERR_NONFINITE and not bool(torch.isfinite(J).any())
        assert bool(torch.isfinite(G).all())  # the returns themselves are finite
    pb = parts.clone()
    pb[5, 2] = float("nan")
    st, J, G = _rollout_status(V, wl, g, R, pb, None, acts)
    assert st == V.ERR_NONFINITE
    assert not bool(torch.isfinite(G[:, 5]).any()) and bool(torch.isfinite(G[:, 6:]).all())
    st, _, _ = _rollout_status(V, wl, g, R, parts, None, acts)
    assert st == V.OK


def test_batched_rollout_reports_nonfinite_weight(V):
    # one planner of three has a NaN weight: the call's status is
    # VOILA_ERR_NONFINITE, and the other planners' J are their single-call bits
    wl = WL.mid_bf16(N=8, K=1, H=1)
    g = V.DeviceMLP.from_spec(wl.g_T)
    R = V.mlp_reward(V.DeviceMLP.from_spec(wl.reward_mlp))
    items = []
    for i, (N, K, H) in enumerate([(200, 3, 2), (130, 2, 4), (64, 5, 1)]):
        parts, acts = WL.planner_inputs(300 + i, N, K, H)
        w = torch.full((N,), 1.0 / N, dtype=torch.float64, device="cuda")
        items.append({"particles": cuda(parts), "actions": cuda(acts), "w": w, "planner_id": 20 + i,
                      "J": torch.empty(K, dtype=torch.float64, device="cuda")})
    refs = []
    for it in items:
        K = it["actions"].shape[0]
        J = torch.empty(K, dtype=torch.float64, device="cuda")
        ws = V.alloc_workspace(V.voila_rollout_workspace_size(g, R, it["particles"].shape[0], K,
                                                              it["actions"].shape[1]))
        V.voila_rollout(g, R, it["particles"], it["w"], it["actions"], wl.d_omega, wl.gamma, wl.seed,
                        it["planner_id"], J, None, None, ws)
        assert V.workspace_status(ws) == V.OK
        refs.append(J)
    pl = V.make_planners(items)
    ws = V.alloc_workspace(V.voila_rollout_batched_workspace_size(g, R, pl))
    V.voila_rollout_batched(g, R, pl, wl.d_s, wl.d_a, wl.d_omega, wl.gamma, wl.seed, 0, ws)
    assert V.workspace_status(ws) == V.OK
    items[1]["w"][17] = float("nan")
    V.voila_rollout_batched(g, R, pl, wl.d_s, wl.d_a, wl.d_omega, wl.gamma, wl.seed, 0, ws)
    assert V.workspace_status(ws) == V.ERR_NONFINITE
    assert torch.isnan(items[1]["J"]).all()
    assert torch.equal(items[0]["J"], refs[0]) and torch.equal(items[2]["J"], refs[2])
