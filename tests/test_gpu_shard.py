"""voila_rollout_shard: a rollout split by sequences or by particles gives the
unsharded call's results (Sec. 2.2: the simulations are independent).

Split by sequences: J, G and best_k of the whole problem, bit for bit. Split by
particles: every shard's G is the matching block of the whole G bit for bit,
and the shards' partial J added in rank order equal the whole J within FP64
rounding. Every form that takes a different kernel (FP32 CUDA cores, BF16 and
FP8 tensor cores, the one-tile kernel of the 512-wide generator), ragged shard
sizes, and the offsets checked against the
oracle's counters (a shard is not the whole problem's first block)."""
import numpy as np
import pytest
import torch

from oracle import voila_oracle as O
from paper_2606_19729_b300 import shard as S
from paper_2606_19729_b300 import workloads as WL
from tests.helpers import cuda, oracle_mlp, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def V():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_19729_b300 import voila
    return voila


def _setup(V, form):
    if form in ("bf16", "fp8"):
        wl = WL.mid_bf16(N=700, K=37, H=4, prec=WL.PREC_FP8 if form == "fp8" else WL.PREC_BF16)
        R = V.mlp_reward(V.DeviceMLP.from_spec(wl.reward_mlp))
        Ro = O.Reward(O.REWARD_MLP, mlp=oracle_mlp(wl.reward_mlp))
    elif form == "wide":  # the 4 x 512 generator: the one-tile kernel with half-layer pipelining
        wl = WL.sweep(N=300, K=21, H=3)
        R = V.goal_reward([1.0, 1.0])
        Ro = O.Reward(O.REWARD_GOAL, np.array([1.0, 1.0]))
    else:
        wl = WL.small_fp32(N=300, K=21, H=5)
        R = V.goal_reward(list(wl.goal))
        Ro = O.Reward(O.REWARD_GOAL, wl.goal)
    return wl, V.DeviceMLP.from_spec(wl.g_T), R, Ro


def _shard(V, wl, g, R, n0, n1, k0, k1):
    N, K = n1 - n0, k1 - k0
    J = torch.empty(K, dtype=torch.float64, device="cuda")
    G = torch.empty((K, N), dtype=torch.float64, device="cuda")
    best = torch.empty(1, dtype=torch.int32, device="cuda")
    ws = V.alloc_workspace(V.voila_rollout_workspace_size(g, R, N, K, wl.H))
    V.voila_rollout_shard(g, R, cuda(wl.particles[n0:n1]), None, n0, wl.N, cuda(wl.actions[k0:k1]), k0,
                          wl.d_omega, wl.gamma, wl.seed, 2, J, G, best, ws)
    assert V.workspace_status(ws) == V.OK
    return J, G, int(best.item())


@pytest.mark.parametrize("form", ["fp32", "bf16", "fp8", "wide"])
def test_sequence_split_is_bit_identical(V, form):
    wl, g, R, _ = _setup(V, form)
    Jf, Gf, bf = _shard(V, wl, g, R, 0, wl.N, 0, wl.K)
    for cuts in ([0, 17, wl.K], [0, 1, 12, wl.K]):
        parts = [_shard(V, wl, g, R, 0, wl.N, a, b) for a, b in zip(cuts[:-1], cuts[1:])]
        J = S.combine_sequence_shards([p[0] for p in parts])
        assert torch.equal(J, Jf)
        assert torch.equal(torch.cat([p[1] for p in parts], dim=0), Gf)
    assert bf == int(torch.argmax(Jf).item())


@pytest.mark.parametrize("form", ["fp32", "bf16", "fp8", "wide"])
def test_particle_split_matches(V, form):
    wl, g, R, Ro = _setup(V, form)
    Jf, Gf, _ = _shard(V, wl, g, R, 0, wl.N, 0, wl.K)
    cuts = [0, 129, wl.N - 3, wl.N]
    parts = [_shard(V, wl, g, R, a, b, 0, wl.K) for a, b in zip(cuts[:-1], cuts[1:])]
    assert torch.equal(torch.cat([p[1] for p in parts], dim=1), Gf)
    J = S.combine_particle_shards([p[0] for p in parts])
    np.testing.assert_allclose(J.cpu().numpy(), Jf.cpu().numpy(), rtol=1e-13, atol=1e-15)
    # a shard in the middle of both axes, against the oracle's counters
    n0, n1, k0, k1 = 129, 300 if wl.N > 300 else 250, 5, 16
    Js, Gs, _ = _shard(V, wl, g, R, n0, n1, k0, k1)
    Jo, Go = O.rollout(oracle_mlp(wl.g_T), Ro, wl.particles[n0:n1], wl.actions, wl.d_omega, wl.gamma, wl.seed,
                       planner=2, w=np.full(n1 - n0, 1.0 / wl.N), k_index=list(range(k0, k1)), n_offset=n0)
    tol = {"fp32": 1e-5, "bf16": 2e-2, "wide": 2e-2, "fp8": 6e-2}[form]
    assert rel_err(Gs.cpu().numpy(), Go) < tol
    assert rel_err(Js.cpu().numpy(), Jo) < tol


def test_shard_arguments_checked(V):
    wl, g, R, _ = _setup(V, "fp32")
    J = torch.empty(wl.K, dtype=torch.float64, device="cuda")
    ws = V.alloc_workspace(V.voila_rollout_workspace_size(g, R, 10, wl.K, wl.H))
    for n_off, n_total in [(-1, wl.N), (wl.N - 5, wl.N), (0, 0)]:
        with pytest.raises(V.VoilaError) as e:
            V.voila_rollout_shard(g, R, cuda(wl.particles[:10]), None, n_off, n_total, cuda(wl.actions), 0,
                                  wl.d_omega, wl.gamma, wl.seed, 0, J, None, None, ws)
        assert e.value.code == V.ERR_ARG
    with pytest.raises(V.VoilaError) as e:
        V.voila_rollout_shard(g, R, cuda(wl.particles[:10]), None, 0, wl.N, cuda(wl.actions), -2,
                              wl.d_omega, wl.gamma, wl.seed, 0, J, None, None, ws)
    assert e.value.code == V.ERR_ARG


def test_shard_zero_horizon_and_empty_blocks(V):
    wl, g, R, _ = _setup(V, "bf16")
    # an empty sequence block is a no-op; a zero horizon gives zero returns
    J = torch.full((1,), 7.0, dtype=torch.float64, device="cuda")
    ws = V.alloc_workspace(V.voila_rollout_workspace_size(g, R, wl.N, 1, wl.H))
    V.voila_rollout_shard(g, R, cuda(wl.particles), None, 0, wl.N, cuda(wl.actions[:0]), 3, wl.d_omega, wl.gamma,
                          wl.seed, 0, torch.empty(0, dtype=torch.float64, device="cuda"), None, None, ws)
    acts0 = torch.empty((2, 0, wl.d_a), dtype=torch.float32, device="cuda")
    J2 = torch.full((2,), 7.0, dtype=torch.float64, device="cuda")
    G2 = torch.full((2, 64), 7.0, dtype=torch.float64, device="cuda")
    V.voila_rollout_shard(g, R, cuda(wl.particles[64:128]), None, 64, wl.N, acts0, 5, wl.d_omega, wl.gamma,
                          wl.seed, 0, J2, G2, None, ws)
    torch.cuda.synchronize()
    assert torch.all(G2 == 0) and torch.all(J2 == 0)
    assert J.item() == 7.0
