"""Batched multi-planner rollout: one launch over planners with uneven N, K, H.

With the two-tile shape every planner's returns equal what voila_rollout
computes for it alone (the same rows, noise counters, arithmetic and reduction
order, so bit-identical) for every work order (static or the atomic queue) and
number of CTA pairs, inside a captured CUDA graph, and match the FP64 oracle;
the one-tile shape (reward output as an MMA) matches the oracle within the
BF16 tolerance and gives the same bits with and without the queue."""
import numpy as np
import pytest
import torch

from oracle import voila_oracle as O
from paper_2606_19729_b300 import workloads as WL
from tests.helpers import cuda, oracle_mlp, rel_err

pytestmark = pytest.mark.gpu
TOL_BF16 = 2e-2
SIZES = [(300, 3, 4), (64, 5, 2), (1000, 2, 7), (129, 1, 1), (7, 4, 0), (513, 2, 3)]


@pytest.fixture(scope="module")
def V():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_19729_b300 import voila
    return voila


def _setup(V, prec=WL.PREC_BF16, sizes=SIZES):
    wl = WL.mid_bf16(N=8, K=1, H=1, prec=prec)
    g = V.DeviceMLP.from_spec(wl.g_T)
    rm = V.DeviceMLP.from_spec(wl.reward_mlp)
    R = V.mlp_reward(rm)
    items, host = [], []
    for i, (N, K, H) in enumerate(sizes):
        parts, acts = WL.planner_inputs(100 + i, N, K, H)
        host.append((parts, acts))
        items.append({"particles": cuda(parts), "actions": cuda(acts), "planner_id": 10 + i,
                      "J": torch.empty(K, dtype=torch.float64, device="cuda"),
                      "G": torch.empty((K, N), dtype=torch.float64, device="cuda"),
                      "best_k": torch.empty(1, dtype=torch.int32, device="cuda")})
    return wl, g, rm, R, items, host


def _single(V, wl, g, R, it):
    N, K, H = it["particles"].shape[0], it["actions"].shape[0], it["actions"].shape[1]
    J = torch.empty(K, dtype=torch.float64, device="cuda")
    G = torch.empty((K, N), dtype=torch.float64, device="cuda")
    ws = V.alloc_workspace(V.voila_rollout_workspace_size(g, R, N, K, H))
    V.voila_rollout(g, R, it["particles"], None, it["actions"], wl.d_omega, wl.gamma, wl.seed, it["planner_id"], J, G,
                    None, ws)
    return J, G


QUEUE, ONE_TILE = 2, 4  # VOILA_SCHED_QUEUE, VOILA_SCHED_ONE_TILE


@pytest.mark.parametrize("schedule", [0, 1, 1 | (40 << 8), 3 << 8, QUEUE, 1 | QUEUE, 1 | QUEUE | (5 << 8),
                                      QUEUE | (1 << 8)])
def test_batched_equals_single_calls(V, schedule):
    wl, g, rm, R, items, _ = _setup(V)
    pl = V.make_planners(items)
    ws = V.alloc_workspace(V.voila_rollout_batched_workspace_size(g, R, pl))
    V.voila_rollout_batched(g, R, pl, wl.d_s, wl.d_a, wl.d_omega, wl.gamma, wl.seed, schedule, ws)
    assert V.workspace_status(ws) == V.OK
    for it in items:
        J, G = _single(V, wl, g, R, it)
        assert torch.equal(it["G"], G)
        assert torch.equal(it["J"], J)
        assert int(it["best_k"].item()) == int(torch.argmax(J).item())


def test_batched_matches_oracle(V):
    wl, g, rm, R, items, host = _setup(V)
    pl = V.make_planners(items)
    ws = V.alloc_workspace(V.voila_rollout_batched_workspace_size(g, R, pl))
    V.voila_rollout_batched(g, R, pl, wl.d_s, wl.d_a, wl.d_omega, wl.gamma, wl.seed, 1, ws)
    torch.cuda.synchronize()
    Ro = O.Reward(O.REWARD_MLP, mlp=oracle_mlp(wl.reward_mlp))
    for i in [0, 2, 5]:
        parts, acts = host[i]
        Jo, Go = O.rollout(oracle_mlp(wl.g_T), Ro, parts, acts, wl.d_omega, wl.gamma, wl.seed, planner=10 + i)
        assert rel_err(items[i]["G"].cpu().numpy(), Go) < TOL_BF16
        assert rel_err(items[i]["J"].cpu().numpy(), Jo) < TOL_BF16
    assert torch.all(items[4]["G"] == 0)  # H = 0


def test_batched_in_cuda_graph_and_autotune(V):
    wl, g, rm, R, items, _ = _setup(V)
    pl = V.make_planners(items)
    ws = V.alloc_workspace(V.voila_rollout_batched_workspace_size(g, R, pl))
    best, ms = V.voila_rollout_batched_autotune(g, R, pl, wl.d_s, wl.d_a, wl.d_omega, wl.gamma, wl.seed, ws)
    assert ms > 0
    V.voila_rollout_batched(g, R, pl, wl.d_s, wl.d_a, wl.d_omega, wl.gamma, wl.seed, best, ws)
    torch.cuda.synchronize()
    ref = [it["J"].clone() for it in items]
    for it in items:
        it["J"].zero_()
    s = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(graph, stream=s):
            V.voila_rollout_batched(g, R, pl, wl.d_s, wl.d_a, wl.d_omega, wl.gamma, wl.seed, best, ws, stream=s)
    graph.replay()
    torch.cuda.synchronize()
    for it, r in zip(items, ref):
        assert torch.equal(it["J"], r)


def test_batched_fp32_form_equals_single_calls(V):
    wl, g, rm, R, items, _ = _setup(V, prec=WL.PREC_FP32, sizes=SIZES[:3])
    pl = V.make_planners(items)
    ws = V.alloc_workspace(V.voila_rollout_batched_workspace_size(g, R, pl))
    V.voila_rollout_batched(g, R, pl, wl.d_s, wl.d_a, wl.d_omega, wl.gamma, wl.seed, 0, ws)
    for it in items:
        J, G = _single(V, wl, g, R, it)
        assert torch.equal(it["G"], G) and torch.equal(it["J"], J)


@pytest.mark.parametrize("schedule", [ONE_TILE | 1, ONE_TILE | QUEUE | 1, ONE_TILE | QUEUE | (3 << 8)])
def test_batched_one_tile_shape_matches_oracle(V, schedule):
    # one 128-row tile per CTA and work item, the reward output as an MMA: the
    # same rows and noise, the reward rounded through BF16 operands
    wl, g, rm, R, items, host = _setup(V)
    pl = V.make_planners(items)
    ws = V.alloc_workspace(V.voila_rollout_batched_workspace_size(g, R, pl))
    V.voila_rollout_batched(g, R, pl, wl.d_s, wl.d_a, wl.d_omega, wl.gamma, wl.seed, schedule, ws)
    assert V.workspace_status(ws) == V.OK
    Ro = O.Reward(O.REWARD_MLP, mlp=oracle_mlp(wl.reward_mlp))
    for i, (parts, acts) in enumerate(host):
        Jo, Go = O.rollout(oracle_mlp(wl.g_T), Ro, parts, acts, wl.d_omega, wl.gamma, wl.seed, planner=10 + i)
        if acts.shape[1] == 0:
            assert torch.all(items[i]["G"] == 0)
            continue
        assert rel_err(items[i]["G"].cpu().numpy(), Go) < TOL_BF16
        assert rel_err(items[i]["J"].cpu().numpy(), Jo) < TOL_BF16
    # the queue does not change the bits of a tile shape
    if schedule & QUEUE:
        ref = [(it["J"].clone(), it["G"].clone()) for it in items]
        V.voila_rollout_batched(g, R, pl, wl.d_s, wl.d_a, wl.d_omega, wl.gamma, wl.seed, ONE_TILE | 1, ws)
        for it, (J, G) in zip(items, ref):
            assert torch.equal(it["J"], J) and torch.equal(it["G"], G)


def test_batched_queue_fp8_and_sweep_dims(V):
    # FP8 form through the queue: the same bits as its single calls; the one-tile
    # shape has no FP8 kernel for these dimensions
    wl, g8, rm8, R8, items, _ = _setup(V, prec=WL.PREC_FP8, sizes=SIZES[:4])
    pl = V.make_planners(items)
    ws = V.alloc_workspace(V.voila_rollout_batched_workspace_size(g8, R8, pl))
    V.voila_rollout_batched(g8, R8, pl, wl.d_s, wl.d_a, wl.d_omega, wl.gamma, wl.seed, QUEUE | 1, ws)
    for it in items:
        J, G = _single(V, wl, g8, R8, it)
        assert torch.equal(it["G"], G) and torch.equal(it["J"], J)
    with pytest.raises(V.VoilaError) as e:
        V.voila_rollout_batched(g8, R8, pl, wl.d_s, wl.d_a, wl.d_omega, wl.gamma, wl.seed, ONE_TILE, ws)
    assert e.value.code == V.ERR_UNSUPPORTED
    # sweep dimensions (12, 3, 16) with the 4x512 generator (wide kernel) through the queue
    sw = WL.sweep(N=300, K=5, H=3)
    gs = V.DeviceMLP.from_spec(sw.g_T)
    Rg = V.goal_reward(list(sw.goal))
    its = [{"particles": cuda(sw.particles), "actions": cuda(sw.actions), "planner_id": 1,
            "J": torch.empty(sw.K, dtype=torch.float64, device="cuda"),
            "G": torch.empty((sw.K, sw.N), dtype=torch.float64, device="cuda")}]
    pls = V.make_planners(its)
    wss = V.alloc_workspace(V.voila_rollout_batched_workspace_size(gs, Rg, pls))
    V.voila_rollout_batched(gs, Rg, pls, sw.d_s, sw.d_a, sw.d_omega, sw.gamma, sw.seed, QUEUE, wss)
    J, G = _single(V, sw, gs, Rg, its[0])
    assert torch.equal(its[0]["G"], G) and torch.equal(its[0]["J"], J)


def test_batched_queue_many_tiny_planners(V):
    # 64 planners of one work item or less each: fewer items than CTA pairs, so
    # most pairs claim the end marker at once; every schedule gives each planner
    # its single-call bits
    rng = np.random.default_rng(11)
    sizes = [(int(rng.integers(1, 40)), int(rng.integers(1, 4)), int(rng.integers(1, 4))) for _ in range(64)]
    wl, g, rm, R, items, _ = _setup(V, sizes=sizes)
    pl = V.make_planners(items)
    ws = V.alloc_workspace(V.voila_rollout_batched_workspace_size(g, R, pl))
    refs = [_single(V, wl, g, R, it) for it in items]
    for schedule in (QUEUE, 1 | QUEUE, 1 | QUEUE | (2 << 8), 1):
        for it in items:
            it["J"].fill_(float("nan"))
        V.voila_rollout_batched(g, R, pl, wl.d_s, wl.d_a, wl.d_omega, wl.gamma, wl.seed, schedule, ws)
        assert V.workspace_status(ws) == V.OK
        for it, (J, G) in zip(items, refs):
            assert torch.equal(it["G"], G) and torch.equal(it["J"], J)
