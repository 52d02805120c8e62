"""Parity of the tensor-core belief update (SIR step of Sec. 3, weights
exp(l / lambda) of Sec. 4.2.3) with the FP64 oracle. With BF16 or FP8 e4m3
generator and likelihood MLPs of the mid-size shapes the proposal runs on the
tensor cores: one kernel computes s'_i = g_T([s_i; a; omega_T(i, 0, step)]) and
l([s'_i; a; o]).

Tolerances follow from the arithmetic: proposals and likelihoods carry the
normwise error of the rollout in the same precision (2e-2 BF16: inputs of every
layer rounded to 8-bit mantissas; 6e-2 FP8 e4m3: hidden activations and weights
with 4-bit mantissas and per-channel scales). A likelihood error of at most
d = tol * max|l| moves every log-weight by at most 2 d / lambda after
normalisation, log Z by at most d / lambda and log ESS by at most 4 d / lambda. The resampled indices are
compared bit for bit with systematic resampling of the device's own weights,
and every output particle with the oracle's proposal of its index."""
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


@pytest.fixture(scope="module", params=[WL.PREC_BF16, WL.PREC_FP8], ids=["bf16", "fp8"])
def wl(request):
    return WL.mid_bf16(N=4096, K=2, H=2, prec=request.param)


def _run(V, wl, N, lam, step, logw=None, planner=0):
    g = V.DeviceMLP.from_spec(wl.g_T)
    lm = V.DeviceMLP.from_spec(wl.ell)
    lik = V.mlp_likelihood(lm)
    parts = wl.particles[:N]
    a = wl.actions[0, 0]
    o = np.linspace(-0.6, 0.5, wl.d_o).astype(np.float32)
    out = torch.empty((N, wl.d_s), dtype=torch.float32, device="cuda")
    idx = torch.empty(N, dtype=torch.int32, device="cuda")
    w = torch.empty(N, dtype=torch.float64, device="cuda")
    lz = torch.empty(1, dtype=torch.float64, device="cuda")
    ess = torch.empty(1, dtype=torch.float64, device="cuda")
    ws = V.alloc_workspace(V.voila_belief_update_workspace_size(g, lik, N))
    V.voila_belief_update(g, lik, cuda(parts), None if logw is None else cuda(logw, torch.float64), cuda(a),
                          cuda(o), wl.d_omega, lam, wl.seed, step, planner, out, idx, w, lz, ess, ws)
    assert V.workspace_status(ws) == V.OK
    res = O.belief_update(oracle_mlp(wl.g_T), O.Likelihood(O.LIK_MLP, mlp=oracle_mlp(wl.ell)), parts, a,
                          o.astype(np.float64), wl.d_omega, lam, wl.seed, step, planner=planner, logw=logw)
    return (out.cpu().numpy(), idx.cpu().numpy(), w.cpu().numpy(), lz.item(), ess.item()), res


def _check(got, res, lam, tol):
    out, idx, w, lz, ess = got
    N = w.shape[0]
    assert abs(np.sum(w) - 1.0) <= N * 2.0 ** -52
    assert np.all(w * 2.0 ** 52 == np.rint(w * 2.0 ** 52))
    d = tol * max(np.max(np.abs(res.ell)), 1e-3)
    big = res.w > 1e-9
    assert np.max(np.abs(np.log(w[big]) - np.log(res.w[big]))) <= 2 * d / lam
    assert abs(lz - res.logZ) <= d / lam
    assert abs(np.log(ess) - np.log(res.ess)) <= 4 * d / lam
    assert np.array_equal(idx, O.systematic_resample(w, res.u0))
    assert rel_err(out, res.s_prop[idx]) < tol


@pytest.mark.parametrize("N", [4096, 1000, 513, 1])
def test_tc_belief_update_mlp_likelihood(V, wl, N):
    got, res = _run(V, wl, N, 1.0, 3)
    _check(got, res, 1.0, TOL[wl.prec])


@pytest.mark.parametrize("lam", [0.5, 0.02])
def test_tc_belief_update_tempered_with_prior(V, wl, lam):
    # lambda = 0.02 spreads l / lambda over several units (|l| < 0.07 at this
    # initialisation): uneven weights, an ESS well below N
    N = 700
    logw = np.random.default_rng(5).normal(0.0, 0.5, size=N)
    got, res = _run(V, wl, N, lam, 11, logw=logw, planner=2)
    if lam < 0.1:
        assert res.ess < 0.8 * N
    _check(got, res, lam, TOL[wl.prec])


def test_tc_belief_update_proposals_match_oracle(V, wl):
    # at a temperature where the weights are almost flat every proposal is
    # gathered somewhere: the gathered rows cover most of the oracle's proposals
    N = 2048
    got, res = _run(V, wl, N, 1e4, 4)
    out, idx = got[0], got[1]
    assert len(np.unique(idx)) > N // 2
    assert rel_err(out, res.s_prop[idx]) < TOL[wl.prec]


def test_fp8_belief_update_other_shapes_unsupported(V):
    # E4M3 MLPs have no CUDA-core form: shapes outside the tensor-core plan are refused
    rng = np.random.default_rng(3)
    g = V.DeviceMLP.from_spec(WL.xavier_mlp(rng, [10, 64, 64, 4], WL.ACT_SILU, WL.PREC_FP8))
    lik = V.gaussian_likelihood(0.5)
    N = 64
    out = torch.empty((N, 4), dtype=torch.float32, device="cuda")
    ws = V.alloc_workspace(V.voila_belief_update_workspace_size(g, lik, N))
    with pytest.raises(RuntimeError, match="unsupported"):
        V.voila_belief_update(g, lik, cuda(np.zeros((N, 4))), None, cuda(np.zeros(2)), cuda(np.zeros(2)), 4, 1.0, 0,
                              0, 0, out, None, None, None, None, ws)


def test_planning_step_in_cuda_graph(V):
    # one planning step (tensor-core belief update with the many-CTA resampling,
    # rollout of the updated belief, PORPP backup) captured in a CUDA graph and
    # replayed: the same bits as the eager calls (every reduction has one order)
    wl = WL.mid_bf16(N=4096, K=16, H=3)
    g = V.DeviceMLP.from_spec(wl.g_T)
    lik = V.mlp_likelihood(V.DeviceMLP.from_spec(wl.ell))
    R = V.mlp_reward(V.DeviceMLP.from_spec(wl.reward_mlp))
    N, K, H = wl.N, wl.K, wl.H
    parts, acts = cuda(wl.particles), cuda(wl.actions)
    a0, obs = cuda(wl.actions[0, 0]), cuda(np.linspace(-0.6, 0.5, wl.d_o))
    p_new = torch.empty_like(parts)
    w = torch.empty(N, dtype=torch.float64, device="cuda")
    J = torch.empty(K, dtype=torch.float64, device="cuda")
    best = torch.empty(1, dtype=torch.int32, device="cuda")
    Vb = torch.empty(1, dtype=torch.float64, device="cuda")
    ws_b = V.alloc_workspace(V.voila_belief_update_workspace_size(g, lik, N))
    ws_r = V.alloc_workspace(V.voila_rollout_workspace_size(g, R, N, K, H))

    def step(stream=None):
        V.voila_belief_update(g, lik, parts, None, a0, obs, wl.d_omega, 0.05, wl.seed, 2, 0, p_new, None, w, None,
                              None, ws_b, stream=stream)
        V.voila_rollout(g, R, p_new, None, acts, wl.d_omega, wl.gamma, wl.seed, 0, J, None, best, ws_r,
                        stream=stream)
        V.voila_preference_backup(J, None, 1.0, Vb, None, stream=stream)

    step()
    torch.cuda.synchronize()
    ref = [t.clone() for t in (p_new, w, J, best, Vb)]
    for t in (p_new, w, J, Vb):
        t.zero_()
    s = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(graph, stream=s):
            step(stream=s)
    graph.replay()
    torch.cuda.synchronize()
    assert V.workspace_status(ws_b) == V.OK and V.workspace_status(ws_r) == V.OK
    for got, r in zip((p_new, w, J, best, Vb), ref):
        assert torch.equal(got, r)
