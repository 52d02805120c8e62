"""Parity of the BF16 belief update (SIR step of Sec. 3, weights exp(l / lambda) of
Sec. 4.2.3) with the FP64 oracle. With BF16 generator and likelihood MLPs of the
mid-size shapes the proposal runs on the tensor cores: one kernel computes
s'_i = g_T([s_i; a; omega_T(i, 0, step)]) and l([s'_i; a; o]).

Tolerances follow from the BF16 arithmetic: proposals and likelihoods carry the
2e-2 normwise error of the BF16 rollout (inputs of every layer rounded to
8-bit mantissas). A likelihood error of at most d = 2e-2 * max|l| moves every
log-weight by at most 2 d / lambda after normalisation, log Z by at most
d / lambda and log ESS by at most 4 d / lambda. The resampled indices are
compared bit for bit with systematic resampling of the device's own weights,
and every output particle with the oracle's proposal of its index."""
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


@pytest.fixture(scope="module")
def wl():
    return WL.mid_bf16(N=4096, K=2, H=2)


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


def _check(got, res, lam):
    out, idx, w, lz, ess = got
    N = w.shape[0]
    assert abs(np.sum(w) - 1.0) <= N * 2.0 ** -52
    assert np.all(w * 2.0 ** 52 == np.rint(w * 2.0 ** 52))
    d = TOL_BF16 * max(np.max(np.abs(res.ell)), 1e-3)
    big = res.w > 1e-9
    assert np.max(np.abs(np.log(w[big]) - np.log(res.w[big]))) <= 2 * d / lam
    assert abs(lz - res.logZ) <= d / lam
    assert abs(np.log(ess) - np.log(res.ess)) <= 4 * d / lam
    assert np.array_equal(idx, O.systematic_resample(w, res.u0))
    assert rel_err(out, res.s_prop[idx]) < TOL_BF16


@pytest.mark.parametrize("N", [4096, 1000, 513, 1])
def test_bf16_belief_update_mlp_likelihood(V, wl, N):
    got, res = _run(V, wl, N, 1.0, 3)
    _check(got, res, 1.0)


def test_bf16_belief_update_tempered_with_prior(V, wl):
    N = 700
    logw = np.random.default_rng(5).normal(0.0, 0.5, size=N)
    got, res = _run(V, wl, N, 0.5, 11, logw=logw, planner=2)
    _check(got, res, 0.5)


def test_bf16_belief_update_proposals_match_oracle(V, wl):
    # at a temperature where the weights are almost flat every proposal is
    # gathered somewhere: the gathered rows cover most of the oracle's proposals
    N = 2048
    got, res = _run(V, wl, N, 1e4, 4)
    out, idx = got[0], got[1]
    assert len(np.unique(idx)) > N // 2
    assert rel_err(out, res.s_prop[idx]) < TOL_BF16
