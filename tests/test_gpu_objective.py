"""Parity of the PORPP preference backup (Sec. 2.2) and the InfoNCE objective
(Eq. 6) with the FP64 oracle.

Tolerances: the backup is FP64 end to end (1e-12 relative). InfoNCE logits:
FP32 arithmetic 1e-4 normwise relative (as the training kernels), BF16 tensor
cores 2e-2 (BF16 activations, as the rollout). The row log-sum-exp and the
loss move by at most the largest logit error, so they are checked against
twice that bound.
"""
import math

import numpy as np
import pytest
import torch

from oracle import voila_oracle as O
from paper_2606_19729_b300 import workloads as WL
from tests.helpers import cuda, oracle_mlp, rel_err

pytestmark = pytest.mark.gpu
TOL_FP32 = 1e-4
TOL_BF16 = 2e-2


@pytest.fixture(scope="module")
def V():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_19729_b300 import voila
    return voila


@pytest.mark.parametrize("K", [1, 37, 1024, 100003])
@pytest.mark.parametrize("eta", [0.5, 20.0])
@pytest.mark.parametrize("with_prior", [False, True])
def test_preference_backup_matches_oracle(V, K, eta, with_prior):
    rng = np.random.default_rng(K)
    J = rng.standard_normal(K) * 3.0 - 10.0
    lp = np.log(rng.dirichlet(np.ones(K))) if with_prior else None
    Vd = torch.empty(1, dtype=torch.float64, device="cuda")
    pi = torch.empty(K, dtype=torch.float64, device="cuda")
    V.voila_preference_backup(cuda(J, torch.float64), None if lp is None else cuda(lp, torch.float64), eta, Vd, pi)
    torch.cuda.synchronize()
    Vo, pio = O.preference_backup(J, eta, lp)
    assert math.isclose(Vd.item(), Vo, rel_tol=1e-12)
    np.testing.assert_allclose(pi.cpu().numpy(), pio, rtol=1e-11, atol=1e-300)
    assert abs(pi.sum().item() - 1.0) < 1e-12


def test_preference_backup_of_a_rollout(V):
    # J straight from the BF16 rollout; the backup sees the device J, the oracle the same values
    wl = WL.mid_bf16(N=512, K=96, H=5)
    g = V.DeviceMLP.from_spec(wl.g_T)
    R = V.mlp_reward(V.DeviceMLP.from_spec(wl.reward_mlp))
    J = torch.empty(wl.K, dtype=torch.float64, device="cuda")
    ws = V.alloc_workspace(V.voila_rollout_workspace_size(g, R, wl.N, wl.K, wl.H))
    V.voila_rollout(g, R, cuda(wl.particles), None, cuda(wl.actions), wl.d_omega, wl.gamma, wl.seed, 0, J, None,
                    None, ws)
    Vd = torch.empty(1, dtype=torch.float64, device="cuda")
    pi = torch.empty(wl.K, dtype=torch.float64, device="cuda")
    V.voila_preference_backup(J, None, 4.0, Vd, pi)
    torch.cuda.synchronize()
    Jh = J.cpu().numpy()
    Vo, pio = O.preference_backup(Jh, 4.0)
    assert math.isclose(Vd.item(), Vo, rel_tol=1e-12)
    assert int(torch.argmax(pi).item()) == int(np.argmax(Jh))


def test_preference_backup_rejects_bad_eta(V):
    J = torch.zeros(4, dtype=torch.float64, device="cuda")
    Vd = torch.empty(1, dtype=torch.float64, device="cuda")
    with pytest.raises(V.VoilaError) as e:
        V.voila_preference_backup(J, None, 0.0, Vd, None)
    assert e.value.code == V.ERR_ARG


def _forward(V, ell_dev, wl, B, with_G=True):
    L = torch.full((B, B), float("nan"), device="cuda")
    lse = torch.empty(B, dtype=torch.float64, device="cuda")
    loss = torch.empty(1, dtype=torch.float64, device="cuda")
    G = torch.empty(B, B, device="cuda") if with_G else None
    ws = V.alloc_workspace(V.voila_infonce_workspace_size(ell_dev, B))
    V.voila_infonce_forward(ell_dev, cuda(wl.S[:B]), cuda(wl.A[:B]), cuda(wl.O[:B]), L, lse, loss, G, ws)
    torch.cuda.synchronize()
    assert V.workspace_status(ws) == V.OK
    return L.cpu().numpy(), lse.cpu().numpy(), loss.item(), None if G is None else G.cpu().numpy()


def _check_against_oracle(wl, B, L, lse, loss, G, tol):
    Lo = O.infonce_logits(oracle_mlp(wl.ell), wl.S[:B], wl.A[:B], wl.O[:B])
    lo, lseo, Go = O.infonce_loss(Lo)
    assert rel_err(L, Lo) < tol
    bound = 2 * tol * np.max(np.abs(Lo)) + 1e-6
    assert np.max(np.abs(lse - lseo)) <= bound
    assert abs(loss - lo) <= bound
    if G is not None:
        np.testing.assert_allclose(G.sum(axis=1), 0.0, atol=1e-5)
        assert np.max(np.abs(G - Go)) <= (math.exp(2 * bound) - 1) / B + 1e-6


@pytest.mark.parametrize("B", [1, 40, 300])
def test_infonce_tensor_cores_match_oracle(V, B):
    # B = 300: 90000 pairs = 175 super-pairs of 512 rows plus a ragged tail
    wl = WL.infonce(B=max(B, 2))
    ell = V.DeviceMLP.from_spec(wl.ell)
    _check_against_oracle(wl, B, *_forward(V, ell, wl, B), TOL_BF16)


@pytest.mark.parametrize("B", [1, 33, 130])
def test_infonce_cuda_cores_match_oracle(V, B):
    wl = WL.infonce(B=max(B, 2), prec=WL.PREC_FP32)
    ell = V.DeviceMLP.from_spec(wl.ell)
    _check_against_oracle(wl, B, *_forward(V, ell, wl, B), TOL_FP32)


def test_infonce_full_batch_sampled_rows(V):
    wl = WL.infonce()
    B = wl.B
    ell = V.DeviceMLP.from_spec(wl.ell)
    L, lse, loss, _ = _forward(V, ell, wl, B, with_G=False)
    rows = np.array([0, 1, 511, 777, B - 1])
    ell_o = oracle_mlp(wl.ell)
    X = O.infonce_pairs(wl.S, wl.A, wl.O).reshape(B, B, -1)[rows].reshape(-1, wl.ell.dims[0])
    Lo = O.mlp_forward(ell_o, X)[:, 0].reshape(len(rows), B)
    assert rel_err(L[rows], Lo) < TOL_BF16
    m = Lo.max(axis=1, keepdims=True)
    lseo = m[:, 0] + np.log(np.exp(Lo - m).sum(axis=1))
    assert np.max(np.abs(lse[rows] - lseo)) <= 2 * TOL_BF16 * np.max(np.abs(Lo)) + 1e-6
    assert np.isfinite(loss) and loss > 0


def test_infonce_step_matches_oracle(V):
    from paper_2606_19729_b300.distill import flat_views
    B = 24
    wl = WL.infonce(B=B, prec=WL.PREC_FP32)
    ell = V.DeviceMLP.from_spec(wl.ell)
    p0 = O.flat_params(oracle_mlp(wl.ell))
    master = cuda(p0)
    m, v = torch.zeros_like(master), torch.zeros_like(master)
    grad = torch.empty_like(master)
    loss = torch.empty(1, dtype=torch.float64, device="cuda")
    ws = V.alloc_workspace(V.voila_infonce_step_workspace_size(ell, B))
    opt = V.voila_adam(wl.lr, 0.9, 0.999, 1e-8, 1)
    V.voila_infonce_step(ell, master, m, v, opt, cuda(wl.S), cuda(wl.A), cuda(wl.O), loss, grad, ws)
    torch.cuda.synchronize()
    lo, _, gW, gb = O.infonce_loss_and_grad(oracle_mlp(wl.ell), wl.S, wl.A, wl.O)
    assert abs(loss.item() - lo) <= TOL_FP32 * abs(lo)
    g_want = np.concatenate([x for l in range(len(gW)) for x in (gW[l].ravel(), gb[l].ravel())])
    assert rel_err(grad.cpu().numpy(), g_want) < TOL_FP32
    got = master.cpu().numpy().astype(np.float64)
    p1 = O.adam_step([p0], [g_want], O.adam_init([p0]), lr=wl.lr)[0]
    big = np.abs(g_want) > 1e-3 * np.max(np.abs(g_want))
    assert np.max(np.abs(got - p1)[big]) < 1e-3 * wl.lr + 1e-6
    assert np.max(np.abs(got - p0)) <= wl.lr * (1 + 1e-5) + 1e-6
    for (w, b), (Wm, bm) in zip(zip(ell.W, ell.b), flat_views(master, ell.dims)):
        assert torch.equal(w, Wm) and torch.equal(b, bm)


def test_infonce_step_loss_decreases_deterministically(V):
    B = 256
    wl = WL.infonce(B=B)
    S, A, Ob = cuda(wl.S), cuda(wl.A), cuda(wl.O)

    def run(steps):
        ell = V.DeviceMLP.from_spec(wl.ell)
        master = cuda(O.flat_params(oracle_mlp(wl.ell)))
        m, v = torch.zeros_like(master), torch.zeros_like(master)
        ws = V.alloc_workspace(V.voila_infonce_step_workspace_size(ell, B))
        losses = torch.empty(steps, dtype=torch.float64, device="cuda")
        for t in range(steps):
            V.voila_infonce_step(ell, master, m, v, V.voila_adam(1e-3, 0.9, 0.999, 1e-8, t + 1), S, A, Ob,
                                 losses[t:t + 1], None, ws)
        torch.cuda.synchronize()
        return losses.cpu().numpy(), master.clone()

    l1, m1 = run(5)
    l2, m2 = run(5)
    assert np.array_equal(l1, l2) and torch.equal(m1, m2)
    assert np.all(np.isfinite(l1)) and l1[-1] < l1[0]
    assert l1[0] <= math.log(B) + 5.0
