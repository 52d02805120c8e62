"""Parity of the vectorised progressive widening (Sec. 4.3) with the FP64 oracle.

Integer results are bit-exact: widening decisions, branch choices, visit and
branch counts (the threshold k_o n^alpha_o is evaluated in FP64 on both sides;
each test first checks that no threshold lies within 1e-9 of an integer, so
the last-bit differences of pow cannot flip a decision). New observations and
likelihood values of FP32 models are FP32 CUDA-core arithmetic (1e-5
normwise relative, the FP32 tolerance); a BF16 f_Z or likelihood of the
planning shapes runs on the tensor cores with BF16 activations (2e-2, the
BF16 tolerance of the rollout; the likelihood then inherits the observations'
error). Resampling
indices are checked as the function of the device's own quantised weights and
the group's u0 (several index vectors are valid up to rounding of the weights).
"""
import numpy as np
import pytest
import torch

from oracle import voila_oracle as O
from paper_2606_19729_b300 import workloads as WL
from tests.helpers import cuda, oracle_mlp, rel_err

pytestmark = pytest.mark.gpu
TOL = 1e-5
TOL_BF16 = 2e-2


@pytest.fixture(scope="module")
def V():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_19729_b300 import voila
    return voila


def _no_ties(k_o, alpha, n_max):
    n = np.arange(1, n_max + 1, dtype=np.float64)
    thr = k_o * np.power(n, alpha)
    return np.min(np.abs(thr - np.rint(thr))) > 1e-9


def _run(V, wl, node, s_next, tree, lik_dev, step, planner=0):
    M = node.shape[0]
    g_Z = V.DeviceMLP.from_spec(wl.g_Z)
    branch = torch.full((M,), -1, dtype=torch.int32, device="cuda")
    widened = torch.empty(M, dtype=torch.uint8, device="cuda")
    ell = torch.empty(M, device="cuda")
    w = torch.empty(M, dtype=torch.float64, device="cuda")
    idx = torch.empty(M, dtype=torch.int32, device="cuda")
    s_out = torch.empty(M, wl.d_s, device="cuda")
    ws = V.alloc_workspace(V.voila_progressive_widening_workspace_size(tree, g_Z, lik_dev, M))
    V.voila_progressive_widening(tree, cuda(node, torch.int32), cuda(s_next), g_Z, lik_dev, wl.d_omega, wl.k_o,
                                 wl.alpha_o, wl.lam, wl.seed, step, planner, branch, s_out, ws, widened, ell, w, idx)
    torch.cuda.synchronize()
    status = V.workspace_status(ws)
    return status, {k: v.cpu().numpy() for k, v in dict(branch=branch, widened=widened, ell=ell, w=w, idx=idx,
                                                        s_out=s_out).items()}


def _trees(V, wl):
    dev = V.PWTree(torch.from_numpy(wl.act), torch.from_numpy(wl.N0), torch.from_numpy(wl.C0),
                   torch.from_numpy(wl.obs0))
    ora = O.PWTree(wl.act.copy(), wl.N0.copy(), wl.C0.copy(), wl.obs0.copy())
    return dev, ora


def _check(wl, got, res, tree_dev, tree_o, node, s_next, step, nodes=None, planner=0, tol_ell=TOL, tol_obs=TOL):
    sel = np.ones(node.shape[0], bool) if nodes is None else np.isin(node, nodes)
    np.testing.assert_array_equal(got["branch"][sel], res.branch)
    np.testing.assert_array_equal(got["widened"][sel].astype(bool), res.widened)
    N = tree_dev.N.cpu().numpy()
    C = tree_dev.C.cpu().numpy()
    obs = tree_dev.obs.cpu().numpy()
    keep = np.arange(wl.n_nodes) if nodes is None else np.asarray(nodes)
    np.testing.assert_array_equal(N[keep], tree_o.N[keep])
    np.testing.assert_array_equal(C[keep], tree_o.C[keep])
    assert rel_err(obs[keep], tree_o.obs[keep]) < tol_obs
    assert rel_err(got["ell"][sel], res.ell) < tol_ell
    if tol_ell <= TOL:
        assert np.max(np.abs(got["w"][sel] - res.w)) < TOL
    # resampling within each (node, branch) group: the device's indices are the
    # systematic resampling of its own weights with the group's u0
    ms_all = np.nonzero(sel)[0]
    for key in set(zip(node[sel].tolist(), got["branch"][sel].tolist())):
        ms = ms_all[(node[sel] == key[0]) & (got["branch"][sel] == key[1])]
        q = got["w"][ms]
        assert abs(q.sum() - 1.0) <= len(ms) * 2.0 ** -52
        u0 = O.pw_group_uniform(wl.seed, key[0], key[1], step, planner)
        np.testing.assert_array_equal(got["idx"][ms], ms[O.systematic_resample(q, u0)])
    np.testing.assert_array_equal(got["s_out"][sel], s_next[got["idx"][sel]].astype(np.float32))


@pytest.mark.parametrize("M,n_nodes", [(1, 3), (700, 40), (3001, 64)])
def test_pw_mlp_matches_oracle(V, M, n_nodes):
    wl = WL.pw(M=M, n_nodes=n_nodes, C_max=16, prec=WL.PREC_FP32)
    assert _no_ties(wl.k_o, wl.alpha_o, 200 + M)
    tree_dev, tree_o = _trees(V, wl)
    ell_dev = V.DeviceMLP.from_spec(wl.ell)
    status, got = _run(V, wl, wl.node, wl.s_next, tree_dev, V.mlp_likelihood(ell_dev), step=3)
    assert status == V.OK
    res = O.progressive_widening(tree_o, wl.node, wl.s_next, oracle_mlp(wl.g_Z),
                                 O.Likelihood(O.LIK_MLP, mlp=oracle_mlp(wl.ell)), wl.d_omega, wl.k_o, wl.alpha_o,
                                 wl.lam, wl.seed, 3)
    _check(wl, got, res, tree_dev, tree_o, wl.node, wl.s_next, 3)


def test_pw_gaussian_two_steps_and_cap(V):
    # fresh nodes with a small cap and fast widening, two consecutive batches
    wl = WL.pw(M=1500, n_nodes=20, C_max=5, prec=WL.PREC_BF16, k_o=1.7, alpha_o=0.45)
    assert _no_ties(wl.k_o, wl.alpha_o, 3000)
    wl.N0[:] = 0
    wl.C0[:] = 0
    wl.obs0[:] = 0.0
    tree_dev, tree_o = _trees(V, wl)
    lik = O.Likelihood(O.LIK_GAUSSIAN, sigma=0.6)
    for step, part in ((0, slice(0, 800)), (1, slice(800, 1500))):
        node, s = wl.node[part], wl.s_next[part]
        status, got = _run(V, wl, node, s, tree_dev, V.gaussian_likelihood(0.6), step=step)
        assert status == V.OK
        res = O.progressive_widening(tree_o, node, s, oracle_mlp(wl.g_Z), lik, wl.d_omega, wl.k_o, wl.alpha_o,
                                     wl.lam, wl.seed, step)
        # BF16 f_Z of the planning shapes: tensor-core observations
        _check(wl, got, res, tree_dev, tree_o, node, s, step, tol_ell=TOL_BF16, tol_obs=TOL_BF16)
    assert tree_dev.C.cpu().numpy().max() <= 5


@pytest.mark.parametrize("M", [65536, 150000])  # 150000: more than 64 radix tiles (the separate scan)
def test_pw_full_batch_sampled_nodes(V, M):
    wl = WL.pw(M=M)
    assert _no_ties(wl.k_o, wl.alpha_o, 200 + wl.M)
    tree_dev, tree_o = _trees(V, wl)
    ell_dev = V.DeviceMLP.from_spec(wl.ell)
    status, got = _run(V, wl, wl.node, wl.s_next, tree_dev, V.mlp_likelihood(ell_dev), step=7)
    assert status == V.OK
    counts = np.bincount(wl.node, minlength=wl.n_nodes)
    np.testing.assert_array_equal(tree_dev.N.cpu().numpy(), wl.N0 + counts)
    # the threshold grows by less than one per visit and the prior counts are
    # consistent, so the branch count follows ceil(k_o n^alpha_o) (capped)
    n1 = (wl.N0 + counts).astype(np.float64)
    expect = np.where(counts > 0, np.minimum(wl.C_max, np.ceil(wl.k_o * np.power(n1, wl.alpha_o))), wl.C0)
    np.testing.assert_array_equal(tree_dev.C.cpu().numpy(), expect)
    # the busiest node, the quietest visited one and three random ones, replayed by the oracle
    nodes = sorted({int(np.argmax(counts)), int(np.argmin(np.where(counts > 0, counts, M + 1)))}
                   | set(np.random.default_rng(3).choice(np.nonzero(counts)[0], 3, replace=False).tolist()))
    sel = np.isin(wl.node, nodes)
    res = O.progressive_widening(tree_o, wl.node[sel], wl.s_next[sel], oracle_mlp(wl.g_Z),
                                 O.Likelihood(O.LIK_MLP, mlp=oracle_mlp(wl.ell)), wl.d_omega, wl.k_o, wl.alpha_o,
                                 wl.lam, wl.seed, 7, sim_index=np.nonzero(sel)[0])
    # BF16 f_Z and likelihood of the planning shapes: tensor cores, BF16 activations
    # (about 2150 widened simulations: five observation items, the last one ragged)
    _check(wl, got, res, tree_dev, tree_o, wl.node, wl.s_next, 7, nodes=nodes, tol_ell=TOL_BF16, tol_obs=TOL_BF16)


def test_pw_tensor_core_likelihood_small(V):
    # BF16 likelihood -> tensor-core gather rows; several 512-row items and a ragged tail
    wl = WL.pw(M=1300, n_nodes=30, C_max=16, prec=WL.PREC_BF16)
    assert _no_ties(wl.k_o, wl.alpha_o, 200 + wl.M)
    tree_dev, tree_o = _trees(V, wl)
    ell_dev = V.DeviceMLP.from_spec(wl.ell)
    status, got = _run(V, wl, wl.node, wl.s_next, tree_dev, V.mlp_likelihood(ell_dev), step=2)
    assert status == V.OK
    res = O.progressive_widening(tree_o, wl.node, wl.s_next, oracle_mlp(wl.g_Z),
                                 O.Likelihood(O.LIK_MLP, mlp=oracle_mlp(wl.ell)), wl.d_omega, wl.k_o, wl.alpha_o,
                                 wl.lam, wl.seed, 2)
    _check(wl, got, res, tree_dev, tree_o, wl.node, wl.s_next, 2, tol_ell=TOL_BF16, tol_obs=TOL_BF16)


def test_pw_tensor_core_observations_many_items(V):
    # fresh nodes that widen on most visits: thousands of widened simulations,
    # several 512-row observation items on the tensor cores and a ragged tail;
    # every node's observations are compared
    wl = WL.pw(M=3000, n_nodes=600, C_max=8, prec=WL.PREC_BF16, k_o=1.7, alpha_o=0.45)
    assert _no_ties(wl.k_o, wl.alpha_o, 3000)
    wl.N0[:] = 0
    wl.C0[:] = 0
    wl.obs0[:] = 0.0
    tree_dev, tree_o = _trees(V, wl)
    ell_dev = V.DeviceMLP.from_spec(wl.ell)
    status, got = _run(V, wl, wl.node, wl.s_next, tree_dev, V.mlp_likelihood(ell_dev), step=5)
    assert status == V.OK
    assert got["widened"].sum() > 3 * 512
    res = O.progressive_widening(tree_o, wl.node, wl.s_next, oracle_mlp(wl.g_Z),
                                 O.Likelihood(O.LIK_MLP, mlp=oracle_mlp(wl.ell)), wl.d_omega, wl.k_o, wl.alpha_o,
                                 wl.lam, wl.seed, 5)
    _check(wl, got, res, tree_dev, tree_o, wl.node, wl.s_next, 5, tol_ell=TOL_BF16, tol_obs=TOL_BF16)


def test_pw_invalid_node_sets_status(V):
    wl = WL.pw(M=64, n_nodes=8, C_max=4, prec=WL.PREC_FP32)
    node = wl.node.copy()
    node[5] = 8
    tree_dev, _ = _trees(V, wl)
    status, _ = _run(V, wl, node, wl.s_next, tree_dev, V.gaussian_likelihood(1.0), step=0)
    assert status == V.ERR_ARG
