"""Edge cases and error paths of the training, objective and widening entry
points: empty batches, too-small workspaces, unsupported precisions and shapes
(the library must refuse them before any device work, with its status codes)."""
import numpy as np
import pytest
import torch

from paper_2606_19729_b300 import workloads as WL
from tests.helpers import cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def V():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_19729_b300 import voila
    return voila


def _code(V, fn, *args, **kw):
    with pytest.raises(V.VoilaError) as e:
        fn(*args, **kw)
    return e.value.code


def test_distill_step_empty_batch_and_small_workspace(V):
    from paper_2606_19729_b300.distill import Distiller
    wl = WL.distill(B=16, teacher_prec=WL.PREC_BF16)
    teacher = V.DeviceMLP.from_spec(wl.teacher)
    d = Distiller(teacher, [torch.from_numpy(w) for w in wl.student.W], [torch.from_numpy(b) for b in wl.student.b],
                  wl.student.act, WL.PREC_BF16, 16)
    before = d.master.clone()
    e = torch.empty(0, 8, device="cuda")
    d.step(e, torch.empty(0, 2, device="cuda"), e)  # B = 0: nothing happens
    torch.cuda.synchronize()
    assert torch.equal(before, d.master)
    small = V.alloc_workspace(1024)
    opt = V.voila_adam(1e-3, 0.9, 0.999, 1e-8, 1)
    assert _code(V, V.voila_distill_step, teacher, d.student, d.ddim, d.master, d.m, d.v, opt, cuda(wl.S), cuda(wl.A),
                 cuda(wl.omega), d.loss, None, small) == V.ERR_WORKSPACE


def test_training_refuses_fp8_and_bad_shapes(V):
    wl = WL.distill(B=16)
    st = V.DeviceMLP([torch.from_numpy(WL.round_bf16(w)) for w in wl.student.W],
                     [torch.from_numpy(b) for b in wl.student.b], wl.student.act, V.FP8E4M3)
    X = cuda(np.zeros((4, 18)))
    Y = torch.empty(4, 8, device="cuda")
    ws = V.alloc_workspace(1 << 20)
    assert _code(V, V.voila_generator_fwd_train, st, X, Y, None, ws) == V.ERR_UNSUPPORTED
    teacher = V.DeviceMLP.from_spec(wl.teacher)
    # omega of the wrong width: the teacher's input is [s; a; x; e] = 82
    Yd = torch.empty(4, 6, device="cuda")
    assert _code(V, V.voila_ddim_sample, teacher, cuda(wl.S[:4]), cuda(wl.A[:4]), cuda(np.zeros((4, 6))), 32, 1e-4,
                 0.02, 64, Yd) == V.ERR_SHAPE


def test_adam_rejects_bad_hyperparameters(V):
    p = torch.zeros(8, device="cuda")
    g = torch.ones(8, device="cuda")
    m, v = torch.zeros_like(p), torch.zeros_like(p)
    assert _code(V, V.voila_adam_step, p, g, m, v, 1e-3, 1.0, 0.999, 1e-8, 1) == V.ERR_ARG  # beta1 = 1
    assert _code(V, V.voila_adam_step, p, g, m, v, 1e-3, 0.9, 0.999, 1e-8, 0) == V.ERR_ARG  # step 0
    assert _code(V, V.voila_adam_step, p, g, m, v, 1e-3, 0.9, 0.999, 0.0, 1) == V.ERR_ARG  # eps 0


def test_infonce_empty_and_shape_errors(V):
    wl = WL.infonce(B=8)
    ell = V.DeviceMLP.from_spec(wl.ell)
    loss = torch.full((1,), 7.0, dtype=torch.float64, device="cuda")
    ws = V.alloc_workspace(V.voila_infonce_workspace_size(ell, 0))
    e = torch.empty(0, 8, device="cuda")
    V.voila_infonce_forward(ell, e, torch.empty(0, 2, device="cuda"), torch.empty(0, 6, device="cuda"), None, None,
                            loss, None, ws)
    torch.cuda.synchronize()
    assert loss.item() == 0.0  # B = 0: the loss of no tuples
    ws = V.alloc_workspace(V.voila_infonce_workspace_size(ell, 8))
    # observation width that does not match the likelihood's input
    assert _code(V, V.voila_infonce_forward, ell, cuda(wl.S), cuda(wl.A), cuda(np.zeros((8, 5))), None, None, loss,
                 None, ws) == V.ERR_SHAPE


def test_widening_empty_batch_and_errors(V):
    wl = WL.pw(M=64, n_nodes=8, C_max=4, prec=WL.PREC_FP32)
    tree = V.PWTree(torch.from_numpy(wl.act), torch.from_numpy(wl.N0), torch.from_numpy(wl.C0),
                    torch.from_numpy(wl.obs0))
    N0 = tree.N.clone()
    g_Z = V.DeviceMLP.from_spec(wl.g_Z)
    lik = V.gaussian_likelihood(1.0)
    ws = V.alloc_workspace(V.voila_progressive_widening_workspace_size(tree, g_Z, lik, 0))
    V.voila_progressive_widening(tree, torch.empty(0, dtype=torch.int32, device="cuda"),
                                 torch.empty(0, wl.d_s, device="cuda"), g_Z, lik, wl.d_omega, wl.k_o, wl.alpha_o,
                                 wl.lam, wl.seed, 0, 0, torch.empty(0, dtype=torch.int32, device="cuda"),
                                 torch.empty(0, wl.d_s, device="cuda"), ws)
    torch.cuda.synchronize()
    assert torch.equal(tree.N, N0)  # no simulations, no visits
    ws = V.alloc_workspace(V.voila_progressive_widening_workspace_size(tree, g_Z, lik, 64))
    branch = torch.empty(64, dtype=torch.int32, device="cuda")
    s_out = torch.empty(64, wl.d_s, device="cuda")
    node = cuda(wl.node, torch.int32)
    s = cuda(wl.s_next)
    # non-positive widening constants
    assert _code(V, V.voila_progressive_widening, tree, node, s, g_Z, lik, wl.d_omega, 0.0, wl.alpha_o, wl.lam,
                 wl.seed, 0, 0, branch, s_out, ws) == V.ERR_ARG
    # f_Z whose output width is not the tree's observation width
    bad = V.DeviceMLP.from_spec(WL.xavier_mlp(np.random.default_rng(0), [18, 16, 5], WL.ACT_SILU, WL.PREC_FP32))
    assert _code(V, V.voila_progressive_widening, tree, node, s, bad, lik, wl.d_omega, wl.k_o, wl.alpha_o, wl.lam,
                 wl.seed, 0, 0, branch, s_out, ws) == V.ERR_SHAPE
    # a workspace sized for fewer simulations
    small = V.alloc_workspace(V.voila_progressive_widening_workspace_size(tree, g_Z, lik, 8))
    assert _code(V, V.voila_progressive_widening, tree, node, s, g_Z, lik, wl.d_omega, wl.k_o, wl.alpha_o, wl.lam,
                 wl.seed, 0, 0, branch, s_out, small) == V.ERR_WORKSPACE


def test_backup_single_sequence(V):
    J = cuda(np.array([-4.25]), torch.float64)
    Vd = torch.empty(1, dtype=torch.float64, device="cuda")
    pi = torch.empty(1, dtype=torch.float64, device="cuda")
    V.voila_preference_backup(J, None, 3.0, Vd, pi)
    torch.cuda.synchronize()
    assert Vd.item() == -4.25 and pi.item() == 1.0  # log of one exponential, uniform prior log 1 = 0
