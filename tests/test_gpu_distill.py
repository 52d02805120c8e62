"""Parity of the distillation-step kernels (Eq. 3) with the FP64 oracle.

The training path computes in FP32 on CUDA cores (weights FP32 or BF16), so
the tolerance is normwise relative 1e-4 (||got - want||_inf / ||want||_inf):
with K <= 512-term FP32 dot products the rounding error is below 512 * 2^-24
= 3e-5 of the operand scale, and the DDIM chain of 32 teacher calls stays
within the same bound on these weights.
"""
import numpy as np
import pytest
import torch

from oracle import voila_oracle as O
from paper_2606_19729_b300 import workloads as WL
from tests.helpers import cuda, oracle_mlp, rel_err

pytestmark = pytest.mark.gpu
TOL = 1e-4
# tensor-core teacher: BF16 operands and activations (relative rounding 2^-9 per
# layer) through 4 layers x 32 steps, FP32 accumulation and state
TOL_BF16 = 2e-2


@pytest.fixture(scope="module")
def V():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_19729_b300 import voila
    return voila


def _student(V, spec, prec):
    """Device student whose forward copy is `spec` rounded to `prec`, and its oracle MLP."""
    W = [WL.round_to(w, prec) for w in spec.W]
    dev = V.DeviceMLP([torch.from_numpy(w) for w in W], [torch.from_numpy(b) for b in spec.b], spec.act, prec)
    return dev, O.MLP(W, [np.asarray(b, np.float64) for b in spec.b], spec.act)


def _x(wl, B):
    return np.concatenate([wl.S[:B], wl.A[:B], wl.omega[:B]], axis=-1)


@pytest.mark.parametrize("prec", [WL.PREC_FP32, WL.PREC_BF16])
@pytest.mark.parametrize("B", [1, 77, 1300])
def test_fwd_train_saves_preactivations(V, prec, B):
    wl = WL.distill(B=max(B, 16))
    dev, om = _student(V, wl.student, prec)
    X = _x(wl, B)
    Xd = cuda(X)
    Y = torch.empty(B, wl.d_x, device="cuda")
    saved = torch.empty(B, 3 * 256, device="cuda")
    ws = V.alloc_workspace(2 * B * 256 * 4)
    V.voila_generator_fwd_train(dev, Xd, Y, saved, ws)
    torch.cuda.synchronize()
    y, zs = O.mlp_forward_saved(om, X)
    assert rel_err(Y.cpu().numpy(), y) < TOL
    z = np.concatenate(zs[:-1], axis=-1)
    assert rel_err(saved.cpu().numpy(), z) < TOL


@pytest.mark.parametrize("prec", [WL.PREC_FP32, WL.PREC_BF16])
@pytest.mark.parametrize("B", [16, 1, 2500])
def test_bwd_matches_oracle_gradient(V, prec, B):
    # B = 16 is the gradient-check batch; 2500 spans three 1024-row chunks with a ragged tail
    wl = WL.distill(B=max(B, 16))
    dev, om = _student(V, wl.student, prec)
    X = _x(wl, B)
    rng = np.random.default_rng(11)
    dY = rng.standard_normal((B, wl.d_x)).astype(np.float32).astype(np.float64)
    Xd, dYd = cuda(X), cuda(dY)
    Y = torch.empty(B, wl.d_x, device="cuda")
    saved = torch.empty(B, 3 * 256, device="cuda")
    V.voila_generator_fwd_train(dev, Xd, Y, saved, V.alloc_workspace(2 * B * 256 * 4))
    dims = dev.dims
    dW = [torch.full((o, i), float("nan"), device="cuda") for i, o in zip(dims[:-1], dims[1:])]
    db = [torch.full((o,), float("nan"), device="cuda") for o in dims[1:]]
    dX = torch.empty(B, dims[0], device="cuda")
    ws = V.alloc_workspace(V.voila_generator_bwd_workspace_size(dev, B))
    V.voila_generator_bwd(dev, Xd, saved, dYd, dX, dW, db, ws)
    torch.cuda.synchronize()
    gX, gW, gb = O.mlp_backward(om, X, dY)
    assert rel_err(dX.cpu().numpy(), gX) < TOL
    for l in range(len(dW)):
        assert rel_err(dW[l].cpu().numpy(), gW[l]) < TOL, l
        assert rel_err(db[l].cpu().numpy(), gb[l]) < TOL, l


def test_bwd_is_deterministic_and_skips_dx(V):
    wl = WL.distill(B=4096)
    dev, _ = _student(V, wl.student, WL.PREC_BF16)
    B = 4096
    Xd = cuda(_x(wl, B))
    dYd = torch.randn(B, wl.d_x, device="cuda", generator=torch.Generator("cuda").manual_seed(3))
    saved = torch.empty(B, 3 * 256, device="cuda")
    V.voila_generator_fwd_train(dev, Xd, torch.empty(B, wl.d_x, device="cuda"), saved,
                                V.alloc_workspace(2 * B * 256 * 4))
    ws = V.alloc_workspace(V.voila_generator_bwd_workspace_size(dev, B))
    outs = []
    for _ in range(2):
        dW = [torch.empty(o, i, device="cuda") for i, o in zip(dev.dims[:-1], dev.dims[1:])]
        db = [torch.empty(o, device="cuda") for o in dev.dims[1:]]
        V.voila_generator_bwd(dev, Xd, saved, dYd, None, dW, db, ws)
        outs.append(torch.cat([t.reshape(-1) for t in dW + db]))
    torch.cuda.synchronize()
    assert torch.equal(outs[0], outs[1])


def test_bwd_full_batch_65536(V):
    # the bench's student and batch; the oracle gradient over all rows
    wl = WL.distill()
    B = wl.B
    dev, om = _student(V, wl.student, WL.PREC_BF16)
    X = _x(wl, B)
    dY = np.random.default_rng(12).standard_normal((B, wl.d_x)).astype(np.float32).astype(np.float64) / B
    Xd, dYd = cuda(X), cuda(dY)
    saved = torch.empty(B, 3 * 256, device="cuda")
    Y = torch.empty(B, wl.d_x, device="cuda")
    V.voila_generator_fwd_train(dev, Xd, Y, saved, V.alloc_workspace(2 * B * 256 * 4))
    dW = [torch.empty(o, i, device="cuda") for i, o in zip(dev.dims[:-1], dev.dims[1:])]
    db = [torch.empty(o, device="cuda") for o in dev.dims[1:]]
    V.voila_generator_bwd(dev, Xd, saved, dYd, None, dW, db,
                          V.alloc_workspace(V.voila_generator_bwd_workspace_size(dev, B)))
    torch.cuda.synchronize()
    y, _ = O.mlp_forward_saved(om, X)
    assert rel_err(Y.cpu().numpy(), y) < TOL
    _, gW, gb = O.mlp_backward(om, X, dY)
    for l in range(len(dW)):
        assert rel_err(dW[l].cpu().numpy(), gW[l]) < TOL, l
        assert rel_err(db[l].cpu().numpy(), gb[l]) < TOL, l


@pytest.mark.parametrize("B,T", [(70, 32), (1, 32), (33, 1), (40, 5)])
def test_ddim_matches_oracle(V, B, T):
    wl = WL.distill(B=max(B, 16))
    teacher = V.DeviceMLP.from_spec(wl.teacher)
    S, A, om = wl.S[:B], wl.A[:B], wl.omega[:B]
    Y = torch.empty(B, wl.d_x, device="cuda")
    V.voila_ddim_sample(teacher, cuda(S), cuda(A), cuda(om), T, wl.beta0, wl.beta1, wl.emb_dim, Y)
    torch.cuda.synchronize()
    want = O.distill_targets(oracle_mlp(wl.teacher), S, A, om, T, wl.beta0, wl.beta1, wl.emb_dim)
    assert rel_err(Y.cpu().numpy(), want) < TOL


def test_ddim_full_batch_sampled_rows(V):
    wl = WL.distill()
    teacher = V.DeviceMLP.from_spec(wl.teacher)
    Y = torch.empty(wl.B, wl.d_x, device="cuda")
    V.voila_ddim_sample(teacher, cuda(wl.S), cuda(wl.A), cuda(wl.omega), wl.T, wl.beta0, wl.beta1, wl.emb_dim, Y)
    torch.cuda.synchronize()
    rows = np.unique(np.concatenate([[0, wl.B - 1], np.random.default_rng(5).integers(0, wl.B, 126)]))
    want = O.distill_targets(oracle_mlp(wl.teacher), wl.S[rows], wl.A[rows], wl.omega[rows], wl.T, wl.beta0,
                             wl.beta1, wl.emb_dim)
    assert rel_err(Y.cpu().numpy()[rows], want) < TOL


@pytest.mark.parametrize("B,T", [(300, 32), (1, 32), (257, 1), (1000, 5)])
def test_ddim_tensor_core_matches_oracle(V, B, T):
    # B = 300 and 1000: several 256-row items with a ragged tail; 1: a single row
    wl = WL.distill(B=max(B, 16), teacher_prec=WL.PREC_BF16)
    teacher = V.DeviceMLP.from_spec(wl.teacher)
    S, A, om = wl.S[:B], wl.A[:B], wl.omega[:B]
    Y = torch.full((B, wl.d_x), float("nan"), device="cuda")
    ws = V.alloc_workspace(V.voila_ddim_sample_workspace_size(teacher, T))
    V.voila_ddim_sample(teacher, cuda(S), cuda(A), cuda(om), T, wl.beta0, wl.beta1, wl.emb_dim, Y, ws)
    torch.cuda.synchronize()
    assert V.workspace_status(ws) == V.OK
    want = O.distill_targets(oracle_mlp(wl.teacher), S, A, om, T, wl.beta0, wl.beta1, wl.emb_dim)
    assert rel_err(Y.cpu().numpy(), want) < TOL_BF16


def test_ddim_tensor_core_full_batch_sampled_rows(V):
    wl = WL.distill(teacher_prec=WL.PREC_BF16)
    teacher = V.DeviceMLP.from_spec(wl.teacher)
    Y = torch.full((wl.B, wl.d_x), float("nan"), device="cuda")
    V.voila_ddim_sample(teacher, cuda(wl.S), cuda(wl.A), cuda(wl.omega), wl.T, wl.beta0, wl.beta1, wl.emb_dim, Y)
    torch.cuda.synchronize()
    assert bool(torch.isfinite(Y).all())
    rows = np.unique(np.concatenate([[0, 255, 256, wl.B - 1], np.random.default_rng(6).integers(0, wl.B, 124)]))
    want = O.distill_targets(oracle_mlp(wl.teacher), wl.S[rows], wl.A[rows], wl.omega[rows], wl.T, wl.beta0,
                             wl.beta1, wl.emb_dim)
    assert rel_err(Y.cpu().numpy()[rows], want) < TOL_BF16


def test_ddim_rejects_bad_shapes(V):
    wl = WL.distill(B=16)
    teacher = V.DeviceMLP.from_spec(wl.teacher)
    Y = torch.empty(16, wl.d_x, device="cuda")
    with pytest.raises(V.VoilaError) as e:  # embedding width does not match the teacher's input
        V.voila_ddim_sample(teacher, cuda(wl.S), cuda(wl.A), cuda(wl.omega), 32, 1e-4, 0.02, 32, Y)
    assert e.value.code == V.ERR_SHAPE
    with pytest.raises(V.VoilaError) as e:
        V.voila_ddim_sample(teacher, cuda(wl.S), cuda(wl.A), cuda(wl.omega), 65, 1e-4, 0.02, 64, Y)
    assert e.value.code == V.ERR_ARG


def test_adam_matches_oracle(V):
    rng = np.random.default_rng(9)
    n = 10007
    p0 = rng.standard_normal(n).astype(np.float32).astype(np.float64)
    p, m, v = cuda(p0), torch.zeros(n, device="cuda"), torch.zeros(n, device="cuda")
    st = O.adam_init([p0])
    want = [p0]
    for t in range(1, 4):
        g = rng.standard_normal(n).astype(np.float32).astype(np.float64)
        V.voila_adam_step(p, cuda(g), m, v, 1e-2, 0.9, 0.999, 1e-8, t)
        want = O.adam_step(want, [g], st, lr=1e-2, beta1=0.9, beta2=0.999, eps=1e-8)
    torch.cuda.synchronize()
    # the update is lr * O(1); FP32 error relative to lr
    assert np.max(np.abs(p.cpu().numpy() - want[0])) < 1e-6 + 1e-4 * 1e-2


@pytest.mark.parametrize("prec", [WL.PREC_FP32, WL.PREC_BF16])
def test_distill_step_matches_oracle(V, prec):
    from paper_2606_19729_b300.distill import Distiller
    B = 300
    wl = WL.distill(B=B)
    teacher = V.DeviceMLP.from_spec(wl.teacher)
    d = Distiller(teacher, [torch.from_numpy(w) for w in wl.student.W], [torch.from_numpy(b) for b in wl.student.b],
                  wl.student.act, prec, B, wl.T, wl.beta0, wl.beta1, wl.emb_dim, lr=wl.lr)
    grad = torch.empty_like(d.master)
    loss = d.step(cuda(wl.S), cuda(wl.A), cuda(wl.omega), grad_out=grad)
    torch.cuda.synchronize()
    # oracle: the same step on the forward copy's values, Adam on the FP32 master
    fwd = O.MLP([WL.round_to(w, prec) for w in wl.student.W], [np.asarray(b, np.float64) for b in wl.student.b],
                wl.student.act)
    s_hat = O.distill_targets(oracle_mlp(wl.teacher), wl.S, wl.A, wl.omega, wl.T, wl.beta0, wl.beta1, wl.emb_dim)
    L, gW, gb = O.distill_loss_and_grad(fwd, wl.S, wl.A, wl.omega, s_hat)
    # FP32 student: CUDA-core FP32 training; BF16 student: tensor cores with BF16
    # activations and deltas (the BF16 tolerance)
    tol = TOL if prec == WL.PREC_FP32 else TOL_BF16
    assert abs(loss.item() - L) <= tol * L
    g_want = np.concatenate([x for l in range(len(gW)) for x in (gW[l].ravel(), gb[l].ravel())])
    g_got = grad.cpu().numpy().astype(np.float64)
    assert rel_err(g_got, g_want) < tol
    p0 = O.flat_params(oracle_mlp(wl.student))
    p1 = O.adam_step([p0], [g_want], O.adam_init([p0]), lr=wl.lr, beta1=0.9, beta2=0.999, eps=1e-8)[0]
    got = d.master.cpu().numpy().astype(np.float64)
    # first Adam step: -lr g / (|g| + eps); where |g| is well above the gradient
    # error the updates agree, elsewhere the step is bounded by lr
    big = np.abs(g_want) > (1e-3 if prec == WL.PREC_FP32 else 0.1) * np.max(np.abs(g_want))
    assert np.max(np.abs(got - p1)[big]) < 1e-3 * wl.lr + 1e-6
    assert np.max(np.abs(got - p0)) <= wl.lr * (1 + 1e-5) + 1e-6
    # the forward copy is the updated master in the forward precision
    from paper_2606_19729_b300.distill import flat_views
    for (w, b), (Wm, bm) in zip(zip(d.student.W, d.student.b), flat_views(d.master, d.dims)):
        assert torch.equal(w, Wm.to(w.dtype)) and torch.equal(b, bm)


@pytest.mark.parametrize("B", [1, 129, 1000])
def test_tensor_core_training_gradient(V, B):
    # BF16 student -> tensor-core forward/backward: ragged batches (tiles of 128
    # rows, split-K chunks of 64) against the FP64 gradient of the same loss
    from paper_2606_19729_b300.distill import Distiller
    wl = WL.distill(B=max(B, 16))
    teacher = V.DeviceMLP.from_spec(wl.teacher)
    d = Distiller(teacher, [torch.from_numpy(w) for w in wl.student.W], [torch.from_numpy(b) for b in wl.student.b],
                  wl.student.act, WL.PREC_BF16, B, wl.T, wl.beta0, wl.beta1, wl.emb_dim, lr=wl.lr)
    grad = torch.empty_like(d.master)
    S, A, om = wl.S[:B], wl.A[:B], wl.omega[:B]
    loss = d.step(cuda(S), cuda(A), cuda(om), grad_out=grad)
    torch.cuda.synchronize()
    assert V.workspace_status(d.ws) == V.OK
    fwd = O.MLP([WL.round_bf16(w) for w in wl.student.W], [np.asarray(b, np.float64) for b in wl.student.b],
                wl.student.act)
    s_hat = O.distill_targets(oracle_mlp(wl.teacher), S, A, om, wl.T, wl.beta0, wl.beta1, wl.emb_dim)
    L, gW, gb = O.distill_loss_and_grad(fwd, S, A, om, s_hat)
    assert abs(loss.item() - L) <= TOL_BF16 * L
    g_want = np.concatenate([x for l in range(len(gW)) for x in (gW[l].ravel(), gb[l].ravel())])
    assert rel_err(grad.cpu().numpy(), g_want) < TOL_BF16
    # per layer too: no layer's gradient hides behind a larger one
    o = 0
    for l in range(len(gW)):
        n = gW[l].size
        assert rel_err(grad.cpu().numpy()[o:o + n], gW[l].ravel()) < TOL_BF16, l
        o += n
        assert rel_err(grad.cpu().numpy()[o:o + gb[l].size], gb[l]) < TOL_BF16, l
        o += gb[l].size


def test_distill_full_batch_loss_decreases_deterministically(V):
    # the bench's configuration: tensor-core teacher, BF16 student forward copy
    from paper_2606_19729_b300.distill import Distiller
    wl = WL.distill(teacher_prec=WL.PREC_BF16)
    teacher = V.DeviceMLP.from_spec(wl.teacher)
    S, A, om = cuda(wl.S), cuda(wl.A), cuda(wl.omega)

    def run(steps):
        d = Distiller(teacher, [torch.from_numpy(w) for w in wl.student.W],
                      [torch.from_numpy(b) for b in wl.student.b], wl.student.act, WL.PREC_BF16, wl.B, wl.T,
                      wl.beta0, wl.beta1, wl.emb_dim, lr=wl.lr)
        losses = torch.empty(steps, dtype=torch.float64, device="cuda")
        for i in range(steps):
            d.step(S, A, om, loss_out=losses[i:i + 1])
        torch.cuda.synchronize()
        return losses.cpu().numpy(), d.master.clone()

    l1, m1 = run(6)
    l2, m2 = run(6)
    assert np.array_equal(l1, l2) and torch.equal(m1, m2)
    assert np.all(np.isfinite(l1)) and l1[-1] < l1[0]


def test_autograd_function_matches_oracle(V):
    from paper_2606_19729_b300.distill import generator
    wl = WL.distill(B=64)
    dev, om = _student(V, wl.student, WL.PREC_FP32)
    X = _x(wl, 64)
    Xd = cuda(X).requires_grad_(True)
    params = [torch.zeros_like(t, requires_grad=True) for pair in zip(dev.W, dev.b) for t in pair]
    Y = generator(Xd, dev, *params)
    (Y * Y).sum().backward()
    y = O.mlp_forward(om, X)
    gX, gW, gb = O.mlp_backward(om, X, 2.0 * y)
    assert rel_err(Xd.grad.cpu().numpy(), gX) < TOL
    for l in range(len(gW)):
        assert rel_err(params[2 * l].grad.cpu().numpy(), gW[l]) < TOL
        assert rel_err(params[2 * l + 1].grad.cpu().numpy(), gb[l]) < TOL


@pytest.mark.parametrize("prec", [WL.PREC_BF16, WL.PREC_FP32])
def test_overlapped_steps_equal_plain_steps(V, prec):
    # the sampler of the next batch on its own stream while the student trains
    # (tensor-core GEMMs spread one CTA per tile): the same losses, gradients
    # and weights, bit for bit, as the plain steps; four batches, then one
    # batch again without a look-ahead
    from paper_2606_19729_b300.distill import Distiller
    B, nb = 1000, 4
    wl = WL.distill(B=B * nb, teacher_prec=WL.PREC_BF16)
    teacher = V.DeviceMLP.from_spec(wl.teacher)
    S, A, om = cuda(wl.S), cuda(wl.A), cuda(wl.omega)
    batches = [(S[i * B:(i + 1) * B], A[i * B:(i + 1) * B], om[i * B:(i + 1) * B]) for i in range(nb)]
    batches.append(batches[1])

    def make():
        return Distiller(teacher, [torch.from_numpy(w) for w in wl.student.W],
                         [torch.from_numpy(b) for b in wl.student.b], wl.student.act, prec, B, wl.T, wl.beta0,
                         wl.beta1, wl.emb_dim, lr=wl.lr)

    plain, ovl = make(), make()
    n = len(batches)
    lp = torch.empty(n, dtype=torch.float64, device="cuda")
    lo = torch.empty(n, dtype=torch.float64, device="cuda")
    gp = [torch.empty_like(plain.master) for _ in range(n)]
    go = [torch.empty_like(plain.master) for _ in range(n)]
    for i, b in enumerate(batches):
        plain.step(*b, loss_out=lp[i:i + 1], grad_out=gp[i])
    for i, b in enumerate(batches):
        nxt = batches[i + 1] if i + 1 < nb else (None, None, None)
        ovl.step_overlapped(*b, *nxt, loss_out=lo[i:i + 1], grad_out=go[i])
    ovl.join()
    torch.cuda.synchronize()
    assert V.workspace_status(ovl._ov["train_ws"]) == V.OK
    assert torch.equal(lp, lo)
    for a, b in zip(gp, go):
        assert torch.equal(a, b)
    assert torch.equal(plain.master, ovl.master)
    for wa, wb in zip(plain.student.W, ovl.student.W):
        assert torch.equal(wa, wb)


@pytest.mark.parametrize("act", [WL.ACT_TANH, WL.ACT_IDENTITY])
def test_tensor_core_training_gradient_other_activations(V, act):
    # the training GEMM's tanh and identity epilogues (act and act' of the
    # forward, the delta of the backward) against the FP64 gradient
    from paper_2606_19729_b300.distill import Distiller
    B = 1000
    wl = WL.distill(B=B)
    teacher = V.DeviceMLP.from_spec(wl.teacher)
    d = Distiller(teacher, [torch.from_numpy(w) for w in wl.student.W], [torch.from_numpy(b) for b in wl.student.b],
                  act, WL.PREC_BF16, B, wl.T, wl.beta0, wl.beta1, wl.emb_dim, lr=wl.lr)
    grad = torch.empty_like(d.master)
    loss = d.step(cuda(wl.S), cuda(wl.A), cuda(wl.omega), grad_out=grad)
    torch.cuda.synchronize()
    assert V.workspace_status(d.ws) == V.OK
    fwd = O.MLP([WL.round_bf16(w) for w in wl.student.W], [np.asarray(b, np.float64) for b in wl.student.b], act)
    s_hat = O.distill_targets(oracle_mlp(wl.teacher), wl.S, wl.A, wl.omega, wl.T, wl.beta0, wl.beta1, wl.emb_dim)
    L, gW, gb = O.distill_loss_and_grad(fwd, wl.S, wl.A, wl.omega, s_hat)
    assert abs(loss.item() - L) <= TOL_BF16 * L
    o = 0
    for l in range(len(gW)):
        n = gW[l].size
        assert rel_err(grad.cpu().numpy()[o:o + n], gW[l].ravel()) < TOL_BF16, l
        o += n
        assert rel_err(grad.cpu().numpy()[o:o + gb[l].size], gb[l]) < TOL_BF16, l
        o += gb[l].size


def test_ddim_tensor_core_mixed_width_teacher(V):
    # 82 -> 512 -> 256 -> 512 -> 8: the sampler's swapped A halves (a layer with
    # K <= 256 writes its first output half into the A half it does not read)
    # across a 256-wide layer, which flips the swap back, against the oracle
    import dataclasses
    B, T = 600, 8
    wl = WL.distill(B=B, teacher_prec=WL.PREC_BF16)
    rng = np.random.default_rng(31)
    wl = dataclasses.replace(wl, teacher=WL.xavier_mlp(rng, [82, 512, 256, 512, 8], WL.ACT_SILU, WL.PREC_BF16))
    teacher = V.DeviceMLP.from_spec(wl.teacher)
    ws = V.alloc_workspace(V.voila_ddim_sample_workspace_size(teacher, T))
    Y = torch.empty(B, wl.d_x, device="cuda")
    V.voila_ddim_sample(teacher, cuda(wl.S), cuda(wl.A), cuda(wl.omega), T, wl.beta0, wl.beta1, wl.emb_dim, Y, ws)
    torch.cuda.synchronize()
    assert V.workspace_status(ws) == V.OK
    want = O.distill_targets(oracle_mlp(wl.teacher), wl.S, wl.A, wl.omega, T, wl.beta0, wl.beta1, wl.emb_dim)
    assert rel_err(Y.cpu().numpy(), want) < TOL_BF16


def test_overlapped_steps_equal_plain_steps_full_batch(V):
    # the bench's configuration (65,536 samples, tensor-core teacher and student):
    # six overlapped steps on the same batch give the plain steps' losses and
    # weights bit for bit (the spread GEMMs run 512 one-tile CTAs per launch)
    from paper_2606_19729_b300.distill import Distiller
    wl = WL.distill(teacher_prec=WL.PREC_BF16)
    teacher = V.DeviceMLP.from_spec(wl.teacher)
    S, A, om = cuda(wl.S), cuda(wl.A), cuda(wl.omega)

    def make():
        return Distiller(teacher, [torch.from_numpy(w) for w in wl.student.W],
                         [torch.from_numpy(b) for b in wl.student.b], wl.student.act, WL.PREC_BF16, wl.B, wl.T,
                         wl.beta0, wl.beta1, wl.emb_dim, lr=wl.lr)

    plain, ovl = make(), make()
    n = 6
    lp = torch.empty(n, dtype=torch.float64, device="cuda")
    lo = torch.empty(n, dtype=torch.float64, device="cuda")
    for i in range(n):
        plain.step(S, A, om, loss_out=lp[i:i + 1])
        ovl.step_overlapped(S, A, om, S, A, om, loss_out=lo[i:i + 1])
    ovl.join()
    torch.cuda.synchronize()
    assert V.workspace_status(ovl._ov["train_ws"]) == V.OK and V.workspace_status(plain.ws) == V.OK
    assert torch.equal(lp, lo)
    assert torch.equal(plain.master, ovl.master)


@pytest.mark.parametrize("prec", [WL.PREC_BF16, WL.PREC_FP32])
def test_checkpoint_resume_continues_bit_for_bit(V, prec):
    # three steps, a checkpoint through torch.save / torch.load, then two more
    # steps: a fresh Distiller (other initial weights) restored from the
    # checkpoint reproduces the last two steps' losses, gradients, weights and
    # moments exactly
    import io
    from paper_2606_19729_b300.distill import Distiller
    B, nb = 2048, 5
    wl = WL.distill(B=B * nb)
    teacher = V.DeviceMLP.from_spec(wl.teacher)
    S, A, om = cuda(wl.S), cuda(wl.A), cuda(wl.omega)
    batches = [(S[i * B:(i + 1) * B], A[i * B:(i + 1) * B], om[i * B:(i + 1) * B]) for i in range(nb)]

    def make(scale):
        return Distiller(teacher, [torch.from_numpy(w * scale) for w in wl.student.W],
                         [torch.from_numpy(b) for b in wl.student.b], wl.student.act, prec, B, wl.T, wl.beta0,
                         wl.beta1, wl.emb_dim, lr=wl.lr)

    run = make(1.0)
    for b in batches[:3]:
        run.step(*b)
    buf = io.BytesIO()
    torch.save(run.state_dict(), buf)
    la = torch.empty(2, dtype=torch.float64, device="cuda")
    ga = [torch.empty_like(run.master) for _ in range(2)]
    for i, b in enumerate(batches[3:]):
        run.step(*b, loss_out=la[i:i + 1], grad_out=ga[i])

    res = make(0.5)
    res.step(*batches[4])  # a different history, overwritten by the checkpoint
    buf.seek(0)
    res.load_state_dict(torch.load(buf))
    assert res.t == 3
    lb = torch.empty(2, dtype=torch.float64, device="cuda")
    gb = [torch.empty_like(res.master) for _ in range(2)]
    for i, b in enumerate(batches[3:]):
        res.step(*b, loss_out=lb[i:i + 1], grad_out=gb[i])
    torch.cuda.synchronize()
    assert V.workspace_status(res.ws) == V.OK
    assert torch.equal(la, lb)
    for a, b in zip(ga, gb):
        assert torch.equal(a, b)
    for x, y in ((run.master, res.master), (run.m, res.m), (run.v, res.v)):
        assert torch.equal(x, y)
    for wa, wb in zip(run.student.W, res.student.W):
        assert torch.equal(wa, wb)
    with pytest.raises(ValueError):
        bad = run.state_dict()
        bad["dims"] = bad["dims"][:-1] + [bad["dims"][-1] + 1]
        res.load_state_dict(bad)
