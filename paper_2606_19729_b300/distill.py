"""Distillation of the transition generator (Eq. 3) on the library's kernels.

``GeneratorFn`` wraps ``voila_generator_fwd_train`` / ``voila_generator_bwd``
as a ``torch.autograd.Function`` for callers that build their own loss.
``Distiller`` keeps the FP32 master weights, the Adam moments and the
forward copy of a student generator and runs whole training steps through
``voila_distill_step`` (teacher DDIM targets, forward, MSE, backward, Adam).
"""
from __future__ import annotations

from typing import List, Optional, Sequence, Tuple

import torch

from . import voila as V


def flat_views(flat: torch.Tensor, dims: Sequence[int]) -> List[Tuple[torch.Tensor, torch.Tensor]]:
    """(W_l, b_l) views of a flat vector laid out [W_0, b_0, W_1, b_1, ...]."""
    out, o = [], 0
    for din, dout in zip(dims[:-1], dims[1:]):
        W = flat[o:o + din * dout].view(dout, din)
        o += din * dout
        b = flat[o:o + dout]
        o += dout
        out.append((W, b))
    if o != flat.numel():
        raise ValueError("flat vector does not match the layer widths")
    return out


def _aliases(t: torch.Tensor, base: torch.Tensor) -> bool:
    """Whether t is a view into base's storage (an FP32 student's weights are)."""
    return t.untyped_storage().data_ptr() == base.untyped_storage().data_ptr()


def n_params(dims: Sequence[int]) -> int:
    return sum(din * dout + dout for din, dout in zip(dims[:-1], dims[1:]))


class GeneratorFn(torch.autograd.Function):
    """Y = mlp(X) with the hand-written backward.

    ``params`` are tensors shaped like W_0, b_0, W_1, b_1, ... (for example FP32
    master weights); they receive the gradients. The forward reads the weights
    held by ``mlp`` (its FP32 or BF16 copy), which the caller keeps in step
    with ``params``.
    """

    @staticmethod
    def forward(ctx, X: torch.Tensor, mlp: V.DeviceMLP, *params: torch.Tensor) -> torch.Tensor:
        X = X.contiguous()
        B = X.shape[0]
        dims = mlp.dims
        Y = torch.empty(B, dims[-1], device=X.device, dtype=torch.float32)
        saved = torch.empty(B, max(sum(dims[1:-1]), 1), device=X.device, dtype=torch.float32)
        ws = V.alloc_workspace(2 * B * max(dims) * 4)
        V.voila_generator_fwd_train(mlp, X, Y, saved, ws)
        ctx.save_for_backward(X, saved)
        ctx.mlp = mlp
        return Y

    @staticmethod
    def backward(ctx, dY: torch.Tensor):
        X, saved = ctx.saved_tensors
        mlp = ctx.mlp
        dims = mlp.dims
        dev = X.device
        dW = [torch.empty(dout, din, device=dev) for din, dout in zip(dims[:-1], dims[1:])]
        db = [torch.empty(dout, device=dev) for dout in dims[1:]]
        dX = torch.empty_like(X) if ctx.needs_input_grad[0] else None
        ws = V.alloc_workspace(V.voila_generator_bwd_workspace_size(mlp, X.shape[0]))
        V.voila_generator_bwd(mlp, X, saved, dY.contiguous().float(), dX, dW, db, ws)
        grads = [g for pair in zip(dW, db) for g in pair]
        return (dX, None, *grads)


def generator(X: torch.Tensor, mlp: V.DeviceMLP, *params: torch.Tensor) -> torch.Tensor:
    return GeneratorFn.apply(X, mlp, *params)


class Distiller:
    """Distillation training state of one student generator (Eq. 3).

    teacher      DeviceMLP of the denoiser v_T([s; a; x_t; e(t)]).
    W, b         the student's initial FP32 weights (host or device tensors).
    prec         precision of the student's forward copy (FP32 or BF16).
    """

    def __init__(self, teacher: V.DeviceMLP, W: Sequence[torch.Tensor], b: Sequence[torch.Tensor], act: int,
                 prec: int, B: int, T: int = 32, beta0: float = 1e-4, beta1: float = 0.02, emb_dim: int = 64,
                 lr: float = 1e-3, betas=(0.9, 0.999), eps: float = 1e-8):
        self.teacher = teacher
        dims = [W[0].shape[1]] + [w.shape[0] for w in W]
        self.dims = dims
        self.master = torch.cat([t for l in range(len(W)) for t in
                                 (torch.as_tensor(W[l]).reshape(-1), torch.as_tensor(b[l]).reshape(-1))]
                                ).to(device="cuda", dtype=torch.float32).contiguous()
        self.m = torch.zeros_like(self.master)
        self.v = torch.zeros_like(self.master)
        views = flat_views(self.master, dims)
        self.student = V.DeviceMLP([w for w, _ in views], [bb for _, bb in views], act, prec)
        self.ddim = V.voila_ddim(T, beta0, beta1, emb_dim)
        self.lr, self.betas, self.eps = lr, betas, eps
        self.t = 0
        self.B = B
        self.d_x = dims[-1]
        self.ws = V.alloc_workspace(V.voila_distill_step_workspace_size(teacher, self.student, B, self.d_x, T))
        self.loss = torch.zeros(1, dtype=torch.float64, device="cuda")

    def step(self, S: torch.Tensor, A: torch.Tensor, omega: torch.Tensor, grad_out: Optional[torch.Tensor] = None,
             loss_out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
        """One step; returns the (device) loss before the update."""
        if omega.shape[0] > self.B:
            raise ValueError("batch larger than the workspace was sized for")
        self.t += 1
        opt = V.voila_adam(self.lr, self.betas[0], self.betas[1], self.eps, self.t)
        out = self.loss if loss_out is None else loss_out
        V.voila_distill_step(self.teacher, self.student, self.ddim, self.master, self.m, self.v, opt, S, A, omega,
                             out, grad_out, self.ws, stream)
        return out

    # ---- checkpoint and resume ----------------------------------------------
    # The training state is the FP32 master weights, Adam's two moment vectors
    # and its step count, and (BF16 students) the forward copy the next step's
    # forward pass reads. Restoring all of them exactly makes a resumed run
    # continue bit for bit; the dictionary holds host tensors and plain values,
    # so torch.save / torch.load store it.

    def state_dict(self) -> dict:
        """The training state as host tensors and plain values."""
        self.join()
        return {
            "dims": list(self.dims), "act": self.student.act, "prec": self.student.prec,
            "master": self.master.cpu(), "m": self.m.cpu(), "v": self.v.cpu(), "t": self.t,
            "lr": self.lr, "betas": tuple(self.betas), "eps": self.eps,
            "forward_W": [w.cpu() for w in self.student.W],
        }

    def load_state_dict(self, sd: dict) -> None:
        """Restores a state_dict() of a Distiller of the same student shape.

        Samples an overlapped step prepared for a following batch are
        dropped (that batch is sampled again)."""
        if list(sd["dims"]) != list(self.dims) or sd["act"] != self.student.act or sd["prec"] != self.student.prec:
            raise ValueError("checkpoint of a different student")
        self.join()
        # in place: the device descriptors keep pointing at these buffers
        self.master.copy_(sd["master"])
        self.m.copy_(sd["m"])
        self.v.copy_(sd["v"])
        for w, src in zip(self.student.W, sd["forward_W"]):
            if not _aliases(w, self.master):  # a BF16 forward copy; FP32 weights are views of master
                w.copy_(src)
        self.t = int(sd["t"])
        self.lr, self.betas, self.eps = sd["lr"], tuple(sd["betas"]), sd["eps"]
        ov = getattr(self, "_ov", None)
        if ov is not None:
            ov["pending"] = None

    # ---- overlapped steps --------------------------------------------------
    # The teacher does not depend on the student, so the targets of the next
    # batch can be sampled while the student trains on the current one. The
    # sampler runs on a high-priority stream and takes every SM first; the
    # student's kernels (their GEMMs launched one CTA per tile) fill the SMs
    # the sampler's last round of work items leaves idle. Two target buffers
    # alternate; events order each sampler after the training that last read
    # its buffer, and each training after the sampler that filled its buffer.

    def _overlap_state(self):
        if getattr(self, "_ov", None) is None:
            T = self.ddim.T
            self._ov = {
                "stream": torch.cuda.Stream(priority=-100),
                "targets": [torch.empty(self.B, self.d_x, device="cuda") for _ in range(2)],
                "ddim_ws": V.alloc_workspace(V.voila_ddim_sample_workspace_size(self.teacher, T)),
                "train_ws": V.alloc_workspace(V.voila_distill_train_step_workspace_size(self.student, self.B,
                                                                                        self.d_x)),
                "sampled": [torch.cuda.Event(), torch.cuda.Event()],
                "trained": [torch.cuda.Event(), torch.cuda.Event()],
                "used": [False, False],  # the slot's buffer has been read by a training
                "pending": None,         # (slot, key) of targets sampled for a batch not yet trained on
                "slot": 0,
            }
        return self._ov

    @staticmethod
    def _key(S, A, omega):
        return tuple((t.data_ptr(), tuple(t.shape)) for t in (S, A, omega))

    def _sample(self, ov, slot, S, A, omega):
        st = ov["stream"]
        for t in (S, A, omega):  # the caching allocator keeps them until the sampler has read them
            t.record_stream(st)
        if ov["used"][slot]:
            st.wait_event(ov["trained"][slot])
        V.voila_ddim_sample(self.teacher, S, A, omega, self.ddim.T, self.ddim.beta0, self.ddim.beta1,
                            self.ddim.emb_dim, ov["targets"][slot], ov["ddim_ws"], stream=st)
        ov["sampled"][slot].record(st)

    def step_overlapped(self, S: torch.Tensor, A: torch.Tensor, omega: torch.Tensor,
                        S_next: Optional[torch.Tensor] = None, A_next: Optional[torch.Tensor] = None,
                        omega_next: Optional[torch.Tensor] = None, grad_out: Optional[torch.Tensor] = None,
                        loss_out: Optional[torch.Tensor] = None) -> torch.Tensor:
        """One step on (S, A, omega), the same results as `step`, with the
        teacher targets of (S_next, A_next, omega_next), when given, sampled
        meanwhile for the following call. Runs on the current stream (the
        training) and an internal high-priority stream (the sampler); the
        returned loss is ordered on the current stream."""
        if omega.shape[0] > self.B:
            raise ValueError("batch larger than the workspace was sized for")
        ov = self._overlap_state()
        cur = torch.cuda.current_stream()
        key = self._key(S, A, omega)
        if ov["pending"] is not None and ov["pending"][1] == key:
            slot = ov["pending"][0]
        else:  # nothing sampled for this batch yet
            slot = ov["slot"]
            ov["stream"].wait_stream(cur)
            self._sample(ov, slot, S, A, omega)
        ov["pending"] = None
        if S_next is not None:
            nxt = 1 - slot
            ov["stream"].wait_stream(cur)  # the next batch's inputs as the caller wrote them
            self._sample(ov, nxt, S_next, A_next, omega_next)
            ov["pending"] = (nxt, self._key(S_next, A_next, omega_next))
            ov["slot"] = slot
        self.t += 1
        opt = V.voila_adam(self.lr, self.betas[0], self.betas[1], self.eps, self.t)
        out = self.loss if loss_out is None else loss_out
        cur.wait_event(ov["sampled"][slot])
        V.voila_distill_train_step(self.student, self.master, self.m, self.v, opt, S, A, omega, ov["targets"][slot],
                                   V.TRAIN_SPREAD, out, grad_out, ov["train_ws"], stream=cur)
        ov["trained"][slot].record(cur)
        ov["used"][slot] = True
        return out

    def join(self):
        """Orders the current stream after every overlapped sampler issued so far."""
        ov = getattr(self, "_ov", None)
        if ov is not None:
            torch.cuda.current_stream().wait_stream(ov["stream"])
