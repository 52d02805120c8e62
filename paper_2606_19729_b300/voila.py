"""Thin ctypes binding of the C-ABI in include/voila.h.

Argument marshalling only: every step of the path runs in the library's
kernels. Tensors must be CUDA tensors of the dtype the header names; the
library is loaded from this package's lib/ folder and importing this module
raises if it is missing.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_double, c_float, c_int32, c_int64, c_size_t, c_uint32, c_uint64, c_void_p
from typing import List, Optional, Sequence

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libvoila.so")
if not os.path.exists(LIB_PATH):
    raise ImportError(f"VOiLA CUDA library not built: {LIB_PATH} is missing "
                      "(run __graft_entry__.build())")
_lib = ctypes.CDLL(LIB_PATH)

MAX_LAYERS = 8
MAX_GOAL = 4
OK, ERR_ARG, ERR_SHAPE, ERR_CUDA, ERR_NONFINITE, ERR_DEGENERATE, ERR_TIMEOUT, ERR_UNSUPPORTED, ERR_WORKSPACE = \
    0, -1, -2, -3, -4, -5, -6, -7, -8
ACT_IDENTITY, ACT_TANH, ACT_SILU = 0, 1, 2
FP32, BF16, FP8E4M3 = 0, 1, 2
REWARD_GOAL, REWARD_MLP = 0, 1
LIK_MLP, LIK_GAUSSIAN = 0, 1
STREAM_ROLLOUT_OMEGA, STREAM_BELIEF_OMEGA, STREAM_RESAMPLE, STREAM_OBS_OMEGA = 0, 1, 2, 3


class voila_mlp(ctypes.Structure):
    _fields_ = [("n_layers", c_int32), ("dims", c_int32 * (MAX_LAYERS + 1)), ("act", c_int32),
                ("prec", c_int32), ("W", c_void_p * MAX_LAYERS), ("b", c_void_p * MAX_LAYERS),
                ("w_scale", c_void_p * MAX_LAYERS)]


class voila_reward(ctypes.Structure):
    _fields_ = [("kind", c_int32), ("goal_dims", c_int32), ("goal", c_float * MAX_GOAL),
                ("mlp", POINTER(voila_mlp))]


class voila_planner(ctypes.Structure):
    _fields_ = [("particles", c_void_p), ("w", c_void_p), ("actions", c_void_p), ("N", c_int32), ("K", c_int32),
                ("H", c_int32), ("planner_id", c_uint32), ("J", c_void_p), ("G", c_void_p), ("best_k", c_void_p)]


class voila_likelihood(ctypes.Structure):
    _fields_ = [("kind", c_int32), ("sigma", c_float), ("mlp", POINTER(voila_mlp))]


class voila_ddim(ctypes.Structure):
    _fields_ = [("T", c_int32), ("beta0", c_double), ("beta1", c_double), ("emb_dim", c_int32)]


class voila_adam(ctypes.Structure):
    _fields_ = [("lr", c_float), ("beta1", c_float), ("beta2", c_float), ("eps", c_float), ("step", c_int32)]


class voila_pw_tree(ctypes.Structure):
    _fields_ = [("n_nodes", c_int32), ("d_a", c_int32), ("d_o", c_int32), ("C_max", c_int32), ("act", c_void_p),
                ("N", c_void_p), ("C", c_void_p), ("obs", c_void_p)]


def _sig(name, res, *args):
    f = getattr(_lib, name)
    f.restype = res
    f.argtypes = list(args)
    return f


_P = c_void_p
_lib_status_string = _sig("voila_status_string", ctypes.c_char_p, c_int32)
_lib_workspace_status = _sig("voila_workspace_status", c_int32, _P, _P)
_lib_rollout_ws = _sig("voila_rollout_workspace_size", c_int32, POINTER(voila_mlp), POINTER(voila_reward),
                       c_int32, c_int32, c_int32, POINTER(c_size_t))
_lib_rollout = _sig("voila_rollout", c_int32, POINTER(voila_mlp), POINTER(voila_reward), _P, _P, c_int32,
                    c_int32, _P, c_int32, c_int32, c_int32, c_int32, c_double, c_uint64, c_uint32, _P, _P,
                    _P, _P, c_size_t, _P)
_lib_rollout_shard = _sig("voila_rollout_shard", c_int32, POINTER(voila_mlp), POINTER(voila_reward), _P, _P,
                          c_int32, c_int32, c_int32, c_int32, _P, c_int32, c_int32, c_int32, c_int32, c_int32,
                          c_double, c_uint64, c_uint32, _P, _P, _P, _P, c_size_t, _P)
_lib_batched_ws = _sig("voila_rollout_batched_workspace_size", c_int32, POINTER(voila_mlp), POINTER(voila_reward),
                       POINTER(voila_planner), c_int32, POINTER(c_size_t))
_lib_batched = _sig("voila_rollout_batched", c_int32, POINTER(voila_mlp), POINTER(voila_reward), POINTER(voila_planner),
                    c_int32, c_int32, c_int32, c_int32, c_double, c_uint64, c_int32, _P, c_size_t, _P)
_lib_batched_tune = _sig("voila_rollout_batched_autotune", c_int32, POINTER(voila_mlp), POINTER(voila_reward),
                         POINTER(voila_planner), c_int32, c_int32, c_int32, c_int32, c_double, c_uint64, _P, c_size_t,
                         POINTER(c_int32), POINTER(c_float), _P)
_lib_belief_ws = _sig("voila_belief_update_workspace_size", c_int32, POINTER(voila_mlp),
                      POINTER(voila_likelihood), c_int32, POINTER(c_size_t))
_lib_belief = _sig("voila_belief_update", c_int32, POINTER(voila_mlp), POINTER(voila_likelihood), _P, _P,
                   c_int32, c_int32, _P, _P, c_int32, c_int32, c_int32, c_float, c_uint64, c_uint32,
                   c_uint32, _P, _P, _P, _P, _P, _P, c_size_t, _P)
_lib_belief_noalloc = _sig("voila_belief_update_noalloc", c_int32, POINTER(voila_mlp), POINTER(voila_likelihood),
                           _P, _P, c_int32, c_int32, _P, _P, c_int32, c_int32, c_int32, c_float, c_uint64,
                           c_uint32, c_uint32, _P, _P, _P, _P, _P, _P, _P)
_lib_fwd = _sig("voila_generator_fwd", c_int32, POINTER(voila_mlp), _P, c_int32, _P, _P)
_lib_fwd_seeded = _sig("voila_generator_fwd_seeded", c_int32, POINTER(voila_mlp), _P, _P, c_int32, c_int32,
                       c_int32, c_int32, c_int32, c_uint64, c_uint32, c_uint32, c_uint32, _P, _P)
_lib_fwd_train = _sig("voila_generator_fwd_train", c_int32, POINTER(voila_mlp), _P, c_int32, _P, _P, _P, c_size_t,
                      _P)
_lib_bwd_ws = _sig("voila_generator_bwd_workspace_size", c_int32, POINTER(voila_mlp), c_int32, POINTER(c_size_t))
_lib_bwd = _sig("voila_generator_bwd", c_int32, POINTER(voila_mlp), _P, _P, _P, c_int32, _P, POINTER(c_void_p),
                POINTER(c_void_p), _P, c_size_t, _P)
_lib_ddim_ws = _sig("voila_ddim_sample_workspace_size", c_int32, POINTER(voila_mlp), c_int32, POINTER(c_size_t))
_lib_ddim = _sig("voila_ddim_sample", c_int32, POINTER(voila_mlp), _P, _P, _P, c_int32, c_int32, c_int32, c_int32,
                 c_int32, c_double, c_double, c_int32, _P, _P, c_size_t, _P)
_lib_adam = _sig("voila_adam_step", c_int32, _P, _P, _P, _P, c_int64, c_float, c_float, c_float, c_float, c_int32, _P)
_lib_distill_ws = _sig("voila_distill_step_workspace_size", c_int32, POINTER(voila_mlp), POINTER(voila_mlp), c_int32,
                       c_int32, c_int32, POINTER(c_size_t))
_lib_distill = _sig("voila_distill_step", c_int32, POINTER(voila_mlp), POINTER(voila_mlp), POINTER(voila_ddim), _P, _P,
                    _P, POINTER(voila_adam), _P, _P, _P, c_int32, c_int32, c_int32, c_int32, _P, _P, _P, c_size_t, _P)
_lib_dtrain_ws = _sig("voila_distill_train_step_workspace_size", c_int32, POINTER(voila_mlp), c_int32, c_int32,
                      POINTER(c_size_t))
_lib_dtrain = _sig("voila_distill_train_step", c_int32, POINTER(voila_mlp), _P, _P, _P, POINTER(voila_adam), _P, _P,
                   _P, _P, c_int32, c_int32, c_int32, c_int32, c_int32, _P, _P, _P, c_size_t, _P)
_lib_load_flat = _sig("voila_mlp_load_flat", c_int32, POINTER(voila_mlp), _P, _P)
_lib_backup = _sig("voila_preference_backup", c_int32, _P, _P, c_int32, c_double, _P, _P, _P)
_lib_nce_ws = _sig("voila_infonce_workspace_size", c_int32, POINTER(voila_mlp), c_int32, POINTER(c_size_t))
_lib_nce_fwd = _sig("voila_infonce_forward", c_int32, POINTER(voila_mlp), _P, _P, _P, c_int32, c_int32, c_int32,
                    c_int32, _P, _P, _P, _P, _P, c_size_t, _P)
_lib_nce_step_ws = _sig("voila_infonce_step_workspace_size", c_int32, POINTER(voila_mlp), c_int32, POINTER(c_size_t))
_lib_nce_step = _sig("voila_infonce_step", c_int32, POINTER(voila_mlp), _P, _P, _P, POINTER(voila_adam), _P, _P, _P,
                     c_int32, c_int32, c_int32, c_int32, _P, _P, _P, c_size_t, _P)
_lib_pw_ws = _sig("voila_progressive_widening_workspace_size", c_int32, POINTER(voila_pw_tree), _P,
                  POINTER(voila_likelihood), c_int32, POINTER(c_size_t))
_lib_pw = _sig("voila_progressive_widening", c_int32, POINTER(voila_pw_tree), _P, _P, c_int32, c_int32,
               POINTER(voila_mlp), POINTER(voila_likelihood), c_int32, c_double, c_double, c_float, c_uint64,
               c_uint32, c_uint32, _P, _P, _P, _P, _P, _P, _P, c_size_t, _P)
_lib_philox = _sig("voila_philox_fill", c_int32, c_uint64, c_uint32, c_uint32, c_uint32, _P, c_int64, _P)
_lib_selftest_wait = _sig("voila_selftest_wait_timeout", c_int32, _P, c_int64, _P)
_lib_normal = _sig("voila_normal_fill", c_int32, c_uint64, c_uint32, c_uint32, c_uint32, c_uint32, c_int32,
                   _P, c_int64, _P)


class VoilaError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {status_string(code)} ({code})")


def status_string(code: int) -> str:
    return _lib_status_string(code).decode()


def _check(code: int, where: str):
    if code != OK:
        raise VoilaError(code, where)


def _ptr(t: Optional[torch.Tensor], dtype=None):
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"expected {dtype}, got {t.dtype}")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream) -> c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class DeviceMLP:
    """An MLP's weights on the device plus its voila_mlp descriptor.

    W[l] is [out, in] (float32 for FP32, bfloat16 for BF16), b[l] float32.
    """

    def __init__(self, W: Sequence[torch.Tensor], b: Sequence[torch.Tensor], act: int, prec: int):
        if len(W) != len(b) or not 1 <= len(W) <= MAX_LAYERS:
            raise ValueError("bad layer count")
        # the FP8 form takes BF16 weights; the library quantises its hidden layers
        wdt = {FP32: torch.float32, BF16: torch.bfloat16, FP8E4M3: torch.bfloat16}[prec]
        self.W = [w.to(device="cuda", dtype=wdt).contiguous() for w in W]
        self.b = [v.to(device="cuda", dtype=torch.float32).contiguous() for v in b]
        self.act, self.prec = act, prec
        self.desc = voila_mlp()
        self.desc.n_layers = len(W)
        dims = [self.W[0].shape[1]] + [w.shape[0] for w in self.W]
        for i, d in enumerate(dims):
            self.desc.dims[i] = d
        self.desc.act = act
        self.desc.prec = prec
        for l in range(len(W)):
            self.desc.W[l] = self.W[l].data_ptr()
            self.desc.b[l] = self.b[l].data_ptr()
        self.dims = dims

    @classmethod
    def from_spec(cls, spec) -> "DeviceMLP":
        """From an object with W, b (numpy FP64 arrays already rounded), act, prec."""
        return cls([torch.from_numpy(w) for w in spec.W], [torch.from_numpy(v) for v in spec.b],
                   spec.act, spec.prec)


def goal_reward(goal: Sequence[float]) -> voila_reward:
    r = voila_reward()
    r.kind = REWARD_GOAL
    r.goal_dims = len(goal)
    for i, g in enumerate(goal):
        r.goal[i] = float(g)
    return r


def mlp_reward(mlp: DeviceMLP) -> voila_reward:
    r = voila_reward()
    r.kind = REWARD_MLP
    r.mlp = ctypes.pointer(mlp.desc)
    r._keep = mlp
    return r


def mlp_likelihood(mlp: DeviceMLP) -> voila_likelihood:
    l = voila_likelihood()
    l.kind = LIK_MLP
    l.mlp = ctypes.pointer(mlp.desc)
    l._keep = mlp
    return l


def gaussian_likelihood(sigma: float) -> voila_likelihood:
    l = voila_likelihood()
    l.kind = LIK_GAUSSIAN
    l.sigma = sigma
    return l


def workspace_status(ws: torch.Tensor, stream=None) -> int:
    return _lib_workspace_status(_ptr(ws), _stream(stream))


def alloc_workspace(nbytes: int) -> torch.Tensor:
    """A 1024-byte aligned device workspace (a view into a slightly larger allocation)."""
    n = max(int(nbytes), 256)
    buf = torch.empty(n + 1024, dtype=torch.uint8, device="cuda")
    off = (-buf.data_ptr()) % 1024
    return buf[off:off + n]


# ---------------------------------------------------------------------------
# Entry points (same names as the C-ABI).
# ---------------------------------------------------------------------------
def voila_rollout_workspace_size(g_T: DeviceMLP, R: voila_reward, N: int, K: int, H: int) -> int:
    n = c_size_t(0)
    _check(_lib_rollout_ws(ctypes.byref(g_T.desc), ctypes.byref(R), N, K, H, ctypes.byref(n)),
           "voila_rollout_workspace_size")
    return n.value


def voila_rollout(g_T: DeviceMLP, R: voila_reward, particles: torch.Tensor, w: Optional[torch.Tensor],
                  actions: torch.Tensor, d_omega: int, gamma: float, seed: int, planner_id: int,
                  J: torch.Tensor, G: Optional[torch.Tensor], best_k: Optional[torch.Tensor],
                  workspace: torch.Tensor, stream=None):
    N, d_s = particles.shape
    K, H, d_a = actions.shape
    code = _lib_rollout(ctypes.byref(g_T.desc), ctypes.byref(R), _ptr(particles, torch.float32),
                        _ptr(w, torch.float64), N, d_s, _ptr(actions, torch.float32), K, H, d_a,
                        d_omega, gamma, seed, planner_id, _ptr(J, torch.float64),
                        _ptr(G, torch.float64), _ptr(best_k, torch.int32), _ptr(workspace),
                        workspace.numel(), _stream(stream))
    _check(code, "voila_rollout")


def voila_rollout_shard(g_T: DeviceMLP, R: voila_reward, particles: torch.Tensor, w: Optional[torch.Tensor],
                        n_offset: int, N_total: int, actions: torch.Tensor, k_offset: int, d_omega: int,
                        gamma: float, seed: int, planner_id: int, J: torch.Tensor, G: Optional[torch.Tensor],
                        best_k: Optional[torch.Tensor], workspace: torch.Tensor, stream=None):
    N, d_s = particles.shape
    K, H, d_a = actions.shape
    code = _lib_rollout_shard(ctypes.byref(g_T.desc), ctypes.byref(R), _ptr(particles, torch.float32),
                              _ptr(w, torch.float64), N, n_offset, N_total, d_s, _ptr(actions, torch.float32), K,
                              k_offset, H, d_a, d_omega, gamma, seed, planner_id, _ptr(J, torch.float64),
                              _ptr(G, torch.float64), _ptr(best_k, torch.int32), _ptr(workspace),
                              workspace.numel(), _stream(stream))
    _check(code, "voila_rollout_shard")


SCHED_LONGEST_FIRST = 1


def make_planners(items) -> "ctypes.Array":
    """items: sequence of dicts with particles, actions, J (tensors) and optional w, G, best_k, planner_id."""
    arr = (voila_planner * len(items))()
    for i, it in enumerate(items):
        N = it["particles"].shape[0]
        K, H = it["actions"].shape[0], it["actions"].shape[1]
        arr[i].particles = _ptr(it["particles"], torch.float32)
        arr[i].w = _ptr(it.get("w"), torch.float64)
        arr[i].actions = _ptr(it["actions"], torch.float32)
        arr[i].N, arr[i].K, arr[i].H = N, K, H
        arr[i].planner_id = it.get("planner_id", i)
        arr[i].J = _ptr(it["J"], torch.float64)
        arr[i].G = _ptr(it.get("G"), torch.float64)
        arr[i].best_k = _ptr(it.get("best_k"), torch.int32)
    return arr


def voila_rollout_batched_workspace_size(g_T: DeviceMLP, R: voila_reward, planners) -> int:
    n = c_size_t(0)
    _check(_lib_batched_ws(ctypes.byref(g_T.desc), ctypes.byref(R), planners, len(planners), ctypes.byref(n)),
           "voila_rollout_batched_workspace_size")
    return n.value


def voila_rollout_batched(g_T: DeviceMLP, R: voila_reward, planners, d_s: int, d_a: int, d_omega: int,
                          gamma: float, seed: int, schedule: int, workspace: torch.Tensor, stream=None):
    _check(_lib_batched(ctypes.byref(g_T.desc), ctypes.byref(R), planners, len(planners), d_s, d_a, d_omega, gamma,
                        seed, schedule, _ptr(workspace), workspace.numel(), _stream(stream)), "voila_rollout_batched")


def voila_rollout_batched_autotune(g_T: DeviceMLP, R: voila_reward, planners, d_s: int, d_a: int, d_omega: int,
                                   gamma: float, seed: int, workspace: torch.Tensor, stream=None):
    best = c_int32(0)
    ms = c_float(0.0)
    _check(_lib_batched_tune(ctypes.byref(g_T.desc), ctypes.byref(R), planners, len(planners), d_s, d_a, d_omega,
                             gamma, seed, _ptr(workspace), workspace.numel(), ctypes.byref(best), ctypes.byref(ms),
                             _stream(stream)), "voila_rollout_batched_autotune")
    return best.value, ms.value


def voila_belief_update_workspace_size(g_T: DeviceMLP, ell: voila_likelihood, N: int) -> int:
    n = c_size_t(0)
    _check(_lib_belief_ws(ctypes.byref(g_T.desc), ctypes.byref(ell), N, ctypes.byref(n)),
           "voila_belief_update_workspace_size")
    return n.value


def voila_belief_update(g_T: DeviceMLP, ell: voila_likelihood, particles_in: torch.Tensor,
                        logw_in: Optional[torch.Tensor], action: torch.Tensor, obs: torch.Tensor,
                        d_omega: int, lam: float, seed: int, step: int, planner_id: int,
                        particles_out: torch.Tensor, idx_out: Optional[torch.Tensor],
                        w_out: Optional[torch.Tensor], logZ_out: Optional[torch.Tensor],
                        ess_out: Optional[torch.Tensor], workspace: torch.Tensor, stream=None):
    N, d_s = particles_in.shape
    code = _lib_belief(ctypes.byref(g_T.desc), ctypes.byref(ell), _ptr(particles_in, torch.float32),
                       _ptr(logw_in, torch.float64), N, d_s, _ptr(action, torch.float32),
                       _ptr(obs, torch.float32), action.numel(), obs.numel(), d_omega, lam, seed, step,
                       planner_id, _ptr(particles_out, torch.float32), _ptr(idx_out, torch.int32),
                       _ptr(w_out, torch.float64), _ptr(logZ_out, torch.float64),
                       _ptr(ess_out, torch.float64), _ptr(workspace), workspace.numel(), _stream(stream))
    _check(code, "voila_belief_update")


def voila_belief_update_noalloc(g_T: DeviceMLP, ell: voila_likelihood, particles_in: torch.Tensor,
                                logw_in: Optional[torch.Tensor], action: torch.Tensor, obs: torch.Tensor,
                                d_omega: int, lam: float, seed: int, step: int, planner_id: int,
                                particles_out: torch.Tensor, idx_out: Optional[torch.Tensor],
                                w_out: Optional[torch.Tensor], logZ_out: Optional[torch.Tensor],
                                ess_out: Optional[torch.Tensor], status_out: Optional[torch.Tensor],
                                stream=None):
    """voila_belief_update without a workspace: the library's fixed device scratch is used."""
    N, d_s = particles_in.shape
    code = _lib_belief_noalloc(ctypes.byref(g_T.desc), ctypes.byref(ell), _ptr(particles_in, torch.float32),
                               _ptr(logw_in, torch.float64), N, d_s, _ptr(action, torch.float32),
                               _ptr(obs, torch.float32), action.numel(), obs.numel(), d_omega, lam, seed,
                               step, planner_id, _ptr(particles_out, torch.float32), _ptr(idx_out, torch.int32),
                               _ptr(w_out, torch.float64), _ptr(logZ_out, torch.float64),
                               _ptr(ess_out, torch.float64), _ptr(status_out, torch.int32), _stream(stream))
    _check(code, "voila_belief_update_noalloc")


def voila_generator_fwd(mlp: DeviceMLP, X: torch.Tensor, Y: torch.Tensor, stream=None):
    _check(_lib_fwd(ctypes.byref(mlp.desc), _ptr(X, torch.float32), X.shape[0], _ptr(Y, torch.float32),
                    _stream(stream)), "voila_generator_fwd")


def voila_generator_fwd_seeded(mlp: DeviceMLP, S: torch.Tensor, A: torch.Tensor, a_stride: int,
                               d_omega: int, seed: int, stream_id: int, step: int, planner_id: int,
                               Y: torch.Tensor, stream=None):
    B, d_s = S.shape
    d_a = A.shape[-1]
    _check(_lib_fwd_seeded(ctypes.byref(mlp.desc), _ptr(S, torch.float32), _ptr(A, torch.float32), a_stride,
                           B, d_s, d_a, d_omega, seed, stream_id, step, planner_id, _ptr(Y, torch.float32),
                           _stream(stream)), "voila_generator_fwd_seeded")


def voila_selftest_wait_timeout(workspace: torch.Tensor, limit_cycles: int, stream=None):
    """A bounded wait that nothing completes; afterwards the workspace status is VOILA_ERR_TIMEOUT."""
    _check(_lib_selftest_wait(_ptr(workspace), limit_cycles, _stream(stream)), "voila_selftest_wait_timeout")


def voila_philox_fill(seed: int, c1: int, c2: int, c3: int, out: torch.Tensor, stream=None):
    _check(_lib_philox(seed, c1, c2, c3, _ptr(out, torch.int32), out.numel() // 4, _stream(stream)),
           "voila_philox_fill")


def voila_normal_fill(seed: int, c1: int, c2: int, stream_id: int, planner_id: int, out: torch.Tensor,
                      stream=None):
    n, dim = out.shape
    _check(_lib_normal(seed, c1, c2, stream_id, planner_id, dim, _ptr(out, torch.float32), n, _stream(stream)),
           "voila_normal_fill")


def voila_generator_fwd_train(mlp: DeviceMLP, X: torch.Tensor, Y: torch.Tensor, saved: Optional[torch.Tensor],
                              workspace: torch.Tensor, stream=None):
    _check(_lib_fwd_train(ctypes.byref(mlp.desc), _ptr(X, torch.float32), X.shape[0], _ptr(Y, torch.float32),
                          _ptr(saved, torch.float32), _ptr(workspace), workspace.numel(), _stream(stream)),
           "voila_generator_fwd_train")


def voila_generator_bwd_workspace_size(mlp: DeviceMLP, B: int) -> int:
    n = c_size_t(0)
    _check(_lib_bwd_ws(ctypes.byref(mlp.desc), B, ctypes.byref(n)), "voila_generator_bwd_workspace_size")
    return n.value


def voila_generator_bwd(mlp: DeviceMLP, X: torch.Tensor, saved: Optional[torch.Tensor], dY: torch.Tensor,
                        dX: Optional[torch.Tensor], dW: Sequence[torch.Tensor], db: Sequence[torch.Tensor],
                        workspace: torch.Tensor, stream=None):
    L = len(mlp.W)
    if len(dW) != L or len(db) != L:
        raise ValueError("one dW and one db per layer")
    pw = (c_void_p * L)(*[_ptr(x, torch.float32).value for x in dW])
    pb = (c_void_p * L)(*[_ptr(x, torch.float32).value for x in db])
    _check(_lib_bwd(ctypes.byref(mlp.desc), _ptr(X, torch.float32), _ptr(saved, torch.float32),
                    _ptr(dY, torch.float32), X.shape[0], _ptr(dX, torch.float32), pw, pb, _ptr(workspace),
                    workspace.numel(), _stream(stream)), "voila_generator_bwd")


def voila_ddim_sample_workspace_size(teacher: DeviceMLP, T: int) -> int:
    n = c_size_t(0)
    _check(_lib_ddim_ws(ctypes.byref(teacher.desc), T, ctypes.byref(n)), "voila_ddim_sample_workspace_size")
    return n.value


def voila_ddim_sample(teacher: DeviceMLP, S: torch.Tensor, A: torch.Tensor, omega: torch.Tensor, T: int,
                      beta0: float, beta1: float, emb_dim: int, Y: torch.Tensor,
                      workspace: Optional[torch.Tensor] = None, stream=None):
    """Teacher DDIM targets; allocates the workspace when none is given."""
    B, d_x = omega.shape
    if workspace is None:
        workspace = alloc_workspace(voila_ddim_sample_workspace_size(teacher, T))
    _check(_lib_ddim(ctypes.byref(teacher.desc), _ptr(S, torch.float32), _ptr(A, torch.float32),
                     _ptr(omega, torch.float32), B, S.shape[1], A.shape[1], d_x, T, beta0, beta1, emb_dim,
                     _ptr(Y, torch.float32), _ptr(workspace), workspace.numel(), _stream(stream)),
           "voila_ddim_sample")


def voila_adam_step(params: torch.Tensor, grads: torch.Tensor, m: torch.Tensor, v: torch.Tensor, lr: float,
                    beta1: float, beta2: float, eps: float, step: int, stream=None):
    _check(_lib_adam(_ptr(params, torch.float32), _ptr(grads, torch.float32), _ptr(m, torch.float32),
                     _ptr(v, torch.float32), params.numel(), lr, beta1, beta2, eps, step, _stream(stream)),
           "voila_adam_step")


def voila_distill_step_workspace_size(teacher: DeviceMLP, student: DeviceMLP, B: int, d_x: int, T: int) -> int:
    n = c_size_t(0)
    _check(_lib_distill_ws(ctypes.byref(teacher.desc), ctypes.byref(student.desc), B, d_x, T, ctypes.byref(n)),
           "voila_distill_step_workspace_size")
    return n.value


def voila_distill_step(teacher: DeviceMLP, student: DeviceMLP, ddim: voila_ddim, master: torch.Tensor,
                       adam_m: torch.Tensor, adam_v: torch.Tensor, opt: voila_adam, S: torch.Tensor,
                       A: torch.Tensor, omega: torch.Tensor, loss_out: torch.Tensor,
                       grad_out: Optional[torch.Tensor], workspace: torch.Tensor, stream=None):
    B, d_x = omega.shape
    _check(_lib_distill(ctypes.byref(teacher.desc), ctypes.byref(student.desc), ctypes.byref(ddim),
                        _ptr(master, torch.float32), _ptr(adam_m, torch.float32), _ptr(adam_v, torch.float32),
                        ctypes.byref(opt), _ptr(S, torch.float32), _ptr(A, torch.float32),
                        _ptr(omega, torch.float32), B, S.shape[1], A.shape[1], d_x, _ptr(loss_out, torch.float64),
                        _ptr(grad_out, torch.float32), _ptr(workspace), workspace.numel(), _stream(stream)),
           "voila_distill_step")


TRAIN_SPREAD = 1  # VOILA_TRAIN_SPREAD


def voila_distill_train_step_workspace_size(student: DeviceMLP, B: int, d_x: int) -> int:
    n = c_size_t(0)
    _check(_lib_dtrain_ws(ctypes.byref(student.desc), B, d_x, ctypes.byref(n)),
           "voila_distill_train_step_workspace_size")
    return n.value


def voila_distill_train_step(student: DeviceMLP, master: torch.Tensor, adam_m: torch.Tensor, adam_v: torch.Tensor,
                             opt: voila_adam, S: torch.Tensor, A: torch.Tensor, omega: torch.Tensor,
                             s_hat: torch.Tensor, flags: int, loss_out: torch.Tensor,
                             grad_out: Optional[torch.Tensor], workspace: torch.Tensor, stream=None):
    B, d_x = omega.shape
    _check(_lib_dtrain(ctypes.byref(student.desc), _ptr(master, torch.float32), _ptr(adam_m, torch.float32),
                       _ptr(adam_v, torch.float32), ctypes.byref(opt), _ptr(S, torch.float32),
                       _ptr(A, torch.float32), _ptr(omega, torch.float32), _ptr(s_hat, torch.float32), B,
                       S.shape[1], A.shape[1], d_x, flags, _ptr(loss_out, torch.float64),
                       _ptr(grad_out, torch.float32), _ptr(workspace), workspace.numel(), _stream(stream)),
           "voila_distill_train_step")


def voila_mlp_load_flat(mlp: DeviceMLP, flat: torch.Tensor, stream=None):
    _check(_lib_load_flat(ctypes.byref(mlp.desc), _ptr(flat, torch.float32), _stream(stream)), "voila_mlp_load_flat")


def voila_preference_backup(J: torch.Tensor, log_pi0: Optional[torch.Tensor], eta: float, V: torch.Tensor,
                            pi: Optional[torch.Tensor], stream=None):
    _check(_lib_backup(_ptr(J, torch.float64), _ptr(log_pi0, torch.float64), J.numel(), eta, _ptr(V, torch.float64),
                       _ptr(pi, torch.float64), _stream(stream)), "voila_preference_backup")


def voila_infonce_workspace_size(ell: DeviceMLP, B: int) -> int:
    n = c_size_t(0)
    _check(_lib_nce_ws(ctypes.byref(ell.desc), B, ctypes.byref(n)), "voila_infonce_workspace_size")
    return n.value


def voila_infonce_forward(ell: DeviceMLP, S: torch.Tensor, A: torch.Tensor, Ob: torch.Tensor,
                          L: Optional[torch.Tensor], lse: Optional[torch.Tensor], loss: torch.Tensor,
                          G: Optional[torch.Tensor], workspace: torch.Tensor, stream=None):
    B = S.shape[0]
    _check(_lib_nce_fwd(ctypes.byref(ell.desc), _ptr(S, torch.float32), _ptr(A, torch.float32),
                        _ptr(Ob, torch.float32), B, S.shape[1], A.shape[1], Ob.shape[1], _ptr(L, torch.float32),
                        _ptr(lse, torch.float64), _ptr(loss, torch.float64), _ptr(G, torch.float32),
                        _ptr(workspace), workspace.numel(), _stream(stream)), "voila_infonce_forward")


def voila_infonce_step_workspace_size(ell: DeviceMLP, B: int) -> int:
    n = c_size_t(0)
    _check(_lib_nce_step_ws(ctypes.byref(ell.desc), B, ctypes.byref(n)), "voila_infonce_step_workspace_size")
    return n.value


def voila_infonce_step(ell: DeviceMLP, master: torch.Tensor, adam_m: torch.Tensor, adam_v: torch.Tensor,
                       opt: voila_adam, S: torch.Tensor, A: torch.Tensor, Ob: torch.Tensor, loss: torch.Tensor,
                       grad_out: Optional[torch.Tensor], workspace: torch.Tensor, stream=None):
    B = S.shape[0]
    _check(_lib_nce_step(ctypes.byref(ell.desc), _ptr(master, torch.float32), _ptr(adam_m, torch.float32),
                         _ptr(adam_v, torch.float32), ctypes.byref(opt), _ptr(S, torch.float32),
                         _ptr(A, torch.float32), _ptr(Ob, torch.float32), B, S.shape[1], A.shape[1], Ob.shape[1],
                         _ptr(loss, torch.float64), _ptr(grad_out, torch.float32), _ptr(workspace),
                         workspace.numel(), _stream(stream)), "voila_infonce_step")


class PWTree:
    """Device action-node tensors for progressive widening (act, N, C, obs)."""

    def __init__(self, act: torch.Tensor, N: torch.Tensor, C: torch.Tensor, obs: torch.Tensor):
        self.act = act.to(device="cuda", dtype=torch.float32).contiguous()
        self.N = N.to(device="cuda", dtype=torch.int64).contiguous()
        self.C = C.to(device="cuda", dtype=torch.int32).contiguous()
        self.obs = obs.to(device="cuda", dtype=torch.float32).contiguous()
        self.desc = voila_pw_tree()
        self.desc.n_nodes = self.act.shape[0]
        self.desc.d_a = self.act.shape[1]
        self.desc.d_o = self.obs.shape[2]
        self.desc.C_max = self.obs.shape[1]
        self.desc.act = self.act.data_ptr()
        self.desc.N = self.N.data_ptr()
        self.desc.C = self.C.data_ptr()
        self.desc.obs = self.obs.data_ptr()


def voila_progressive_widening_workspace_size(tree: "PWTree", g_Z: Optional[DeviceMLP], ell: voila_likelihood,
                                              M: int) -> int:
    n = c_size_t(0)
    gz = ctypes.cast(ctypes.byref(g_Z.desc), ctypes.c_void_p) if g_Z is not None else None
    _check(_lib_pw_ws(ctypes.byref(tree.desc), gz, ctypes.byref(ell), M, ctypes.byref(n)),
           "voila_progressive_widening_workspace_size")
    return n.value


def voila_progressive_widening(tree: PWTree, node: torch.Tensor, s_next: torch.Tensor, g_Z: DeviceMLP,
                               ell: voila_likelihood, d_omega: int, k_o: float, alpha_o: float, lam: float, seed: int,
                               step: int, planner_id: int, branch: torch.Tensor, s_out: torch.Tensor,
                               workspace: torch.Tensor, widened: Optional[torch.Tensor] = None,
                               ell_out: Optional[torch.Tensor] = None, w: Optional[torch.Tensor] = None,
                               idx: Optional[torch.Tensor] = None, stream=None):
    M, d_s = s_next.shape
    _check(_lib_pw(ctypes.byref(tree.desc), _ptr(node, torch.int32), _ptr(s_next, torch.float32), M, d_s,
                   ctypes.byref(g_Z.desc), ctypes.byref(ell), d_omega, k_o, alpha_o, lam, seed, step, planner_id,
                   _ptr(branch, torch.int32), _ptr(widened, torch.uint8), _ptr(ell_out, torch.float32),
                   _ptr(w, torch.float64), _ptr(idx, torch.int32), _ptr(s_out, torch.float32), _ptr(workspace),
                   workspace.numel(), _stream(stream)), "voila_progressive_widening")
