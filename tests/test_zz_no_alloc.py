"""The allocation-free belief update (voila_belief_update_noalloc).

Some callers cannot allocate device memory, for example a control loop that
forbids allocation once it runs or a plug-in inside a framework that owns all
device memory. They call the variant that keeps its scratch in a fixed array
inside the library. These tests check, through the C-ABI, that it returns what
the workspace entry point returns on the same inputs, for two calls in a row
(the second call must not see the first call's leftovers), and that sizes
beyond the fixed array are refused before any device work.

This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

from oracle import voila_oracle as O
from paper_2606_19729_b300 import workloads as WL
from tests.helpers import cuda, oracle_mlp

TOL_FP32 = 1e-5


@pytest.fixture(scope="module")
def V():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_19729_b300 import voila
    return voila


def _outputs(N, d_s):
    return (torch.empty((N, d_s), dtype=torch.float32, device="cuda"),
            torch.empty(N, dtype=torch.int32, device="cuda"),
            torch.empty(N, dtype=torch.float64, device="cuda"),
            torch.empty(1, dtype=torch.float64, device="cuda"),
            torch.empty(1, dtype=torch.float64, device="cuda"))


def _case(V, wl, lik, N, lam, step, logw=None):
    g = V.DeviceMLP.from_spec(wl.g_T)
    parts = cuda(wl.particles[:N])
    a = cuda(wl.actions[0, 0])
    o = cuda(np.linspace(-0.3, 0.4, wl.d_o))
    lw = None if logw is None else cuda(logw, torch.float64)
    ref = _outputs(N, wl.d_s)
    ws = V.alloc_workspace(V.voila_belief_update_workspace_size(g, lik, N))
    V.voila_belief_update(g, lik, parts, lw, a, o, wl.d_omega, lam, wl.seed, step, 0, *ref, ws)
    assert V.workspace_status(ws) == V.OK
    got = _outputs(N, wl.d_s)
    status = torch.full((1,), 99, dtype=torch.int32, device="cuda")
    V.voila_belief_update_noalloc(g, lik, parts, lw, a, o, wl.d_omega, lam, wl.seed, step, 0, *got, status)
    torch.cuda.synchronize()
    assert int(status.item()) == V.OK
    return [t.cpu().numpy() for t in ref], [t.cpu().numpy() for t in got]


def _same(ref, got):
    for r, g in zip(ref, got):
        if r.dtype.kind in "iu":
            assert np.array_equal(r, g)
        else:
            np.testing.assert_allclose(g, r, rtol=TOL_FP32, atol=1e-12)


@pytest.mark.gpu
def test_noalloc_matches_workspace_entry_point_twice(V):
    wl = WL.small_fp32(N=1500)
    # first call: Gaussian likelihood, sharp weights, with prior log-weights
    logw = np.log(np.random.default_rng(4).dirichlet(np.ones(1500)))
    ref, got = _case(V, wl, V.gaussian_likelihood(0.3), 1500, 1.0, 2, logw)
    _same(ref, got)
    # second call in a row: smaller N and an MLP likelihood on the same scratch
    ell = V.DeviceMLP.from_spec(wl.ell)
    ref2, got2 = _case(V, wl, V.mlp_likelihood(ell), 257, 1.25, 3)
    _same(ref2, got2)
    # and the result is the oracle's (weights within FP32 tolerance, indices exact given them)
    res = O.belief_update(oracle_mlp(wl.g_T), O.Likelihood(O.LIK_MLP, mlp=oracle_mlp(wl.ell)),
                          wl.particles[:257], wl.actions[0, 0], np.linspace(-0.3, 0.4, wl.d_o).astype(np.float32),
                          wl.d_omega, 1.25, wl.seed, 3)
    assert np.max(np.abs(got2[2] - res.w)) < TOL_FP32
    assert np.array_equal(got2[1], O.systematic_resample(got2[2], res.u0))


@pytest.mark.gpu
def test_noalloc_reports_device_status_and_refuses_oversize(V):
    wl = WL.small_fp32(N=64)
    g = V.DeviceMLP.from_spec(wl.g_T)
    lik = V.gaussian_likelihood(0.5)
    out = _outputs(64, wl.d_s)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    logw = torch.full((64,), -float("inf"), dtype=torch.float64, device="cuda")
    V.voila_belief_update_noalloc(g, lik, cuda(wl.particles), logw, cuda(wl.actions[0, 0]), cuda(np.zeros(4)),
                                  wl.d_omega, 1.0, 0, 0, 0, *out, status)
    torch.cuda.synchronize()
    assert int(status.item()) == V.ERR_DEGENERATE
    # more particles than the fixed scratch holds: refused on the host
    N_big = 200000
    big = torch.zeros((N_big, wl.d_s), dtype=torch.float32, device="cuda")
    outs = _outputs(N_big, wl.d_s)
    with pytest.raises(V.VoilaError) as e:
        V.voila_belief_update_noalloc(g, lik, big, None, cuda(wl.actions[0, 0]), cuda(np.zeros(4)), wl.d_omega,
                                      1.0, 0, 0, 0, *outs, status)
    assert e.value.code == V.ERR_WORKSPACE


def _largest_n(V, g, lik, cap):
    """The largest particle count whose belief-update workspace fits `cap` bytes."""
    lo, hi = 1, 1 << 20
    while lo < hi:
        mid = (lo + hi + 1) // 2
        if V.voila_belief_update_workspace_size(g, lik, mid) <= cap:
            lo = mid
        else:
            hi = mid - 1
    return lo


@pytest.mark.gpu
def test_noalloc_bf16_tensor_core_proposal_up_to_the_limit(V):
    # BF16 generator and likelihood of the tensor-core shapes: the packed weights
    # share the fixed array with the particle scratch, and above 2048 particles
    # the resampling runs in many CTAs; both run here through the fixed array,
    # twice in a row, at the largest N it holds and one particle more
    wl = WL.mid_bf16(N=80000, K=1, H=1)
    g = V.DeviceMLP.from_spec(wl.g_T)
    lik = V.mlp_likelihood(V.DeviceMLP.from_spec(wl.ell))
    cap = 4 << 20  # VOILA_NOALLOC_SCRATCH_BYTES
    n_max = _largest_n(V, g, lik, cap)
    assert 50000 < n_max < 80000
    for N, lam, step in ((4096, 1.0, 1), (n_max, 0.5, 2)):
        ref, got = _case(V, wl, lik, N, lam, step)
        _same(ref, got)
        # indices: the systematic resampling of the device's own weights
        u0 = O.resample_uniform(wl.seed, step, 0)
        assert np.array_equal(got[1], O.systematic_resample(got[2], u0))
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    outs = _outputs(n_max + 1, wl.d_s)
    with pytest.raises(V.VoilaError) as e:
        V.voila_belief_update_noalloc(g, lik, cuda(wl.particles[:n_max + 1]), None, cuda(wl.actions[0, 0]),
                                      cuda(np.zeros(wl.d_o)), wl.d_omega, 1.0, wl.seed, 3, 0, *outs, status)
    assert e.value.code == V.ERR_WORKSPACE
