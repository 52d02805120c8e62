"""Stored oracle fixtures (tests/golden/, written by tests/golden/make_golden.py
from the FP64 oracle alone).

CPU: the oracle reproduces every stored value (integers and random words bit
for bit, floats to 1e-12), so an edit that changes its arithmetic has to come
with regenerated fixtures (and a stated reason). GPU: the device path against the stored values, with no oracle run:
the FP32 rollout and belief update (1e-5 relative, the FP32 bound) and the
Philox words (bit-exact)."""
import json
import os

import numpy as np
import pytest
import torch

from oracle import voila_oracle as O
from paper_2606_19729_b300 import workloads as WL
from tests.golden import make_golden as MG
from tests.helpers import cuda

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
TOL_FP32 = 1e-5


def _load(name):
    with open(os.path.join(HERE, name)) as f:
        return json.load(f)


def _unhex(xs):
    return np.array([float.fromhex(x) for x in xs], np.float64)


def test_golden_step_reproduced_by_oracle():
    # floats to 1e-12 relative: the library matmul's summation order may differ
    # between CPUs in the last bits; the indices exactly
    now, ref = MG.small_fp32_step(), _load("small_fp32_step.json")
    assert now["case"] == ref["case"] and now["G_shape"] == ref["G_shape"] and now["idx"] == ref["idx"]
    for key in ("J", "G", "w", "s_prop"):
        np.testing.assert_allclose(_unhex(now[key]), _unhex(ref[key]), rtol=1e-12, atol=1e-15)
    for key in ("logZ", "ess", "u0"):
        assert abs(float.fromhex(now[key]) - float.fromhex(ref[key])) <= 1e-12 * abs(float.fromhex(ref[key]))
    assert now["u0"] == ref["u0"]  # 53 random bits, exact


def test_golden_philox_reproduced_by_oracle():
    assert MG.philox_words() == _load("philox_words.json")


def test_golden_step_invariants():
    g = _load("small_fp32_step.json")
    w = _unhex(g["w"])
    assert abs(w.sum() - 1.0) <= len(w) * 2.0 ** -52
    assert np.all(w * 2.0 ** 52 == np.rint(w * 2.0 ** 52))
    assert g["idx"] == sorted(g["idx"])  # systematic resampling returns a non-decreasing index list
    assert 1.0 <= float.fromhex(g["ess"]) <= len(w)


@pytest.fixture(scope="module")
def V():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_19729_b300 import voila
    return voila


@pytest.mark.gpu
def test_golden_device_rollout_and_belief(V):
    g = _load("small_fp32_step.json")
    c = g["case"]
    wl = WL.small_fp32(N=c["N"], K=c["K"], H=c["H"])
    gm = V.DeviceMLP.from_spec(wl.g_T)
    rm = V.DeviceMLP.from_spec(wl.reward_mlp)
    R = V.mlp_reward(rm)
    N, K, H = c["N"], c["K"], c["H"]
    J = torch.empty(K, dtype=torch.float64, device="cuda")
    G = torch.empty((K, N), dtype=torch.float64, device="cuda")
    ws = V.alloc_workspace(V.voila_rollout_workspace_size(gm, R, N, K, H))
    V.voila_rollout(gm, R, cuda(wl.particles), None, cuda(wl.actions), wl.d_omega, wl.gamma, wl.seed, 0, J, G,
                    None, ws)
    assert V.workspace_status(ws) == V.OK
    Jg, Gg = _unhex(g["J"]), _unhex(g["G"]).reshape(g["G_shape"])
    np.testing.assert_allclose(J.cpu().numpy(), Jg, rtol=TOL_FP32, atol=TOL_FP32 * np.max(np.abs(Jg)))
    np.testing.assert_allclose(G.cpu().numpy(), Gg, rtol=TOL_FP32, atol=TOL_FP32 * np.max(np.abs(Gg)))

    lm = V.DeviceMLP.from_spec(wl.ell)
    lik = V.mlp_likelihood(lm)
    out = torch.empty((N, wl.d_s), dtype=torch.float32, device="cuda")
    idx = torch.empty(N, dtype=torch.int32, device="cuda")
    w = torch.empty(N, dtype=torch.float64, device="cuda")
    lz = torch.empty(1, dtype=torch.float64, device="cuda")
    ess = torch.empty(1, dtype=torch.float64, device="cuda")
    wsb = V.alloc_workspace(V.voila_belief_update_workspace_size(gm, lik, N))
    V.voila_belief_update(gm, lik, cuda(wl.particles), None, cuda(wl.actions[0, 0]), cuda(np.array(c["obs"])),
                          wl.d_omega, c["lam"], wl.seed, c["step"], 0, out, idx, w, lz, ess, wsb)
    assert V.workspace_status(wsb) == V.OK
    wd = w.cpu().numpy()
    np.testing.assert_allclose(wd, _unhex(g["w"]), rtol=TOL_FP32, atol=TOL_FP32 / N)
    assert abs(lz.item() - float.fromhex(g["logZ"])) <= TOL_FP32 * max(1.0, abs(float.fromhex(g["logZ"])))
    assert abs(ess.item() - float.fromhex(g["ess"])) <= 10 * TOL_FP32 * float.fromhex(g["ess"])
    # indices: systematic resampling of the device's own weights with the stored u0
    assert np.array_equal(idx.cpu().numpy(), O.systematic_resample(wd, float.fromhex(g["u0"])))
    s_prop = _unhex(g["s_prop"]).reshape(N, wl.d_s)
    np.testing.assert_allclose(out.cpu().numpy(), s_prop[idx.cpu().numpy()], rtol=TOL_FP32, atol=TOL_FP32)


@pytest.mark.gpu
def test_golden_device_philox_words(V):
    for case in _load("philox_words.json"):
        if case["c0"] >= 65536:
            continue  # the fill call covers counter words 0 .. n - 1
        c3 = O.counter_word3(case["stream"], case["planner"], case["block"])
        out = torch.empty(4 * (case["c0"] + 1), dtype=torch.int32, device="cuda")
        V.voila_philox_fill(case["seed"], case["c1"], case["c2"], c3, out)
        got = out.cpu().numpy().view(np.uint32)[4 * case["c0"]: 4 * case["c0"] + 4]
        assert [int(x) for x in got] == case["words"]
