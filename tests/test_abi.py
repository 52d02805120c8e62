"""The C-ABI library loads and exports every entry point include/voila.h declares
(CPU only: no call here reaches the device)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "voila.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(voila_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ["voila_rollout", "voila_belief_update", "voila_generator_fwd", "voila_philox_fill",
              "voila_rollout_workspace_size", "voila_belief_update_workspace_size"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2606_19729_b300 import voila as V
    lib = ctypes.CDLL(V.LIB_PATH)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_and_host_validation():
    from paper_2606_19729_b300 import voila as V
    assert V.status_string(V.OK) == "ok"
    assert "workspace" in V.status_string(V.ERR_WORKSPACE)
    m = V.voila_mlp()
    m.n_layers = 0   # invalid descriptor: rejected on the host
    r = V.goal_reward([1.0, 1.0])
    n = ctypes.c_size_t(0)
    assert V._lib_rollout_ws(ctypes.byref(m), ctypes.byref(r), 4, 4, 4, ctypes.byref(n)) == V.ERR_ARG
    assert V._lib_rollout(ctypes.byref(m), ctypes.byref(r), None, None, 4, 4, None, 4, 4, 2, 4, 0.9, 0, 0,
                          None, None, None, None, 0, None) == V.ERR_ARG
    assert V._lib_philox(0, 0, 0, 0, None, -1, None) == V.ERR_ARG
    assert V._lib_selftest_wait(None, 5, None) == V.ERR_ARG
    assert V._lib_normal(0, 0, 0, 0, 0, 0, None, 1, None) == V.ERR_ARG


def test_workspace_sizes_are_host_computable():
    from paper_2606_19729_b300 import voila as V
    m = V.voila_mlp()
    m.n_layers = 3
    for i, d in enumerate([10, 64, 64, 4]):
        m.dims[i] = d
    m.act, m.prec = V.ACT_TANH, V.FP32
    for l in range(3):
        m.W[l] = 16  # never dereferenced on the host
        m.b[l] = 16
    r = V.goal_reward([1.0, 1.0])
    n = ctypes.c_size_t(0)
    assert V._lib_rollout_ws(ctypes.byref(m), ctypes.byref(r), 256, 64, 10, ctypes.byref(n)) == V.OK
    assert n.value >= 256 * 64 * 8
    lik = V.gaussian_likelihood(0.5)
    assert V._lib_belief_ws(ctypes.byref(m), ctypes.byref(lik), 256, ctypes.byref(n)) == V.OK
    assert n.value >= 256 * (4 * 4 + 16)


def test_distill_train_step_host_validation():
    # the student's half of a distillation step: workspace size computable on the
    # host, unknown flags and missing pointers refused before any device work
    from paper_2606_19729_b300 import voila as V
    m = V.voila_mlp()
    m.n_layers = 4
    for i, d in enumerate([18, 256, 256, 256, 8]):
        m.dims[i] = d
    m.act, m.prec = V.ACT_SILU, V.BF16
    for l in range(4):
        m.W[l] = 16  # never dereferenced on the host
        m.b[l] = 16
    n = ctypes.c_size_t(0)
    assert V._lib_dtrain_ws(ctypes.byref(m), 65536, 8, ctypes.byref(n)) == V.OK
    small = n.value
    assert V._lib_dtrain_ws(ctypes.byref(m), 131072, 8, ctypes.byref(n)) == V.OK and n.value > small
    assert V._lib_dtrain_ws(ctypes.byref(m), -1, 8, ctypes.byref(n)) == V.ERR_ARG
    opt = V.voila_adam(1e-3, 0.9, 0.999, 1e-8, 1)
    p = ctypes.c_void_p(16)
    args = [ctypes.byref(m), p, p, p, ctypes.byref(opt), p, p, p, p, 64, 8, 2, 8]
    # unknown flag bits
    assert V._lib_dtrain(*args, 2, p, None, p, small, None) == V.ERR_ARG
    # no loss output
    assert V._lib_dtrain(*args, V.TRAIN_SPREAD, None, None, p, small, None) == V.ERR_ARG
    # widths that do not match the student
    bad = [ctypes.byref(m), p, p, p, ctypes.byref(opt), p, p, p, p, 64, 8, 3, 8]
    assert V._lib_dtrain(*bad, 0, p, None, p, small, None) == V.ERR_SHAPE
