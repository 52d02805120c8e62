"""Shared test helpers: map the seeded workloads onto the oracle and the device."""
import numpy as np
import torch

from oracle import voila_oracle as O


def oracle_mlp(spec):
    return O.MLP([np.asarray(w, np.float64) for w in spec.W], [np.asarray(b, np.float64) for b in spec.b],
                 spec.act)


def rel_err(got, want):
    """Normwise relative error ||got - want||_inf / ||want||_inf."""
    got = np.asarray(got, np.float64)
    want = np.asarray(want, np.float64)
    return float(np.max(np.abs(got - want)) / max(np.max(np.abs(want)), 1e-300))


def cuda(x, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(x)).to(device="cuda", dtype=dtype).contiguous()
