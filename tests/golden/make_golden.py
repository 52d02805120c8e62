"""Writes the stored oracle fixtures of this folder. It calls only the FP64
oracle and the seeded input generators (no device code), so every stored value
is the oracle's. Run from the repository root:

    python tests/golden/make_golden.py

The fixtures pin the oracle against later edits (tests/test_golden.py re-runs
the oracle on the same inputs and requires the stored integers and random
words bit for bit and the floats to 1e-12) and
give the GPU tests expected values that need no oracle run. Floats are stored
as hexadecimal strings (float.hex), so the files round-trip exactly.

Fixtures:
* small_fp32_step.json: the FP32 workload (2x64 tanh MLPs; Sec. 5.2's
  generator shape family) at N = 32 particles, K = 4 sequences, H = 3 steps:
  the rollout's J_k and G (Sec. 2.1 return, Eq. 1 estimate), then one SIR
  belief update (Sec. 3, weights of Sec. 4.2.3) with the MLP likelihood,
  lambda = 0.5, step 7: resampled indices, quantised weights, log Z, ESS, u0.
* philox_words.json: Philox4x32-10 words (Salmon et al., SC'11) of the
  oracle for eight counters of the streams the path draws from.
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import voila_oracle as O  # noqa: E402
from paper_2606_19729_b300 import workloads as WL  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
STEP_CASE = dict(N=32, K=4, H=3, lam=0.5, step=7, obs=[0.25, -0.5, 0.125, 0.75])
PHILOX_CASES = [
    # (c0, c1, c2, stream, planner, block, seed)
    (0, 0, 0, O.STREAM_ROLLOUT_OMEGA, 0, 0, 0),
    (5, 3, 2, O.STREAM_ROLLOUT_OMEGA, 1, 1, 1),
    (4095, 1023, 19, O.STREAM_ROLLOUT_OMEGA, 0, 1, 1),
    (17, 0, 9, O.STREAM_BELIEF_OMEGA, 2, 0, 3),
    (0, 0, 7, O.STREAM_RESAMPLE, 0, 0, 0),
    (65535, 0, 4, O.STREAM_OBS_OMEGA, 65535, 3, 2**40 + 5),
    (1, 2, 3, O.STREAM_TRUE_STATE, 0, 0, 12345),
    (2**32 - 1, 2**32 - 1, 2**32 - 1, O.STREAM_ROLLOUT_OMEGA, 4095, 4095, 2**64 - 1),
]


def _mlp(spec):
    return O.MLP([np.asarray(w, np.float64) for w in spec.W], [np.asarray(b, np.float64) for b in spec.b],
                 spec.act)


def _hex(a):
    return [float(x).hex() for x in np.asarray(a, np.float64).ravel()]


def small_fp32_step():
    c = STEP_CASE
    wl = WL.small_fp32(N=c["N"], K=c["K"], H=c["H"])
    J, G = O.rollout(_mlp(wl.g_T), O.Reward(O.REWARD_MLP, mlp=_mlp(wl.reward_mlp)), wl.particles, wl.actions,
                     wl.d_omega, wl.gamma, wl.seed)
    obs = np.asarray(c["obs"], np.float64)
    res = O.belief_update(_mlp(wl.g_T), O.Likelihood(O.LIK_MLP, mlp=_mlp(wl.ell)), wl.particles,
                          wl.actions[0, 0], obs, wl.d_omega, c["lam"], wl.seed, c["step"])
    return {
        "case": dict(c, workload="small_fp32", seed=wl.seed, d_omega=wl.d_omega, gamma=wl.gamma,
                     reward="mlp", action="actions[0, 0]"),
        "J": _hex(J), "G_shape": list(G.shape), "G": _hex(G),
        "idx": [int(i) for i in res.idx], "w": _hex(res.w), "logZ": float(res.logZ).hex(),
        "ess": float(res.ess).hex(), "u0": float(res.u0).hex(), "s_prop": _hex(res.s_prop),
    }


def philox_words():
    out = []
    for (c0, c1, c2, stream, planner, block, seed) in PHILOX_CASES:
        k0, k1 = O.seed_key(seed)
        c3 = O.counter_word3(stream, planner, block)
        w = O.philox4x32_10(np.uint64(c0), np.uint64(c1), np.uint64(c2), np.uint64(c3), k0, k1)
        out.append({"c0": c0, "c1": c1, "c2": c2, "stream": stream, "planner": planner, "block": block,
                    "seed": seed, "words": [int(x) for x in np.asarray(w, np.uint64).ravel()]})
    return out


def main():
    with open(os.path.join(HERE, "small_fp32_step.json"), "w") as f:
        json.dump(small_fp32_step(), f, indent=0)
    with open(os.path.join(HERE, "philox_words.json"), "w") as f:
        json.dump(philox_words(), f, indent=1)


if __name__ == "__main__":
    main()
