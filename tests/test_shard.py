"""Rollout split over ranks by particles and by sequences (host side).

The simulations are independent (Sec. 2.2), so the rollout splits into
shards whose noise counters are those of the whole problem. On the CPU: the
oracle's particle offset reproduces the whole problem's returns block by
block, the partition covers every index once, and two gloo ranks each
computing a shard with the oracle, gathered with the package's host logic,
give the unsharded oracle's returns (each rank's block of G bit for bit; J
within FP64 rounding, the particle split as the rank-order sum of partials).
"""
import os
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import voila_oracle as O  # noqa: E402
from paper_2606_19729_b300 import shard as S  # noqa: E402
from paper_2606_19729_b300 import workloads as WL  # noqa: E402


def _problem():
    wl = WL.small_fp32(N=37, K=6, H=3)
    g = O.MLP(wl.g_T.W, wl.g_T.b, wl.g_T.act)
    R = O.Reward(O.REWARD_GOAL, wl.goal)
    return wl, g, R


@pytest.mark.parametrize("total,world", [(0, 1), (5, 1), (5, 2), (37, 2), (37, 4), (3, 4), (1024, 3)])
def test_shard_range_partitions_every_index_once(total, world):
    seen = []
    for r in range(world):
        off, cnt = S.shard_range(total, world, r)
        assert cnt >= 0 and off == len(seen)
        seen.extend(range(off, off + cnt))
    assert seen == list(range(total))
    counts = [S.shard_range(total, world, r)[1] for r in range(world)]
    assert max(counts) - min(counts) <= 1


def test_shard_range_rejects_bad_geometry():
    for args in [(5, 0, 0), (5, 2, 2), (5, 2, -1), (-1, 2, 0)]:
        with pytest.raises(ValueError):
            S.shard_range(*args)


def test_oracle_particle_offset_reproduces_the_whole_problem():
    wl, g, R = _problem()
    J, G = O.rollout(g, R, wl.particles, wl.actions, wl.d_omega, wl.gamma, wl.seed)
    cut = 16
    Ja, Ga = O.rollout(g, R, wl.particles[:cut], wl.actions, wl.d_omega, wl.gamma, wl.seed,
                       w=np.full(cut, 1.0 / wl.N))
    Jb, Gb = O.rollout(g, R, wl.particles[cut:], wl.actions, wl.d_omega, wl.gamma, wl.seed,
                       w=np.full(wl.N - cut, 1.0 / wl.N), n_offset=cut)
    assert np.array_equal(np.concatenate([Ga, Gb], axis=1), G)
    np.testing.assert_allclose(Ja + Jb, J, rtol=1e-13, atol=1e-15)
    # without the offset the second block would draw the first block's noise
    _, Gwrong = O.rollout(g, R, wl.particles[cut:], wl.actions, wl.d_omega, wl.gamma, wl.seed)
    assert not np.array_equal(Gwrong, Gb)


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    wl, g, R = _problem()
    # by sequences
    k0, kc = S.shard_range(wl.K, world, rank)
    Jk, Gk = O.rollout(g, R, wl.particles, wl.actions, wl.d_omega, wl.gamma, wl.seed,
                       k_index=list(range(k0, k0 + kc)))
    J_seq = S.gather_sequence_shards(torch.from_numpy(Jk), wl.K)
    # by particles
    n0, nc = S.shard_range(wl.N, world, rank)
    Jn, Gn = O.rollout(g, R, wl.particles[n0:n0 + nc], wl.actions, wl.d_omega, wl.gamma, wl.seed,
                       w=np.full(nc, 1.0 / wl.N), n_offset=n0)
    J_part = S.reduce_particle_shards(torch.from_numpy(Jn))
    dist.barrier()
    out[rank] = (J_seq.numpy().tolist(), J_part.numpy().tolist(), Gk.tolist(), Gn.tolist())
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_gather():
    world = 2
    port = 29600 + (os.getpid() % 1000)
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    wl, g, R = _problem()
    J, G = O.rollout(g, R, wl.particles, wl.actions, wl.d_omega, wl.gamma, wl.seed)
    # every rank's block of G is the whole problem's, bit for bit
    assert np.array_equal(np.concatenate([np.array(res[r][2]) for r in range(world)], axis=0), G)
    assert np.array_equal(np.concatenate([np.array(res[r][3]) for r in range(world)], axis=1), G)
    for r in range(world):
        J_seq, J_part = np.array(res[r][0]), np.array(res[r][1])
        # (the oracle's J is one library matrix-vector product, whose summation order
        # may depend on the shape, so J is compared within FP64 rounding here; the
        # device's sequence split is bit-exact and tested on the GPU)
        np.testing.assert_allclose(J_seq, J, rtol=1e-14, atol=1e-15)
        np.testing.assert_allclose(J_part, J, rtol=1e-13, atol=1e-15)
    assert res[0][:2] == res[1][:2]
