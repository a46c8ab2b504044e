"""The row-sharded algebra of Alg. 1 (oracle/sharded.py) on gloo ranks on
CPU against the single-process oracle: each rank holds a block of rows of S,
every pass ends in one sum over ranks of its small result, and the gathered
U, the singular values and the coefficients equal the oracle's on the whole
matrix (CholeskyQR2 there against Householder QR here: same basis, signs
fixed by the same rule)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle.rpod import rpod
from oracle.sharded import rpod_rows
from paper_2504_15350_gb300.shard import row_blocks
from synth import make_recipe, snapshot_matrix


def test_row_blocks_cover_and_align():
    for n, world in ((1000, 3), (64, 4), (0, 2), (262144, 8), (130, 2), (5, 1)):
        blocks = row_blocks(n, world)
        assert len(blocks) == world
        assert sum(c for _, c in blocks) == n
        r = 0
        for r0, c in blocks:
            assert r0 == r
            r += c
        for r0, c in blocks[:-1]:
            assert r0 % 64 == 0 and (c % 64 == 0 or r0 + c == n)
        counts = [c for _, c in blocks]
        assert max(counts) - min(counts) <= 64


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _problem():
    rec = make_recipe(16, 20, 150, 80, ("power", 1.2), seed=3, noise=1e-6)
    return snapshot_matrix(rec).numpy()          # 320 x 150


def _worker(rank, world, port, align, q, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        S = _problem()
        r0, nr = row_blocks(S.shape[0], world, align)[rank]

        def allreduce(a):
            t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64))
            dist.all_reduce(t)
            return t.numpy()

        def allgather(obj):
            got = [None] * world
            dist.all_gather_object(got, obj)
            return got

        res = rpod_rows(S[r0:r0 + nr], r0, 12, 8, q, 5, allreduce, allgather)
        blocks = allgather((r0, res.U))
        out[rank] = (blocks, res.sigma, res.C, res.Uhat)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,align,q", [(2, 64, 1), (3, 32, 2), (3, 256, 0)])
def test_row_sharded_rpod_equals_oracle(world, align, q):
    # (3, 256, 0): 320 rows in two 256-row tiles, so rank 0 holds no rows
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, port, align, q, out), nprocs=world, join=True)
        res = dict(out)
    S = _problem()
    ref = rpod(S, 12, 8, q, seed=5)
    for rank in range(world):
        blocks, sigma, C, Uhat = res[rank]
        U = np.concatenate([u for _, u in sorted(blocks, key=lambda b: b[0])], axis=0)
        assert U.shape == ref.U.shape
        assert np.allclose(sigma, ref.sigma, rtol=1e-11, atol=1e-13 * ref.sigma[0])
        # distinct singular values: every column equal, signs by the same rule
        assert np.abs(U - ref.U).max() <= 1e-8
        assert np.abs(C - ref.C).max() <= 1e-9 * np.abs(ref.C).max()
        # replicated quantities agree across ranks exactly
        assert np.array_equal(sigma, res[0][1]) and np.array_equal(C, res[0][2])
