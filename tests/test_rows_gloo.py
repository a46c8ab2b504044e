"""Host logic of the row-sharded exchange (paper_2504_15350_gb300/rows.py)
on two gloo CPU ranks: the C callback that rpod_basis_rows calls is built by
make_exchange over a workspace tensor and TorchComm; called here directly
with addresses inside a CPU stand-in for the workspace, it must combine the
ranks' values in place (sum, max, min; FP64 and FP32) and report a buffer
outside the workspace as a failed exchange.  No GPU and no library: only
ctypes and torch.distributed."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import paper_2504_15350_gb300.rpod as R
from paper_2504_15350_gb300.rows import TorchComm, make_exchange


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ws = torch.zeros(4096, dtype=torch.uint8)
        errors = []
        cb = make_exchange(ws, TorchComm(), errors)
        res = {}
        # FP64 sum at byte 256, FP64 max at 1024, FP64 min at 2048, FP32 sum at 3072
        a = ws[256:256 + 8 * 10].view(torch.float64)
        a.copy_(torch.arange(10, dtype=torch.float64) * (rank + 1))
        assert cb(None, ws.data_ptr() + 256, 10, R.RPOD_F64, R.RPOD_REDUCE_SUM, None) == 0
        res["sum"] = a.clone().numpy()
        b = ws[1024:1024 + 8 * 5].view(torch.float64)
        b.copy_(torch.tensor([rank, -rank, 3.0, rank * 10.0, -1.0], dtype=torch.float64))
        assert cb(None, ws.data_ptr() + 1024, 5, R.RPOD_F64, R.RPOD_REDUCE_MAX, None) == 0
        res["max"] = b.clone().numpy()
        c = ws[2048:2048 + 8 * 3].view(torch.float64)
        c.copy_(torch.tensor([1e300 if rank == 0 else 7.0, rank + 0.5, 2.0], dtype=torch.float64))
        assert cb(None, ws.data_ptr() + 2048, 3, R.RPOD_F64, R.RPOD_REDUCE_MIN, None) == 0
        res["min"] = c.clone().numpy()
        d = ws[3072:3072 + 4 * 6].view(torch.float32)
        d.copy_(torch.full((6,), float(rank + 1)))
        assert cb(None, ws.data_ptr() + 3072, 6, R.RPOD_F32, R.RPOD_REDUCE_SUM, None) == 0
        res["f32"] = d.clone().numpy()
        # a buffer that leaves the workspace: refused without a collective
        res["bad"] = cb(None, ws.data_ptr() + 4090, 4, R.RPOD_F64, R.RPOD_REDUCE_SUM, None)
        res["errors"] = len(errors)
        out[rank] = res
    finally:
        dist.destroy_process_group()


def test_exchange_callback_two_gloo_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
    for r in range(world):
        res = out[r]
        assert np.array_equal(res["sum"], np.arange(10) * 3.0)
        assert np.array_equal(res["max"], np.array([1.0, 0.0, 3.0, 10.0, -1.0]))
        assert np.array_equal(res["min"], np.array([7.0, 0.5, 2.0]))
        assert np.array_equal(res["f32"], np.full(6, 3.0, dtype=np.float32))
        assert res["bad"] == 1 and res["errors"] == 1
