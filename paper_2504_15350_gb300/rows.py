"""Row-sharded randomized POD through librpod's rpod_basis_rows (ctypes).

Each call holds one contiguous block of the rows (grid cells) of S and runs
Alg. 1's passes over it; the library hands every quantity of the whole
matrix -- the CholeskyQR Grams, Z = S^T Q, T = Q^T S and the sign rule's
candidates -- to an exchange callback, which this module builds from a
communicator object with one method, ``allreduce(tensor, op)`` (op "sum",
"max" or "min", in place on a tensor that views the library's buffer).

* TorchComm: torch.distributed (NCCL between GPUs of one node; the tensors
  are device views of the plan's workspace, the collective runs on the
  current stream).
* ThreadComm: several row blocks on one GPU, one host thread each; the
  exchange synchronises the block's stream, combines on the host and
  writes back (used by the tests).

The C callback receives a device pointer into the plan's workspace; the
adapter turns it into a tensor view of that workspace (no copy), so the
combination happens in place."""
from __future__ import annotations

import ctypes
import threading

import numpy as np
import torch

from . import rpod as R

EXCHANGE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                               ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p)
_OPS = {R.RPOD_REDUCE_SUM: "sum", R.RPOD_REDUCE_MAX: "max", R.RPOD_REDUCE_MIN: "min"}
_DTYPES = {R.RPOD_F64: torch.float64, R.RPOD_F32: torch.float32}


def rpod_rows_plan_create(n_total, row0, n_rows, m, k, p, q, seed, compute, flags=0) -> int:
    h = ctypes.c_void_p()
    R._check(R.load().rpod_rows_plan_create(ctypes.byref(h), n_total, row0, n_rows, m, k, p, q, seed,
                                            compute, flags), "rpod_rows_plan_create")
    return h.value


def rpod_basis_rows(plan, S, lds, s_dtype, U, ldu, sigma, C, ldc, ws, ws_bytes, stream, exchange,
                    ctx=None):
    return R.load().rpod_basis_rows(plan, S, lds, s_dtype, U, ldu, sigma, C, ldc, ws, ws_bytes, stream,
                                    ctypes.cast(exchange, ctypes.c_void_p), ctx)


def buffer_view(base: torch.Tensor, ptr: int, count: int, dtype: torch.dtype) -> torch.Tensor:
    """`count` elements of `dtype` at address ptr inside the uint8 tensor
    `base`, as a view (raises if the range is not inside it)."""
    off = ptr - base.data_ptr()
    nbytes = count * torch.tensor([], dtype=dtype).element_size()
    if off < 0 or off + nbytes > base.numel() or off % torch.tensor([], dtype=dtype).element_size():
        raise ValueError("exchange buffer outside the workspace")
    return base[off:off + nbytes].view(dtype)


def make_exchange(base: torch.Tensor, comm, errors: list):
    """C exchange callback over the workspace tensor `base`: views the buffer
    and calls comm.allreduce(view, op).  Python errors are recorded in
    `errors` and reported to the library as a failed exchange."""
    def cb(ctx, buf, count, dtype, op, stream):
        try:
            view = buffer_view(base, int(buf), int(count), _DTYPES[int(dtype)])
            comm.allreduce(view, _OPS[int(op)])
            return 0
        except Exception as e:  # reported as RPOD_ERR_EXCHANGE
            errors.append(e)
            return 1
    return EXCHANGE_FN(cb)


class TorchComm:
    """Exchange over a torch.distributed process group."""

    def __init__(self, group=None):
        self.group = group

    def allreduce(self, t: torch.Tensor, op: str):
        import torch.distributed as dist
        red = {"sum": dist.ReduceOp.SUM, "max": dist.ReduceOp.MAX, "min": dist.ReduceOp.MIN}[op]
        dist.all_reduce(t, op=red, group=self.group)


class ThreadComm:
    """Exchange among `world` host threads (one row block each) of one
    process: each thread's view is copied to the host after its stream is
    synchronised, the values are combined in rank order, and every thread
    copies the result back.  A broken barrier (a thread that failed) makes
    the others fail too."""

    def __init__(self, world: int, timeout: float = 120.0):
        self.world = world
        self.bar = threading.Barrier(world, timeout=timeout)
        self.slots = [None] * world
        self.local = threading.local()

    def rank(self, r: int):
        self.local.rank = r
        return self

    def allreduce(self, t: torch.Tensor, op: str):
        r = self.local.rank
        if t.is_cuda:
            torch.cuda.current_stream(t.device).synchronize()
        self.slots[r] = t.cpu().numpy().copy()
        self.bar.wait()
        vals = np.stack(self.slots)
        res = {"sum": vals.sum(0), "max": vals.max(0), "min": vals.min(0)}[op]
        self.bar.wait()
        t.copy_(torch.from_numpy(res))
        if t.is_cuda:
            torch.cuda.current_stream(t.device).synchronize()


class RowsPlan:
    """rPOD plan for the row block row0 .. row0 + n_rows - 1 of an n_total x m
    matrix, with its own workspace on `device`."""

    def __init__(self, n_total, row0, n_rows, m, k, p, q, seed=0, compute="f64", flags=0,
                 device="cuda"):
        self.compute = {"f64": R.RPOD_F64, "f32": R.RPOD_F32}[compute] if isinstance(compute, str) \
            else int(compute)
        self.n_total, self.row0, self.n_rows, self.m = n_total, row0, n_rows, m
        self.k, self.p, self.q, self.l = k, p, q, k + p
        self.flags = flags
        self.device = torch.device(device)
        self.handle = rpod_rows_plan_create(n_total, row0, n_rows, m, k, p, q, seed, self.compute, flags)
        self.ws_bytes = R.rpod_workspace_bytes(self.handle)
        self.ws = torch.empty(self.ws_bytes + 256, dtype=torch.uint8, device=self.device)
        off = (-self.ws.data_ptr()) % 256
        self.ws_ptr = self.ws.data_ptr() + off
        self.ws[off:off + 256].zero_()
        self.out_dtype = torch.float64 if self.compute == R.RPOD_F64 else torch.float32

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            try:
                R.rpod_plan_destroy(h)
            except Exception:
                pass
            self.handle = None

    def basis(self, S_rows, comm):
        """Alg. 1 on this block (column-major n_rows x m tensor).  Returns
        (U_rows, sigma, C); sigma and C are the same on every block."""
        ku = self.l if (self.flags & R.RPOD_FLAG_RETURN_ALL_L) else self.k
        U = R.empty_colmajor(self.n_rows, ku, self.out_dtype, self.device)
        sigma = torch.empty(self.l, dtype=torch.float64, device=self.device)
        C = R.empty_colmajor(self.k, self.m, self.out_dtype, self.device)
        errors = []
        cb = make_exchange(self.ws, comm, errors)
        stream = torch.cuda.current_stream(self.device).cuda_stream
        rc = rpod_basis_rows(self.handle, S_rows.data_ptr(), R.colmajor_ld(S_rows), R.dtype_code(S_rows.dtype),
                             U.data_ptr(), R.colmajor_ld(U), sigma.data_ptr(), C.data_ptr(),
                             R.colmajor_ld(C), self.ws_ptr, self.ws_bytes, stream, cb)
        if errors:
            raise R.RpodError(R.RPOD_ERR_EXCHANGE, f"rpod_basis_rows exchange: {errors[0]!r}")
        R._check(rc, "rpod_basis_rows")
        return U, sigma, C

    def status(self):
        return R.rpod_status_sync(self.handle, self.ws_ptr,
                                  torch.cuda.current_stream(self.device).cuda_stream)
