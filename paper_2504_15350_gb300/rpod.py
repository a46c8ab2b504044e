"""ctypes binding of librpod's C ABI (include/rpod.h).

Every function of the header is exposed under the same name with the same
arguments (device pointers as Python ints, the stream as its integer
handle).  `Plan` adds torch-tensor marshalling: it reads data pointers,
leading dimensions and the current CUDA stream from tensors and allocates
the outputs and the workspace with torch; all arithmetic runs in the
library's kernels.
"""
from __future__ import annotations

import ctypes
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "librpod.so")

RPOD_F64, RPOD_F32, RPOD_BF16, RPOD_F16 = 0, 1, 2, 3
RPOD_OK = 0
RPOD_ERR_INVALID_ARG = 1
RPOD_ERR_UNSUPPORTED = 2
RPOD_ERR_NONFINITE = 3
RPOD_ERR_BREAKDOWN = 4
RPOD_ERR_NO_CONVERGENCE = 5
RPOD_ERR_TIMEOUT = 6
RPOD_ERR_CUDA = 7
RPOD_ERR_WORKSPACE = 8
RPOD_ERR_IO = 9
RPOD_ERR_EXCHANGE = 10
RPOD_REDUCE_SUM, RPOD_REDUCE_MAX, RPOD_REDUCE_MIN = 0, 1, 2
RPOD_WARN_RANK_DEFICIENT = 1
RPOD_FLAG_REFINE_FP32 = 1
RPOD_FLAG_RETURN_ALL_L = 4
RPOD_FLAG_HOST_IO = 8

_c_i64, _c_i32, _c_u64, _c_u32, _p = (ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64,
                                      ctypes.c_uint32, ctypes.c_void_p)

class Instance(ctypes.Structure):
    """rpod_instance of include/rpod.h."""
    _fields_ = [("n", _c_i64), ("m", _c_i64), ("k", _c_i32), ("p", _c_i32), ("q", _c_i32),
                ("seed", _c_u64), ("S", _p), ("lds", _c_i64), ("S_refine", _p), ("ldr", _c_i64),
                ("U", _p), ("ldu", _c_i64), ("sigma", _p), ("C", _p), ("ldc", _c_i64)]


_pi32 = ctypes.POINTER(_c_i32)

# name -> (restype, argtypes); mirrors include/rpod.h
SIGNATURES = {
    "rpod_batch_create": (ctypes.c_int, [ctypes.POINTER(_p), _c_i32, ctypes.POINTER(Instance), _c_i32,
                                         _c_u32, _c_i32]),
    "rpod_batch_workspace_bytes": (ctypes.c_int, [_p, ctypes.POINTER(ctypes.c_size_t)]),
    "rpod_batch_run": (ctypes.c_int, [_p, _p, ctypes.c_size_t, _p]),
    "rpod_batch_tune": (ctypes.c_int, [_p, _p, ctypes.c_size_t, _p, _c_i32, _pi32, _pi32, _pi32]),
    "rpod_batch_set_pass_stages": (ctypes.c_int, [_p, _c_i32]),
    "rpod_batch_configure": (ctypes.c_int, [_p, _c_i32, _c_i32]),
    "rpod_batch_status_sync": (ctypes.c_int, [_p, _p, _p, _pi32, ctypes.POINTER(_c_u32)]),
    "rpod_batch_last_launch_count": (ctypes.c_int, [_p]),
    "rpod_batch_destroy": (None, [_p]),
    "rpod_lstm_create": (ctypes.c_int, [ctypes.POINTER(_p), _c_i32, _c_i32, _c_i32, _c_i32, _c_i32,
                                        _c_i32, _c_u32]),
    "rpod_lstm_param_count": (_c_i64, [_p]),
    "rpod_lstm_workspace_bytes": (ctypes.c_int, [_p, ctypes.POINTER(ctypes.c_size_t)]),
    "rpod_lstm_set_params": (ctypes.c_int, [_p, _p, _p, ctypes.c_size_t, _p]),
    "rpod_lstm_get_params": (ctypes.c_int, [_p, _p, _p, ctypes.c_size_t, _p]),
    "rpod_lstm_forward": (ctypes.c_int, [_p, _p, _c_i32, _p, _p, ctypes.c_size_t, _p]),
    "rpod_lstm_loss_grad": (ctypes.c_int, [_p, _p, _p, _c_i32, _p, _p, _p, ctypes.c_size_t, _p]),
    "rpod_lstm_train_step": (ctypes.c_int, [_p, _p, _p, _c_i32, ctypes.c_float, ctypes.c_float, _p, _p,
                                            ctypes.c_size_t, _p]),
    "rpod_lstm_gather": (ctypes.c_int, [_p, _p, _p, _c_i32, _c_i32, _c_i32, _p, _c_i32, _p, _p, _p]),
    "rpod_lstm_rollout": (ctypes.c_int, [_p, _p, _c_i32, _c_i32, _c_i32, _p, _p, ctypes.c_size_t, _p]),
    "rpod_lstm_set_dropout": (ctypes.c_int, [_p, ctypes.c_double, _c_u64]),
    "rpod_lstm_train_epoch": (ctypes.c_int, [_p, _p, _p, _c_i32, _c_i32, _c_i32, _p, _c_i32, _c_i32,
                                             ctypes.c_float, ctypes.c_float, _p, _p, ctypes.c_size_t,
                                             _p]),
    "rpod_lstm_save": (ctypes.c_int, [_p, ctypes.c_char_p, _p, ctypes.c_size_t, _p]),
    "rpod_lstm_load": (ctypes.c_int, [ctypes.POINTER(_p), ctypes.c_char_p]),
    "rpod_lstm_restore": (ctypes.c_int, [_p, _p, ctypes.c_size_t, _p]),
    "rpod_lstm_dims": (ctypes.c_int, [_p, _pi32]),
    "rpod_lstm_last_launch_count": (ctypes.c_int, [_p]),
    "rpod_lstm_status_sync": (ctypes.c_int, [_p, _p, _p]),
    "rpod_selftest_grid_barrier": (ctypes.c_int, [ctypes.c_double, _p]),
    "rpod_lstm_destroy": (None, [_p]),
    "rpod_plan_create": (ctypes.c_int, [ctypes.POINTER(_p), _c_i64, _c_i64, _c_i32, _c_i32, _c_i32,
                                        _c_u64, _c_i32, _c_u32]),
    "rpod_workspace_bytes": (ctypes.c_int, [_p, ctypes.POINTER(ctypes.c_size_t)]),
    "rpod_plan_set_svd_sweeps": (ctypes.c_int, [_p, _c_i32]),
    "rpod_plan_set_graph": (ctypes.c_int, [_p, _c_i32]),
    "rpod_rows_plan_create": (ctypes.c_int, [ctypes.POINTER(_p), _c_i64, _c_i64, _c_i64, _c_i64, _c_i32,
                                             _c_i32, _c_i32, _c_u64, _c_i32, _c_u32]),
    "rpod_basis_rows": (ctypes.c_int, [_p, _p, _c_i64, _c_i32, _p, _c_i64, _p, _p, _c_i64, _p,
                                       ctypes.c_size_t, _p, _p, _p]),
    "rpod_basis": (ctypes.c_int, [_p, _p, _c_i64, _c_i32, _p, _c_i64, _p, _c_i64, _p, _p, _c_i64,
                                  _p, ctypes.c_size_t, _p]),
    "rpod_project": (ctypes.c_int, [_p, _p, _c_i64, _c_i32, _p, _c_i64, _c_i64, _c_i32, _p, _c_i64,
                                    _p, ctypes.c_size_t, _p]),
    "rpod_status_sync": (ctypes.c_int, [_p, _p, _p, ctypes.POINTER(_c_u32)]),
    "rpod_plan_destroy": (None, [_p]),
    "rpod_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "rpod_last_launch_count": (ctypes.c_int, [_p]),
    "rpod_sketch": (ctypes.c_int, [_p, _p, _c_i64, _c_i32, _p]),
    "rpod_sample": (ctypes.c_int, [_p, _p, _c_i64, _p, _c_i64, _c_i32, _p, _c_i64, _p,
                                   ctypes.c_size_t, _p]),
    "rpod_project_static": (ctypes.c_int, [_p, _p, _c_i64, _c_i32, _p, _c_i64, _c_i64, _c_i32, _p,
                                           _c_i64, _p]),
    "rpod_fluctuations": (ctypes.c_int, [_c_i64, _c_i64, _c_i64, _p, _c_i64, _c_i32, _p, _c_i64,
                                         _c_i32, _p, _c_i64, _c_i32, _p, _c_i64, _p]),
    "rpod_energy_rank": (ctypes.c_int, [_p, _c_i32, ctypes.c_double, _p, _p]),
    "rpod_selftest_wait_timeout": (ctypes.c_int, [ctypes.c_double, _p]),
    "rpod_basis_save": (ctypes.c_int, [_p, ctypes.c_char_p, _p, _c_i64, _p, _p, _c_i64, _p]),
    "rpod_basis_file_info": (ctypes.c_int, [ctypes.c_char_p, ctypes.POINTER(_c_i64)]),
    "rpod_basis_load": (ctypes.c_int, [ctypes.c_char_p, _p, _c_i64, _p, _p, _c_i64, _p]),
    "rpod_profile_enable": (ctypes.c_int, [_p, ctypes.c_int]),
    "rpod_profile_read": (ctypes.c_int, [_p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Loads librpod.so (built by paper_2504_15350_gb300.build) and declares
    its signatures.  Raises if the library is missing: there is no fallback."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"librpod.so not built ({path}); run paper_2504_15350_gb300.build.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class RpodError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        msg = load().rpod_strerror(code).decode()
        super().__init__(f"{what}: {msg} (status {code})" if what else f"{msg} (status {code})")


def _check(code: int, what: str):
    if code != RPOD_OK:
        raise RpodError(code, what)


# ---- same-name wrappers --------------------------------------------------
def rpod_plan_create(n, m, k, p, q, seed, compute, flags=0) -> int:
    h = _p()
    _check(load().rpod_plan_create(ctypes.byref(h), n, m, k, p, q, seed, compute, flags),
           "rpod_plan_create")
    return h.value


def rpod_workspace_bytes(plan) -> int:
    b = ctypes.c_size_t()
    _check(load().rpod_workspace_bytes(plan, ctypes.byref(b)), "rpod_workspace_bytes")
    return b.value


def rpod_plan_set_svd_sweeps(plan, max_sweeps):
    return load().rpod_plan_set_svd_sweeps(plan, max_sweeps)


def rpod_plan_set_graph(plan, enable):
    return load().rpod_plan_set_graph(plan, enable)


def rpod_basis(plan, S, lds, s_dtype, S_refine, ldr, U, ldu, sigma, C, ldc, ws, ws_bytes, stream):
    return load().rpod_basis(plan, S, lds, s_dtype, S_refine, ldr, U, ldu, sigma, C, ldc, ws,
                             ws_bytes, stream)


def rpod_project(plan, U, ldu, kc, S_new, lds, m_new, s_dtype, C, ldc, ws, ws_bytes, stream):
    return load().rpod_project(plan, U, ldu, kc, S_new, lds, m_new, s_dtype, C, ldc, ws, ws_bytes,
                               stream)


def rpod_status_sync(plan, ws, stream):
    f = _c_u32()
    rc = load().rpod_status_sync(plan, ws, stream, ctypes.byref(f))
    return rc, f.value


def rpod_plan_destroy(plan):
    load().rpod_plan_destroy(plan)


def rpod_strerror(code):
    return load().rpod_strerror(code).decode()


def rpod_last_launch_count(plan):
    return load().rpod_last_launch_count(plan)


def rpod_sketch(plan, Lam, ld, dtype, stream):
    return load().rpod_sketch(plan, Lam, ld, dtype, stream)


def rpod_sample(plan, A, lda, S, lds, s_dtype, Y, ldy, ws, ws_bytes, stream):
    return load().rpod_sample(plan, A, lda, S, lds, s_dtype, Y, ldy, ws, ws_bytes, stream)


def rpod_project_static(plan, U, ldu, kc, S_new, lds, m_new, s_dtype, C, ldc, stream):
    """Allocation-free projection: same result as rpod_project, with the
    split-K scratch in a fixed 16 MiB device array of the library (for
    callers that cannot allocate device memory or hand out a workspace)."""
    return load().rpod_project_static(plan, U, ldu, kc, S_new, lds, m_new, s_dtype, C, ldc, stream)


def rpod_fluctuations(n, m, nt, S, lds, s_dtype, F, ldf, f_dtype, H, ldh, h_dtype, Sbar, ldb,
                      stream):
    return load().rpod_fluctuations(n, m, nt, S, lds, s_dtype, F, ldf, f_dtype, H, ldh, h_dtype,
                                    Sbar, ldb, stream)


def rpod_selftest_wait_timeout(seconds, stream):
    return load().rpod_selftest_wait_timeout(float(seconds), stream)


def rpod_energy_rank(sigma, count, delta, rank, stream):
    return load().rpod_energy_rank(sigma, count, delta, rank, stream)


def rpod_basis_save(plan, path, U, ldu, sigma, C, ldc, stream):
    return load().rpod_basis_save(plan, os.fsencode(path), U, ldu, sigma, C, ldc, stream)


def rpod_basis_file_info(path):
    """(n, m, k, p, q, seed, compute, flags, ku) of a basis file."""
    v = (_c_i64 * 9)()
    _check(load().rpod_basis_file_info(os.fsencode(path), v), "rpod_basis_file_info")
    out = [int(x) for x in v]
    out[5] &= (1 << 64) - 1
    return tuple(out)


def rpod_basis_load(path, U, ldu, sigma, C, ldc, stream):
    return load().rpod_basis_load(os.fsencode(path), U, ldu, sigma, C, ldc, stream)


def load_basis(path, device="cuda"):
    """(Plan, U, sigma, C) from a basis file: the plan recreated from the
    file's parameters, the arrays on `device`."""
    torch = _torch()
    n, m, k, p, q, seed, compute, flags, ku = rpod_basis_file_info(path)
    plan = Plan(n, m, k, p, q, seed=seed, compute=compute, flags=flags, device=device)
    U = empty_colmajor(n, ku, plan.out_dtype, plan.device)
    sigma = torch.empty(k + p, dtype=torch.float64, device=plan.device)
    C = empty_colmajor(k, m, plan.out_dtype, plan.device)
    _check(rpod_basis_load(path, U.data_ptr(), colmajor_ld(U), sigma.data_ptr(), C.data_ptr(),
                           colmajor_ld(C), plan._stream()), "rpod_basis_load")
    return plan, U, sigma, C


def rpod_profile_enable(plan, enable):
    return load().rpod_profile_enable(plan, int(enable))


def rpod_profile_read(plan):
    n = ctypes.c_int(); ms = ctypes.c_double(); b = ctypes.c_double(); f = ctypes.c_double()
    _check(load().rpod_profile_read(plan, ctypes.byref(n), ctypes.byref(ms), ctypes.byref(b),
                                    ctypes.byref(f)), "rpod_profile_read")
    return n.value, ms.value, b.value, f.value


def rpod_batch_create(instances, compute, flags, s_dtype) -> int:
    arr = (Instance * len(instances))(*instances)
    h = _p()
    _check(load().rpod_batch_create(ctypes.byref(h), len(instances), arr, compute, flags, s_dtype),
           "rpod_batch_create")
    return h.value


def rpod_batch_workspace_bytes(batch) -> int:
    b = ctypes.c_size_t()
    _check(load().rpod_batch_workspace_bytes(batch, ctypes.byref(b)), "rpod_batch_workspace_bytes")
    return b.value


def rpod_batch_run(batch, ws, ws_bytes, stream):
    return load().rpod_batch_run(batch, ws, ws_bytes, stream)


def rpod_batch_tune(batch, ws, ws_bytes, stream, trials):
    """(streams, split_pct, stages) of the fastest configuration."""
    s, p, g = _c_i32(), _c_i32(), _c_i32()
    _check(load().rpod_batch_tune(batch, ws, ws_bytes, stream, trials, ctypes.byref(s), ctypes.byref(p),
                                  ctypes.byref(g)), "rpod_batch_tune")
    return s.value, p.value, g.value


def rpod_batch_set_pass_stages(batch, stages):
    return load().rpod_batch_set_pass_stages(batch, stages)


def rpod_batch_configure(batch, streams, split_pct):
    return load().rpod_batch_configure(batch, streams, split_pct)


def rpod_batch_status_sync(batch, ws, stream):
    bad, fl = _c_i32(), _c_u32()
    rc = load().rpod_batch_status_sync(batch, ws, stream, ctypes.byref(bad), ctypes.byref(fl))
    return rc, bad.value, fl.value


def rpod_batch_last_launch_count(batch):
    return load().rpod_batch_last_launch_count(batch)


def rpod_batch_destroy(batch):
    load().rpod_batch_destroy(batch)


# ---- torch marshalling ------------------------------------------------------
def _torch():
    import torch
    return torch


def dtype_code(t) -> int:
    torch = _torch()
    return {torch.float64: RPOD_F64, torch.float32: RPOD_F32, torch.bfloat16: RPOD_BF16,
            torch.float16: RPOD_F16}[t]


def colmajor_ld(A) -> int:
    """Leading dimension of a column-major 2-D view (stride (1, ld))."""
    if A.dim() != 2 or A.stride(0) != 1:
        raise ValueError("expected a column-major matrix view (stride(0) == 1); use X.t() of a "
                         "row-major (m, n) tensor")
    return max(A.stride(1), A.shape[0])


def empty_colmajor(rows, cols, dtype, device):
    torch = _torch()
    return torch.empty((cols, rows), dtype=dtype, device=device).t()


def fluctuations(S, nt, f_dtype="same", h_dtype=None, in_place=False, out=None):
    """Per-sample time averages and fluctuation snapshots (Eqs. (time_av),
    (fluct_q)) of the column-major n x m tensor S holding m / nt samples of nt
    snapshots.  Returns (F, H, Sbar): F in `f_dtype` ("same" for S's dtype, a
    torch dtype, or None for no F; S itself when in_place), H a 16-bit copy
    (h_dtype a torch dtype or None), Sbar n x (m / nt) (float64 for a float64
    S, float32 otherwise).  `out` = (F, H, Sbar) reuses caller tensors."""
    torch = _torch()
    n, m = S.shape
    if nt < 1 or m % nt:
        raise ValueError("nt must divide the number of snapshots")
    dev = S.device
    if f_dtype == "same":
        f_dtype = S.dtype
    sb_dtype = torch.float64 if S.dtype == torch.float64 else torch.float32
    if out is not None:
        F, H, Sbar = out
    else:
        Sbar = empty_colmajor(n, m // nt, sb_dtype, dev)
        if in_place:
            F = S
        else:
            F = empty_colmajor(n, m, f_dtype, dev) if f_dtype is not None else None
        H = empty_colmajor(n, m, h_dtype, dev) if h_dtype is not None else None
    rc = rpod_fluctuations(n, m, nt, S.data_ptr(), colmajor_ld(S), dtype_code(S.dtype),
                           F.data_ptr() if F is not None else None,
                           colmajor_ld(F) if F is not None else 0,
                           dtype_code(F.dtype) if F is not None else 0,
                           H.data_ptr() if H is not None else None,
                           colmajor_ld(H) if H is not None else 0,
                           dtype_code(H.dtype) if H is not None else 0,
                           Sbar.data_ptr(), colmajor_ld(Sbar),
                           torch.cuda.current_stream(dev).cuda_stream)
    _check(rc, "rpod_fluctuations")
    return F, H, Sbar


def energy_rank(sigma, delta, out=None):
    """Eq. (energy) on the device: a 1-element int32 tensor holding the
    smallest N whose leading singular values retain the fraction delta of the
    sum of all values given (0 for a spectrum with no positive sum)."""
    torch = _torch()
    if sigma.dtype != torch.float64 or not sigma.is_contiguous():
        raise ValueError("sigma must be a contiguous float64 tensor")
    rank = out if out is not None else torch.empty(1, dtype=torch.int32, device=sigma.device)
    _check(rpod_energy_rank(sigma.data_ptr(), sigma.numel(), float(delta), rank.data_ptr(),
                            torch.cuda.current_stream(sigma.device).cuda_stream),
           "rpod_energy_rank")
    return rank


class Plan:
    """An rPOD plan plus its workspace, for tensors on one CUDA device."""

    def __init__(self, n, m, k, p, q, seed=0, compute="f32", flags=0, device="cuda"):
        torch = _torch()
        self.compute = {"f64": RPOD_F64, "f32": RPOD_F32, "bf16": RPOD_BF16,
                        "f16": RPOD_F16}[compute] if isinstance(compute, str) else int(compute)
        self.n, self.m, self.k, self.p, self.q, self.l = n, m, k, p, q, k + p
        self.flags = flags
        self.device = torch.device(device)
        self.handle = rpod_plan_create(n, m, k, p, q, seed, self.compute, flags)
        self.ws_bytes = rpod_workspace_bytes(self.handle)
        self.ws = torch.empty(self.ws_bytes + 256, dtype=torch.uint8, device=self.device)
        off = (-self.ws.data_ptr()) % 256
        self.ws_ptr = self.ws.data_ptr() + off
        self.ws[off:off + 256].zero_()
        self.out_dtype = torch.float64 if self.compute == RPOD_F64 else torch.float32

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            try:
                rpod_plan_destroy(h)
            except Exception:
                pass
            self.handle = None

    def _stream(self):
        return _torch().cuda.current_stream(self.device).cuda_stream

    def basis(self, S, S_refine=None, out=None):
        """Alg. 1 on the column-major n x m tensor S.  Returns (U, sigma, C):
        U n x k (or n x l), sigma (l,) float64, C k x m (column-major views)."""
        torch = _torch()
        ku = self.l if (self.flags & RPOD_FLAG_RETURN_ALL_L) else self.k
        if out is None and (self.flags & RPOD_FLAG_HOST_IO):
            # host outputs (pinned) for a plan that takes host buffers
            U = torch.empty((ku, self.n), dtype=self.out_dtype, pin_memory=True).t()
            sigma = torch.empty(self.l, dtype=torch.float64, pin_memory=True)
            C = torch.empty((self.m, self.k), dtype=self.out_dtype, pin_memory=True).t()
        elif out is None:
            U = empty_colmajor(self.n, ku, self.out_dtype, self.device)
            sigma = torch.empty(self.l, dtype=torch.float64, device=self.device)
            C = empty_colmajor(self.k, self.m, self.out_dtype, self.device)
        else:
            U, sigma, C = out
        ref_ptr, ldr = (0, 0)
        if S_refine is not None:
            ref_ptr, ldr = S_refine.data_ptr(), colmajor_ld(S_refine)
        rc = rpod_basis(self.handle, S.data_ptr(), colmajor_ld(S), dtype_code(S.dtype), ref_ptr or None,
                        ldr, U.data_ptr(), colmajor_ld(U), sigma.data_ptr(), C.data_ptr(),
                        colmajor_ld(C), self.ws_ptr, self.ws_bytes, self._stream())
        _check(rc, "rpod_basis")
        return U, sigma, C

    def project(self, U, S_new, out=None):
        """C' = U^T S' (kc x m_new, column-major)."""
        kc = U.shape[1]
        m_new = S_new.shape[1]
        C = out if out is not None else empty_colmajor(kc, m_new, self.out_dtype, self.device)
        rc = rpod_project(self.handle, U.data_ptr(), colmajor_ld(U), kc, S_new.data_ptr(),
                          colmajor_ld(S_new), m_new, dtype_code(S_new.dtype), C.data_ptr(),
                          colmajor_ld(C), self.ws_ptr, self.ws_bytes, self._stream())
        _check(rc, "rpod_project")
        return C

    def save_basis(self, path, U, sigma, C):
        """Writes the plan's parameters and the outputs of basis() to a file
        (read back by load_basis)."""
        _check(rpod_basis_save(self.handle, path, U.data_ptr(), colmajor_ld(U), sigma.data_ptr(),
                               C.data_ptr(), colmajor_ld(C), self._stream()), "rpod_basis_save")

    def status(self):
        """(status code, warning flags) after synchronising the stream."""
        return rpod_status_sync(self.handle, self.ws_ptr, self._stream())

    def launches(self):
        return rpod_last_launch_count(self.handle)

    def set_graph(self, enable):
        """Graph replay of repeated basis calls with unchanged buffers
        (rpod_plan_set_graph; on by default)."""
        _check(rpod_plan_set_graph(self.handle, 1 if enable else 0), "rpod_plan_set_graph")

    def set_svd_sweeps(self, max_sweeps):
        """Caps the FP64 form's one-sided Jacobi sweeps (rpod_plan_set_svd_sweeps)."""
        _check(rpod_plan_set_svd_sweeps(self.handle, max_sweeps), "rpod_plan_set_svd_sweeps")

    def svd_sweeps(self):
        """Jacobi sweeps the last FP64 basis call ran (diagnostic word 5 of the
        workspace's status block); synchronises the device."""
        torch = _torch()
        torch.cuda.synchronize(self.device)
        off = self.ws_ptr - self.ws.data_ptr()
        return int(self.ws[off + 20:off + 24].cpu().view(torch.int32).item())

    def sketch(self, dtype=None):
        """The plan's Gaussian sketch Lambda (m x l, column-major)."""
        torch = _torch()
        dtype = dtype or self.out_dtype
        Lam = empty_colmajor(self.m, self.l, dtype, self.device)
        _check(rpod_sketch(self.handle, Lam.data_ptr(), colmajor_ld(Lam), dtype_code(dtype),
                           self._stream()), "rpod_sketch")
        return Lam

    def profile(self, enable=True):
        _check(rpod_profile_enable(self.handle, enable), "rpod_profile_enable")

    def profile_read(self):
        """(passes, summed pass ms, algorithmic bytes, flops) of the last basis call."""
        return rpod_profile_read(self.handle)


class Batch:
    """A batch of independent rPOD instances over column-major torch tensors
    S_b (n_b x m_b) on one device; outputs U_b, sigma_b, C_b are allocated
    here and stay fixed (the captured graph writes into them)."""

    def __init__(self, S_list, ks, p, q, seeds, compute="f32", flags=0, S_refine=None,
                 device="cuda"):
        torch = _torch()
        self.device = torch.device(device)
        self.compute = {"f64": RPOD_F64, "f32": RPOD_F32, "bf16": RPOD_BF16,
                        "f16": RPOD_F16}[compute] if isinstance(compute, str) else int(compute)
        out_dt = torch.float64 if self.compute == RPOD_F64 else torch.float32
        self.S = list(S_list)
        self.S_refine = list(S_refine) if S_refine is not None else [None] * len(self.S)
        self.U, self.sigma, self.C, insts = [], [], [], []
        for b, S in enumerate(self.S):
            n, m = S.shape
            k = int(ks[b])
            l = k + p
            ku = l if (flags & RPOD_FLAG_RETURN_ALL_L) else k
            U = empty_colmajor(n, ku, out_dt, self.device)
            sg = torch.empty(l, dtype=torch.float64, device=self.device)
            C = empty_colmajor(k, m, out_dt, self.device)
            self.U.append(U)
            self.sigma.append(sg)
            self.C.append(C)
            R = self.S_refine[b]
            insts.append(Instance(n, m, k, p, q, int(seeds[b]), S.data_ptr(), colmajor_ld(S),
                                  R.data_ptr() if R is not None else None,
                                  colmajor_ld(R) if R is not None else 0, U.data_ptr(),
                                  colmajor_ld(U), sg.data_ptr(), C.data_ptr(), colmajor_ld(C)))
        self.s_dtype = dtype_code(self.S[0].dtype)
        self.flags = flags
        self.shapes = [[int(S.shape[0]), int(S.shape[1]), int(ks[b]), int(p), int(q)]
                       for b, S in enumerate(self.S)]
        self.handle = rpod_batch_create(insts, self.compute, flags, self.s_dtype)
        self.ws_bytes = rpod_batch_workspace_bytes(self.handle)
        self.ws = torch.empty(self.ws_bytes + 256, dtype=torch.uint8, device=self.device)
        self.ws_ptr = self.ws.data_ptr() + (-self.ws.data_ptr()) % 256

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            try:
                rpod_batch_destroy(h)
            except Exception:
                pass
            self.handle = None

    def _stream(self):
        return _torch().cuda.current_stream(self.device).cuda_stream

    def run(self):
        _check(rpod_batch_run(self.handle, self.ws_ptr, self.ws_bytes, self._stream()),
               "rpod_batch_run")

    def tune(self, trials=3, cache=None):
        """Autotunes the launch configuration (rpod_batch_tune) and returns
        (streams, split_pct, stages).  With `cache` (a JSON file path) a
        configuration tuned before for the same instance shapes, form, GPU
        and library build is applied without timing, and a new one is
        stored."""
        key = self._tune_key() if cache else None
        if cache:
            import json
            try:
                with open(cache) as f:
                    hit = json.load(f).get(key)
            except (OSError, ValueError):
                hit = None
            if hit:
                self.configure(hit[0], hit[1], hit[2])
                return tuple(hit)
        best = rpod_batch_tune(self.handle, self.ws_ptr, self.ws_bytes, self._stream(), trials)
        if cache:
            import json
            try:
                with open(cache) as f:
                    db = json.load(f)
            except (OSError, ValueError):
                db = {}
            db[key] = list(best)
            tmp = f"{cache}.tmp{os.getpid()}"
            with open(tmp, "w") as f:
                json.dump(db, f, indent=1, sort_keys=True)
            os.replace(tmp, cache)
        return best

    def _tune_key(self):
        import hashlib
        import json
        torch = _torch()
        with open(LIB_PATH, "rb") as f:
            lib = hashlib.sha256(f.read()).hexdigest()[:16]
        desc = {"compute": self.compute, "flags": self.flags, "s_dtype": self.s_dtype,
                "shapes": self.shapes, "gpu": torch.cuda.get_device_name(self.device), "lib": lib}
        return hashlib.sha256(json.dumps(desc, sort_keys=True).encode()).hexdigest()[:24]

    def configure(self, streams, split_pct, stages=None):
        _check(rpod_batch_configure(self.handle, streams, split_pct), "rpod_batch_configure")
        if stages is not None:
            _check(rpod_batch_set_pass_stages(self.handle, stages), "rpod_batch_set_pass_stages")

    def status(self):
        return rpod_batch_status_sync(self.handle, self.ws_ptr, self._stream())

    def launches(self):
        return rpod_batch_last_launch_count(self.handle)


# ---- LSTM (same-name wrappers and a torch convenience class) ---------------
RPOD_LSTM_FP32_WEIGHTS = 1


def rpod_lstm_create(in_dim, hidden, layers, out_dim, window, max_batch, flags=0):
    h = _p()
    _check(load().rpod_lstm_create(ctypes.byref(h), in_dim, hidden, layers, out_dim, window, max_batch,
                                   flags), "rpod_lstm_create")
    return h.value


def rpod_lstm_param_count(net):
    return load().rpod_lstm_param_count(net)


def rpod_lstm_workspace_bytes(net):
    b = ctypes.c_size_t()
    _check(load().rpod_lstm_workspace_bytes(net, ctypes.byref(b)), "rpod_lstm_workspace_bytes")
    return b.value


def rpod_lstm_set_params(net, theta, ws, ws_bytes, stream):
    return load().rpod_lstm_set_params(net, theta, ws, ws_bytes, stream)


def rpod_lstm_get_params(net, theta, ws, ws_bytes, stream):
    return load().rpod_lstm_get_params(net, theta, ws, ws_bytes, stream)


def rpod_lstm_forward(net, X, B, Y, ws, ws_bytes, stream):
    return load().rpod_lstm_forward(net, X, B, Y, ws, ws_bytes, stream)


def rpod_lstm_loss_grad(net, X, Yt, B, loss, grad, ws, ws_bytes, stream):
    return load().rpod_lstm_loss_grad(net, X, Yt, B, loss, grad, ws, ws_bytes, stream)


def rpod_lstm_train_step(net, X, Yt, B, lr, wd, loss, ws, ws_bytes, stream):
    return load().rpod_lstm_train_step(net, X, Yt, B, lr, wd, loss, ws, ws_bytes, stream)


def rpod_lstm_gather(net, series, mu, n_series, t_len, d, idx, B, X, Y, stream):
    return load().rpod_lstm_gather(net, series, mu, n_series, t_len, d, idx, B, X, Y, stream)


def rpod_lstm_rollout(net, window, B, mu_cols, steps, out, ws, ws_bytes, stream):
    return load().rpod_lstm_rollout(net, window, B, mu_cols, steps, out, ws, ws_bytes, stream)


def rpod_lstm_set_dropout(net, p, seed):
    return load().rpod_lstm_set_dropout(net, float(p), int(seed))


def rpod_lstm_train_epoch(net, series, mu, n_series, t_len, d, idx, n_windows, batch, lr, wd,
                          loss_out, ws, ws_bytes, stream):
    return load().rpod_lstm_train_epoch(net, series, mu, n_series, t_len, d, idx, n_windows, batch,
                                        lr, wd, loss_out, ws, ws_bytes, stream)


def rpod_lstm_save(net, path, ws, ws_bytes, stream):
    return load().rpod_lstm_save(net, os.fsencode(path), ws, ws_bytes, stream)


def rpod_lstm_load(path) -> int:
    h = _p()
    _check(load().rpod_lstm_load(ctypes.byref(h), os.fsencode(path)), "rpod_lstm_load")
    return h.value


def rpod_lstm_restore(net, ws, ws_bytes, stream):
    return load().rpod_lstm_restore(net, ws, ws_bytes, stream)


def rpod_lstm_dims(net):
    d = (_c_i32 * 7)()
    _check(load().rpod_lstm_dims(net, d), "rpod_lstm_dims")
    return tuple(int(v) for v in d)


def rpod_lstm_last_launch_count(net):
    return load().rpod_lstm_last_launch_count(net)


def rpod_lstm_status_sync(net, ws, stream):
    return load().rpod_lstm_status_sync(net, ws, stream)


def rpod_selftest_grid_barrier(seconds, stream):
    return load().rpod_selftest_grid_barrier(seconds, stream)


def rpod_lstm_destroy(net):
    load().rpod_lstm_destroy(net)


class LSTM:
    """An rpod_lstm plus its workspace on one CUDA device (torch tensors in,
    torch tensors out; all arithmetic in the library's kernels)."""

    def __init__(self, in_dim, hidden, layers, out_dim, window, max_batch, theta=None, device="cuda",
                 fp32_weights=False, _handle=None):
        torch = _torch()
        self.device = torch.device(device)
        self.dims = (in_dim, hidden, layers, out_dim, window)
        self.max_batch = max_batch
        self.fp32_weights = fp32_weights
        self.handle = _handle if _handle is not None else rpod_lstm_create(
            in_dim, hidden, layers, out_dim, window, max_batch,
            RPOD_LSTM_FP32_WEIGHTS if fp32_weights else 0)
        self.P = rpod_lstm_param_count(self.handle)
        self.ws_bytes = rpod_lstm_workspace_bytes(self.handle)
        self.ws = torch.empty(self.ws_bytes + 256, dtype=torch.uint8, device=self.device)
        self.ws_ptr = self.ws.data_ptr() + (-self.ws.data_ptr()) % 256
        self.loss = torch.zeros(1, dtype=torch.float32, device=self.device)
        if theta is not None:
            self.set_params(theta)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            try:
                rpod_lstm_destroy(h)
            except Exception:
                pass
            self.handle = None

    def _stream(self):
        return _torch().cuda.current_stream(self.device).cuda_stream

    def set_params(self, theta):
        torch = _torch()
        t = torch.as_tensor(theta, dtype=torch.float32).to(self.device).contiguous()
        assert t.numel() == self.P
        self._theta_in = t
        _check(rpod_lstm_set_params(self.handle, t.data_ptr(), self.ws_ptr, self.ws_bytes, self._stream()),
               "rpod_lstm_set_params")

    @classmethod
    def load(cls, path, device="cuda"):
        """A network from a model file written by save(), with its
        parameters, Adam state and dropout settings restored."""
        h = rpod_lstm_load(path)
        I, H, L, O, T, Bmax, flags = rpod_lstm_dims(h)
        net = cls(I, H, L, O, T, Bmax, device=device,
                  fp32_weights=bool(flags & RPOD_LSTM_FP32_WEIGHTS), _handle=h)
        _check(rpod_lstm_restore(h, net.ws_ptr, net.ws_bytes, net._stream()), "rpod_lstm_restore")
        return net

    def save(self, path):
        _check(rpod_lstm_save(self.handle, path, self.ws_ptr, self.ws_bytes, self._stream()),
               "rpod_lstm_save")

    def train_epoch(self, series, mu, idx, batch, lr=1e-3, weight_decay=1e-5):
        """One epoch over the window list idx ((n, 2) int32 device tensor of
        (series, first step), in training order); returns the mean batch
        loss as a 1-element device tensor."""
        torch = _torch()
        series, mu, idx = series.contiguous(), mu.contiguous(), idx.contiguous()
        n_series, t_len = series.shape[0], series.shape[1]
        d = mu.shape[1] if mu.dim() == 2 else 0
        out = torch.empty(1, dtype=torch.float32, device=self.device)
        _check(rpod_lstm_train_epoch(self.handle, series.data_ptr(), mu.data_ptr() if d else None,
                                     n_series, t_len, d, idx.data_ptr(), idx.shape[0], batch, lr,
                                     weight_decay, out.data_ptr(), self.ws_ptr, self.ws_bytes,
                                     self._stream()), "rpod_lstm_train_epoch")
        return out

    def set_dropout(self, p, seed=0):
        """Dropout between stacked layers in later training passes (the
        mask definition is in include/rpod.h); p = 0 switches it off."""
        _check(rpod_lstm_set_dropout(self.handle, p, seed), "rpod_lstm_set_dropout")

    def get_params(self):
        torch = _torch()
        t = torch.empty(self.P, dtype=torch.float32, device=self.device)
        _check(rpod_lstm_get_params(self.handle, t.data_ptr(), self.ws_ptr, self.ws_bytes, self._stream()),
               "rpod_lstm_get_params")
        return t

    def forward(self, X):
        torch = _torch()
        X = X.contiguous()
        B = X.shape[0]
        Y = torch.empty((B, self.dims[3]), dtype=torch.float32, device=self.device)
        _check(rpod_lstm_forward(self.handle, X.data_ptr(), B, Y.data_ptr(), self.ws_ptr, self.ws_bytes,
                                 self._stream()), "rpod_lstm_forward")
        return Y

    def loss_grad(self, X, Yt):
        torch = _torch()
        X, Yt = X.contiguous(), Yt.contiguous()
        g = torch.empty(self.P, dtype=torch.float32, device=self.device)
        _check(rpod_lstm_loss_grad(self.handle, X.data_ptr(), Yt.data_ptr(), X.shape[0], self.loss.data_ptr(),
                                   g.data_ptr(), self.ws_ptr, self.ws_bytes, self._stream()),
               "rpod_lstm_loss_grad")
        return self.loss.clone(), g

    def train_step(self, X, Yt, lr=1e-3, weight_decay=1e-5):
        _check(rpod_lstm_train_step(self.handle, X.data_ptr(), Yt.data_ptr(), X.shape[0], lr, weight_decay,
                                    self.loss.data_ptr(), self.ws_ptr, self.ws_bytes, self._stream()),
               "rpod_lstm_train_step")
        return self.loss

    def gather(self, series, mu, idx):
        """Windows (X, Y) for rows idx (B, 2) = (series, first step) of
        series (n_series, t_len, out_dim) and mu (n_series, d)."""
        torch = _torch()
        series, idx = series.contiguous(), idx.to(torch.int32).contiguous()
        n_series, t_len, _ = series.shape
        d = 0 if mu is None else mu.shape[1]
        B = idx.shape[0]
        X = torch.empty((B, self.dims[4], self.dims[0]), dtype=torch.float32, device=self.device)
        Y = torch.empty((B, self.dims[3]), dtype=torch.float32, device=self.device)
        mptr = mu.contiguous().data_ptr() if mu is not None else None
        _check(rpod_lstm_gather(self.handle, series.data_ptr(), mptr, n_series, t_len, d, idx.data_ptr(), B,
                                X.data_ptr(), Y.data_ptr(), self._stream()), "rpod_lstm_gather")
        return X, Y

    def rollout(self, window, mu_cols, steps):
        torch = _torch()
        window = window.contiguous()
        B = window.shape[0]
        out = torch.empty((B, steps, self.dims[3]), dtype=torch.float32, device=self.device)
        _check(rpod_lstm_rollout(self.handle, window.data_ptr(), B, mu_cols, steps, out.data_ptr(), self.ws_ptr,
                                 self.ws_bytes, self._stream()), "rpod_lstm_rollout")
        return out

    def launches(self):
        return rpod_lstm_last_launch_count(self.handle)

    def status(self):
        """Device status of the last persistent rollout (RPOD_OK or
        RPOD_ERR_TIMEOUT); synchronises the stream."""
        return rpod_lstm_status_sync(self.handle, self.ws_ptr, self._stream())
