"""The allocation-free projection rpod_project_static, through the C ABI.

It serves callers that cannot allocate device memory or hand the library a
workspace (a framework that owns all device memory through its own pool, a
plugin callback that may not allocate, a loop that must not risk the
synchronisation an allocation can cause): its scratch is a fixed 16 MiB array
inside the library.  The test checks its output against rpod_project (the
workspace entry point) on two calls in a row, so the array's leftover
contents from one call cannot leak into the next, and that a request larger
than the array is refused.  This file is collected last on purpose."""
import pytest
import torch

import paper_2504_15350_gb300.rpod as R

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2504_15350_gb300.build import build
    build()
    R.load()


def _colmajor(rows, cols, dtype, gen):
    return torch.randn((cols, rows), generator=gen, dtype=torch.float64).to(dtype).cuda().t()


@pytest.mark.parametrize("compute,dtype,rel", [("f32", torch.float32, 1e-5), ("f64", torch.float64, 1e-12),
                                               ("bf16", torch.float32, 1e-5)])
def test_static_projection_matches_workspace_projection(compute, dtype, rel):
    """A 16-bit plan projects FP32 U and S' (its FP32 branch) like the F32 one."""
    g = torch.Generator().manual_seed(11)
    n, m, k, p = 20000, 3000, 24, 8
    plan = R.Plan(n, m, k, p, 1, compute=compute)
    stream = torch.cuda.current_stream().cuda_stream
    code = R.dtype_code(dtype)
    for call, (kc, m_new) in enumerate([(24, 3001), (32, 777)]):
        U = _colmajor(n, kc, dtype, g)
        S = _colmajor(n, m_new, dtype, g)
        ref = plan.project(U, S)
        C = torch.full((m_new, kc), float("nan"), dtype=dtype, device="cuda").t()
        rc = R.rpod_project_static(plan.handle, U.data_ptr(), R.colmajor_ld(U), kc, S.data_ptr(),
                                   R.colmajor_ld(S), m_new, code, C.data_ptr(), R.colmajor_ld(C),
                                   stream)
        assert rc == R.RPOD_OK, (call, R.rpod_strerror(rc))
        torch.cuda.synchronize()
        err = float((C.double() - ref.double()).abs().max() / ref.double().abs().max())
        assert err <= rel, (call, err)


def test_static_projection_rejects_oversized_request():
    plan = R.Plan(4096, 512, 100, 20, 1, compute="f32")
    U = torch.zeros((100, 4096), device="cuda").t()
    m_new = (16 << 20) // (4 * 100) + 1          # one column more than the array holds
    S = torch.zeros((m_new, 4096), device="cuda").t()
    C = torch.zeros((m_new, 100), device="cuda").t()
    rc = R.rpod_project_static(plan.handle, U.data_ptr(), 4096, 100, S.data_ptr(), 4096, m_new,
                               R.RPOD_F32, C.data_ptr(), 100, torch.cuda.current_stream().cuda_stream)
    assert rc == R.RPOD_ERR_UNSUPPORTED
    rc = R.rpod_project_static(plan.handle, U.data_ptr(), 4096, 100, S.data_ptr(), 4096, m_new,
                               R.RPOD_F64, C.data_ptr(), 100, torch.cuda.current_stream().cuda_stream)
    assert rc == R.RPOD_ERR_INVALID_ARG


def test_static_projection_rejects_16bit_snapshots():
    """Only FP32 (or FP64 for an FP64 plan) operands: 16-bit S' is refused
    before anything is enqueued."""
    plan = R.Plan(4096, 512, 16, 8, 1, compute="bf16")
    U = torch.zeros((16, 4096), device="cuda").t()
    S = torch.zeros((512, 4096), dtype=torch.bfloat16, device="cuda").t()
    C = torch.zeros((512, 16), device="cuda").t()
    rc = R.rpod_project_static(plan.handle, U.data_ptr(), 4096, 16, S.data_ptr(), 4096, 512,
                               R.RPOD_BF16, C.data_ptr(), 16, torch.cuda.current_stream().cuda_stream)
    assert rc == R.RPOD_ERR_INVALID_ARG
