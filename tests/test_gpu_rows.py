"""Row-sharded Alg. 1 through the C ABI (rpod_rows_plan_create,
rpod_basis_rows): two and three row blocks of one matrix on one GPU, one
host thread per block, the exchanges combined on the host.  The blocks'
results must equal the row-sharded oracle (oracle/sharded.py, the same
algebra in numpy), the single-process oracle on the whole matrix and the
library's single-block rpod_basis.  No kernel waits on another block: every
exchange goes through the host."""
import threading

import numpy as np
import pytest
import torch

import paper_2504_15350_gb300.rpod as R
from oracle.rpod import rpod as oracle_rpod
from oracle.sharded import rpod_rows as oracle_rows
from paper_2504_15350_gb300.rows import RowsPlan, ThreadComm
from paper_2504_15350_gb300.shard import row_blocks
from synth import make_recipe, snapshot_matrix
from tests.rpod_checks import F64_FLOOR, max_angle, orth_err, sigma_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2504_15350_gb300.build import build
    build()
    R.load()


def _run_threads(world, fn):
    out, err = [None] * world, []

    def body(r):
        try:
            out[r] = fn(r)
        except Exception as e:  # surfaced below
            err.append(e)

    th = [threading.Thread(target=body, args=(r,)) for r in range(world)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    if err:
        raise err[0]
    return out


def _gpu_rows(S, blocks, k, p, q, seed, flags=0):
    world = len(blocks)
    comm = ThreadComm(world)
    Sd = S.t().contiguous().cuda().t()

    def one(r):
        r0, nr = blocks[r]
        st = torch.cuda.Stream()
        with torch.cuda.stream(st):
            plan = RowsPlan(S.shape[0], r0, nr, S.shape[1], k, p, q, seed=seed, compute="f64", flags=flags)
            U, sig, C = plan.basis(Sd[r0:r0 + nr], comm.rank(r))
            rc, warn = plan.status()
            st.synchronize()
            return U.cpu().numpy(), sig.cpu().numpy(), C.cpu().numpy(), rc, warn
    return _run_threads(world, one)


def _oracle_rows(S, blocks, k, p, q, seed):
    """oracle/sharded.py on the same blocks, one host thread per block."""
    world = len(blocks)
    comm = ThreadComm(world)
    box = [None] * world

    def one(r):
        r0, nr = blocks[r]
        loc = comm.rank(r)

        def allreduce(a):
            t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64))
            loc.allreduce(t, "sum")
            return t.numpy()

        def allgather(obj):
            box[r] = obj
            comm.bar.wait()
            gathered = list(box)
            comm.bar.wait()
            return gathered
        return oracle_rows(S[r0:r0 + nr], r0, k, p, q, seed, allreduce, allgather)
    return _run_threads(world, one)


@pytest.mark.parametrize("world,align", [(2, 64), (3, 64), (3, 512)])
def test_rows_match_sharded_and_single_process_oracles(world, align):
    rec = make_recipe(64, 64, 500, 400, ("power", 1.5), seed=0, noise=1e-6)
    S = snapshot_matrix(rec).numpy()                      # 4096 x 500, FP64
    k, p, q, seed = 20, 10, 1, 0
    blocks = row_blocks(S.shape[0], world, align)
    res = _gpu_rows(torch.from_numpy(S).t().contiguous().t(), blocks, k, p, q, seed)
    for r in range(world):
        assert res[r][3] == R.RPOD_OK, (r, R.rpod_strerror(res[r][3]))
    U = np.concatenate([res[r][0] for r in range(world)], 0)
    sig, C = res[0][1], res[0][2]
    for r in range(1, world):                             # replicated results agree bit for bit
        assert np.array_equal(res[r][1], sig) and np.array_equal(res[r][2], C)
    o = oracle_rpod(S, k, p, q, seed=seed)
    ok, er, ea = sigma_close(sig, o.sigma, 1e-10, 1e-12, floor=F64_FLOOR)
    assert ok, (er, ea)
    assert max_angle(o.U[:, :k], U) <= 1e-8
    assert orth_err(U) <= 1e-12
    idx = np.argmax(np.abs(U), axis=0)
    assert np.all(U[idx, np.arange(k)] > 0)               # sign rule over the whole U
    assert np.abs(C - o.C).max() <= 1e-9 * o.sigma[0]
    # the row-sharded oracle (same blocks, same algebra)
    orr = _oracle_rows(S, blocks, k, p, q, seed)
    Uo = np.concatenate([x.U[:, :k] for x in orr], 0)
    assert np.allclose(sig, orr[0].sigma, rtol=1e-10, atol=1e-12 * sig[0])
    assert np.abs(U - Uo).max() <= 1e-8
    # and the library's single-block form
    plan = R.Plan(S.shape[0], S.shape[1], k, p, q, seed=seed, compute="f64")
    U1, s1, C1 = plan.basis(torch.from_numpy(S).t().contiguous().cuda().t())
    assert np.allclose(sig, s1.cpu().numpy(), rtol=1e-12, atol=1e-14 * sig[0])
    assert np.abs(U - U1.cpu().numpy()).max() <= 1e-10


def test_rows_graded_spectrum_and_return_all_l():
    """Three blocks of an eight-decade spectrum with all l columns returned:
    the same relative accuracy as the single-block FP64 form."""
    rng = np.random.default_rng(9)
    n, m, l, k = 3000, 400, 40, 30
    U0, _ = np.linalg.qr(rng.standard_normal((n, l)))
    V0, _ = np.linalg.qr(rng.standard_normal((m, l)))
    s = np.logspace(0, -8, l)
    S = (U0 * s) @ V0.T
    blocks = row_blocks(n, 3, 64)
    res = _gpu_rows(torch.from_numpy(S).t().contiguous().t(), blocks, k, l - k, 1, 0,
                    flags=R.RPOD_FLAG_RETURN_ALL_L)
    assert all(x[3] == R.RPOD_OK for x in res)
    sig = res[0][1]
    U = np.concatenate([x[0] for x in res], 0)
    top = s >= 1e-7 * s[0]
    e = np.abs(sig - s) / s
    assert e[top].max() <= 1e-10 and e.max() <= 1e-9, e.max()
    assert U.shape == (n, l) and orth_err(U) <= 1e-12


def test_rows_failed_exchange_and_wrong_plans():
    class Failing:
        calls = 0

        def allreduce(self, t, op):
            Failing.calls += 1
            if Failing.calls == 3:
                raise RuntimeError("link down")
            # one block: the combination is the identity

    rng = np.random.default_rng(1)
    S = torch.from_numpy(rng.standard_normal((600, 200))).t().contiguous().cuda().t()
    plan = RowsPlan(600, 0, 600, 200, 8, 4, 1, compute="f64")
    with pytest.raises(R.RpodError) as e:
        plan.basis(S, Failing())
    assert e.value.code == R.RPOD_ERR_EXCHANGE and Failing.calls == 3
    # rpod_basis refuses a row plan; row plans support the FP64 form only
    U = torch.empty(1, device="cuda")
    rc = R.rpod_basis(plan.handle, S.data_ptr(), 600, R.RPOD_F64, None, 0, U.data_ptr(), 600,
                      U.data_ptr(), U.data_ptr(), 8, plan.ws_ptr, plan.ws_bytes, 0)
    assert rc == R.RPOD_ERR_INVALID_ARG
    with pytest.raises(R.RpodError) as e:
        RowsPlan(600, 0, 300, 200, 8, 4, 1, compute="f32")
    assert e.value.code == R.RPOD_ERR_UNSUPPORTED
    with pytest.raises(R.RpodError) as e:
        RowsPlan(600, 400, 300, 200, 8, 4, 1, compute="f64")      # rows past n_total
    assert e.value.code == R.RPOD_ERR_INVALID_ARG
