"""CPU tests of the C ABI boundary: the library builds, loads and exports
every function declared in include/*.h; host-side argument checks return
their documented codes without touching a GPU."""
import ctypes
import glob
import os
import re

import pytest

import paper_2504_15350_gb300.rpod as R
from paper_2504_15350_gb300.build import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        # function declarations; typedefs of callback types are not symbols
        for m in re.finditer(r"^\s*(?!typedef\b)(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*"
                             r"([a-z][a-z0-9_]*)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    build()
    return R.load()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "rpod_basis" in names and "rpod_plan_create" in names
    for n in names:
        assert hasattr(lib, n), n
    # the binding declares exactly the header's rpod_ functions
    assert {n for n in names if n.startswith("rpod_")} <= set(R.SIGNATURES) | {
        n for n in names if not n.startswith("rpod_")}


def test_plan_argument_checks(lib):
    h = ctypes.c_void_p()
    bad = [(0, 10, 1, 0, 1), (10, 0, 1, 0, 1), (100, 50, 0, 5, 1), (100, 50, 5, -1, 1),
           (100, 50, 5, 5, -1), (100, 50, 40, 20, 1), (1000, 1000, 100, 29, 1)]
    for n, m, k, p, q in bad:
        assert lib.rpod_plan_create(ctypes.byref(h), n, m, k, p, q, 0, R.RPOD_F32, 0) == R.RPOD_ERR_INVALID_ARG
    assert lib.rpod_plan_create(ctypes.byref(h), 100, 50, 5, 5, 1, 0, 9, 0) == R.RPOD_ERR_INVALID_ARG
    assert lib.rpod_plan_create(ctypes.byref(h), 100, 50, 5, 5, 1, 0, R.RPOD_F32, 1 << 9) == R.RPOD_ERR_INVALID_ARG
    assert lib.rpod_plan_create(None, 100, 50, 5, 5, 1, 0, R.RPOD_F32, 0) == R.RPOD_ERR_INVALID_ARG
    assert lib.rpod_plan_create(ctypes.byref(h), 100, 50, 100 - 28, 28, 1, 0, R.RPOD_F32, 0) == R.RPOD_ERR_INVALID_ARG


def test_workspace_and_pointer_checks(lib):
    plan = R.rpod_plan_create(4096, 500, 20, 10, 1, 0, R.RPOD_F64)
    try:
        ws = R.rpod_workspace_bytes(plan)
        assert ws > 4096 * 30 * 8
        fake = 1 << 20
        # missing workspace, short workspace, misaligned workspace
        assert R.rpod_basis(plan, fake, 4096, R.RPOD_F64, None, 0, fake, 4096, fake, fake, 20, None, ws, None) == R.RPOD_ERR_WORKSPACE
        assert R.rpod_basis(plan, fake, 4096, R.RPOD_F64, None, 0, fake, 4096, fake, fake, 20, fake, ws - 1, None) == R.RPOD_ERR_WORKSPACE
        assert R.rpod_basis(plan, fake, 4096, R.RPOD_F64, None, 0, fake, 4096, fake, fake, 20, fake + 8, ws, None) == R.RPOD_ERR_WORKSPACE
        # leading dimensions and dtype
        assert R.rpod_basis(plan, fake, 4095, R.RPOD_F64, None, 0, fake, 4096, fake, fake, 20, fake, ws, None) == R.RPOD_ERR_INVALID_ARG
        assert R.rpod_basis(plan, fake, 4096, R.RPOD_F64, None, 0, fake, 4096, fake, fake, 19, fake, ws, None) == R.RPOD_ERR_INVALID_ARG
        assert R.rpod_basis(plan, fake, 4096, R.RPOD_F32, None, 0, fake, 4096, fake, fake, 20, fake, ws, None) == R.RPOD_ERR_INVALID_ARG
        assert R.rpod_basis(plan, None, 4096, R.RPOD_F64, None, 0, fake, 4096, fake, fake, 20, fake, ws, None) == R.RPOD_ERR_INVALID_ARG
        assert R.rpod_project(plan, fake, 4096, 31, fake, 4096, 10, R.RPOD_F64, fake, 31, fake, ws, None) == R.RPOD_ERR_INVALID_ARG
    finally:
        R.rpod_plan_destroy(plan)


def test_strerror_covers_codes(lib):
    for c in range(9):
        assert R.rpod_strerror(c) != "unknown status"
    assert R.rpod_strerror(99) == "unknown status"


def test_fluctuation_and_energy_rank_argument_checks(lib):
    # nt must divide m; S and Sbar must be given; leading dimensions >= n
    assert lib.rpod_fluctuations(10, 9, 2, 1, 10, R.RPOD_F32, None, 0, 0, None, 0, 0, 1, 10,
                                 None) == R.RPOD_ERR_INVALID_ARG
    assert lib.rpod_fluctuations(10, 8, 2, None, 10, R.RPOD_F32, None, 0, 0, None, 0, 0, 1, 10,
                                 None) == R.RPOD_ERR_INVALID_ARG
    assert lib.rpod_fluctuations(10, 8, 2, 1, 10, R.RPOD_F32, None, 0, 0, None, 0, 0, None, 10,
                                 None) == R.RPOD_ERR_INVALID_ARG
    assert lib.rpod_fluctuations(10, 8, 2, 1, 9, R.RPOD_F32, None, 0, 0, None, 0, 0, 1, 10,
                                 None) == R.RPOD_ERR_INVALID_ARG
    assert lib.rpod_fluctuations(10, 8, 0, 1, 10, R.RPOD_F32, None, 0, 0, None, 0, 0, 1, 10,
                                 None) == R.RPOD_ERR_INVALID_ARG
    assert lib.rpod_fluctuations(10, 8, 2, 1, 10, 7, None, 0, 0, None, 0, 0, 1, 10,
                                 None) == R.RPOD_ERR_INVALID_ARG
    # in place with another type, and unsupported type pairs
    assert lib.rpod_fluctuations(10, 8, 2, 64, 10, R.RPOD_F32, 64, 10, R.RPOD_BF16, None, 0, 0,
                                 1, 10, None) == R.RPOD_ERR_INVALID_ARG
    assert lib.rpod_fluctuations(10, 8, 2, 64, 10, R.RPOD_F64, 128, 10, R.RPOD_F32, None, 0, 0,
                                 1, 10, None) == R.RPOD_ERR_UNSUPPORTED
    assert lib.rpod_fluctuations(10, 8, 2, 64, 10, R.RPOD_F64, None, 0, 0, 128, 10, R.RPOD_BF16,
                                 1, 10, None) == R.RPOD_ERR_UNSUPPORTED
    assert lib.rpod_fluctuations(10, 8, 2, 64, 10, R.RPOD_F32, None, 0, 0, 128, 10, R.RPOD_F32,
                                 1, 10, None) == R.RPOD_ERR_UNSUPPORTED
    assert lib.rpod_energy_rank(1, 4, 0.0, 1, None) == R.RPOD_ERR_INVALID_ARG
    assert lib.rpod_energy_rank(1, 4, 1.5, 1, None) == R.RPOD_ERR_INVALID_ARG
    assert lib.rpod_energy_rank(1, 0, 0.5, 1, None) == R.RPOD_ERR_INVALID_ARG
    assert lib.rpod_energy_rank(None, 4, 0.5, 1, None) == R.RPOD_ERR_INVALID_ARG


def test_lstm_file_and_epoch_argument_checks(lib, tmp_path):
    h = ctypes.c_void_p()
    assert lib.rpod_lstm_load(ctypes.byref(h), str(tmp_path / "missing.bin").encode()) == R.RPOD_ERR_IO
    bad = tmp_path / "bad.bin"
    bad.write_bytes(b"not a model file" * 10)
    assert lib.rpod_lstm_load(ctypes.byref(h), str(bad).encode()) == R.RPOD_ERR_IO
    assert lib.rpod_lstm_load(None, str(bad).encode()) == R.RPOD_ERR_INVALID_ARG
    assert R.rpod_strerror(R.RPOD_ERR_IO) == "file could not be read or written"
    net = R.rpod_lstm_create(6, 8, 2, 2, 3, 4)
    try:
        assert R.rpod_lstm_dims(net) == (6, 8, 2, 2, 3, 4, 0)
        # no loaded state to restore
        assert lib.rpod_lstm_restore(net, None, 0, None) == R.RPOD_ERR_INVALID_ARG
        # batch above max_batch, no full batch, d + out_dim != in_dim
        assert lib.rpod_lstm_train_epoch(net, 1, 1, 2, 10, 4, 1, 10, 8, 1e-3, 1e-5, None, None, 0,
                                         None) == R.RPOD_ERR_INVALID_ARG
        assert lib.rpod_lstm_train_epoch(net, 1, 1, 2, 10, 4, 1, 3, 4, 1e-3, 1e-5, None, None, 0,
                                         None) == R.RPOD_ERR_INVALID_ARG
        assert lib.rpod_lstm_train_epoch(net, 1, 1, 2, 10, 3, 1, 10, 4, 1e-3, 1e-5, None, None, 0,
                                         None) == R.RPOD_ERR_INVALID_ARG
        # a valid call without a workspace
        assert lib.rpod_lstm_train_epoch(net, 1, 1, 2, 10, 4, 1, 10, 4, 1e-3, 1e-5, None, None, 0,
                                         None) == R.RPOD_ERR_WORKSPACE
        assert lib.rpod_lstm_save(net, b"x", None, 0, None) == R.RPOD_ERR_WORKSPACE
    finally:
        R.rpod_lstm_destroy(net)


def test_basis_file_errors(lib, tmp_path):
    info = (ctypes.c_int64 * 9)()
    assert lib.rpod_basis_file_info(str(tmp_path / "none.bin").encode(), info) == R.RPOD_ERR_IO
    bad = tmp_path / "bad.bin"
    bad.write_bytes(b"RPODBASE" + b"\0" * 100)      # right magic, wrong version
    assert lib.rpod_basis_file_info(str(bad).encode(), info) == R.RPOD_ERR_IO
    assert lib.rpod_basis_file_info(None, info) == R.RPOD_ERR_INVALID_ARG
    assert lib.rpod_basis_load(str(bad).encode(), None, 1, None, None, 1, None) == R.RPOD_ERR_INVALID_ARG
    assert lib.rpod_basis_save(None, b"x", 1, 1, 1, 1, 1, None) == R.RPOD_ERR_INVALID_ARG


def test_selftest_wait_argument_checks(lib):
    for bad in (0.0, -1.0, 3.0, float("nan")):
        assert lib.rpod_selftest_wait_timeout(bad, None) == R.RPOD_ERR_INVALID_ARG


def test_host_io_plan_workspace_and_batch_rejection(lib):
    p0 = R.rpod_plan_create(5000, 300, 10, 5, 1, 0, R.RPOD_F32, 0)
    p1 = R.rpod_plan_create(5000, 300, 10, 5, 1, 0, R.RPOD_F32, R.RPOD_FLAG_HOST_IO)
    try:
        # room for S (16-element-aligned columns) plus U, sigma and C
        assert R.rpod_workspace_bytes(p1) >= R.rpod_workspace_bytes(p0) + 4 * 5008 * 300
    finally:
        R.rpod_plan_destroy(p0)
        R.rpod_plan_destroy(p1)
    inst = R.Instance(n=100, m=50, k=5, p=2, q=1, seed=0, S=1, lds=100, S_refine=None, ldr=0,
                      U=1, ldu=100, sigma=1, C=1, ldc=5)
    h = ctypes.c_void_p()
    arr = (R.Instance * 1)(inst)
    assert lib.rpod_batch_create(ctypes.byref(h), 1, arr, R.RPOD_F32, R.RPOD_FLAG_HOST_IO,
                                 R.RPOD_F32) == R.RPOD_ERR_UNSUPPORTED
