"""Regression pin: the oracle reproduces the stored small-case output written
by tests/golden/make_golden.py (which calls only the oracle)."""
import json
import os

import numpy as np

from tests.golden.make_golden import compute

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_oracle_reproduces_golden():
    ref = json.load(open(os.path.join(HERE, "rpod_small.json")))
    now = compute()
    assert np.allclose(now["sigma"], ref["sigma"], rtol=1e-12)
    assert np.allclose(now["C_row0"], ref["C_row0"], rtol=1e-9, atol=1e-12 * ref["sigma"][0])
    assert np.allclose(now["U_col0"], ref["U_col0"], atol=1e-11)
