"""Writes tests/golden/rpod_small.json from the FP64 oracle only.

Case: synthetic recipe on an 8 x 16 grid (n = 128), m = 60 snapshots,
J = 40 modes with amplitudes j^-1.5, noise 1e-6, seed 7; Alg. 1 with
k = 6, p = 4, q = 1, sketch seed 11.  Stored: the l singular values, the
first row of the modal coefficients and the first basis column.

Run from the repository root:  python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle.rpod import rpod  # noqa: E402
from synth import make_recipe, snapshot_matrix  # noqa: E402

CASE = dict(nx=8, ny=16, m=60, J=40, decay=("power", 1.5), seed=7, noise=1e-6,
            k=6, p=4, q=1, sketch_seed=11)


def compute():
    c = CASE
    rec = make_recipe(c["nx"], c["ny"], c["m"], c["J"], c["decay"], seed=c["seed"], noise=c["noise"])
    S = snapshot_matrix(rec).numpy()
    r = rpod(S, c["k"], c["p"], c["q"], seed=c["sketch_seed"])
    return {"case": {**c, "decay": list(c["decay"])}, "sigma": r.sigma.tolist(),
            "C_row0": r.C[0].tolist(), "U_col0": r.U[:, 0].tolist()}


if __name__ == "__main__":
    with open(os.path.join(HERE, "rpod_small.json"), "w") as f:
        json.dump(compute(), f, indent=1)
