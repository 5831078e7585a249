"""Writes the stored expected values under tests/golden/ from the oracle alone.

Run from the repository root:  python tests/golden/make_golden.py
It imports only ``oracle`` (and numpy); nothing here touches the CUDA path.
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle.problems import BakeoffProblem  # noqa: E402


def manufactured():
    dims, amp, tol = (2, 2, 2), 0.05, 1e-12
    orders = [2, 3, 4, 5, 6, 7]
    errs = []
    for N in orders:
        prob = BakeoffProblem(5, *dims, N, amp=amp)
        b, u_exact = prob.manufactured_rhs()
        x, _ = prob.solve(b, tol=tol)
        errs.append(float(np.max(np.abs(x - u_exact))))
    return {"source": "BP5 (Table 1) on the deformed unit cube, f = 3 pi^2 sin sin sin, "
                      "u = sin(pi x) sin(pi y) sin(pi z); max nodal error of the PCG solution",
            "dims": list(dims), "amp": amp, "tol": tol, "orders": orders,
            "max_nodal_error": errs}


if __name__ == "__main__":
    out = manufactured()
    with open(os.path.join(HERE, "manufactured_bp5.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out))
