"""Writes the stored expected values of tests/golden/ by calling only the FP64
oracle (no value here comes from the CUDA path).

    python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle.fe import Mesh  # noqa: E402
from oracle.efe import EFESystem  # noqa: E402
from oracle import scf as S  # noqa: E402
from paper_2607_06848_gb300 import workloads as W  # noqa: E402


def dimer_scf():
    """The 2-atom workload (8^3 cells, p = 4, 8 states, degree 20) SCF to 1e-8."""
    w = W.dimer()
    m = Mesh(w["h"], w["ncell"], w["p"])
    s = EFESystem(m, w["atoms"], enrich=dict(alpha=1.2, r0=5.0 * 0.33 / 1.33, t=0.33),
                  proj=dict(rc=1.0, rtrunc=6.0, h=w["hproj"]))
    rows = s.nn + s.n_enr
    X0 = W.random_block(rows, w["nstates"], 1)
    u0 = W.random_block(rows, 1, 2)
    X0[:s.nn] *= s.mask[:, None]
    u0[:s.nn] *= s.mask[:, None]
    out = S.scf(s, w["Z"], X0, u0, cheb_degree=w["cheb_degree"])
    return dict(source="oracle.scf.scf on workloads.dimer(); X0 = random_block(rows, 8, 1), "
                       "u0 = random_block(rows, 1, 2), boundary rows zeroed",
                E=out["E"], F=out["F"], mu=out["mu"], eig=[float(x) for x in out["eig"]],
                iters=out["iters"], history=[{k: float(v) for k, v in h.items()} for h in out["history"]])


if __name__ == "__main__":
    with open(os.path.join(HERE, "dimer_scf.json"), "w") as f:
        json.dump(dimer_scf(), f, indent=1)
    print("wrote dimer_scf.json")
