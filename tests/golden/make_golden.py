"""Writes the stored expected values of tests/golden/ by calling only the FP64
oracle (no value here comes from the CUDA path).

    python tests/golden/make_golden.py [dimer] [atom]     (default: all)
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


def atom_scf():
    """One atom on the centre node of the dimer's mesh (8 states, degree 20): its
    Fermi level lies in the 3-fold p shell, so F != E.  SCF to 1e-8."""
    w = W.single_atom()
    m = Mesh(w["h"], w["ncell"], w["p"])
    s = EFESystem(m, w["atoms"], enrich=dict(alpha=1.2, r0=5.0 * 0.33 / 1.33, t=0.33),
                  proj=dict(rc=1.0, rtrunc=6.0, h=w["hproj"]))
    rows = s.nn + s.n_enr
    X0 = W.random_block(rows, w["nstates"], 1)
    u0 = W.random_block(rows, 1, 2)
    X0[:s.nn] *= s.mask[:, None]
    u0[:s.nn] *= s.mask[:, None]
    out = S.scf(s, w["Z"], X0, u0, cheb_degree=w["cheb_degree"])
    return dict(source="oracle.scf.scf on workloads.single_atom(); X0 = random_block(rows, 8, 1), "
                       "u0 = random_block(rows, 1, 2), boundary rows zeroed",
                E=out["E"], F=out["F"], mu=out["mu"], eig=[float(x) for x in out["eig"]],
                occ=[float(x) for x in out["occ"]], iters=out["iters"],
                history=[{k: float(v) for k, v in h.items()} for h in out["history"]])


CASES = {"dimer": dimer_scf, "atom": atom_scf}

if __name__ == "__main__":
    for name in (sys.argv[1:] or list(CASES)):
        with open(os.path.join(HERE, name + "_scf.json"), "w") as f:
            json.dump(CASES[name](), f, indent=1)
        print("wrote %s_scf.json" % name)
