"""Standard against residual Chebyshev filtering with the approximate M~^-1
(Sec. III.B, Fig. 1) on the GPU.

Orchestration only: every computation is a libefe call (efe_atomic_density,
efe_smeared_charge, efe_poisson, efe_xc, efe_set_potential, efe_chfsi_kind).
For each workload the operator is the non-self-consistent (Harris) potential
of the superposed atomic densities; from the same seeded start vectors and
Lanczos vector the multipass eigensolver runs with each filter in each
precision and records, after every pass, the largest residual
||H psi - eps M^E psi|| of the occupied states.  bf16 runs keep bf16 in every
pass (no switch to FP32).  The occupied eigenvalues of every run are compared
with those of the FP64 residual run (or, where FP64 is not run, the FP32
residual run).

Usage: python -m paper_2607_06848_gb300.ablation [--workloads dimer cluster8 cluster64]
       [--passes 25] [--tol 1e-10] [--precisions fp64 fp32 bf16]
"""
import argparse
import json
import time

from . import workloads as W
from .efe import (EFE, EFE_FILTER_KEEP_PRECISION, EFE_FILTER_RESIDUAL, EFE_FILTER_STANDARD,
                  EFEError, PRECISIONS)

ENRICH = dict(alpha=1.2, r_end=5.0, t=0.33)
WORKLOADS = dict(dimer=W.dimer, cluster8=W.cluster8, cluster64=W.cluster64)


def harris_system(w):
    """The EFE system of workload w with v = v_xc[rho0] + phi[rho0 + b_sm] set."""
    import torch
    g = EFE(w["h"], w["ncell"], w["p"], w["atoms"], w["Z"], enrich=ENRICH,
            psp=dict(rc=1.0, r_trunc=6.0, h=w["hproj"], rloc=0.8))
    d = g.dims
    rho0 = torch.empty(d["n_quad"], dtype=torch.float64, device="cuda")
    bq = torch.empty_like(rho0)
    g.efe_atomic_density(2.4, rho0)
    g.efe_smeared_charge(bq)
    phi = torch.empty(d["n_nodes"], dtype=torch.float64, device="cuda")
    phq = torch.empty_like(rho0)
    g.efe_poisson(rho0 + bq, phi, phq, tol=1e-10)
    v = torch.empty_like(rho0)
    g.efe_xc(rho0, v, None)
    v += phq
    g.efe_set_potential(v)
    return g


def run(g, w, kind, precision, passes, tol, seed=1234):
    import torch
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    rows, N = g.dims["n_rows"], w["nstates"]
    X = torch.randn((rows, N), generator=gen, dtype=torch.float64, device="cuda")
    u0 = torch.randn((rows, 1), generator=gen, dtype=torch.float64, device="cuda")
    nocc = int(round(float(sum(w["Z"])) / 2))
    flags = kind | (EFE_FILTER_KEEP_PRECISION if precision == "bf16" else 0)
    rec = dict(workload=w["name"], filter="standard" if kind == EFE_FILTER_STANDARD else "residual",
               precision=precision)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    try:
        eig, res, npass, ok, hist = g.efe_chfsi_kind(X, w["cheb_degree"], kind=flags, u0=u0, max_pass=passes,
                                                     tol=tol, nconv=nocc, prec=PRECISIONS[precision])
    except EFEError as exc:
        # a run whose vectors blow up ends in a failed Rayleigh-Ritz: a result of the ablation
        torch.cuda.synchronize()
        rec.update(failed=str(exc), seconds=time.perf_counter() - t0, eig_occ=None)
        return rec
    torch.cuda.synchronize()
    rec.update(passes=npass, converged=bool(ok), seconds=time.perf_counter() - t0,
               min_resid=float(min(hist)) if len(hist) else None, history=[float(x) for x in hist],
               eig_occ=[float(x) for x in eig[:nocc]])
    return rec


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workloads", nargs="+", default=["dimer", "cluster8", "cluster64"])
    ap.add_argument("--passes", type=int, default=25)
    ap.add_argument("--tol", type=float, default=1e-10)
    ap.add_argument("--precisions", nargs="+", default=None,
                    help="default: fp64 fp32 bf16 (cluster64: fp32 bf16)")
    args = ap.parse_args(argv)
    out = []
    for name in args.workloads:
        w = WORKLOADS[name]()
        g = harris_system(w)
        precs = args.precisions or (["fp32", "bf16"] if name == "cluster64" else ["fp64", "fp32", "bf16"])
        runs = [run(g, w, kind, p, args.passes, args.tol)
                for p in precs for kind in (EFE_FILTER_RESIDUAL, EFE_FILTER_STANDARD)]
        ref = next(r for r in runs if r["filter"] == "residual" and r["eig_occ"])
        key = "max_eig_err_vs_" + ref["precision"] + "_residual"
        for r in runs:
            if r["eig_occ"]:
                r[key] = max(abs(a - b) for a, b in zip(r["eig_occ"], ref["eig_occ"]))
        for r in runs:
            del r["eig_occ"]
            print(json.dumps(r), flush=True)
        out += runs
        g.close()
    return out


if __name__ == "__main__":
    main()
