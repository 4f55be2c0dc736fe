#!/usr/bin/env python
"""Residual Chebyshev filter throughput on one GB300 (GDOF*vec*deg/s).

Workload (default): 64-atom seeded cluster (Z = 4, >= 4.2 bohr apart) in a
40-bohr cube, 24^3 cells of degree 6 (145^3 GLL grid, 2.92M interior FE DOF)
+ 256 enrichment DOF, 154 vectors, filter degree 30, bounds from a 10-step
Lanczos.  One step = one residual filter pass (eigen-residual G, 29 steps of
the recurrence with H M~^-1, V_out) -- the "filter" of the metric.
value = (FE DOF + enriched DOF) * vectors * degree / step time.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Multi-GPU runs are independent replicas (one per rank), weak scaling.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ChFSI GDOF·vec·deg/s, mixed vs FP64 at |ΔE|≤1e-5 Ha/atom; SCF time-to-solution"
UNIT = "GDOF*vec*deg/s"
T_ENR, R_END, ALPHA = 0.33, 5.0, 1.2


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = []
        with open(self.f.name) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def max_over_ranks(value, dist=None, device="cpu"):
    """The largest value over all ranks (the step time of the slowest replica)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_rank, world, ms_per_step):
    """Whole-job throughput in G-units/s: every rank runs its own replica (weak scaling)."""
    return units_per_rank * world / (ms_per_step / 1e3) / 1e9


def workload(name):
    from paper_2607_06848_gb300 import workloads as W
    if name == "cluster64":
        return W.cluster64()
    if name == "dimer":
        return W.dimer()
    if name == "cluster8":
        return W.cluster8()
    raise SystemExit("unknown workload " + name)


def cpu_sample(steps=1, warmup=0):
    """The FP64 oracle, as it stands, on a bounded sample of the same workload:
    the 64-atom cluster's discretisation (h = 40/24 bohr, degree 6, Gauss 8^3)
    on a 6^3-cell sub-box around one atom, 16 vectors, filter degree 30.
    Returns (GDOF*vec*deg/s, seconds per step, description, threads)."""
    from oracle.fe import Mesh
    from oracle.efe import EFESystem
    from oracle import chfsi as OC
    from paper_2607_06848_gb300 import workloads as W
    h = 40.0 / 24.0
    mesh = Mesh(h, (6, 6, 6), 6)
    atom = np.array([[5.0, 5.0, 5.0]])
    osys = EFESystem(mesh, atom, enrich=dict(alpha=ALPHA, r0=R_END * T_ENR / (1 + T_ENR), t=T_ENR),
                     proj=dict(rc=1.0, rtrunc=6.0, h=np.array([[1.0, -0.5]])))
    osys.set_potential(W.soft_coulomb_potential(mesh.all_quad_points(), atom))
    N, m = 16, 30
    V = W.random_block(osys.nn + osys.n_enr, N, 7)
    V[:osys.nn] *= osys.mask[:, None]
    lam, V, HV = OC.rayleigh_ritz(osys, V)
    b = OC.lanczos_bounds(osys, W.random_block(osys.nn + osys.n_enr, 1, 8), 10)[2]
    for _ in range(warmup):
        OC.residual_filter(osys, V, lam, m, lam[-1], b, lam[0], HV=HV)
    t0 = time.perf_counter()
    for _ in range(steps):
        OC.residual_filter(osys, V, lam, m, lam[-1], b, lam[0], HV=HV)
    dt = (time.perf_counter() - t0) / max(steps, 1)
    M = int(osys.mask.sum()) + osys.n_enr
    desc = ("oracle residual filter (FP64 NumPy/SciPy) on a 6^3-cell sub-box of the cluster64 "
            "discretisation around one atom: %d DOF x %d vectors x degree %d, %d steps"
            % (M, N, m, steps))
    return M * N * m / dt / 1e9, dt, desc, os.cpu_count()


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    val, dt, desc, cores = cpu_sample(steps=args.steps, warmup=args.warmup)
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "cluster64 (sampled sub-box for the CPU oracle)", "vectors": 16,
                       "filter_degree": 30},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _traffic_per_unit(name, key):
    """A per-unit DRAM traffic figure recorded from an ncu capture (profiles/<name>)."""
    try:
        with open(os.path.join(ROOT, "profiles", name)) as f:
            for line in f:
                if line.startswith(key):
                    return float(line.split()[1])
    except OSError:
        pass
    return None


def algorithmic_bytes_bf16(w, d, N, m):
    """Algorithmic HBM bytes of the bf16 filter, following the scope table's
    measurement rule: per recurrence step 4 arrays x 2 B per DOF x vector (read
    Y_{k-1} = M~^-1 Z_{k-1}, Y_{k-2}, Ghat; write Y_k -- bf16 storage; the first
    step has no Y_{k-2}) plus the per-cell bf16 H_e stream (n_cells n_e^2 x 2 B,
    unpadded).  Around the m - 1 steps: M V (read V, write MV), the start (read
    HV, MV; write Ghat, Y_1) and V_out (read Y_m, V; write V_out): 54 B per
    DOF x vector.  Returns per-launch bytes of the two kernels and the total of
    one filter.  DOF = interior FE nodes + enriched rows."""
    M = d["n_fe_dof"] + d["n_enr"]
    z0 = (m - 2) / (m - 1)                    # share of the steps that read Y_{k-2}
    rec = 2.0 * N * (3.0 + z0) * d["n_fe_dof"]
    he = 2.0 * d["n_cells"] * d["ne"] ** 2
    total = (m - 1) * (2.0 * N * (3.0 + z0) * M + he) + 54.0 * M * N
    return rec, he, total


def roofline_bf16(w, d, N, m, ms_cell_launch, ms_rec_launch, ms_filter, pk, pk_kind):
    """HBM rooflines of the bf16 filter from live CUDA-event times: the whole
    filter pass, and its two heaviest kernels (k_gather_rec_c: the FE-node
    recurrence with the gather of the cell products; k_cell_mma: the tcgen05
    cell products), with the algorithmic bytes of algorithmic_bytes_bf16 (the
    recurrence's four arrays go to the node kernel, the H_e stream to the cell
    kernel; what either moves beyond that -- the per-cell product round trip,
    the operand gather, tile padding -- is excess, visible in 'traffic' where
    an ncu summary of the current kernel exists).  Sorted by share of the pass:
    the dominant kernel first, the whole pass last."""
    hbm = pk["hbm_gbs"]
    rec_b, he_b, total_b = algorithmic_bytes_bf16(w, d, N, m)
    out = []
    for name, bytes_, ms, traffic_file, key, per in (
            ("k_gather_rec_c (FE-node recurrence: gather of cell products, coupling, Eq. residualapprox)",
             rec_b, ms_rec_launch, "k_gather_rec_c_traffic.txt", "traffic_over_algorithmic", rec_b),
            ("k_cell_mma (tcgen05 cell products, one launch per H apply)", he_b, ms_cell_launch,
             "k_cell_mma_traffic.txt", "bytes_per_cell", d["n_cells"])):
        achieved = bytes_ / (ms / 1e3) / 1e9 if ms and ms > 0 else None
        traffic = None
        if d["ne"] == 343 and N == 154:      # counters taken on these kernels at this shape (p = 6, N = 154)
            f = _traffic_per_unit(traffic_file, key)
            traffic = f * per if f else None
        out.append({"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                    "frac": achieved / hbm if achieved else None, "traffic": traffic,
                    "algorithmic_bytes": bytes_, "peak_kind": pk_kind + " (burst copy)", "kernel": name,
                    "ms_per_launch": ms, "ms_per_step": ms * (m - 1) if ms else None})
    out.sort(key=lambda r: -(r["ms_per_step"] or 0.0))
    achieved = total_b / (ms_filter / 1e3) / 1e9 if ms_filter > 0 else None
    out.append({"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm if achieved else None, "traffic": None, "algorithmic_bytes": total_b,
                "peak_kind": pk_kind + " (burst copy)",
                "kernel": "whole filter pass (m - 1 recurrence steps + G, V_out)", "ms_per_step": ms_filter,
                "bound_value": M_N_m(d, N, m) / (total_b / (hbm * 1e9)) / 1e9})
    return out


def M_N_m(d, N, m):
    """The metric's units of one filter pass: (FE DOF + enriched DOF) x vectors x degree."""
    return (d["n_fe_dof"] + d["n_enr"]) * N * m


def roofline_rr(d, N, ms_rr, pk):
    """Rayleigh-Ritz at the benchmark's size in FP64 on the CUDA cores: the FP64
    H^E X (2 n_e^2 N flop per cell), the Grams X^T M X and X^T H X (2 M N^2
    each) and the rotation of X, HX, MX (3 x 2 M N^2); the generalized N x N
    eigensolve is not counted.  Peak: 152 SMs x 2 FP64 FMA lanes x 2 flop x max
    clock (the nominal ~1.25 TFLOP/s of GB300's FP64)."""
    M = d["n_rows"]
    flops = 2.0 * d["ne"] ** 2 * N * d["n_cells"] + 5 * 2.0 * M * N * N
    peak = 152 * 2 * 2 * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    achieved = flops / (ms_rr / 1e3) / 1e12 if ms_rr > 0 else None
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak if achieved else None, "traffic": None, "flops": flops,
            "peak_kind": "derived from SM count, FP64 lanes and max clock", "ms": ms_rr,
            "kernel": "Rayleigh-Ritz (FP64 H^E X, Grams, rotation; cuSOLVER sygvd not counted)"}


def roofline_simt(head, d, N, ms_sweep, pk):
    """SIMT cell products: FP32 (or FP64) FMA pipes, 152 SMs x lanes x 2 flop x max clock."""
    lanes = 128 if head == "fp32" else 2
    peak = 152 * lanes * 2 * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    flops = d["n_cells"] * 2.0 * d["ne"] ** 2 * N
    achieved = flops / (ms_sweep / 1e3) / 1e12 if ms_sweep > 0 else None
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak if achieved else None, "traffic": None,
            "peak_kind": "derived from SM count and max clock",
            "kernel": "k_cell_apply (SIMT cell products, 8 colour launches per H apply)",
            "ms_per_launch": ms_sweep}


def scf_time_to_solution(torch, dev):
    """SCF time-to-solution, FP64 and mixed (every filter pass in bf16), from the
    same start vectors, with |dE| per atom of mixed against FP64:
    the 2-atom workload (8^3 cells, p = 4, 8 states, degree 20) and an 8-atom cluster
    at the same resolution (12x13x11 cells, 20 states)."""
    from paper_2607_06848_gb300 import EFE, workloads as W, EFE_FP64, EFE_BF16
    out = {}
    for key, w in (("dimer", W.dimer()), ("cluster8_h2p4", W.ws_cluster(8, 1008))):
        g = EFE(w["h"], w["ncell"], w["p"], w["atoms"], w["Z"], enrich=dict(alpha=ALPHA, r_end=R_END, t=T_ENR),
                psp=dict(rc=1.0, r_trunc=6.0, h=w["hproj"], rloc=0.8))
        rows = g.dims["n_rows"]
        rec = {}
        for name, prec in (("fp64", EFE_FP64), ("mixed_bf16", EFE_BF16)):
            X = torch.tensor(W.random_block(rows, w["nstates"], 1), device=dev)
            u0 = torch.tensor(W.random_block(rows, 1, 2), device=dev)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = g.efe_scf(X, u0, cheb_degree=w["cheb_degree"], precision=prec)
            torch.cuda.synchronize()
            rec[name] = {"seconds": time.perf_counter() - t0, "iters": r["iters"], "converged": r["converged"],
                         "E_Ha": r["E"], "poisson_cg_iters": r["poisson_iters"]}
        rec["dE_mixed_vs_fp64_Ha_per_atom"] = abs(rec["mixed_bf16"]["E_Ha"] - rec["fp64"]["E_Ha"]) / len(w["atoms"])
        d = g.dims
        rec["workload"] = "%d atoms, %dx%dx%d cells p=%d (%d FE DOF + %d enriched), %d states, degree %d" % (
            len(w["atoms"]), *w["ncell"], w["p"], d["n_fe_dof"], d["n_enr"], w["nstates"], w["cheb_degree"])
        out[key] = rec
        g.close()
    return out


def scf_cluster64(torch, dev):
    """SCF time-to-solution at the benchmark's own size (24^3 cells p = 6, 154 states,
    degree 30) on the 64-atom cluster with one element's projector strengths: mixed
    (every filter pass in bf16) from seeded vectors, then FP64 continued from the mixed
    fixed point (its vectors and density), whose energy the mixed one is compared with.
    Phase times: potential, eigensolver, density, energy, mixing (ms)."""
    from paper_2607_06848_gb300 import EFE, workloads as W, EFE_FP64, EFE_BF16
    w = W.cluster64_species()
    g = EFE(w["h"], w["ncell"], w["p"], w["atoms"], w["Z"], enrich=dict(alpha=ALPHA, r_end=R_END, t=T_ENR),
            psp=dict(rc=1.0, r_trunc=6.0, h=w["hproj"], rloc=0.8))
    rows = g.dims["n_rows"]
    X = torch.tensor(W.random_block(rows, w["nstates"], 1), device=dev)
    u0 = torch.tensor(W.random_block(rows, 1, 2), device=dev)
    rho = torch.empty(g.dims["n_quad"], dtype=torch.float64, device=dev)
    rec = {}
    for name, prec, it in (("mixed_bf16", EFE_BF16, 100), ("fp64_continued", EFE_FP64, 10)):
        start = rho.clone() if name == "fp64_continued" else None
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = g.efe_scf(X, u0, rho0_q=start, rho_out=rho, cheb_degree=w["cheb_degree"], precision=prec,
                      max_iter=it, profile=1)
        torch.cuda.synchronize()
        rec[name] = {"seconds": time.perf_counter() - t0, "iters": r["iters"], "converged": r["converged"],
                     "E_Ha": r["E"], "ms_phase": [round(x, 1) for x in r["ms_phase"]]}
    rec["dE_mixed_vs_fp64_Ha_per_atom"] = abs(rec["mixed_bf16"]["E_Ha"] - rec["fp64_continued"]["E_Ha"]) / 64
    d = g.dims
    rec["workload"] = "64 atoms (one element), 24^3 cells p=6 (%d FE DOF + %d enriched), %d states, degree %d" % (
        d["n_fe_dof"], d["n_enr"], w["nstates"], w["cheb_degree"])
    g.close()
    return rec


def run_ours(args):
    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2607_06848_gb300 import EFE, workloads as W, EFE_FP64, EFE_FP32, EFE_BF16
    w = workload(args.workload)
    t_setup = time.perf_counter()
    g = EFE(w["h"], w["ncell"], w["p"], w["atoms"], w["Z"], enrich=dict(alpha=ALPHA, r_end=R_END, t=T_ENR),
            psp=dict(rc=1.0, r_trunc=6.0, h=w["hproj"]))
    d = g.dims
    # non-self-consistent (Harris) potential of the superposed atomic densities:
    # v = v_xc[rho0] + phi[rho0 + b_sm], all through the library's SCF pieces
    nq = d["n_quad"]
    rho0 = torch.empty(nq, dtype=torch.float64, device=dev)
    bq = torch.empty_like(rho0)
    g.efe_atomic_density(2.4, rho0)
    g.efe_smeared_charge(bq)
    phi = torch.empty(d["n_nodes"], dtype=torch.float64, device=dev)
    phq = torch.empty_like(rho0)
    poisson_its, _ = g.efe_poisson(rho0 + bq, phi, phq, tol=1e-10)
    v = torch.empty_like(rho0)
    g.efe_xc(rho0, v, None)
    v += phq
    del phi, phq, bq, rho0
    g.efe_set_potential(v)
    rows, N, m = d["n_rows"], w["nstates"], w["cheb_degree"]
    gen = torch.Generator(device=dev)
    gen.manual_seed(1234)
    X = torch.randn((rows, N), generator=gen, dtype=torch.float64, device=dev)
    HX = torch.empty_like(X)
    eig, res = g.efe_rayleigh_ritz(X, HX)
    u0 = torch.randn((rows, 1), generator=gen, dtype=torch.float64, device=dev)
    tmin, tmax, b = g.efe_lanczos(u0, 10)
    bounds = (float(eig[0]), float(eig[-1]), float(b))
    lam = torch.tensor(eig, device=dev)
    Vout = torch.empty_like(X)
    t_setup = time.perf_counter() - t_setup
    M = d["n_fe_dof"] + d["n_enr"]
    units = M * N * m

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def timed(prec, steps, warmup):
        for _ in range(warmup):
            g.efe_filter(X, HX, lam, m, bounds, Vout, prec=prec)
        barrier()
        s = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        cells_ms = rec_ms = 0.0
        launches = rec_n = 0
        e0.record(s)
        for _ in range(steps):
            g.efe_filter(X, HX, lam, m, bounds, Vout, prec=prec)
            st = g.stats()
            cells_ms += st["ms_cell"]
            rec_ms += st["ms_rec"]
            rec_n += st["rec_launches"]
            launches += st["launches"]
        e1.record(s)
        barrier()
        ms = max_over_ranks(e0.elapsed_time(e1) / steps, dist, dev)
        return ms, cells_ms / steps, launches, (rec_ms / rec_n if rec_n else None)

    precs = {"fp64": EFE_FP64, "fp32": EFE_FP32, "bf16": EFE_BF16}
    head = args.prec
    clk = ClockSampler(local)
    ms, cell_ms, launches, rec_ms_launch = timed(precs[head], args.steps, args.warmup)
    clocks = clk.stop()
    by_prec = {head: {"ms_per_step": ms, "value": units / (ms / 1e3) / 1e9, "steps": args.steps,
                      "warmup": args.warmup}}
    for extra in args.also:
        if extra != head:
            mse, _, _, _ = timed(precs[extra], 1, 1)
            by_prec[extra] = {"ms_per_step": mse, "value": units / (mse / 1e3) / 1e9, "steps": 1, "warmup": 1}
    # Rayleigh-Ritz at this size (one warm call, then one timed; its FP64 H^E X dominates)
    Xr = X.clone()
    HXr = torch.empty_like(Xr)
    g.efe_rayleigh_ritz(Xr, HXr)
    Xr.copy_(X)
    torch.cuda.synchronize()
    g.efe_rayleigh_ritz(Xr, HXr)
    ms_rr = g.stats()["ms_rr"]
    del Xr, HXr

    # end to end through the public call with host buffers (pinned)
    Vh = torch.empty((rows, N), dtype=torch.float64, pin_memory=True)
    HVh = torch.empty((rows, N), dtype=torch.float64, pin_memory=True)
    lamh = torch.tensor(eig, dtype=torch.float64).contiguous()
    Vh.copy_(X.cpu())
    HVh.copy_(HX.cpu())
    Oh = torch.empty((rows, N), dtype=torch.float64, pin_memory=True)   # pinned output
    e2e_steps = max(1, min(args.steps, 3))
    g.efe_filter_host(Vh.numpy(), HVh.numpy(), lamh.numpy(), m, bounds, prec=precs[head], out=Oh.numpy())
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        out_h = g.efe_filter_host(Vh.numpy(), HVh.numpy(), lamh.numpy(), m, bounds, prec=precs[head],
                                  out=Oh.numpy())
    barrier()
    e2e_ms = max_over_ranks((time.perf_counter() - t0) / e2e_steps * 1e3, dist, dev)
    h2d = (2 * rows * N + N) * 8
    d2h = rows * N * 8
    del out_h

    pk, pk_kind = peaks()
    ms_sweep = cell_ms / (m - 1)          # m - 1 H applies per filter pass
    if head == "bf16":
        rl = roofline_bf16(w, d, N, m, ms_sweep, rec_ms_launch, ms, pk, pk_kind)
    else:
        rl = [roofline_simt(head, d, N, ms_sweep, pk)]
    line = {
        "metric": METRIC, "value": job_value(units, world, ms), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": {"fp64": "f64", "fp32": "f32", "bf16": "bf16"}[head],
        "data": "synthetic",
        "config": {"workload": "%s: %d atoms, %dx%dx%d cells p=%d (%d FE DOF + %d enriched), %d vectors, "
                               "filter degree %d" % (w["name"], len(w["atoms"]), *w["ncell"], w["p"],
                                                     d["n_fe_dof"], d["n_enr"], N, m),
                   "precision": head, "l2": "inputs larger than L2 (%.2f GB per block)" % (rows * N * 8 / 1e9),
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "potential": "Harris v_xc[rho0] + phi[rho0 + b_sm] of superposed atomic densities "
                                "(Poisson CG %d iterations)" % poisson_its},
        "by_precision": by_prec,
        "roofline": rl[0],
        "roofline_kernels": rl,
        "rayleigh_ritz": roofline_rr(d, N, ms_rr, pk),
        "e2e": {"value": job_value(units, world, e2e_ms), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "clocks": clocks,
        "setup_s": t_setup,
    }
    if not args.no_scf:
        line["scf"] = scf_time_to_solution(torch, dev)
        if args.scf_c1:
            line["scf"]["cluster64_species"] = scf_cluster64(torch, dev)
    if rank == 0 and world == 1 and not args.no_cpu:
        val, dt, desc, cores = cpu_sample(steps=6, warmup=0)
        line["cpu_baseline"] = {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc}
    if rank == 0:
        print(json.dumps(line), flush=True)
    g.close()
    if dist is not None:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="bf16", choices=["fp64", "fp32", "bf16"])
    ap.add_argument("--also", nargs="*", default=["fp32", "fp64"],
                    help="other precisions timed once for the by_precision table")
    ap.add_argument("--workload", default="cluster64")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-scf", action="store_true")
    ap.add_argument("--scf-c1", action="store_true",
                    help="add the SCF at the benchmark's own size (64 atoms, ~7 minutes)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
