"""The benchmark's roofline arithmetic on the host (no GPU).

The algorithmic bytes of the bf16 filter follow the scope table's rule: per
recurrence step four arrays of 2 bytes per DOF x vector (read Y_{k-1},
Y_{k-2} -- absent in the first step -- and Ghat, write Y_k) plus the unpadded
bf16 cell-matrix stream; around the steps the FP64 interface (M V, the start,
V_out).  The figures here are counted step by step from the grid,
independently of the benchmark's closed form, and the DRAM traffic comes from
the committed ncu summaries when one exists for the current kernel.
"""
import os

import pytest

import bench
from paper_2607_06848_gb300 import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))


def _dims(w):
    n = w["ncell"][0]
    p = w["p"]
    G = n * p + 1
    return {"n_fe_dof": (G - 2) ** 3, "n_nodes": G ** 3, "n_cells": n ** 3, "ne": (p + 1) ** 3,
            "n_enr": 4 * len(w["atoms"]), "n_rows": G ** 3 + 4 * len(w["atoms"])}


def test_algorithmic_bytes_of_the_benchmark():
    w = W.cluster64()
    d = _dims(w)
    N, m = w["nstates"], w["cheb_degree"]
    fe, M = d["n_fe_dof"], d["n_fe_dof"] + d["n_enr"]
    he = 2.0 * d["n_cells"] * d["ne"] ** 2           # bf16 cell matrices, unpadded
    assert he == pytest.approx(3.253e9, rel=1e-3)
    rec_launches, total = [], 0.0
    for k in range(2, m + 1):
        arrays = 4 if k > 2 else 3                    # Y_{k-1}, Ghat, Y_k (+ Y_{k-2})
        rec_launches.append(2.0 * N * arrays * fe)
        total += 2.0 * N * arrays * M + he
    total += (16 + 20 + 18) * M * N                   # M V; start (HV, MV -> Ghat, Y_1); V_out
    rec, he_b, tot = bench.algorithmic_bytes_bf16(w, d, N, m)
    assert rec == pytest.approx(sum(rec_launches) / len(rec_launches), rel=1e-12)
    assert he_b == pytest.approx(he, rel=1e-12)
    assert tot == pytest.approx(total, rel=1e-12)
    assert tot == pytest.approx(29 * (3.59e9 + 3.253e9) + 24.3e9, rel=5e-3)
    # 1 ms per launch at 1000 GB/s: achieved = bytes / 1e6, fraction achieved / 1000
    out = bench.roofline_bf16(w, d, N, m, 1.0, 1.0, 29.0, {"hbm_gbs": 1000.0}, "test")
    for r in out:
        ms = r.get("ms_per_launch") or r["ms_per_step"]
        assert r["achieved"] == pytest.approx(r["algorithmic_bytes"] / 1e6 / ms, rel=1e-12)
        assert r["frac"] == pytest.approx(r["achieved"] / 1000.0, rel=1e-12)
    whole = out[-1]
    assert whole["kernel"].startswith("whole filter")
    # the bound implied by the bytes: units / (bytes / peak)
    units = M * N * m
    assert whole["bound_value"] == pytest.approx(units / (tot / 1e12) / 1e9, rel=1e-12)


def test_traffic_comes_from_the_ncu_summaries():
    w = W.cluster64()
    d = _dims(w)
    N, m = w["nstates"], w["cheb_degree"]
    out = bench.roofline_bf16(w, d, N, m, 1.0, 1.0, 29.0, {"hbm_gbs": 1.0}, "test")
    by = {r["kernel"].split()[0]: r for r in out}
    for name, f, key, per in (("k_gather_rec_c", "k_gather_rec_c_traffic.txt", "traffic_over_algorithmic",
                               by["k_gather_rec_c"]["algorithmic_bytes"]),
                              ("k_cell_mma", "k_cell_mma_traffic.txt", "bytes_per_cell", d["n_cells"])):
        v = bench._traffic_per_unit(f, key)
        if v is None:
            assert by[name]["traffic"] is None
        else:
            assert by[name]["traffic"] == pytest.approx(v * per)
    # other shapes carry no counters
    out8 = bench.roofline_bf16(w, d, 64, 30, 1.0, 1.0, 29.0, {"hbm_gbs": 1.0}, "test")
    assert all(r["traffic"] is None for r in out8)


def test_rayleigh_ritz_flops():
    w = W.cluster64()
    d = _dims(w)
    N = w["nstates"]
    r = bench.roofline_rr(d, N, 1000.0, {"sm_max_mhz": 2070.0})
    flops = 2.0 * 343 ** 2 * N * 24 ** 3 + 10.0 * d["n_rows"] * N * N
    assert r["flops"] == pytest.approx(flops, rel=1e-12)
    assert r["peak"] == pytest.approx(1.2586, rel=1e-3)
    assert r["achieved"] == pytest.approx(flops / 1e12, rel=1e-12)


def test_job_value_counts_every_replica():
    # units per rank x ranks / seconds, in G-units per second
    assert bench.job_value(2e9, 4, 500.0) == pytest.approx(16.0)
