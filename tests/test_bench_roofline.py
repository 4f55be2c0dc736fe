"""The benchmark's roofline arithmetic on the host (no GPU).

The algorithmic bytes of the two heaviest kernels of the mixed filter follow
from the mesh alone: the node recurrence reads one cell row per (cell, node)
incidence, Z_{k-1}, Z_{k-2} (absent in the first step) and G, and writes Z_k
at every interior node, and zeros at the Dirichlet nodes; the cell products
stream the bf16 cell matrix and operand and write the FP32 products.  The
figures here are counted independently from the grid, and the DRAM traffic
comes from the committed ncu summaries.
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
    return {"n_fe_dof": (G - 2) ** 3, "n_nodes": G ** 3, "n_cells": n ** 3, "ne": (p + 1) ** 3}


def test_recurrence_and_cell_bytes_of_the_benchmark():
    w = W.cluster64()
    d = _dims(w)
    N, m = w["nstates"], w["cheb_degree"]
    pk = {"hbm_gbs": 1000.0}
    out = bench.roofline_bf16(w, d, N, m, 1.0, 1.0, pk, "test")
    by = {r["kernel"].split()[0]: r for r in out}
    # count the (cell, node) incidences of interior nodes directly: along an
    # axis an interior node index i in 1..G-2 lies in two cells if i % p == 0
    n, p = w["ncell"][0], w["p"]
    per_axis = sum(2 if i % p == 0 else 1 for i in range(1, n * p))
    inc = per_axis ** 3
    fe, bnd = d["n_fe_dof"], d["n_nodes"] - d["n_fe_dof"]
    steps_with_z0 = (m - 2) / (m - 1)
    rec = 4.0 * N * (inc + (3.0 + steps_with_z0) * fe + bnd)
    assert by["k_gather_rec_w"]["algorithmic_bytes"] == pytest.approx(rec, rel=1e-12)
    assert rec == pytest.approx(10.04e9, rel=1e-3)           # the figure quoted for cluster64
    cell = d["n_cells"] * (2.0 * d["ne"] ** 2 + 6.0 * d["ne"] * N)
    assert by["k_cell_mma"]["algorithmic_bytes"] == pytest.approx(cell, rel=1e-12)
    assert cell == pytest.approx(7.634e9, rel=1e-3)
    # 1 ms per launch at 1000 GB/s: achieved = bytes / 1e6, fraction achieved / 1000
    for r in out:
        assert r["achieved"] == pytest.approx(r["algorithmic_bytes"] / 1e6, rel=1e-12)
        assert r["frac"] == pytest.approx(r["achieved"] / 1000.0, rel=1e-12)


def test_traffic_comes_from_the_ncu_summaries():
    w = W.cluster64()
    d = _dims(w)
    out = bench.roofline_bf16(w, d, w["nstates"], w["cheb_degree"], 1.0, 1.0, {"hbm_gbs": 1.0}, "test")
    by = {r["kernel"].split()[0]: r for r in out}
    ratio = bench._traffic_per_unit("k_gather_rec_w_traffic.txt", "traffic_over_algorithmic")
    per_cell = bench._traffic_per_unit("k_cell_mma_traffic.txt", "bytes_per_cell")
    assert ratio is not None and 1.0 <= ratio < 1.2
    assert per_cell is not None
    assert by["k_gather_rec_w"]["traffic"] == pytest.approx(ratio * by["k_gather_rec_w"]["algorithmic_bytes"])
    assert by["k_cell_mma"]["traffic"] == pytest.approx(per_cell * d["n_cells"])
    # the cell kernel's traffic stays within a few percent of its algorithmic bytes
    assert 1.0 <= by["k_cell_mma"]["traffic"] / by["k_cell_mma"]["algorithmic_bytes"] < 1.1
    # other shapes carry no counters
    w8 = dict(w, nstates=64)
    out8 = bench.roofline_bf16(w8, d, 64, 30, 1.0, 1.0, {"hbm_gbs": 1.0}, "test")
    assert all(r["traffic"] is None for r in out8)


def test_job_value_counts_every_replica():
    # units per rank x ranks / seconds, in G-units per second
    assert bench.job_value(2e9, 4, 500.0) == pytest.approx(16.0)
