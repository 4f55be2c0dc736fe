"""Pins for the oracle's finite-element layer (Sec. III.A): quadrature
exactness, Lagrange basis identities, cell matrices against closed forms and
the harmonic-oscillator spectrum 1.5, 2.5 (x3), 3.5 (x6) with its h-rate."""
import math

import numpy as np
import pytest
import scipy.linalg as sla

from oracle.fe import Mesh, gauss_rule, gll_rule, lagrange_deriv, lagrange_eval
from oracle.efe import EFESystem


def _mono_int(k):
    return 0.0 if k % 2 else 2.0 / (k + 1)


@pytest.mark.parametrize("p", range(1, 9))
def test_gll_exact_to_2p_minus_1(p):
    x, w = gll_rule(p)
    assert len(x) == p + 1 and abs(x[0] + 1) < 1e-15 and abs(x[-1] - 1) < 1e-15
    for k in range(2 * p):
        assert abs(np.sum(w * x ** k) - _mono_int(k)) < 1e-13
    # and not exact one degree higher (it is the Lobatto rule, not Gauss)
    assert abs(np.sum(w * x ** (2 * p)) - _mono_int(2 * p)) > 1e-6


@pytest.mark.parametrize("n", range(1, 11))
def test_gauss_exact_to_2n_minus_1(n):
    x, w = gauss_rule(n)
    for k in range(2 * n):
        assert abs(np.sum(w * x ** k) - _mono_int(k)) < 1e-13
    assert abs(np.sum(w * x ** (2 * n)) - _mono_int(2 * n)) > 1e-8


@pytest.mark.parametrize("p", [1, 2, 4, 6])
def test_lagrange_identities(p):
    xg, _ = gll_rule(p)
    assert np.allclose(lagrange_eval(xg, xg), np.eye(p + 1), atol=1e-13)
    t = np.linspace(-1, 1, 37)
    L = lagrange_eval(xg, t)
    D = lagrange_deriv(xg, t)
    assert np.allclose(L.sum(axis=1), 1.0, atol=1e-12)
    assert np.allclose(D.sum(axis=1), 0.0, atol=1e-10)
    # reproduces x^p exactly and its derivative
    assert np.allclose(L @ xg ** p, t ** p, atol=1e-12)
    assert np.allclose(D @ xg ** p, p * t ** (p - 1), atol=1e-10)
    eps = 1e-6
    fd = (lagrange_eval(xg, t + eps) - lagrange_eval(xg, t - eps)) / (2 * eps)
    assert np.allclose(D, fd, atol=1e-6)


@pytest.mark.parametrize("p,h", [(2, 1.0), (4, 2.0), (6, 1.5)])
def test_cell_matrices_closed_forms(p, h):
    m = Mesh(h, (1, 1, 1), p)
    K = m.stiffness_cell()
    ones = np.ones(m.ne)
    assert np.allclose(K @ ones, 0.0, atol=1e-11)
    X = m.node_xyz()
    for g in ([1.0, 0, 0], [0.3, -1.2, 0.5]):
        u = X @ np.array(g)
        # int |grad u|^2 = |g|^2 * h^3 for a linear u
        assert abs(u @ K @ u - np.dot(g, g) * h ** 3) < 1e-10 * max(1, h ** 3)
    Mc = m.potential_cell(np.ones(m.nq ** 3))
    assert abs(ones @ Mc @ ones - h ** 3) < 1e-12
    assert abs(m.lumped_mass().sum() - h ** 3) < 1e-12
    # consistent mass integrates x*y exactly
    u = X[:, 0]
    v = X[:, 1]
    assert abs(u @ Mc @ v - (h ** 2 / 2) * (h ** 2 / 2) * h) < 1e-10


def _ho_eigs(n, p, k=10, box=12.0):
    m = Mesh(box / n, (n, n, n), p)
    ctr = np.full(3, box / 2)
    s = EFESystem(m, ctr[None, :])
    s.set_potential(0.5 * np.sum((m.all_quad_points() - ctr) ** 2, axis=1))
    rows = s.dof_rows()
    E = np.zeros((s.nn, len(rows)))
    E[rows, np.arange(len(rows))] = 1.0
    H = s.apply_H(E)[rows]
    M = s.apply_M(E)[rows]
    return sla.eigh(H, M, eigvals_only=True, subset_by_index=[0, k - 1])


EXACT_HO = np.array([1.5, 2.5, 2.5, 2.5, 3.5, 3.5, 3.5, 3.5, 3.5, 3.5])


def test_harmonic_oscillator_p_convergence():
    errs = [np.max(np.abs(_ho_eigs(6, p) - EXACT_HO)) for p in (2, 3)]
    assert errs[1] < errs[0] / 5
    assert errs[1] < 0.08
    e = _ho_eigs(6, 3)
    # cubic symmetry keeps the 3-fold degeneracy of the first excited level
    assert np.ptp(e[1:4]) < 1e-9


@pytest.mark.slow
def test_harmonic_oscillator_h_rate():
    # spectral elements with GLL lumping: ground-state error ~ h^(2p); p = 2
    e4 = abs(_ho_eigs(4, 2, k=1)[0] - 1.5)
    e8 = abs(_ho_eigs(8, 2, k=1)[0] - 1.5)
    rate = math.log(e4 / e8, 2)
    assert 3.0 < rate < 5.5, rate
