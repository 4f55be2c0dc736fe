"""Pins for the oracle eigensolver (Sec. III.B): Chebyshev scalars in closed
form, the residual filter equal to the plain filter when M~ = M, converged
Ritz pairs equal to a dense generalized eigensolve, the Lanczos bound above
the spectrum, and the qualitative Fig. 1 behaviour (the plain filter with
M~^-1 stalls where the residual filter converges)."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle.chfsi import (cheb_scalars, chfsi, lanczos_bounds, rayleigh_ritz,
                          residual_filter, residual_norms, standard_filter)
from oracle.efe import EFESystem
from oracle.fe import Mesh

R0 = 5.0 * 0.33 / 1.33


def test_cheb_scalars_closed_form():
    a, b, a0 = -1.0, 7.0, -3.0
    lam = np.concatenate([np.linspace(-3, -1, 7), np.linspace(-1, 7, 9)])
    m = 25
    C = cheb_scalars(lam, m, a, b, a0)
    e, c = (b - a) / 2, (b + a) / 2

    def T(k, x):
        x = np.asarray(x, float)
        out = np.empty_like(x)
        big = np.abs(x) > 1
        out[big] = np.sign(x[big]) ** k * np.cosh(k * np.arccosh(np.abs(x[big])))
        out[~big] = np.cos(k * np.arccos(x[~big]))
        return out

    for k in range(m + 1):
        ref = T(k, (lam - c) / e) / T(k, np.array([(a0 - c) / e]))[0]
        assert np.allclose(C[k], ref, rtol=1e-11, atol=1e-14)
    assert abs(C[m][0] - 1.0) < 1e-12
    bound = 1.0 / abs(T(m, np.array([(a0 - c) / e]))[0])
    assert np.all(np.abs(C[m][lam >= a]) <= bound * (1 + 1e-9))


def _system(atoms, n=3, p=2, box=12.0, hp=None):
    m = Mesh(box / n, (n, n, n), p)
    atoms = np.asarray(atoms, float)
    if hp is None:
        hp = np.tile([[1.0, -0.5]], (len(atoms), 1))
    s = EFESystem(m, atoms, enrich=dict(alpha=1.2, r0=R0, t=0.33),
                  proj=dict(rc=1.0, rtrunc=6.0, h=hp))
    q = m.all_quad_points()
    v = -np.sum([3.0 / np.sqrt(0.5 + np.sum((q - a) ** 2, axis=1)) for a in atoms], axis=0)
    s.set_potential(v)
    return s


def _dense(s):
    rows = s.dof_rows()
    E = np.zeros((s.nn + s.n_enr, len(rows)))
    E[rows, np.arange(len(rows))] = 1.0
    return rows, s.apply_H(E)[rows], s.apply_M(E)[rows]


def _rand(s, N, seed):
    X = np.random.default_rng(seed).standard_normal((s.nn + s.n_enr, N))
    X[:s.nn] *= s.mask[:, None]
    return X


def test_residual_equals_standard_when_Mtilde_exact():
    s = _system([[6.0, 6.0, 6.0]])                  # one atom: M~ = M exactly
    X = _rand(s, 6, 1)
    lam, V, HV = rayleigh_ritz(s, X)
    a0, a, b = lam[0], lam[-1], 60.0
    V1 = residual_filter(s, V, lam, 12, a, b, a0, HV=HV)
    V2 = standard_filter(s, V, 12, a, b, a0)
    assert np.allclose(V1, V2, atol=1e-9 * np.abs(V2).max())


def test_chfsi_matches_dense_eigh():
    s = _system([[5.0, 6.0, 6.0], [7.2, 6.1, 5.8]])
    rows, H, M = _dense(s)
    ref = sla.eigh(H, M, eigvals_only=True, subset_by_index=[0, 7])
    X = _rand(s, 8, 5)
    u0 = _rand(s, 1, 6)
    out = chfsi(s, X, 16, 1e-10, 60, u0, nconv=6)
    assert out["history"][-1] < 1e-10
    assert np.allclose(out["lam"][:6], ref[:6], atol=1e-10)
    V = out["V"]
    assert np.allclose(V.T @ s.apply_M(V), np.eye(8), atol=1e-11)
    # boundary rows stay zero
    assert np.abs(V[:s.nn][~s.mask]).max() == 0.0


def test_lanczos_upper_bound():
    s = _system([[5.0, 6.0, 6.0], [7.2, 6.1, 5.8]])
    rows, H, M = _dense(s)
    ni = int(s.mask.sum())
    Mt = M.copy()
    Mt[ni:ni + 4, ni + 4:] = 0
    Mt[ni + 4:, ni:ni + 4] = 0
    lmax = sla.eigh(H, Mt, eigvals_only=True)[-1]
    lmin = sla.eigh(H, Mt, eigvals_only=True)[0]
    tmin, tmax, b = lanczos_bounds(s, _rand(s, 1, 9), 10)
    assert b >= lmax * (1 - 1e-12)
    assert tmax <= lmax + 1e-9 and tmin >= lmin - 1e-9
    assert b < 1.5 * lmax


@pytest.mark.slow
def test_standard_filter_stalls_residual_converges():
    # qualitative repeat of Fig. 1: with the atom-block M~^-1 the plain filter
    # cannot reach a tight residual, the residual filter can.
    s = _system([[5.3, 6.0, 6.0], [6.9, 6.0, 6.0]], n=3, p=2)
    X = _rand(s, 8, 11)
    u0 = _rand(s, 1, 12)
    res = chfsi(s, X, 12, 1e-11, 25, u0, nconv=5, residual=True)
    std = chfsi(s, X, 12, 1e-11, 25, u0, nconv=5, residual=False)
    assert res["history"][-1] < 1e-10
    assert min(std["history"]) > 1e3 * res["history"][-1]
