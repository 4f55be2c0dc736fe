"""Pins of oracle parts that the other oracle tests only use, never fix:

* the Gaussian-overlap correction of the ion-ion energy (Sec. II.A, Eqs.
  EZZbmsear/EellocReform; our reading of the smeared charges b_sm) against
  the FE electrostatics of two Gaussian charges: 1/2 int b phi[b] - E_self +
  dE_ZZ must be the point-charge energy Z_I Z_J / R;
* the smearing entropy of the 500 K occupations (Sec. IV) against the
  half-filled level and the grand-potential identity of Fermi-Dirac
  occupations;
* the quadrature assembly of the projector overlaps P_c (nodal basis) and P_a
  (enrichment) against the radial integrals of the projectors (nodal
  interpolation of 1 and of x is exact);
* the hydrogen-like closed form: with the 1s orbital exp(-Z r) in the span of
  the enrichment, the lowest eigenvalue of -1/2 Lap - Z/r tends to -Z^2/2 as
  the quadrature is refined (Sec. II.B: atomic orbitals as enrichment);
* the SCF of one atom whose Fermi level lies inside its 3-fold p shell: F - E
  is the closed-form entropy of occupations 2/3.

Each pin is also run against a plausible mistake (a flipped sign, erf for
erfc, a dropped term) to show that it would catch it."""
import json
import math
import os

import numpy as np
import pytest
import scipy.linalg as sla
from scipy.integrate import quad
from scipy.special import erf

from oracle import scf as S
from oracle.efe import EFESystem, Y00, Y1C, dense_raw_matrices
from oracle.fe import Mesh

HERE = os.path.dirname(os.path.abspath(__file__))


# --- ion-ion overlap correction ------------------------------------------------
def _two_gaussian_electrostatics():
    """1/2 int b phi[b] for b = -Z_1 g(r - R_1) - Z_2 g(r - R_2) (alpha = 0.8) by the
    FE Poisson solve with the exact potential on the box faces (the erf potentials
    of the two charges), on 6^3 cells of degree 6 in a 12-bohr cube."""
    alpha, Z = 0.8, np.array([4.0, 3.0])
    L, n, p = 12.0, 6, 6
    m = Mesh(L / n, (n, n, n), p)
    atoms = np.array([[L / 2 - 0.8, L / 2, L / 2], [L / 2 + 0.8, L / 2 + 0.3, L / 2 - 0.2]])
    b = S.gaussian_charge(m.all_quad_points(), atoms, Z, alpha)
    X = m.node_xyz()
    exact = np.zeros(len(X))
    for a, z in zip(atoms, Z):
        r = np.linalg.norm(X - a, axis=1)
        exact -= z * erf(r / alpha) / r          # no node sits on a centre
    phi, _ = S.poisson_solve(m, b, tol=1e-13, boundary=exact)
    phq = m.interpolate(phi[:, None])[:, 0]
    return 0.5 * m.integrate(b * phq), atoms, Z, alpha


def test_zz_overlap_correction_pinned_by_fe_electrostatics():
    half_bphi, atoms, Z, alpha = _two_gaussian_electrostatics()
    R = float(np.linalg.norm(atoms[0] - atoms[1]))
    point = Z[0] * Z[1] / R

    def residual(corr):
        return abs(half_bphi - S.self_energy(Z, alpha) + corr - point)

    good = S.zz_overlap_correction(atoms, Z, alpha)
    assert good > 0.25                              # the overlap is far from negligible here
    assert residual(good) < 3e-4, residual(good)    # FE error of this mesh ~8e-5
    # plausible mistakes in the correction all miss by far more than the FE error
    s2a = math.sqrt(2.0) * alpha
    for bad in (-good,                                           # sign
                Z[0] * Z[1] * math.erf(R / s2a) / R,             # erf for erfc
                Z[0] * Z[1] * math.erfc(R / alpha) / R,          # width alpha, not sqrt(2) alpha
                0.0):                                            # no correction
        assert residual(bad) > 100 * residual(good), bad


# --- smearing entropy ------------------------------------------------------------
def test_entropy_term_half_filled_level():
    kT = S.KB_HA * 500.0
    assert abs(S.entropy_term(np.array([0.5]), kT) + 2.0 * kT * math.log(2.0)) < 1e-18
    assert abs(S.entropy_term(np.array([0.5, 0.5, 1.0, 0.0]), kT) + 4.0 * kT * math.log(2.0)) < 1e-18
    assert S.entropy_term(np.array([1.0, 1.0, 0.0]), kT) == 0.0


def test_entropy_term_grand_potential_identity():
    # for Fermi-Dirac occupations f_i = 1/(1 + exp((eps_i - mu)/kT)) of a
    # spin-degenerate spectrum the band free energy satisfies
    #   2 sum f eps - T S = mu N_e - 2 kT sum ln(1 + exp(-(eps - mu)/kT)),
    # which fixes the sign, the factor 2 and both logarithms of the entropy
    kT = S.KB_HA * 500.0
    eig = np.array([-1.0, -0.8, -0.6, -0.4, -0.4, -0.4, -0.2, -0.196, 0.0, 0.1])
    # N_e = 8, 9: the Fermi level inside the 3-fold level; 13.3: between two
    # levels 2.5 kT apart -- partial occupations in every case
    for ne in (8.0, 9.0, 13.3):
        mu, f = S.fermi_level(eig, ne, kT)
        assert -S.entropy_term(f, kT) > 1e-3 * kT
        x = (eig - mu) / kT
        grand = mu * ne - 2.0 * kT * float(np.sum(np.logaddexp(0.0, -x)))

        def lhs(ent):
            return 2.0 * float(np.sum(f * eig)) + ent(f)

        good = lhs(lambda ff: S.entropy_term(ff, kT))
        assert abs(good - grand) < 1e-12, (ne, good, grand)

        def ent_without_hole_term(ff):
            return 2.0 * kT * float(sum(v * math.log(v) for v in ff if 0 < v < 1))

        for bad in (lambda ff: -S.entropy_term(ff, kT),
                    lambda ff: 0.5 * S.entropy_term(ff, kT),
                    ent_without_hole_term):
            assert abs(lhs(bad) - grand) > 1e-6, ne


# --- projector assembly ----------------------------------------------------------
def _radial(fn, R):
    return quad(fn, 0.0, R, epsabs=0.0, epsrel=1e-13, limit=200)[0]


def test_projector_assembly_moments():
    # h = 1.6: the cell Jacobian (h/2)^3 differs from 1, so a dropped Jacobian or
    # quadrature weight changes every value
    h, n, p, rc, rt = 1.6, 10, 5, 1.0, 6.0
    L = h * n
    ctr = np.array([L / 2 + 0.13, L / 2 - 0.21, L / 2 + 0.07])
    m = Mesh(h, (n, n, n), p)
    assert abs(m.J - 1.0) > 0.4
    s = EFESystem(m, ctr[None, :], proj=dict(rc=rc, rtrunc=rt, h=np.array([[1.0, 1.0]])))
    As = (math.pi * rc * rc) ** -0.75
    Ap = As * math.sqrt(2.0) / rc
    g = lambda r: math.exp(-r * r / (2 * rc * rc))          # noqa: E731
    # int beta_s over the truncated ball, and int x_m beta_pm = A_p int x_m^2 g = A_p (1/3) int r^2 g
    ref_s = As * 4.0 * math.pi * _radial(lambda r: r * r * g(r), rt)
    ref_p = Ap * (4.0 * math.pi / 3.0) * _radial(lambda r: r ** 4 * g(r), rt)
    one = s.mask.astype(float)                # the box faces are far outside the ball
    X = m.node_xyz()
    v = s.Pc @ one
    assert abs(v[0] - ref_s) < 1e-8 * ref_s, (v[0], ref_s)
    assert np.abs(v[1:]).max() < 1e-8 * ref_s
    for k in range(3):
        v = s.Pc @ ((X[:, k] - ctr[k]) * one)
        assert abs(v[1 + k] - ref_p) < 1e-8 * ref_p, (k, v[1 + k], ref_p)
        assert max(abs(v[j]) for j in range(4) if j != 1 + k) < 1e-8 * ref_p
    # P_a with the uncut Gaussian enrichment r^l exp(-alpha r^2) Y_lm: Gaussian
    # products with exponent a = alpha + 1/(2 rc^2) in closed form
    alpha = 1.2
    s2 = EFESystem(m, ctr[None, :], enrich=dict(alpha=alpha, r0=None),
                   proj=dict(rc=rc, rtrunc=rt, h=np.array([[1.0, 1.0]])))
    a = alpha + 1.0 / (2 * rc * rc)
    ref_ss = As * Y00 * (math.pi / a) ** 1.5
    ref_pp = Ap * Y1C * (math.pi / a) ** 1.5 / (2.0 * a)
    Pa = s2.Pa
    assert abs(Pa[0, 0] - ref_ss) < 1e-6 * ref_ss, (Pa[0, 0], ref_ss)
    assert np.abs(np.diag(Pa)[1:] - ref_pp).max() < 1e-6 * ref_pp
    assert np.abs(Pa - np.diag(np.diag(Pa))).max() < 1e-6 * ref_pp


# --- hydrogen-like closed form -----------------------------------------------------
@pytest.mark.parametrize("Z", [1.0, 2.0])
def test_hydrogen_like_lowest_eigenvalue(Z):
    # nucleus on a node (no Gauss point at r = 0); the 1s function exp(-Z r)
    # (and its p partners r Y_1m exp(-Z r)) as uncut enrichment; -Z/r at the
    # Gauss points.  The error is the quadrature of the cusp and of the 1/r
    # singularity in the 8 cells at the nucleus: it falls as n_q grows
    L = 16.0 / Z
    errs = []
    for nq in (8, 16, 24):
        m = Mesh(L / 4, (4, 4, 4), 2, nq)
        ctr = np.full(3, L / 2)
        s = EFESystem(m, ctr[None, :], enrich=dict(alpha=Z, r0=None, radial="slater"))
        s.set_potential(-Z / np.linalg.norm(m.all_quad_points() - ctr, axis=1))
        H, M = dense_raw_matrices(s)
        lam = sla.eigh(H, M, eigvals_only=True, subset_by_index=[0, 0])[0]
        errs.append(abs(lam + 0.5 * Z * Z) / (0.5 * Z * Z))
    assert errs[0] > errs[1] > errs[2], errs
    assert errs[2] < 5e-4, errs
    assert errs[0] / errs[2] > 20.0, errs


# --- SCF with a partially filled shell ---------------------------------------------
def _atom_scf_inputs():
    from paper_2607_06848_gb300 import workloads as W
    w = W.single_atom()
    m = Mesh(w["h"], w["ncell"], w["p"])
    s = EFESystem(m, w["atoms"], enrich=dict(alpha=1.2, r0=5.0 * 0.33 / 1.33, t=0.33),
                  proj=dict(rc=1.0, rtrunc=6.0, h=w["hproj"]))
    rows = s.nn + s.n_enr
    X0 = W.random_block(rows, w["nstates"], 1)
    u0 = W.random_block(rows, 1, 2)
    X0[:s.nn] *= s.mask[:, None]
    u0[:s.nn] *= s.mask[:, None]
    return w, s, X0, u0


@pytest.mark.slow
def test_atom_scf_partial_shell_entropy():
    ref = json.load(open(os.path.join(HERE, "golden", "atom_scf.json")))
    w, s, X0, u0 = _atom_scf_inputs()
    out = S.scf(s, w["Z"], X0, u0, cheb_degree=w["cheb_degree"])
    assert out["history"][-1]["drho"] < 1e-8
    kT = S.KB_HA * 500.0
    f = out["occ"]
    # the 3-fold p shell is lowest and holds the 4 electrons: f = 2/3 each
    assert np.allclose(f[:3], 2.0 / 3.0, atol=1e-6) and np.all(f[3:] < 1e-12)
    assert np.ptp(out["eig"][:3]) < 1e-8
    ts = 3 * 2.0 * kT * ((2.0 / 3.0) * math.log(2.0 / 3.0) + (1.0 / 3.0) * math.log(1.0 / 3.0))
    assert abs((out["F"] - out["E"]) - ts) < 1e-9, (out["F"] - out["E"], ts)
    assert abs(out["E"] - ref["E"]) < 1e-9 and abs(out["F"] - ref["F"]) < 1e-9
