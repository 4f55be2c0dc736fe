"""Pins for the oracle's SCF pieces (Sec. II.A): PW92 against its limits and
its own derivative, the FE Poisson solve against the erf potential of a
Gaussian charge and its closed-form self energy, the Fermi level, Anderson
mixing on a linear map, and a full dimer SCF (energy decreases, the raw
density integrates to N_e up to the lumping error)."""
import math

import numpy as np
import pytest
from scipy.special import erf

from oracle import scf as S
from oracle.efe import EFESystem
from oracle.fe import Mesh


def test_pw92_exchange_closed_form_and_derivative():
    rho = np.logspace(-6, 2, 200)
    eps, v = S.lda_pw92(rho)
    ex = -0.75 * (3 / math.pi) ** (1 / 3) * rho ** (1 / 3)
    ec = eps - ex
    assert np.all(ec < 0) and np.all(ec > ex)               # correlation smaller than exchange
    h = 1e-6 * rho
    e1, _ = S.lda_pw92(rho + h)
    e0, _ = S.lda_pw92(rho - h)
    fd = ((rho + h) * e1 - (rho - h) * e0) / (2 * h)
    assert np.allclose(v, fd, rtol=1e-8)
    e, vv = S.lda_pw92(np.array([0.0, 1e-15, -1e-3]))
    assert np.all(e == 0) and np.all(vv == 0)


def test_pw92_high_density_limit():
    # eps_c -> c0 ln rs - c1, c0 = (1 - ln 2)/pi^2, c1 = 0.046644 (RPA limit)
    c0 = (1 - math.log(2)) / math.pi ** 2
    rs = np.array([1e-6, 1e-7])
    rho = 3 / (4 * math.pi * rs ** 3)
    eps, _ = S.lda_pw92(rho)
    ex = -0.75 * (3 / math.pi) ** (1 / 3) * rho ** (1 / 3)
    ec = eps - ex
    slope = (ec[0] - ec[1]) / (math.log(rs[0]) - math.log(rs[1]))
    assert abs(slope - c0) < 2e-5
    assert abs((ec[1] - c0 * math.log(rs[1])) + 0.046644) < 2e-4
    # textbook values of the uniform gas correlation energy (Ha)
    for r, ref in [(1.0, -0.0598), (2.0, -0.0448), (5.0, -0.0282), (10.0, -0.0186)]:
        rho = 3 / (4 * math.pi * r ** 3)
        e, _ = S.lda_pw92(np.array([rho]))
        ecv = e[0] + 0.75 * (3 / math.pi) ** (1 / 3) * rho ** (1 / 3)
        assert abs(ecv - ref) < 3e-4, (r, ecv)


def test_fermi_level():
    eig = np.array([-2.0, -1.0, -0.99, -0.5, 0.3])
    kT = S.KB_HA * 500
    for ne in (2.0, 4.0, 5.0, 7.3):
        mu, f = S.fermi_level(eig, ne, kT)
        assert abs(2 * f.sum() - ne) < 1e-11
    mu, f = S.fermi_level(eig, 4.0, 1e-6)
    assert np.allclose(f, [1, 1, 0, 0, 0], atol=1e-12)


@pytest.mark.slow
def test_poisson_gaussian_charge():
    alpha, Z = 0.8, 1.0
    box, ctr = 12.0, np.array([6.0, 6.0, 6.0])
    errs = []
    for n in (6, 12):
        m = Mesh(box / n, (n, n, n), 4)
        q = m.all_quad_points()
        rho = -S.gaussian_charge(q, ctr[None, :], [Z], alpha)    # +Z g_alpha
        X = m.node_xyz()
        r = np.linalg.norm(X - ctr, axis=1)
        with np.errstate(invalid="ignore", divide="ignore"):
            exact = np.where(r > 0, Z * erf(r / alpha) / np.where(r > 0, r, 1), Z * 2 / (math.sqrt(math.pi) * alpha))
        phi, it = S.poisson_solve(m, rho, tol=1e-13, boundary=exact)
        errs.append(np.max(np.abs(phi - exact)))
        if n == 12:
            phq = m.interpolate(phi[:, None])[:, 0]
            e_self = 0.5 * m.integrate(rho * phq)
            assert abs(e_self - S.self_energy([Z], alpha)) < 1e-5
    assert errs[1] < errs[0] / 20 and errs[1] < 1e-4


def test_anderson_linear_fixed_point():
    rng = np.random.default_rng(0)
    n = 30
    A = rng.standard_normal((n, n))
    A = 0.9 * A / np.linalg.norm(A, 2)
    c = rng.standard_normal(n)
    xstar = np.linalg.solve(np.eye(n) - A, c)
    w = np.ones(n)
    hin, hout = [np.zeros(n)], [c.copy()]
    for k in range(40):
        x = S.anderson_mix(hin, hout, w, 0.5)
        hin.append(x)
        hout.append(A @ x + c)
        hin, hout = hin[-9:], hout[-9:]
    assert np.linalg.norm(hin[-1] - xstar) < 1e-8
    # without history it is plain linear mixing
    x = S.anderson_mix([np.zeros(n)], [c], w, 0.3)
    assert np.allclose(x, 0.3 * c)


@pytest.mark.slow
def test_dimer_scf():
    from paper_2607_06848_gb300 import workloads as W
    w = W.dimer()
    m = Mesh(w["h"], w["ncell"], w["p"])
    s = EFESystem(m, w["atoms"], enrich=dict(alpha=1.2, r0=5 * 0.33 / 1.33, t=0.33),
                  proj=dict(rc=1.0, rtrunc=6.0, h=w["hproj"]))
    rows = s.nn + s.n_enr
    X0 = W.random_block(rows, w["nstates"], 1)
    u0 = W.random_block(rows, 1, 2)
    X0[:s.nn] *= s.mask[:, None]
    u0[:s.nn] *= s.mask[:, None]
    out = S.scf(s, w["Z"], X0, u0, cheb_degree=20, renormalize=False)
    hist = out["history"]
    assert hist[-1]["drho"] < 1e-8 and hist[-1]["dE"] < 1e-8
    E = [h["E"] for h in hist]
    assert all(E[i + 1] < E[i] + 1e-7 for i in range(len(E) - 1))
    # 2 sum f = N_e exactly; the raw density integral differs only by lumping
    assert abs(2 * out["occ"].sum() - 8.0) < 1e-11
    assert abs(m.integrate(out["rho"]) - 8.0) < 2e-2
    # the energy by another route: kinetic + nonlocal as orbital expectation
    # values (H^E with v = 0), E_xc and the electrostatics of rho_out directly.
    # With the raw density, 2 sum f eps_i - int rho_out v_eff is exactly that
    # expectation value (same quadrature in V and in rho), so the two agree to
    # rounding at any iteration; a dropped or mis-signed term would not
    V, f, rho = out["V"], out["occ"], out["rho"]
    Z = np.asarray(w["Z"], float)
    s.set_potential(np.zeros(len(rho)))
    tnl = 2.0 * float(np.sum(f * np.sum(V * s.apply_H(V), axis=0)))
    eps, _ = S.lda_pw92(rho)
    bq = S.gaussian_charge(m.all_quad_points(), s.atoms, Z, 0.8)
    _, phq, _ = S.hartree_potential(m, rho, bq)
    E_direct = (tnl + m.integrate(rho * eps) + 0.5 * m.integrate((rho + bq) * phq)
                - S.self_energy(Z, 0.8) + S.zz_overlap_correction(s.atoms, Z, 0.8))
    assert abs(E_direct - out["E"]) < 1e-10, (E_direct, out["E"])


def test_kerker_factor_on_sine_modes():
    # the Kerker step multiplies each mode of the residual by q^2 / (q^2 + k2):
    # sin(a pi x/L) sin(b pi y/L) sin(c pi z/L) vanishes on the box and has
    # q^2 = (a^2 + b^2 + c^2) pi^2 / L^2; the FE solve converges to it in h and p
    L = 8.0
    errs = {}
    for n, p in ((4, 4), (8, 4), (4, 6)):
        m = Mesh(L / n, (n, n, n), p)
        q = m.all_quad_points()
        for (a, b, c) in ((1, 1, 1), (2, 1, 1)):
            R = (np.sin(a * math.pi * q[:, 0] / L) * np.sin(b * math.pi * q[:, 1] / L)
                 * np.sin(c * math.pi * q[:, 2] / L))
            q2 = (a * a + b * b + c * c) * math.pi ** 2 / L ** 2
            for k2 in (0.64, 2.0):
                fac = q2 / (q2 + k2)
                PR = S.kerker(m, R, k2)
                errs[(n, p, a, k2)] = np.abs(PR - fac * R).max() / np.abs(fac * R).max()
    assert max(v for k, v in errs.items() if k[:2] == (4, 6)) < 2e-6
    for a in (1, 2):
        for k2 in (0.64, 2.0):
            assert errs[(8, 4, a, k2)] < errs[(4, 4, a, k2)] / 16.0


@pytest.mark.slow
def test_kerker_scf_reaches_the_same_fixed_point():
    # a preconditioner of the mixing step changes the path, not the solution:
    # the dimer SCF with the Kerker step ends at the golden FP64 energy
    import json
    import os
    from paper_2607_06848_gb300 import workloads as W
    ref = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "dimer_scf.json")))
    w = W.dimer()
    m = Mesh(w["h"], w["ncell"], w["p"])
    s = EFESystem(m, w["atoms"], enrich=dict(alpha=1.2, r0=5 * 0.33 / 1.33, t=0.33),
                  proj=dict(rc=1.0, rtrunc=6.0, h=w["hproj"]))
    rows = s.nn + s.n_enr
    X0 = W.random_block(rows, w["nstates"], 1)
    u0 = W.random_block(rows, 1, 2)
    X0[:s.nn] *= s.mask[:, None]
    u0[:s.nn] *= s.mask[:, None]
    out = S.scf(s, w["Z"], X0, u0, cheb_degree=20, precond_k2=0.64)
    assert out["history"][-1]["drho"] < 1e-8
    assert abs(out["E"] - ref["E"]) / 2 < 1e-8, (out["E"], ref["E"])
