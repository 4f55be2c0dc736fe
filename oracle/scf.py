"""Oracle: the self-consistent field machinery around the eigensolver (FP64).

TEST INFRASTRUCTURE ONLY (see oracle/fe.py).

Follows Sec. II.A of the paper:
  * Eq. (rhocompute): rho(r) = 2 sum_i f(eps_i, mu) |psi_i(r)|^2, Fermi-Dirac f.
  * Eq. (electronconstraint): 2 sum_i f(eps_i, mu) = N_e fixes mu.
  * Eq. (vKS): v_KS = v_xc + v_el; LDA exchange-correlation of Perdew-Wang
    (PW92) form, spin unpolarised.
  * Eqs. (EZZbmsear), (EellocReform), (poisson): local reformulation of the
    electrostatics; phi solves -1/(4 pi) Lap phi = rho + b_sm.
  * Sec. IV: 500 K smearing and Anderson mixing.
Readings where the paper is silent: the local pseudopotential
v_loc = -Z erf(r/alpha)/r is exactly the potential of the Gaussian charge
-Z g_alpha, so b_sm = sum -Z_I g_alpha(r - R_I) and v_loc - v_sm = 0; the
self energy is E_self = sum Z_I^2 / (sqrt(2 pi) alpha) and the Gaussian
overlap correction dE_ZZ = sum_{I<J} Z_I Z_J erfc(R_IJ/(sqrt(2) alpha))/R_IJ.
"""
import math

import numpy as np

from .chfsi import chfsi, lanczos_bounds, residual_filter, rayleigh_ritz, residual_norms

KB_HA = 3.166811563e-6          # Boltzmann constant in Ha/K

# PW92 parameters for eps_c(r_s, zeta = 0)
PW_A, PW_A1 = 0.031091, 0.21370
PW_B = (7.5957, 3.5876, 1.6382, 0.49294)
RHO_FLOOR = 1e-14


def lda_pw92(rho):
    """LDA (Slater exchange + PW92 correlation): returns (eps_xc, v_xc) per point.

    eps_x = -(3/4)(3/pi)^(1/3) rho^(1/3);  eps_c = -2A(1 + a1 rs) ln(1 + 1/(2A(b1 rs^1/2 +
    b2 rs + b3 rs^3/2 + b4 rs^2)));  v_xc = eps_xc - (rs/3) d eps_xc/d rs.
    Points with rho < 1e-14 get zero.
    """
    rho = np.asarray(rho, float)
    eps = np.zeros_like(rho)
    v = np.zeros_like(rho)
    ok = rho >= RHO_FLOOR
    r = rho[ok]
    rs = (3.0 / (4.0 * math.pi * r)) ** (1.0 / 3.0)
    ex = -0.75 * (3.0 / math.pi) ** (1.0 / 3.0) * r ** (1.0 / 3.0)
    vx = 4.0 / 3.0 * ex
    b1, b2, b3, b4 = PW_B
    srs = np.sqrt(rs)
    q0 = -2.0 * PW_A * (1.0 + PW_A1 * rs)
    q1 = 2.0 * PW_A * (b1 * srs + b2 * rs + b3 * rs * srs + b4 * rs * rs)
    dq1 = PW_A * (b1 / srs + 2.0 * b2 + 3.0 * b3 * srs + 4.0 * b4 * rs)
    lg = np.log(1.0 + 1.0 / q1)
    ec = q0 * lg
    dec = -2.0 * PW_A * PW_A1 * lg - q0 * dq1 / (q1 * q1 + q1)
    vc = ec - rs / 3.0 * dec
    eps[ok] = ex + ec
    v[ok] = vx + vc
    return eps, v


def fermi_level(eig, n_elec, kT, tol=1e-12, max_iter=400):
    """Bisection on mu for 2 sum_i f_i = N_e (Eq. electronconstraint); returns (mu, f)."""
    eig = np.asarray(eig, float)

    def count(mu):
        x = (eig - mu) / kT
        return 2.0 * np.sum(0.5 * (1.0 - np.tanh(0.5 * x)))

    lo = float(eig.min()) - 50.0 * kT - 1.0
    hi = float(eig.max()) + 50.0 * kT + 1.0
    mu = 0.5 * (lo + hi)
    for _ in range(max_iter):
        mu = 0.5 * (lo + hi)
        n = count(mu)
        if abs(n - n_elec) < tol:
            break
        if n > n_elec:
            hi = mu
        else:
            lo = mu
    f = 0.5 * (1.0 - np.tanh(0.5 * (eig - mu) / kT))
    return mu, f


def entropy_term(f, kT):
    """-T S = 2 kT sum [f ln f + (1-f) ln(1-f)] (spin-degenerate smearing entropy)."""
    f = np.clip(np.asarray(f, float), 0.0, 1.0)
    s = 0.0
    for x in f:
        if 0.0 < x < 1.0:
            s += x * math.log(x) + (1.0 - x) * math.log(1.0 - x)
    return 2.0 * kT * s


def gaussian_charge(pts, atoms, Z, alpha):
    """b_sm(x) = sum_I -Z_I pi^-3/2 alpha^-3 exp(-|x - R_I|^2 / alpha^2)."""
    out = np.zeros(len(pts))
    c = math.pi ** -1.5 / alpha ** 3
    for R, z in zip(atoms, Z):
        d2 = np.sum((pts - R[None, :]) ** 2, axis=1)
        out -= z * c * np.exp(-d2 / (alpha * alpha))
    return out


def self_energy(Z, alpha):
    return float(sum(z * z for z in Z) / (math.sqrt(2.0 * math.pi) * alpha))


def zz_overlap_correction(atoms, Z, alpha):
    """sum_{I<J} Z_I Z_J erfc(R_IJ / (sqrt 2 alpha)) / R_IJ."""
    e = 0.0
    for i in range(len(Z)):
        for j in range(i + 1, len(Z)):
            R = float(np.linalg.norm(atoms[i] - atoms[j]))
            e += Z[i] * Z[j] * math.erfc(R / (math.sqrt(2.0) * alpha)) / R
    return e


def poisson_solve(mesh, fq, tol=1e-12, max_iter=5000, boundary=None, k2=0.0):
    """FE solution of -1/(4 pi) Lap phi + k2/(4 pi) phi = f (k2 = 0: Poisson, Eq.
    poisson) with phi = 0 (or ``boundary``) on the box.

    Weak form: (1/4pi) (K + k2 M) phi = F, F_j = int N_j f, M the lumped (GLL)
    mass, by Jacobi-preconditioned conjugate gradients to ||r|| < tol ||F||.
    Returns (phi_nodes, iterations).
    """
    Ke = mesh.stiffness_cell() / (4.0 * math.pi)
    mask = mesh.interior_mask()
    shift = (k2 / (4.0 * math.pi)) * mesh.lumped_mass() if k2 else np.zeros(mesh.nnodes)
    F = mesh.integrate_against_basis(fq)
    g = np.zeros(mesh.nnodes)
    if boundary is not None:
        g[~mask] = boundary[~mask]
        F = F - mesh.apply_cells(Ke, g[:, None])[:, 0]
    F = F * mask

    def A(x):
        return (mesh.apply_cells(Ke, (x * mask)[:, None])[:, 0] + shift * x) * mask

    diag = mesh.apply_cells(np.diag(np.diag(Ke)), np.ones((mesh.nnodes, 1)))[:, 0] + shift
    dinv = np.where(mask, 1.0 / diag, 0.0)
    x = np.zeros(mesh.nnodes)
    r = F.copy()
    z = dinv * r
    p = z.copy()
    rz = float(r @ z)
    bnorm = float(np.linalg.norm(F))
    it = 0
    if bnorm == 0.0:
        return x + g, 0
    while it < max_iter:
        Ap = A(p)
        alpha = rz / float(p @ Ap)
        x += alpha * p
        r -= alpha * Ap
        it += 1
        if np.linalg.norm(r) < tol * bnorm:
            break
        z = dinv * r
        rz_new = float(r @ z)
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x + g, it


def density(sysm, V, f):
    """rho(x_q) = 2 sum_i f_i psi_i(x_q)^2 at every Gauss point (Eq. rhocompute)."""
    psi = sysm.values_at_quad(V)
    return 2.0 * np.sum(psi * psi * np.asarray(f)[None, :], axis=1)


def anderson_mix(hist_in, hist_out, w, beta, precond=None):
    """Anderson mixing (Walker-Ni form) on densities at quadrature points.

    hist_in/hist_out: lists of rho_in, rho_out (oldest first); w: quadrature
    weights (the inner product).  gamma minimises ||R_k - dR gamma||_w;
    rho_next = (x_k - dX gamma) + beta P(R_k - dR gamma), P = precond or the
    identity (the paper's plain Anderson).
    """
    P = precond if precond is not None else (lambda r: r)
    xk = hist_in[-1]
    Rk = hist_out[-1] - hist_in[-1]
    m = len(hist_in) - 1
    if m == 0:
        return xk + beta * P(Rk)
    dX = np.stack([hist_in[j + 1] - hist_in[j] for j in range(m)], axis=1)
    R = [hist_out[j] - hist_in[j] for j in range(m + 1)]
    dR = np.stack([R[j + 1] - R[j] for j in range(m)], axis=1)
    A = dR.T @ (w[:, None] * dR)
    b = dR.T @ (w * Rk)
    gamma = np.linalg.lstsq(A, b, rcond=None)[0]
    return (xk - dX @ gamma) + beta * P(Rk - dR @ gamma)


def kerker(mesh, R, k2, tol=1e-12):
    """Kerker preconditioning of a density residual (not in the paper, whose
    mixing is plain Anderson): R - k2 (-Lap + k2)^-1 R, the Fourier factor
    q^2 / (q^2 + k2) of each mode, with the inverse by the FE solve above
    (phi = 4 pi (-Lap + k2)^-1 R, so the correction is k2 phi / (4 pi))."""
    phi, _ = poisson_solve(mesh, R, tol=tol, k2=k2)
    phq = mesh.interpolate(phi[:, None])[:, 0]
    return R - (k2 / (4.0 * math.pi)) * phq


def initial_density(mesh, atoms, Z, kappa=2.4):
    """Superposition of atomic Gaussians Z (kappa/pi)^3/2 exp(-kappa r^2), scaled to N_e."""
    pts = mesh.all_quad_points()
    rho = np.zeros(len(pts))
    for R, z in zip(atoms, Z):
        d2 = np.sum((pts - R[None, :]) ** 2, axis=1)
        rho += z * (kappa / math.pi) ** 1.5 * np.exp(-kappa * d2)
    return rho * (float(np.sum(Z)) / mesh.integrate(rho))


def hartree_potential(mesh, rho_q, bq, tol=1e-12):
    """phi of rho + b_sm (Eq. poisson), nodal and at the Gauss points."""
    phi, it = poisson_solve(mesh, rho_q + bq, tol=tol)
    return phi, mesh.interpolate(phi[:, None])[:, 0], it


def total_energy(mesh, eig, f, kT, rho_out, veff_in, bq, phi_out_q, atoms, Z, alpha):
    """E = 2 sum f eps - int rho_out v_eff[rho_in] + E_xc[rho_out]
         + 1/2 int (rho_out + b_sm) phi[rho_out] - E_self + dE_ZZ; F = E - TS."""
    band = 2.0 * float(np.sum(f * eig))
    exc, _ = lda_pw92(rho_out)
    E = (band - mesh.integrate(rho_out * veff_in) + mesh.integrate(rho_out * exc)
         + 0.5 * mesh.integrate((rho_out + bq) * phi_out_q)
         - self_energy(Z, alpha) + zz_overlap_correction(atoms, Z, alpha))
    return E, E + entropy_term(f, kT)


def scf(sysm, Z, X0, lanczos_u0, *, cheb_degree=20, temperature=500.0, alpha_loc=0.8,
        mix_beta=0.5, mix_hist=8, tol_rho=1e-8, tol_e=1e-8, max_iter=60,
        first_tol=1e-2, first_max_pass=20, renormalize=True, rho0=None, log=None, precond_k2=0.0):
    """Self-consistent field loop (Sec. II.A; Sec. IV for 500 K and Anderson).

    Per iteration: phi[rho_in] by Poisson, v_eff = v_xc[rho_in] + phi; cell and
    coupling matrices; eigenpairs by residual ChFSI (first iteration: passes
    until the max residual < first_tol, from X0; later: one pass); mu;
    rho_out; energy; Anderson mixing (precond_k2 > 0: with the Kerker step
    above, an addition to the paper's plain Anderson).  Converged when
    ||rho_out - rho_in||/N_e < tol_rho and |dE| < tol_e per atom.
    """
    mesh = sysm.mesh
    atoms = sysm.atoms
    Z = np.asarray(Z, float)
    ne = float(Z.sum())
    kT = KB_HA * temperature
    pts = mesh.all_quad_points()
    bq = gaussian_charge(pts, atoms, Z, alpha_loc)
    w = np.tile(mesh.quad_weights(), mesh.ncells)
    rho_in = initial_density(mesh, atoms, Z) if rho0 is None else np.asarray(rho0, float)
    N = X0.shape[1]
    nocc = int(math.ceil(ne / 2.0))
    hin, hout = [], []
    E_prev = None
    V = lam = HV = None
    history = []
    for it in range(1, max_iter + 1):
        phi, phi_q, _ = hartree_potential(mesh, rho_in, bq)
        _, vxc = lda_pw92(rho_in)
        veff = vxc + phi_q
        sysm.set_potential(veff)
        if it == 1:
            out = chfsi(sysm, X0, cheb_degree, first_tol, first_max_pass, lanczos_u0,
                        nconv=nocc)
            lam, V, HV = out["lam"], out["V"], out["HV"]
        else:
            _, _, b = lanczos_bounds(sysm, lanczos_u0)
            HV = sysm.apply_H(V)
            Vout = residual_filter(sysm, V, lam, cheb_degree, float(lam[-1]), b, float(lam[0]), HV=HV)
            lam, V, HV = rayleigh_ritz(sysm, Vout)
        mu, f = fermi_level(lam, ne, kT)
        rho_out = density(sysm, V, f)
        if renormalize:
            rho_out = rho_out * (ne / mesh.integrate(rho_out))
        _, phi_out_q, _ = hartree_potential(mesh, rho_out, bq)
        E, F = total_energy(mesh, lam, f, kT, rho_out, veff, bq, phi_out_q, atoms, Z, alpha_loc)
        dr = math.sqrt(mesh.integrate((rho_out - rho_in) ** 2)) / ne
        dE = abs(E - E_prev) / len(Z) if E_prev is not None else np.inf
        res = residual_norms(sysm, V, lam, HV)
        history.append(dict(it=it, E=E, F=F, mu=mu, drho=dr, dE=dE, resid=float(res[:nocc].max())))
        if log is not None:
            log(history[-1])
        if dr < tol_rho and dE < tol_e:
            break
        E_prev = E
        hin.append(rho_in)
        hout.append(rho_out)
        hin, hout = hin[-(mix_hist + 1):], hout[-(mix_hist + 1):]
        pre = (lambda r: kerker(mesh, r, precond_k2)) if precond_k2 > 0.0 else None
        rho_in = anderson_mix(hin, hout, w, mix_beta, precond=pre)
    return dict(E=E, F=F, mu=mu, eig=lam, occ=f, V=V, rho=rho_out, iters=it, history=history)
