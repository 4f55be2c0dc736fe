"""Oracle: residual Chebyshev-filtered subspace iteration (FP64).

TEST INFRASTRUCTURE ONLY (see oracle/fe.py).

Follows Sec. III.B of the paper:
  * Eq. (ChebyRecur): C_m = (2 s_m / e)(x - c) C_{m-1} - s_{m-1} s_m C_{m-2},
    s_m = 1 / (2/s_1 - s_{m-1}), s_1 = e / (a_min - c), c = (a+b)/2,
    e = (b-a)/2, C_0 = 1, C_1 = s_1 (x - c) / e.
  * Eq. (residual) defines Z_k = M~ (C_k(A) V - V C_k(Lambda)).  Eq.
    (residualapprox) as printed is garbled in two places; the recurrence
    derived from Eq. (residual) and Eq. (ChebyRecur) with M~ M^-1 ~ I is
        Z_k = (2 s_k/e)(H M~^-1 Z_{k-1} - c Z_{k-1}) - s_{k-1} s_k Z_{k-2}
              + (2 s_k/e) G diag(C_{k-1}(Lambda)),
        Z_0 = 0,  Z_1 = (s_1/e) G,  G = H V - M V Lambda,
        V_out = M~^-1 Z_m + V diag(C_m(Lambda)).
  * Eq. (projectedKSEig): Rayleigh-Ritz with the exact M^E.
  * Multipass filtering until the eigen-residual falls below a tolerance.
Spectral bounds are not described in the paper; our reading is a k-step
Lanczos on M~^-1 H in the M~ inner product (the same tridiagonal matrix as
Lanczos on M~^-1/2 H M~^-1/2) giving b = theta_max + |beta_k s_k|.
"""
import numpy as np
import scipy.linalg as sla


def lanczos_bounds(sysm, u0, k=10):
    """k-step Lanczos for the spectrum of M~^-1 H^E, started from the vector u0.

    Returns (theta_min, theta_max, upper_bound) with
    upper_bound = theta_max + |beta_k * (last component of its Ritz vector)|.
    """
    u0 = np.asarray(u0, float).reshape(-1, 1)
    Mt = sysm.apply_Mtilde
    q = u0 / np.sqrt(float(np.sum(u0 * Mt(u0))))
    q_prev = np.zeros_like(q)
    alphas, betas = [], []
    beta = 0.0
    for j in range(k):
        w = sysm.apply_H(q)
        a = float(np.sum(q * w))
        r = sysm.apply_Minv_approx(w) - a * q - beta * q_prev
        beta = float(np.sqrt(max(float(np.sum(r * Mt(r))), 0.0)))
        alphas.append(a)
        betas.append(beta)
        if beta == 0.0:
            break
        q_prev, q = q, r / beta
    T = np.diag(alphas) + np.diag(betas[:-1], 1) + np.diag(betas[:-1], -1)
    th, S = np.linalg.eigh(T)
    return float(th[0]), float(th[-1]), float(th[-1] + abs(betas[-1] * S[-1, -1]))


def cheb_scalars(lam, m, a, b, a0):
    """C_k(lambda) for k = 0..m by Eq. (ChebyRecur); returns (m+1, len(lam))."""
    lam = np.asarray(lam, float)
    e = (b - a) / 2.0
    c = (b + a) / 2.0
    s1 = e / (a0 - c)
    out = np.empty((m + 1, len(lam)))
    out[0] = 1.0
    out[1] = s1 * (lam - c) / e
    s_prev = s1
    for k in range(2, m + 1):
        s = 1.0 / (2.0 / s1 - s_prev)
        out[k] = (2.0 * s / e) * (lam - c) * out[k - 1] - s_prev * s * out[k - 2]
        s_prev = s
    return out


def residual_filter(sysm, V, lam, m, a, b, a0, HV=None):
    """One residual Chebyshev filter of degree m (Eqs. residual, residualapprox corrected).

    V: (rows, N) approximate eigenvectors; lam: their Ritz values.  Returns V_out.
    """
    lam = np.asarray(lam, float)
    e = (b - a) / 2.0
    c = (b + a) / 2.0
    s1 = e / (a0 - c)
    if HV is None:
        HV = sysm.apply_H(V)
    G = HV - sysm.apply_M(V) * lam[None, :]
    Ck = cheb_scalars(lam, m, a, b, a0)
    Z_prev = np.zeros_like(G)
    Z = (s1 / e) * G
    s_prev = s1
    for k in range(2, m + 1):
        s = 1.0 / (2.0 / s1 - s_prev)
        HY = sysm.apply_H(sysm.apply_Minv_approx(Z))
        Z_new = (2.0 * s / e) * (HY - c * Z) - s_prev * s * Z_prev \
            + (2.0 * s / e) * G * Ck[k - 1][None, :]
        Z_prev, Z = Z, Z_new
        s_prev = s
    return sysm.apply_Minv_approx(Z) + V * Ck[m][None, :]


def standard_filter(sysm, V, m, a, b, a0):
    """Plain Chebyshev filter C_m(M~^-1 H) V (Eq. ChebyRecur with the approximate inverse)."""
    e = (b - a) / 2.0
    c = (b + a) / 2.0
    s1 = e / (a0 - c)
    Y_prev = V
    Y = (s1 / e) * (sysm.apply_Minv_approx(sysm.apply_H(V)) - c * V)
    s_prev = s1
    for k in range(2, m + 1):
        s = 1.0 / (2.0 / s1 - s_prev)
        Y_new = (2.0 * s / e) * (sysm.apply_Minv_approx(sysm.apply_H(Y)) - c * Y) - s_prev * s * Y_prev
        Y_prev, Y = Y, Y_new
        s_prev = s
    return Y


def rayleigh_ritz(sysm, V):
    """Eq. (projectedKSEig): V^T H V d = eps V^T M V d with the exact M^E.

    Returns (lam ascending, V D, H V D) with (V D)^T M (V D) = I.
    """
    HV = sysm.apply_H(V)
    Hp = V.T @ HV
    S = V.T @ sysm.apply_M(V)
    Hp = 0.5 * (Hp + Hp.T)
    S = 0.5 * (S + S.T)
    lam, D = sla.eigh(Hp, S)
    return lam, V @ D, HV @ D


def residual_norms(sysm, V, lam, HV=None):
    """||H psi_i - eps_i M psi_i||_2 for M-normalised columns."""
    if HV is None:
        HV = sysm.apply_H(V)
    R = HV - sysm.apply_M(V) * lam[None, :]
    return np.sqrt(np.sum(R * R, axis=0))


def chfsi(sysm, X0, m, tol, max_pass, lanczos_u0, nconv=None, lanczos_k=10,
          residual=True, bounds=None):
    """Multipass (residual) ChFSI for the lowest eigenpairs (Sec. III.B).

    Bounds for the first pass: Lanczos theta_min = a0, b = Lanczos upper
    bound, a = a0 + 0.3 (b - a0) (our reading); later passes a = max Ritz
    value, a0 = min Ritz value.  Stops when the residuals of the lowest
    ``nconv`` states are below ``tol``.
    Returns dict(lam, V, HV, resid, passes, history).
    """
    N = X0.shape[1]
    nconv = N if nconv is None else nconv
    if bounds is None:
        tmin, tmax, b = lanczos_bounds(sysm, lanczos_u0, lanczos_k)
        a0 = tmin
        a = tmin + 0.3 * (b - tmin)
    else:
        a0, a, b = bounds
    lam, V, HV = rayleigh_ritz(sysm, X0)
    hist = []
    passes = 0
    res = residual_norms(sysm, V, lam, HV)
    while passes < max_pass:
        if residual:
            Vout = residual_filter(sysm, V, lam, m, a, b, a0, HV=HV)
        else:
            Vout = standard_filter(sysm, V, m, a, b, a0)
        lam, V, HV = rayleigh_ritz(sysm, Vout)
        res = residual_norms(sysm, V, lam, HV)
        passes += 1
        hist.append(float(np.max(res[:nconv])))
        a0, a = float(lam[0]), float(lam[-1])
        if hist[-1] < tol:
            break
    return dict(lam=lam, V=V, HV=HV, resid=res, passes=passes, history=hist, bounds=(a0, a, b))
