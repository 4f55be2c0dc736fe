"""Oracle: the learned density warm start (FP64).

TEST INFRASTRUCTURE ONLY (see oracle/fe.py).

The paper starts each SCF from a superposition of atomic densities (Sec. II.A,
Sec. IV) and has no learned part.  What is written out here is the plain
definition of a learned correction on top of that superposition: a small
per-atom network maps a radial description of each atom's neighbourhood to
the coefficients of a few atom-centred radial functions, whose sum corrects
the superposition.  Every constant below is a choice of this implementation,
not of the paper.

  descriptors  D_Ik = sum_{J != I, r_IJ < R_C} Z_J exp(-(r_IJ - mu_k)^2 / (2 s^2)) f_c(r_IJ)
               mu_k = 2 + 8 k / 31 (k = 0..31), s = 0.4 bohr,
               f_c(r) = (1 + cos(pi r / R_C)) / 2, R_C = 10 bohr
  network      x = (D - x_mean) / x_std
               a1 = silu(W1 x + b1), a2 = silu(W2 a1 + b2), a3 = silu(W3 a2 + b3)
               y = W4 a3 + b4,  c_I = y_mean + y_std * y         (32 -> 128 -> 128 -> 128 -> 8)
               silu(z) = z / (1 + exp(-z))
  basis        g_k(r) = (kappa_k / pi)^{3/2} exp(-kappa_k r^2), kappa_k = 0.5 * 16^{k/7} (k = 0..7);
               per atom the orthonormal combination phi = L^{-1} g, S = L L^T, S_kl = int g_k g_l
  correction   drho(x) = sum_I sum_k c_Ik phi_k(|x - R_I|)  (atoms with |x - R_I| < R_PHI = 8 bohr)
  warm start   rho_0 = max(rho_sup + drho, 0) scaled to N_e; rho_sup alone when no network
               is given or when the result is not a usable density
  targets      c* = argmin_c  || rho_scf - rho_sup - drho(c) ||_q^2 + ridge |c|^2, the norm being
               the mesh's Gauss quadrature (so the normal equations hold the quadrature Gram
               matrix of the phi_Ik, and what the SCF sees -- values at the Gauss points -- is
               what is fitted)
  training     loss = mean over atoms and outputs of (y - (c* - y_mean) / y_std)^2, minimised
               with Adam (Kingma & Ba, 2015)

Parameter vector (one flat array, the same layout on every side):
  W1 [128][32], b1 [128], W2 [128][128], b2 [128], W3 [128][128], b3 [128],
  W4 [8][128], b4 [8]                         -- 38,280 trained values
  x_mean [32], x_std [32], y_mean [8], y_std [8] -- 80 fixed normalisation values
Weights are stored row-major [out][in].
"""
import math

import numpy as np

N_DESC, N_HID, N_OUT = 32, 128, 8
R_C, MU0, MU1, SIGMA = 10.0, 2.0, 10.0, 0.4
R_PHI = 8.0
KAPPA = 0.5 * 16.0 ** (np.arange(N_OUT) / 7.0)
X_STD_FLOOR, Y_STD_FLOOR = 1e-2, 1e-8

LAYERS = ((N_HID, N_DESC), (N_HID, N_HID), (N_HID, N_HID), (N_OUT, N_HID))


def _offsets():
    off, o = [], 0
    for (m, n) in LAYERS:
        off.append((o, o + m * n, m, n))        # (W offset, b offset, out, in)
        o += m * n + m
    return off, o


OFFSETS, N_TRAIN = _offsets()
N_PARAMS = N_TRAIN + 2 * N_DESC + 2 * N_OUT


def unpack(theta):
    """Views (W1, b1, ..., W4, b4), x_mean, x_std, y_mean, y_std of a parameter vector."""
    layers = [(theta[w:w + m * n].reshape(m, n), theta[b:b + m]) for (w, b, m, n) in OFFSETS]
    o = N_TRAIN
    xm, xs = theta[o:o + N_DESC], theta[o + N_DESC:o + 2 * N_DESC]
    ym, ys = theta[o + 2 * N_DESC:o + 2 * N_DESC + N_OUT], theta[o + 2 * N_DESC + N_OUT:N_PARAMS]
    return layers, xm, xs, ym, ys


# --- descriptors ---------------------------------------------------------
def descriptor_centres():
    return MU0 + (MU1 - MU0) * np.arange(N_DESC) / (N_DESC - 1)


def descriptors(atoms, Z):
    """D_Ik of every atom (n, 32), pair by pair."""
    atoms = np.asarray(atoms, float)
    n = len(atoms)
    mu = descriptor_centres()
    D = np.zeros((n, N_DESC))
    for i in range(n):
        for j in range(n):
            if i == j:
                continue
            r = math.sqrt(float(np.sum((atoms[i] - atoms[j]) ** 2)))
            if r >= R_C:
                continue
            fc = 0.5 * (1.0 + math.cos(math.pi * r / R_C))
            D[i] += Z[j] * np.exp(-(r - mu) ** 2 / (2.0 * SIGMA ** 2)) * fc
    return D


# --- network -------------------------------------------------------------
def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def forward(theta, D):
    """Normalised outputs y (n, 8) and the pre-activations of the three hidden layers."""
    layers, xm, xs, _, _ = unpack(theta)
    a = (np.asarray(D, float) - xm) / xs
    acts, pre = [a], []
    for li, (W, b) in enumerate(layers):
        z = a @ W.T + b
        if li < 3:
            pre.append(z)
            a = silu(z)
            acts.append(a)
        else:
            a = z
    return a, acts, pre


def predict(theta, D):
    """Correction coefficients c (n, 8) in physical units."""
    y, _, _ = forward(theta, D)
    _, _, _, ym, ys = unpack(theta)
    return ym + ys * y


def loss_and_grad(theta, D, T):
    """Mean squared error of the normalised outputs and its gradient (N_TRAIN,).

    Back-propagation by the chain rule, layer by layer from the output."""
    layers, _, _, ym, ys = unpack(theta)
    y, acts, pre = forward(theta, D)
    t = (np.asarray(T, float) - ym) / ys
    nel = y.size
    loss = float(np.sum((y - t) ** 2)) / nel
    delta = 2.0 * (y - t) / nel                      # dL/dy
    grad = np.zeros(N_TRAIN)
    for li in range(3, -1, -1):
        w, b, m, n = OFFSETS[li]
        a_in = acts[li]
        grad[w:w + m * n] = (delta.T @ a_in).ravel()
        grad[b:b + m] = delta.sum(axis=0)
        if li > 0:
            delta = (delta @ layers[li][0]) * dsilu(pre[li - 1])
    return loss, grad


def adam_step(theta, m, v, g, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update of the trained part of theta (t counts from 1)."""
    theta, m, v = theta.copy(), m.copy(), v.copy()
    m[:] = beta1 * m + (1.0 - beta1) * g
    v[:] = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    theta[:N_TRAIN] -= lr * mh / (np.sqrt(vh) + eps)
    return theta, m, v


def train(theta, D, T, steps, t0=0, m=None, v=None, **adam):
    """Full-batch Adam for `steps` steps; returns theta, m, v and the loss before each step."""
    m = np.zeros(N_TRAIN) if m is None else m
    v = np.zeros(N_TRAIN) if v is None else v
    hist = []
    for s in range(steps):
        loss, g = loss_and_grad(theta, D, T)
        hist.append(loss)
        theta, m, v = adam_step(theta, m, v, g, t0 + s + 1, **adam)
    return theta, m, v, np.array(hist)


def set_normalisation(theta, D, T):
    """Per-feature mean and standard deviation of the training inputs and targets,
    floored at 1e-2 (inputs) and 1e-8 (targets)."""
    theta = theta.copy()
    D, T = np.asarray(D, float), np.asarray(T, float)
    o = N_TRAIN
    xm, ym = D.mean(axis=0), T.mean(axis=0)
    xs = np.maximum(np.sqrt(np.mean((D - xm) ** 2, axis=0)), X_STD_FLOOR)
    ys = np.maximum(np.sqrt(np.mean((T - ym) ** 2, axis=0)), Y_STD_FLOOR)
    theta[o:o + N_DESC], theta[o + N_DESC:o + 2 * N_DESC] = xm, xs
    theta[o + 2 * N_DESC:o + 2 * N_DESC + N_OUT], theta[o + 2 * N_DESC + N_OUT:] = ym, ys
    return theta


# --- correction basis ----------------------------------------------------
def basis_overlap(R=0.0):
    """S_kl(R) = int g_k(|x|) g_l(|x - R|) dx (closed form for Gaussians)."""
    ka, kb = KAPPA[:, None], KAPPA[None, :]
    red = ka * kb / (ka + kb)
    return (red / math.pi) ** 1.5 * np.exp(-red * R * R)


def basis_transform():
    """L^{-1} with S(0) = L L^T, so that phi = L^{-1} g is orthonormal."""
    L = np.linalg.cholesky(basis_overlap(0.0))
    return np.linalg.inv(L)


def phi_at(points, centre):
    """phi_k(|x - R|) at the points (npts, 8); zero at and beyond R_PHI."""
    d2 = np.sum((np.asarray(points) - np.asarray(centre)[None, :]) ** 2, axis=1)
    g = (KAPPA[None, :] / math.pi) ** 1.5 * np.exp(-KAPPA[None, :] * d2[:, None])
    g[d2 >= R_PHI ** 2] = 0.0
    return g @ basis_transform().T


def density_correction(mesh, atoms, c):
    """drho at every Gauss point of the mesh."""
    pts = mesh.all_quad_points()
    out = np.zeros(len(pts))
    for R, ci in zip(np.asarray(atoms, float), np.asarray(c, float)):
        out += phi_at(pts, R) @ ci
    return out


def fit_correction(mesh, atoms, drho, ridge=1e-3):
    """Least-squares coefficients (n, 8) of a density difference given at the Gauss
    points: (Phi^T W Phi + ridge I) c = Phi^T W drho, Phi the phi_Ik at the points."""
    atoms = np.asarray(atoms, float)
    pts = mesh.all_quad_points()
    wq = np.tile(mesh.quad_weights(), mesh.ncells)
    Phi = np.hstack([phi_at(pts, R) for R in atoms])
    A = Phi.T @ (wq[:, None] * Phi) + ridge * np.eye(Phi.shape[1])
    r = Phi.T @ (wq * drho)
    return np.linalg.solve(A, r).reshape(len(atoms), N_OUT)


def corrected_density(mesh, atoms, Z, c, rho_sup=None, kappa=2.4):
    """max(rho_sup + drho(c), 0) scaled to N_e, or rho_sup when that density is not
    usable (non-finite or without positive charge).  Returns (rho_0, used_fallback)."""
    from .scf import initial_density
    if rho_sup is None:
        rho_sup = initial_density(mesh, atoms, Z, kappa)
    rho = np.maximum(rho_sup + density_correction(mesh, atoms, c), 0.0)
    tot = mesh.integrate(rho)
    if not np.all(np.isfinite(rho)) or not tot > 0.0:
        return rho_sup, True
    return rho * (float(np.sum(Z)) / tot), False


def warm_start_density(mesh, atoms, Z, theta=None, rho_sup=None, kappa=2.4):
    """The corrected density with the network's coefficients, or rho_sup when theta is
    None.  Returns (rho_0, used_fallback)."""
    from .scf import initial_density
    if rho_sup is None:
        rho_sup = initial_density(mesh, atoms, Z, kappa)
    if theta is None:
        return rho_sup, True
    return corrected_density(mesh, atoms, Z, predict(theta, descriptors(atoms, Z)), rho_sup=rho_sup)
