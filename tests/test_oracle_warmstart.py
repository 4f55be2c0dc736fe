"""Pins of the learned warm-start oracle (oracle/warmstart.py) to facts outside it.

* descriptors: a sampled Gaussian comb sums to sqrt(2 pi) s / dmu and its
  centroid is the pair distance (Poisson summation, exact to ~1e-15 inside the
  comb); f_c(R_C / 2) = 1/2; invariance under rotation, translation and
  permutation; additivity over neighbours and linearity in Z_J;
* silu: the identity silu(z) - silu(-z) = z, silu'(0) = 1/2;
* network wiring: a network that passes one input through one unit per layer
  reduces to a scalar composition evaluated with math.exp;
* gradients: central finite differences of the loss (FP64);
* Adam: with a constant gradient the bias-corrected moments equal g and g^2, so
  every step moves each weight by exactly -lr g / (|g| + eps);
* basis: the closed-form Gaussian overlaps against a 1-D Gauss-Legendre
  integration (the 3-D integral factorises), orthonormality of phi under a
  fine FE mesh's quadrature, and a synthesise-then-fit round trip (exact in
  the quadrature norm, on the production resolution h = 2, p = 4);
* warm start: charge N_e, non-negativity, and the superposition when the
  network's output is identically zero.
"""
import math

import numpy as np
import pytest

from oracle import warmstart as O
from oracle.fe import Mesh
from oracle.scf import initial_density
from paper_2607_06848_gb300 import workloads as W


def _rot(seed):
    q, _ = np.linalg.qr(np.random.default_rng(seed).standard_normal((3, 3)))
    return q


def test_descriptor_comb_sum_and_centroid():
    dmu = (O.MU1 - O.MU0) / (O.N_DESC - 1)
    mu = O.descriptor_centres()
    for d in (5.0, 5.7, 6.3, 7.0):      # >= 7.5 s from both ends of the comb
        u = np.random.default_rng(int(d * 10)).standard_normal(3)
        u /= np.linalg.norm(u)
        atoms = np.array([[3.0, 4.0, 5.0], [3.0, 4.0, 5.0] + d * u])
        D = O.descriptors(atoms, np.array([4.0, 2.5]))
        fc = 0.5 * (1 + math.cos(math.pi * d / 10.0))
        assert abs(D[0].sum() - 2.5 * fc * math.sqrt(2 * math.pi) * 0.4 / dmu) < 1e-12 * D[0].sum()
        assert abs(D[1].sum() - 4.0 * fc * math.sqrt(2 * math.pi) * 0.4 / dmu) < 1e-12 * D[1].sum()
        assert abs(np.dot(mu, D[0]) / D[0].sum() - d) < 1e-11
    atoms = np.array([[0.0, 0, 0], [5.0, 0, 0]])
    assert abs(O.descriptors(atoms, np.ones(2))[0].sum() - 0.5 * math.sqrt(2 * math.pi) * 0.4 / dmu) < 1e-12 * 2
    far = np.array([[0.0, 0, 0], [10.0, 0, 0], [0, 10.5, 0]])
    assert np.all(O.descriptors(far, np.ones(3))[0] == 0.0)


def test_descriptor_invariances_and_additivity():
    atoms = W.place_atoms(9, 0.0, 12.0, 4.2, 3)
    Z = np.random.default_rng(4).uniform(1, 5, 9)
    D = O.descriptors(atoms, Z)
    Q = _rot(5)
    D2 = O.descriptors(atoms @ Q.T + np.array([1.5, -7.0, 3.3]), Z)
    assert np.allclose(D, D2, rtol=1e-12, atol=1e-14)
    perm = np.random.default_rng(6).permutation(9)
    assert np.allclose(O.descriptors(atoms[perm], Z[perm]), D[perm], rtol=1e-12, atol=1e-14)
    acc = np.zeros(O.N_DESC)
    for j in range(1, 9):
        acc += O.descriptors(atoms[[0, j]], Z[[0, j]])[0]
    assert np.allclose(acc, D[0], rtol=1e-12, atol=1e-14)
    Z3 = Z.copy()
    Z3[1:] *= 3.0
    assert np.allclose(O.descriptors(atoms, Z3)[0], 3 * D[0], rtol=1e-12, atol=1e-14)


def test_silu_identities():
    z = np.linspace(-30, 30, 601)
    assert np.allclose(O.silu(z) - O.silu(-z), z, rtol=0, atol=1e-13)
    assert O.silu(0.0) == 0.0 and abs(O.dsilu(0.0) - 0.5) < 1e-16
    hh = 1e-6
    assert np.allclose(O.dsilu(z), (O.silu(z + hh) - O.silu(z - hh)) / (2 * hh), atol=1e-8)


def test_network_wiring_scalar_composition():
    th = np.zeros(O.N_PARAMS)
    (w1, b1, _, n1), (w2, b2, _, n2), (w3, b3, _, n3), (w4, b4, _, n4) = O.OFFSETS
    th[w1 + 5 * n1 + 7] = 1.3        # unit 5 of layer 1 reads input 7
    th[b1 + 5] = -0.2
    th[w2 + 9 * n2 + 5] = -0.7       # unit 9 of layer 2 reads unit 5
    th[w3 + 2 * n3 + 9] = 2.0        # unit 2 of layer 3 reads unit 9
    th[b3 + 2] = 0.1
    th[w4 + 6 * n4 + 2] = 1.5        # output 6 reads unit 2
    th[b4 + 6] = 0.25
    o = O.N_TRAIN
    th[o:o + 32] = 1.0               # x_mean
    th[o + 32:o + 64] = 2.0          # x_std
    th[o + 64:o + 72] = 3.0          # y_mean
    th[o + 72:o + 80] = 5.0          # y_std
    D = np.random.default_rng(0).uniform(0, 4, (3, 32))
    c = O.predict(th, D)

    def s(z):
        return z / (1.0 + math.exp(-z))
    for i in range(3):
        x = (D[i, 7] - 1.0) / 2.0
        y6 = 1.5 * s(2.0 * s(-0.7 * s(1.3 * x - 0.2)) + 0.1) + 0.25
        exp = np.full(8, 3.0)
        exp[6] += 5.0 * y6
        assert np.allclose(c[i], exp, rtol=1e-14, atol=1e-14)


def test_gradient_central_differences():
    th = W.mlp_init(11)
    rng = np.random.default_rng(12)
    D = rng.uniform(0, 3, (6, 32))
    T = rng.standard_normal((6, 8))
    th = O.set_normalisation(th, D, T)
    loss, g = O.loss_and_grad(th, D, T)
    idx = np.concatenate([rng.choice(O.N_TRAIN, 300, replace=False),
                          np.arange(O.OFFSETS[3][1], O.OFFSETS[3][1] + 8)])
    hh = 1e-6
    for k in idx:
        tp, tm = th.copy(), th.copy()
        tp[k] += hh
        tm[k] -= hh
        fd = (O.loss_and_grad(tp, D, T)[0] - O.loss_and_grad(tm, D, T)[0]) / (2 * hh)
        assert abs(fd - g[k]) < 1e-7 * max(1.0, abs(g[k])), (k, fd, g[k])
    assert loss > 0


def test_adam_constant_gradient_exact_steps():
    th = W.mlp_init(1)
    g = np.random.default_rng(2).standard_normal(O.N_TRAIN)
    m = np.zeros(O.N_TRAIN)
    v = np.zeros(O.N_TRAIN)
    cur = th.copy()
    lr, eps = 3e-3, 1e-8
    for t in range(1, 6):
        cur, m, v = O.adam_step(cur, m, v, g, t, lr=lr, eps=eps)
        step = lr * g / (np.abs(g) + eps)
        assert np.allclose(cur[:O.N_TRAIN], th[:O.N_TRAIN] - t * step, rtol=0, atol=1e-14)
    assert np.array_equal(cur[O.N_TRAIN:], th[O.N_TRAIN:])


def test_training_reduces_loss_on_teacher_targets():
    rng = np.random.default_rng(3)
    D = rng.uniform(0, 3, (64, 32))
    teacher = W.mlp_init(99)
    T = O.predict(teacher, D)
    th = O.set_normalisation(W.mlp_init(5), D, T)
    th, m, v, hist = O.train(th, D, T, 200, lr=2e-3)
    assert hist[-1] < 0.05 * hist[0]


def _one_d_overlap(ka, kb, R):
    # composite Gauss-Legendre: 400 panels of 8 points on [-20, 20]
    xg, wg = np.polynomial.legendre.leggauss(8)
    a = np.linspace(-20.0, 20.0, 401)
    x = 0.5 * (a[:-1] + a[1:])[:, None] + 0.05 * xg[None, :]
    w = np.broadcast_to(0.05 * wg[None, :], x.shape).ravel()
    x = x.ravel()
    fa = math.sqrt(ka / math.pi) * np.exp(-ka * x * x)
    fb = math.sqrt(kb / math.pi) * np.exp(-kb * (x - R) ** 2)
    return float(np.sum(w * fa * fb))


def test_basis_overlap_closed_form_vs_1d_quadrature():
    for R in (0.0, 1.3, 4.2):
        S = O.basis_overlap(R)
        for a in range(8):
            for b in range(8):
                ka, kb = O.KAPPA[a], O.KAPPA[b]
                q = _one_d_overlap(ka, kb, R) * _one_d_overlap(ka, kb, 0.0) ** 2
                assert abs(S[a, b] - q) < 1e-13 * max(1.0, abs(q))
    for k in O.KAPPA:           # each g_k has unit charge
        assert abs((_one_d_overlap(k, 1e-30, 0.0) / math.sqrt(1e-30 / math.pi)) ** 3 - 1) < 1e-13
    Li = O.basis_transform()
    assert np.allclose(Li @ O.basis_overlap(0.0) @ Li.T, np.eye(8), atol=1e-9)


def test_phi_orthonormal_on_fe_mesh():
    m = Mesh(0.5, (24, 24, 24), 2, nq=6)
    pts = m.all_quad_points()
    wq = np.tile(m.quad_weights(), m.ncells)
    P = O.phi_at(pts, np.array([6.0, 6.0, 6.0]))
    G = P.T @ (wq[:, None] * P)
    # S is ill-conditioned (cond ~2e7, |L^-1| up to ~1e3), so the quadrature error
    # of the narrow Gaussians is amplified in the last combinations; a wrong
    # transform (L^-T for L^-1, a transposed S) is off by O(1)
    assert np.max(np.abs(G - np.eye(8))) < 1e-3
    assert np.max(np.abs(G[:5, :5] - np.eye(5))) < 1e-6


def test_fit_recovers_synthesised_coefficients():
    m = Mesh(2.0, (7, 7, 7), 4)
    atoms = np.array([[5.0, 7.0, 7.0], [9.2, 7.0, 7.0], [7.1, 10.3, 6.4]])
    c = np.random.default_rng(8).standard_normal((3, 8))
    dr = O.density_correction(m, atoms, c)
    cf = O.fit_correction(m, atoms, dr, ridge=0.0)
    assert np.max(np.abs(cf - c)) < 1e-8 * np.max(np.abs(c))
    # the ridge shrinks the coefficients towards zero
    cr = O.fit_correction(m, atoms, dr, ridge=0.1)
    assert np.linalg.norm(cr) < np.linalg.norm(cf)


def test_warm_start_charge_and_fallback():
    w = W.ws_cluster(4, 1000)
    m = Mesh(w["h"], w["ncell"], w["p"])
    sup = initial_density(m, w["atoms"], w["Z"])
    rho, fb = O.warm_start_density(m, w["atoms"], w["Z"], None, rho_sup=sup)
    assert fb and rho is sup
    th = W.mlp_init(2)
    (_, _, _, _), (_, _, _, _), (_, _, _, _), (w4, b4, mo, ni) = O.OFFSETS
    th0 = th.copy()
    th0[w4:w4 + mo * ni + mo] = 0.0           # output layer zero and y_mean = 0: no correction
    rho0, fb0 = O.warm_start_density(m, w["atoms"], w["Z"], th0, rho_sup=sup)
    assert not fb0 and np.allclose(rho0, sup, rtol=1e-14, atol=1e-300)
    th1 = th.copy()
    th1[O.N_TRAIN + 64:O.N_TRAIN + 72] = 0.05   # y_mean: a real correction
    rho1, fb1 = O.warm_start_density(m, w["atoms"], w["Z"], th1, rho_sup=sup)
    assert not fb1 and np.all(rho1 >= 0)
    assert abs(m.integrate(rho1) - 16.0) < 1e-10
    assert np.max(np.abs(rho1 - sup)) > 1e-3
