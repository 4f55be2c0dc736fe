"""Pins for the oracle's EFE operators (Sec. II.B, Eqs. Discrete_Eig_Gen_H/M,
MEInvApprox): the cutoff's defining properties, analytic gradients against
finite differences, the Galerkin harmonic oscillator with the exact s/p
eigenfunctions as enrichment (eigenvalues 1.5, 2.5 x3 on a coarse mesh), and
the orthogonalization identities H^E = T^T H_raw T, M^E = T^T M_raw T, M^ec = 0."""
import math

import numpy as np
import pytest
import scipy.linalg as sla

from oracle.efe import (EFESystem, apply_H_blocks, cutoff, dense_raw_matrices, enrichment_values,
                        orthogonal_blocks,
                        projector_values)
from oracle.fe import Mesh

R0 = 5.0 * 0.33 / 1.33


def test_cutoff_properties():
    r = np.linspace(0, 6, 6001)
    h, dh = cutoff(r, R0, 0.33)
    rend = R0 + R0 / 0.33
    assert abs(rend - 5.0) < 1e-12
    assert np.all(h[r < R0] == 1.0) and np.all(h[r >= rend] == 0.0)
    assert np.all((h >= 0) & (h <= 1))
    assert np.all(np.diff(h) <= 1e-15)                      # monotone
    mid = (r > R0 + 1e-3) & (r < rend - 1e-3)
    eps = 1e-6
    fd = (cutoff(r[mid] + eps, R0, 0.33)[0] - cutoff(r[mid] - eps, R0, 0.33)[0]) / (2 * eps)
    assert np.allclose(dh[mid], fd, atol=1e-7)
    # smooth joins: value and slope continuous at both ends
    assert cutoff(np.array([R0 + 1e-4]), R0, 0.33)[0][0] > 1 - 1e-12
    assert abs(cutoff(np.array([rend - 1e-4]), R0, 0.33)[0][0]) < 1e-12


def test_enrichment_gradients_fd():
    rng = np.random.default_rng(3)
    ctr = np.array([1.0, -0.5, 0.25])
    pts = ctr + rng.uniform(-4.5, 4.5, size=(400, 3))
    v, g = enrichment_values(pts, ctr, 1.2, R0, 0.33)
    eps = 1e-6
    for d in range(3):
        e = np.zeros(3)
        e[d] = eps
        fd = (enrichment_values(pts + e, ctr, 1.2, R0, 0.33)[0]
              - enrichment_values(pts - e, ctr, 1.2, R0, 0.33)[0]) / (2 * eps)
        assert np.allclose(g[:, d, :], fd, atol=1e-7)
    # s function: Y00 exp(-a r^2) inside r0
    inside = np.linalg.norm(pts - ctr, axis=1) < R0
    r2 = np.sum((pts[inside] - ctr) ** 2, axis=1)
    assert np.allclose(v[0, inside], np.exp(-1.2 * r2) / math.sqrt(4 * math.pi), rtol=1e-14)


def test_projectors_unit_norm():
    # fine tensor grid over [-7, 7]^3
    t = np.linspace(-7, 7, 141)
    dx = t[1] - t[0]
    X, Y, Z = np.meshgrid(t, t, t, indexing="ij")
    pts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    b = projector_values(pts, np.zeros(3), 1.0, 6.0)
    G = (b @ b.T) * dx ** 3
    assert np.allclose(np.diag(G), 1.0, atol=1e-6)
    assert np.allclose(G - np.diag(np.diag(G)), 0.0, atol=1e-9)


def _ho_system(n, p, nq, alpha=0.5):
    box = 12.0
    m = Mesh(box / n, (n, n, n), p, nq)
    ctr = np.full(3, box / 2)
    s = EFESystem(m, ctr[None, :], enrich=dict(alpha=alpha, r0=None))
    s.set_potential(0.5 * np.sum((m.all_quad_points() - ctr) ** 2, axis=1))
    return s


def _consistent_raw_mass(s):
    """Gram matrix of {N_j} U {a_k} with every integral by the Gauss rule."""
    m = s.mesh
    idx = np.nonzero(s.mask)[0]
    Mc = m.potential_cell(np.ones(m.nq ** 3))
    Mg = m.apply_cells(Mc, np.eye(m.nnodes)[:, idx])[idx]
    if not s.n_enr:
        return Mg
    B = s.B.toarray()[idx]
    return np.block([[Mg, B], [B.T, s.Aee]])


def test_galerkin_exact_enrichment_harmonic_oscillator():
    # With the exact 1s and 2p eigenfunctions in the span, the Galerkin
    # problem (consistent Gauss mass) is exact up to quadrature even on a
    # mesh that alone is far off.
    s = _ho_system(3, 2, 12)
    H, _ = dense_raw_matrices(s)
    M = _consistent_raw_mass(s)
    w = sla.eigh(H, M, eigvals_only=True, subset_by_index=[0, 4])
    assert np.allclose(w[:4], [1.5, 2.5, 2.5, 2.5], atol=1e-7), w
    # the same mesh without enrichment is far off
    s0 = EFESystem(s.mesh, s.atoms)
    s0.set_potential(s.vq.ravel())
    H0, M0 = dense_raw_matrices(s0)
    w0 = sla.eigh(H0, _consistent_raw_mass(s0), eigvals_only=True, subset_by_index=[0, 0])
    assert w0[0] - 1.5 > 1e-2


def _dimer_system(n=3, p=2):
    box = 12.0
    m = Mesh(box / n, (n, n, n), p)
    atoms = np.array([[5.0, 6.0, 6.0], [7.1, 6.2, 5.9]])
    hp = np.array([[1.3, -0.7], [-1.1, 0.4]])
    s = EFESystem(m, atoms, enrich=dict(alpha=1.2, r0=R0, t=0.33),
                  proj=dict(rc=1.0, rtrunc=6.0, h=hp))
    q = m.all_quad_points()
    v = -np.sum([2.0 / np.sqrt(1.0 + np.sum((q - a) ** 2, axis=1)) for a in atoms], axis=0)
    s.set_potential(v)
    return s


def _efe_dense(s):
    rows = s.dof_rows()
    E = np.zeros((s.nn + s.n_enr, len(rows)))
    E[rows, np.arange(len(rows))] = 1.0
    return s.apply_H(E)[rows], s.apply_M(E)[rows], s.apply_Minv_approx(E)[rows]


def test_orthogonalization_identities():
    s = _dimer_system()
    HE, ME, MtI = _efe_dense(s)
    Hr, Mr = dense_raw_matrices(s)
    ni = int(s.mask.sum())
    C = s.C.toarray()[:, np.nonzero(s.mask)[0]]
    T = np.eye(ni + s.n_enr)
    T[:ni, ni:] = -C.T
    assert np.allclose(HE, T.T @ Hr @ T, atol=1e-11)
    assert np.allclose(ME, T.T @ Mr @ T, atol=1e-13)
    assert np.abs(ME[:ni, ni:]).max() < 1e-14          # M^ec = 0
    assert np.allclose(HE, HE.T, atol=1e-12)
    w1 = sla.eigh(HE, ME, eigvals_only=True, subset_by_index=[0, 5])
    w2 = sla.eigh(Hr, Mr, eigvals_only=True, subset_by_index=[0, 5])
    assert np.allclose(w1, w2, atol=1e-9)
    # approximate inverse: exact on the FE block, atom blocks on the enriched block
    Mt = ME.copy()
    for I in range(s.na):
        for J in range(s.na):
            if I != J:
                Mt[ni + 4 * I:ni + 4 * I + 4, ni + 4 * J:ni + 4 * J + 4] = 0
    assert np.allclose(MtI @ Mt, np.eye(len(Mt)), atol=1e-10)
    assert np.abs(Mt - ME).max() > 1e-8            # the dimer's blocks do couple


def test_nonlocal_is_separable_rank():
    s = _dimer_system()
    HE, _, _ = _efe_dense(s)
    proj = s.proj
    s.proj = None
    s.n_proj_saved, s.n_proj = s.n_proj, 0
    HE0, _, _ = _efe_dense(s)
    s.proj, s.n_proj = proj, s.n_proj_saved
    d = HE - HE0
    sv = np.linalg.svd(d, compute_uv=False)
    assert sv[7] > 1e-6 * sv[0] and sv[8] < 1e-10 * sv[0]   # 2 atoms x 4 projectors


def _one_atom(h, n, p, centre, hp=(0.8, -1.3)):
    m = Mesh(h, (n, n, n), p)
    s = EFESystem(m, np.asarray([centre], float), enrich=dict(alpha=1.2, r0=R0, t=0.33),
                  proj=dict(rc=1.0, rtrunc=6.0, h=np.asarray([hp], float)))
    q = m.all_quad_points()
    s.set_potential(-2.0 / np.sqrt(1.0 + np.sum((q - s.atoms[0]) ** 2, axis=1)))
    return s


def test_block_form_equals_transform_form():
    # H^E through its blocks E = H^ac - C H^cc, H^E_ee = H^aa - C H^ca - E C^T and
    # P^E = P_a - P_c C^T (the mixed filter's form) against T^T H_raw T, on the
    # filter's operands M~^-1 Z: the overlapping dimer and a degree-6 atom whose
    # enrichment is nearly in the FE space (the transform form itself loses
    # ~3 digits there, hence the looser bound)
    for s, tol in ((_dimer_system(), 1e-13), (_one_atom(40.0 / 24.0, 6, 6, (5.0, 5.1, 4.9)), 1e-11)):
        X = np.random.default_rng(3).standard_normal((s.nn + s.n_enr, 4))
        X[:s.nn] *= s.mask[:, None]
        Y = s.apply_Minv_approx(X)
        a, b = s.apply_H(Y), apply_H_blocks(s, Y)
        assert np.abs(a - b).max() < tol * np.abs(a).max()
        # the blocks are those of the dense H^E
        Hcc, E, HEee, PE = orthogonal_blocks(s)
        if s.nn < 1000:
            HE, _, _ = _efe_dense(s)
            ni = int(s.mask.sum())
            idx = np.nonzero(s.mask)[0]
            HP = (PE.T * s.D[None, :]) @ PE
            assert np.allclose(HE[ni:, ni:], HEee + HP, atol=1e-11)
            assert np.allclose(HE[ni:, :ni], E[:, idx] + (PE.T * s.D[None, :]) @ s.Pc.toarray()[:, idx],
                               atol=1e-11)


def test_transform_form_cancels_at_degree_6():
    # why the mixed filter uses the blocks: at degree 6, h = 40/24 the enrichment
    # is nearly representable (M^ee ~ 1e-6 A_ee), the orthogonalized coordinates
    # of M~^-1 Z are large, and the two FE-row terms of T^T H_raw T,
    # H^cc (X_c - C^T X_e) and H^ca X_e, are each tens of times their sum
    ratios = {}
    for key, s in (("p2", _dimer_system()), ("p6", _one_atom(40.0 / 24.0, 6, 6, (5.0, 5.1, 4.9)))):
        X = np.random.default_rng(3).standard_normal((s.nn + s.n_enr, 4))
        X[:s.nn] *= s.mask[:, None]
        Xc, Xe = s.split(s.apply_Minv_approx(X))
        Xcp = (Xc * s.mask[:, None]) - s.C.T @ Xe
        A = s.mesh.apply_cells(s.He, Xcp) * s.mask[:, None]
        B = (s.Hca @ Xe) * s.mask[:, None]
        ratios[key] = np.abs(A).max() / np.abs(A + B).max()
        ratios[key + "_mee"] = np.linalg.eigvalsh(s.Mee).min() / np.linalg.eigvalsh(s.Aee).min()
    assert ratios["p6_mee"] < 1e-4 < ratios["p2_mee"]
    assert ratios["p6"] > 10.0 > 5.0 > ratios["p2"], ratios


def test_E_vanishes_outside_one_cell_dilation():
    # E = H^ac - C H^cc is nonzero only at nodes of cells that share a node with
    # a cell meeting the enrichment ball (r <= r_end): C lives on the nodes of
    # those cells and H^cc reaches one cell further; some nonzeros do lie outside
    # the cells that meet the ball, so the supports must include the layer
    h, n, p = 1.5, 12, 2
    s = _one_atom(h, n, p, (9.1, 8.9, 9.0))
    _, E, _, _ = orthogonal_blocks(s)
    m = s.mesh
    r_end = R0 * (1.0 + 1.0 / 0.33)
    cn = m.cell_nodes()
    X = s.atoms[0]
    meets = np.zeros((n, n, n), bool)
    for c in range(m.ncells):
        cx, cy, cz = m.cell_coords(c)
        lo = np.array([cx, cy, cz]) * h
        d = np.clip(X, lo, lo + h) - X
        meets[cz, cy, cx] = d @ d <= r_end ** 2
    dil = meets.copy()
    for ax in range(3):
        dil = dil | np.roll(dil, 1, axis=ax) | np.roll(dil, -1, axis=ax)   # the ball is far from the box faces
    inner = np.zeros(s.nn, bool)
    outer = np.zeros(s.nn, bool)
    for c in range(m.ncells):
        cx, cy, cz = m.cell_coords(c)
        if meets[cz, cy, cx]:
            inner[cn[c]] = True
        if dil[cz, cy, cx]:
            outer[cn[c]] = True
    nz = np.abs(E).max(axis=0) > 0.0
    assert not np.any(nz & ~outer)
    assert np.any(nz & ~inner)
