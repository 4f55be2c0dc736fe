"""Oracle: the orthogonalized enriched finite element (EFE) operators (FP64).

TEST INFRASTRUCTURE ONLY (see oracle/fe.py).

Follows the paper:
  * Sec. II.B, Eq. (cutoff properties): the smooth cutoff h(r, r0, t) equal to
    1 below r0 and 0 beyond r0 + r0/t.  The paper defers the exact form to its
    earlier work; our reading is the C-infinity step
        s = (r - r0) t / r0,  psi(x) = exp(-1/x) (x > 0),
        h = psi(1-s) / (psi(1-s) + psi(s)).
  * Sec. II.B: enrichment N^E_{k,I} = g_l(r) h(r) Y_lm - sum_j c_j N^C_j with
    real Y_lm, here l = 0, 1 (s, px, py, pz) and g_l(r) = r^l exp(-alpha r^2).
  * Orthogonalization (Sec. II.B; coefficients deferred by the paper): with
    B_jk = int a_k N_j and the GLL-lumped M^cc, c_k = (M^cc)^-1 B_:k, i.e. the
    basis transform T = [[I, -C^T], [0, I]], C = B^T (M^cc)^-1.  Then
    M^E = T^T M_raw T has a zero off-diagonal block (Eq. Discrete_Eig_Gen_M)
    and H^E = T^T H_raw T (Eq. Discrete_Eig_Gen_H).
  * Sec. III.A, Eq. (MEInvApprox): the approximate inverse with diagonal
    (M^cc)^-1 and the atom-block-diagonal (M~^ee)^-1.
  * Sec. II.A, Eq. (KS): H = -1/2 Laplacian + v_eff + nonlocal, the nonlocal
    part separable, sum_I sum_lm |beta_Ilm> h_Il <beta_Ilm|; our reading of
    the projectors: beta_s = A_s exp(-r^2/(2 rc^2)), beta_pm = A_p x_m
    exp(-r^2/(2 rc^2)), unit L2 norm, truncated at r_trunc.
"""
import math

import numpy as np
import scipy.sparse as sp

Y00 = 1.0 / math.sqrt(4.0 * math.pi)
Y1C = math.sqrt(3.0 / (4.0 * math.pi))   # r * Y_1m = Y1C * x_m


def cutoff(r, r0, t):
    """h(r, r0, t) and dh/dr (Sec. II.B, Eq. cutoff properties; our reading of its form)."""
    r = np.asarray(r, float)
    s = (r - r0) * t / r0
    h = np.ones_like(r)
    dh = np.zeros_like(r)
    h[s >= 1.0] = 0.0
    mid = (s > 0.0) & (s < 1.0)
    sm = s[mid]
    u = np.exp(-1.0 / (1.0 - sm))          # psi(1-s)
    w = np.exp(-1.0 / sm)                  # psi(s)
    du = -u / (1.0 - sm) ** 2              # d/ds psi(1-s)
    dw = w / sm ** 2                       # d/ds psi(s)
    h[mid] = u / (u + w)
    dh[mid] = (du * w - u * dw) / (u + w) ** 2 * (t / r0)
    return h, dh


def enrichment_values(pts, center, alpha, r0=None, t=0.33, radial="gauss"):
    """Atomic parts a_f (f = s, px, py, pz) and their gradients at points.

    Returns (vals (4, n), grads (4, 3, n)).  ``r0=None`` switches the cutoff
    off (h = 1), used only by closed-form checks.  The radial part g(r) is
    exp(-alpha r^2) (``radial="gauss"``, the workloads' functions) or the
    hydrogen-like exp(-alpha r) (``radial="slater"``, alpha = Z: the exact
    1s orbital of -Z/r, used by the closed-form check of Sec. II.B's claim
    that atomic orbitals in the span give the atomic eigenvalues).
    """
    d = pts - center[None, :]
    r = np.sqrt(np.sum(d * d, axis=1))
    if radial == "gauss":
        g = np.exp(-alpha * r * r)
        gpr = -2.0 * alpha * g                      # g'(r)/r
    elif radial == "slater":
        g = np.exp(-alpha * r)
        with np.errstate(divide="ignore", invalid="ignore"):
            gpr = np.where(r > 0, -alpha * g / np.where(r > 0, r, 1.0), 0.0)
    else:
        raise ValueError("radial must be 'gauss' or 'slater'")
    if r0 is None:
        h = np.ones_like(r)
        dh = np.zeros_like(r)
    else:
        h, dh = cutoff(r, r0, t)
    f = g * h
    # f'(r)/r = g'(r)/r h + g h'(r)/r, h'/r finite at r = 0 because h' vanishes below r0
    with np.errstate(divide="ignore", invalid="ignore"):
        dh_over_r = np.where(r > 0, dh / np.where(r > 0, r, 1.0), 0.0)
    fpr = gpr * h + g * dh_over_r
    vals = np.empty((4, len(r)))
    grads = np.empty((4, 3, len(r)))
    vals[0] = Y00 * f
    grads[0] = Y00 * fpr[None, :] * d.T
    for m in range(3):
        vals[1 + m] = Y1C * d[:, m] * f
        grads[1 + m] = Y1C * d[:, m][None, :] * fpr[None, :] * d.T
        grads[1 + m, m] += Y1C * f
    return vals, grads


def projector_values(pts, center, rc, rtrunc):
    """beta_s, beta_px, beta_py, beta_pz at points (unit L2 norm before truncation)."""
    d = pts - center[None, :]
    r2 = np.sum(d * d, axis=1)
    g = np.exp(-r2 / (2.0 * rc * rc))
    g[r2 > rtrunc * rtrunc] = 0.0
    As = (math.pi * rc * rc) ** -0.75
    Ap = As * math.sqrt(2.0) / rc
    out = np.empty((4, len(r2)))
    out[0] = As * g
    for m in range(3):
        out[1 + m] = Ap * d[:, m] * g
    return out


class EFESystem:
    """The discrete EFE eigenproblem H^E psi = eps M^E psi on a uniform mesh.

    Unknown vectors hold (nnodes + n_enr) rows: all global FE nodes (boundary
    rows are kept and must stay zero) followed by 4 enrichment rows per atom.
    """

    def __init__(self, mesh, atoms, enrich=None, proj=None):
        self.mesh = mesh
        self.atoms = np.asarray(atoms, float).reshape(-1, 3)
        self.na = len(self.atoms)
        self.enrich = enrich
        self.proj = proj
        self.n_enr = 4 * self.na if enrich is not None else 0
        self.n_proj = 4 * self.na if proj is not None else 0
        nn = mesh.nnodes
        self.nn = nn
        self.mask = mesh.interior_mask()
        m = mesh.lumped_mass()
        self.mcc = np.where(self.mask, m, 0.0)
        self.minv = np.where(self.mask, 1.0 / m, 0.0)
        self.Bq = mesh.basis_at_quad()
        self.Gq = mesh.grad_at_quad()
        self.wq = mesh.quad_weights()
        self.Ke = mesh.stiffness_cell()
        if self.proj is not None:
            self.D = np.repeat(np.asarray(proj["h"], float).reshape(self.na, 2), [1, 3], axis=1).ravel()
        self._static_integrals()
        self.He = None

    # --- static (potential-independent) integrals --------------------
    def _cells_near(self, center, radius):
        """Cells whose box meets the ball (a superset of where the functions are non-zero)."""
        m = self.mesh
        c = np.arange(m.ncells)
        lo = np.stack([c % m.nx, (c // m.nx) % m.ny, c // (m.nx * m.ny)], axis=1) * m.h
        q = np.clip(center[None, :], lo, lo + m.h)
        d2 = np.sum((q - center[None, :]) ** 2, axis=1)
        return list(np.nonzero(d2 <= radius * radius)[0])

    def _support_radius(self):
        r = 0.0
        if self.enrich is not None:
            e = self.enrich
            if e.get("r0") is None:
                r = np.inf
            else:
                r = e["r0"] * (1.0 + 1.0 / e["t"])
        if self.proj is not None:
            r = max(r, self.proj["rtrunc"])
        return r

    def _atom_cells(self):
        R = self._support_radius()
        if not np.isfinite(R):
            return [list(range(self.mesh.ncells))] * self.na
        return [self._cells_near(self.atoms[I], R) for I in range(self.na)]

    def _funcs_at(self, c):
        """Enrichment values/grads and projector values of every atom touching cell c."""
        m = self.mesh
        pts = m.quad_points(c)
        atoms = self.cell_atoms[c]
        A = np.zeros((4 * len(atoms), len(pts)))
        dA = np.zeros((4 * len(atoms), 3, len(pts)))
        P = np.zeros((4 * len(atoms), len(pts)))
        for i, I in enumerate(atoms):
            if self.enrich is not None:
                e = self.enrich
                v, g = enrichment_values(pts, self.atoms[I], e["alpha"], e.get("r0"), e.get("t", 0.33),
                                         e.get("radial", "gauss"))
                A[4 * i:4 * i + 4] = v
                dA[4 * i:4 * i + 4] = g
            if self.proj is not None:
                P[4 * i:4 * i + 4] = projector_values(pts, self.atoms[I], self.proj["rc"], self.proj["rtrunc"])
        return atoms, pts, A, dA, P

    def _static_integrals(self):
        m = self.mesh
        nn, ne = self.nn, self.n_enr
        atom_cells = self._atom_cells()
        self.cell_atoms = [[] for _ in range(m.ncells)]
        for I, cells in enumerate(atom_cells):
            for c in cells:
                self.cell_atoms[c].append(I)
        cn = m.cell_nodes()
        w = self.wq
        rowsB, colsB, valB, valK = [], [], [], []
        rowsP, colsP, valP = [], [], []
        self.Aee = np.zeros((ne, ne))
        self.Kaa = np.zeros((ne, ne))
        self.Pa = np.zeros((self.n_proj, ne))
        self._cache = {}
        for c in range(m.ncells):
            if not self.cell_atoms[c]:
                continue
            atoms, pts, A, dA, P = self._funcs_at(c)
            self._cache[c] = (atoms, A, P)
            kidx = np.concatenate([np.arange(4 * I, 4 * I + 4) for I in atoms])
            nodes = cn[c]
            if ne:
                Bc = self.Bq.T @ (w[None, :] * A).T                       # (ne_cell, k)
                Kc = 0.5 * sum(self.Gq[d].T @ (w[None, :] * dA[:, d, :]).T for d in range(3))
                rowsB.append(np.repeat(nodes, len(kidx)))
                colsB.append(np.tile(kidx, len(nodes)))
                valB.append(Bc.ravel())
                valK.append(Kc.ravel())
                self.Aee[np.ix_(kidx, kidx)] += (A * w[None, :]) @ A.T
                self.Kaa[np.ix_(kidx, kidx)] += 0.5 * sum((dA[:, d, :] * w[None, :]) @ dA[:, d, :].T
                                                          for d in range(3))
            if self.n_proj:
                Pc = (P * w[None, :]) @ self.Bq                            # (k, ne_cell)
                rowsP.append(np.repeat(kidx, len(nodes)))
                colsP.append(np.tile(nodes, len(kidx)))
                valP.append(Pc.ravel())
                if ne:
                    self.Pa[np.ix_(kidx, kidx)] += (P * w[None, :]) @ A.T
        keep = self.mask.astype(float)
        if ne:
            r, cc = np.concatenate(rowsB), np.concatenate(colsB)
            self.B = sp.csr_matrix((np.concatenate(valB), (r, cc)), shape=(nn, ne))
            self.Kca = sp.csr_matrix((np.concatenate(valK), (r, cc)), shape=(nn, ne))
            self.B = sp.diags(keep) @ self.B
            self.Kca = sp.diags(keep) @ self.Kca
            # Orthogonalization: C = B^T (M^cc)^-1 so that M^ec = 0
            self.C = (self.B.T @ sp.diags(self.minv)).tocsr()              # (ne, nn)
            self.Mee = self.Aee - (self.B.T @ (sp.diags(self.minv) @ self.B)).toarray()
            self.Mee = 0.5 * (self.Mee + self.Mee.T)
            self.Mee_blk_inv = np.zeros((self.na, 4, 4))
            for I in range(self.na):
                blk = self.Mee[4 * I:4 * I + 4, 4 * I:4 * I + 4]
                self.Mee_blk_inv[I] = np.linalg.inv(blk)
        if self.n_proj:
            self.Pc = sp.csr_matrix((np.concatenate(valP),
                                     (np.concatenate(rowsP), np.concatenate(colsP))),
                                    shape=(self.n_proj, nn))
            self.Pc = self.Pc @ sp.diags(keep)

    # --- potential-dependent assembly (per SCF step) ---------------------
    def set_potential(self, vq):
        """Cell matrices H_e = 1/2 K_e + V_e and the potential parts of the coupling."""
        m = self.mesh
        nq3 = m.nq ** 3
        vq = np.asarray(vq, float).reshape(m.ncells, nq3)
        self.vq = vq
        He = np.empty((m.ncells, m.ne, m.ne))
        for c in range(m.ncells):
            He[c] = 0.5 * self.Ke + m.potential_cell(vq[c])
        self.He = He
        if self.n_enr:
            ne = self.n_enr
            w = self.wq
            cn = m.cell_nodes()
            rows, cols, vals = [], [], []
            Vaa = np.zeros((ne, ne))
            for c, (atoms, A, P) in self._cache.items():
                kidx = np.concatenate([np.arange(4 * I, 4 * I + 4) for I in atoms])
                wv = w * vq[c]
                Vc = self.Bq.T @ (wv[None, :] * A).T
                rows.append(np.repeat(cn[c], len(kidx)))
                cols.append(np.tile(kidx, m.ne))
                vals.append(Vc.ravel())
                Vaa[np.ix_(kidx, kidx)] += (A * wv[None, :]) @ A.T
            Vca = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                                shape=(self.nn, ne))
            Vca = sp.diags(self.mask.astype(float)) @ Vca
            self.Hca = (self.Kca + Vca).tocsr()
            self.Haa = self.Kaa + Vaa
            self.Haa = 0.5 * (self.Haa + self.Haa.T)

    # --- operators -------------------------------------------------------
    def split(self, X):
        return X[:self.nn], X[self.nn:]

    def apply_H(self, X):
        """H^E X = T^T (H_raw (T X)) (Eqs. Discrete_Eig_Gen_H, KS)."""
        X = np.asarray(X, float)
        Xc, Xe = self.split(X)
        Xc = Xc * self.mask[:, None]
        if self.n_enr:
            Xcp = Xc - self.C.T @ Xe
        else:
            Xcp = Xc
        Yc = self.mesh.apply_cells(self.He, Xcp)
        Ye = np.zeros((self.n_enr, X.shape[1]))
        if self.n_enr:
            Yc = Yc + self.Hca @ Xe
            Ye = self.Hca.T @ Xcp + self.Haa @ Xe
        if self.n_proj:
            Wp = self.Pc @ Xcp
            if self.n_enr:
                Wp = Wp + self.Pa @ Xe
            Wp = self.D[:, None] * Wp
            Yc = Yc + self.Pc.T @ Wp
            if self.n_enr:
                Ye = Ye + self.Pa.T @ Wp
        Yc = Yc * self.mask[:, None]
        if self.n_enr:
            Ye = Ye - self.C @ Yc
        return np.concatenate([Yc, Ye], axis=0)

    def apply_M(self, X):
        """Exact M^E X: diagonal M^cc and the full M^ee (Eq. Discrete_Eig_Gen_M)."""
        Xc, Xe = self.split(X)
        Yc = self.mcc[:, None] * Xc
        Ye = self.Mee @ Xe if self.n_enr else Xe
        return np.concatenate([Yc, Ye], axis=0)

    def apply_Minv_approx(self, X):
        """(M~^E)^-1 X (Eq. MEInvApprox)."""
        Xc, Xe = self.split(X)
        Yc = self.minv[:, None] * Xc
        Ye = np.empty_like(Xe)
        for I in range(self.na if self.n_enr else 0):
            Ye[4 * I:4 * I + 4] = self.Mee_blk_inv[I] @ Xe[4 * I:4 * I + 4]
        return np.concatenate([Yc, Ye], axis=0)

    def apply_Mtilde(self, X):
        """M~^E X (the block-diagonal approximation itself)."""
        Xc, Xe = self.split(X)
        Yc = self.mcc[:, None] * Xc
        Ye = np.empty_like(Xe)
        for I in range(self.na if self.n_enr else 0):
            Ye[4 * I:4 * I + 4] = self.Mee[4 * I:4 * I + 4, 4 * I:4 * I + 4] @ Xe[4 * I:4 * I + 4]
        return np.concatenate([Yc, Ye], axis=0)

    def dof_rows(self):
        """Row indices of the true unknowns: interior FE nodes then enrichment rows."""
        return np.concatenate([np.nonzero(self.mask)[0], self.nn + np.arange(self.n_enr)])

    # --- values of the EFE functions at the quadrature points -----------
    def values_at_quad(self, X):
        """psi(x_q) for every column of X at every Gauss point (Sec. II.B expansion).

        psi = sum_j N_j (X_c - C^T X_e)_j + sum_k a_k X_e,k.
        """
        m = self.mesh
        Xc, Xe = self.split(np.asarray(X, float))
        Xc = Xc * self.mask[:, None]
        Xcp = Xc - self.C.T @ Xe if self.n_enr else Xc
        out = m.interpolate(Xcp)
        if self.n_enr:
            nq3 = m.nq ** 3
            for c, (atoms, A, P) in self._cache.items():
                kidx = np.concatenate([np.arange(4 * I, 4 * I + 4) for I in atoms])
                out[c * nq3:(c + 1) * nq3] += A.T @ Xe[kidx]
        return out


def assembled_fe_hamiltonian(sysm):
    """H^cc over all nodes as a sparse matrix, rows and columns of Dirichlet nodes zero:
    the sum over cells of the cell matrices H_e (Eq. Discrete_Eig_Gen_H, FE block)."""
    m = sysm.mesh
    cn = m.cell_nodes()
    ne = m.ne
    r = np.repeat(cn, ne, axis=1).ravel()
    c = np.tile(cn, (1, ne)).ravel()
    H = sp.csr_matrix((sysm.He.reshape(-1), (r, c)), shape=(sysm.nn, sysm.nn))
    mk = sp.diags(sysm.mask.astype(float))
    return (mk @ H @ mk).tocsr()


def orthogonal_blocks(sysm):
    """The blocks of H^E = T^T H_raw T that touch the enriched rows, written out
    (Sec. II.B orthogonalization, T = [[I, -C^T], [0, I]]):

      FE-enrichment block   E     = H^ac - C H^cc                 (n_enr x nn)
      enriched block        H^E_ee = H^aa - C H^ca - E C^T          (local part)
      projector overlaps    P^E   = P_a - P_c C^T                  (n_proj x n_enr)

    Returns (Hcc, E, HEee, PE); PE is None without projectors."""
    Hcc = assembled_fe_hamiltonian(sysm)
    C = sysm.C.toarray()
    Hca = sysm.Hca.toarray()
    E = Hca.T - C @ Hcc.toarray()
    HEee = sysm.Haa - C @ Hca - E @ C.T
    PE = sysm.Pa - sysm.Pc.toarray() @ C.T if sysm.n_proj else None
    return Hcc, E, HEee, PE


def apply_H_blocks(sysm, X, blocks=None):
    """H^E X from the blocks of H^E (no T transform): FE rows
    H^cc X_c + E^T X_e + P_c^T W, enriched rows E X_c + H^E_ee X_e + P^E^T W with
    W = D (P_c X_c + P^E X_e).  Equal to apply_H in exact arithmetic."""
    Hcc, E, HEee, PE = orthogonal_blocks(sysm) if blocks is None else blocks
    Xc, Xe = sysm.split(np.asarray(X, float))
    Xc = Xc * sysm.mask[:, None]
    Yc = Hcc @ Xc + E.T @ Xe
    Ye = E @ Xc + HEee @ Xe
    if sysm.n_proj:
        W = sysm.D[:, None] * (sysm.Pc @ Xc + PE @ Xe)
        Yc = Yc + sysm.Pc.T @ W
        Ye = Ye + PE.T @ W
    Yc = Yc * sysm.mask[:, None]
    return np.concatenate([Yc, Ye], axis=0)


def dense_raw_matrices(sysm):
    """H_raw and M_raw over (interior nodes + enrichment), assembled entry by entry.

    Independent of the T-transform: the raw basis {N_j} U {a_k}.  Used only for
    tiny meshes to check that (H^E, M^E) and (H_raw, M_raw) share eigenvalues.
    """
    m = sysm.mesh
    idx = np.nonzero(sysm.mask)[0]
    ni = len(idx)
    pos = -np.ones(m.nnodes, dtype=np.int64)
    pos[idx] = np.arange(ni)
    n = ni + sysm.n_enr
    H = np.zeros((n, n))
    M = np.zeros((n, n))
    cn = m.cell_nodes()
    for c in range(m.ncells):
        loc = pos[cn[c]]
        ok = loc >= 0
        H[np.ix_(loc[ok], loc[ok])] += sysm.He[c][np.ix_(ok, ok)]
    M[np.arange(ni), np.arange(ni)] = sysm.mcc[idx]
    if sysm.n_enr:
        e = slice(ni, n)
        Bi = sysm.B.toarray()[idx]
        Hci = sysm.Hca.toarray()[idx]
        M[:ni, e] = Bi
        M[e, :ni] = Bi.T
        M[e, e] = sysm.Aee
        H[:ni, e] = Hci
        H[e, :ni] = Hci.T
        H[e, e] = sysm.Haa
    if sysm.n_proj:
        P = sysm.Pc.toarray()[:, idx]
        if sysm.n_enr:
            P = np.concatenate([P, sysm.Pa], axis=1)
        H += P.T @ (sysm.D[:, None] * P)
    return H, M
