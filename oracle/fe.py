"""Oracle: spectral hexahedral finite elements (FP64, NumPy).

TEST INFRASTRUCTURE ONLY.  This package is the slow, plain CPU statement of the
method that the CUDA path is checked against.  Only the tests, the smoke check
and the CPU-baseline leg of the benchmark may import it; the product path never
does.

What it follows (paper, Sec. III.A "Evaluation of Overlap Matrix Inverse"):
spectral finite elements -- a Lagrange basis on Gauss-Lobatto-Legendre (GLL)
nodes -- combined with GLL quadrature, which makes the classical-classical
overlap block M^cc diagonal.  Every other integral uses a Gauss-Legendre rule
with ``nq`` points per axis per cell (the paper does not say which rule it
uses for those; ``nq = p + 2`` is our reading, which integrates the kinetic
term exactly).

Index conventions (shared by definition with the CUDA path, not by code):
  global node   n = (iz * Gy + iy) * Gx + ix,   G* = ncell* * p + 1
  cell          c = (cz * ny + cy) * nx + cx
  local node    l = (az * (p+1) + ay) * (p+1) + ax
  quad point    q = (qz * nq + qy) * nq + qx
Homogeneous Dirichlet conditions: boundary nodes are not degrees of freedom.
"""
import numpy as np
from numpy.polynomial import legendre as _leg


def gll_rule(p):
    """GLL nodes/weights on [-1, 1] for degree p (p+1 points).

    Nodes: the end points and the roots of P_p'(x).  Weights:
    w_i = 2 / (p (p+1) P_p(x_i)^2).  Exact for polynomials of degree <= 2p-1.
    """
    if p < 1:
        raise ValueError("degree must be >= 1")
    Pp = _leg.Legendre.basis(p)
    inner = np.sort(np.real(Pp.deriv().roots())) if p > 1 else np.array([])
    x = np.concatenate([[-1.0], inner, [1.0]])
    w = 2.0 / (p * (p + 1) * Pp(x) ** 2)
    return x, w


def gauss_rule(n):
    """Gauss-Legendre rule with n points on [-1, 1]; exact to degree 2n-1."""
    x, w = _leg.leggauss(n)
    return x, w


def lagrange_eval(nodes, xi):
    """Values l_a(xi_q) of the Lagrange polynomials on ``nodes``: shape (len(xi), len(nodes))."""
    nodes = np.asarray(nodes, float)
    xi = np.atleast_1d(np.asarray(xi, float))
    k = len(nodes)
    out = np.ones((len(xi), k))
    for a in range(k):
        for b in range(k):
            if b != a:
                out[:, a] *= (xi - nodes[b]) / (nodes[a] - nodes[b])
    return out


def lagrange_deriv(nodes, xi):
    """Derivatives l_a'(xi_q): product rule over the factors, shape (len(xi), len(nodes))."""
    nodes = np.asarray(nodes, float)
    xi = np.atleast_1d(np.asarray(xi, float))
    k = len(nodes)
    out = np.zeros((len(xi), k))
    for a in range(k):
        for c in range(k):
            if c == a:
                continue
            term = np.full(len(xi), 1.0 / (nodes[a] - nodes[c]))
            for b in range(k):
                if b != a and b != c:
                    term = term * (xi - nodes[b]) / (nodes[a] - nodes[b])
            out[:, a] += term
    return out


class Mesh:
    """Uniform mesh of cubic cells of side h over [0, nx h] x [0, ny h] x [0, nz h]."""

    def __init__(self, h, ncell, p, nq=None):
        self.h = float(h)
        self.nx, self.ny, self.nz = (int(v) for v in ncell)
        self.p = int(p)
        self.nq = int(nq) if nq else self.p + 2
        self.ne = (self.p + 1) ** 3
        self.Gx, self.Gy, self.Gz = (self.nx * self.p + 1, self.ny * self.p + 1,
                                     self.nz * self.p + 1)
        self.nnodes = self.Gx * self.Gy * self.Gz
        self.ncells = self.nx * self.ny * self.nz
        self.xg, self.wg = gll_rule(self.p)
        self.xq, self.wq = gauss_rule(self.nq)
        # 1D tables at Gauss points
        self.B1 = lagrange_eval(self.xg, self.xq)     # (nq, p+1)
        self.D1 = lagrange_deriv(self.xg, self.xq)    # d/dxi
        self.J = (self.h / 2.0) ** 3                  # volume Jacobian
        self._cell_nodes = None

    # --- geometry -----------------------------------------------------
    def cell_coords(self, c):
        cx = c % self.nx
        cy = (c // self.nx) % self.ny
        cz = c // (self.nx * self.ny)
        return cx, cy, cz

    def node_xyz(self):
        """Coordinates of all global nodes, shape (nnodes, 3)."""
        def axis(ncell):
            pts = np.empty(ncell * self.p + 1)
            for cidx in range(ncell):
                pts[cidx * self.p: cidx * self.p + self.p + 1] = (
                    cidx * self.h + self.h * (self.xg + 1.0) / 2.0)
            return pts
        x, y, z = axis(self.nx), axis(self.ny), axis(self.nz)
        Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
        return np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)

    def interior_mask(self):
        ix = np.arange(self.Gx)
        iy = np.arange(self.Gy)
        iz = np.arange(self.Gz)
        mx = (ix > 0) & (ix < self.Gx - 1)
        my = (iy > 0) & (iy < self.Gy - 1)
        mz = (iz > 0) & (iz < self.Gz - 1)
        return (mz[:, None, None] & my[None, :, None] & mx[None, None, :]).ravel()

    def cell_nodes(self):
        """Global node index of every (cell, local node): shape (ncells, (p+1)^3)."""
        if self._cell_nodes is None:
            p = self.p
            a = np.arange(p + 1)
            AZ, AY, AX = np.meshgrid(a, a, a, indexing="ij")
            AZ, AY, AX = AZ.ravel(), AY.ravel(), AX.ravel()
            out = np.empty((self.ncells, self.ne), dtype=np.int64)
            for c in range(self.ncells):
                cx, cy, cz = self.cell_coords(c)
                out[c] = ((cz * p + AZ) * self.Gy + (cy * p + AY)) * self.Gx + (cx * p + AX)
            self._cell_nodes = out
        return self._cell_nodes

    def quad_points(self, c):
        """Physical Gauss points of cell c, shape (nq^3, 3), in q order."""
        cx, cy, cz = self.cell_coords(c)
        t = self.h * (self.xq + 1.0) / 2.0
        QZ, QY, QX = np.meshgrid(cz * self.h + t, cy * self.h + t, cx * self.h + t,
                                 indexing="ij")
        return np.stack([QX.ravel(), QY.ravel(), QZ.ravel()], axis=1)

    def quad_weights(self):
        """Physical weights w_qx w_qy w_qz J for one cell, shape (nq^3,)."""
        w = self.wq
        return (w[:, None, None] * w[None, :, None] * w[None, None, :]).ravel() * self.J

    def all_quad_points(self):
        return np.concatenate([self.quad_points(c) for c in range(self.ncells)], axis=0)

    # --- reference-cell matrices -------------------------------------
    def basis_at_quad(self):
        """3D basis values N_l(x_q) for the reference cell: (nq^3, (p+1)^3)."""
        B = self.B1
        return np.einsum("ia,jb,kc->kjicba", B, B, B).reshape(self.nq ** 3, self.ne)

    def grad_at_quad(self):
        """Physical gradients dN_l/dx_d at quad points: (3, nq^3, (p+1)^3)."""
        B, D = self.B1, self.D1
        s = 2.0 / self.h
        gx = np.einsum("ia,jb,kc->kjicba", D, B, B).reshape(self.nq ** 3, self.ne) * s
        gy = np.einsum("ia,jb,kc->kjicba", B, D, B).reshape(self.nq ** 3, self.ne) * s
        gz = np.einsum("ia,jb,kc->kjicba", B, B, D).reshape(self.nq ** 3, self.ne) * s
        return np.stack([gx, gy, gz])

    def stiffness_cell(self):
        """K_e[i,j] = int_cell grad N_i . grad N_j, by the Gauss rule (exact)."""
        G = self.grad_at_quad()
        w = self.quad_weights()
        return sum(G[d].T @ (w[:, None] * G[d]) for d in range(3))

    def potential_cell(self, vq):
        """V_e[i,j] = int_cell v N_i N_j by the Gauss rule; vq: values at the nq^3 points."""
        B = self.basis_at_quad()
        w = self.quad_weights()
        return B.T @ ((w * vq)[:, None] * B)

    def lumped_mass(self):
        """Diagonal M^cc from GLL quadrature (Sec. III.A), over all global nodes."""
        wg = self.wg
        we = (wg[:, None, None] * wg[None, :, None] * wg[None, None, :]).ravel() * self.J
        m = np.zeros(self.nnodes)
        cn = self.cell_nodes()
        for c in range(self.ncells):
            np.add.at(m, cn[c], we)
        return m

    # --- operators on nodal arrays -----------------------------------
    def apply_cells(self, mats, X, chunk=4096):
        """Assembly by definition: Y = sum_e P_e^T A_e P_e X.

        ``mats`` is either one (ne, ne) matrix shared by every cell or a
        (ncells, ne, ne) array; X is (nnodes, N).  Boundary rows are not
        masked here.  Cells are processed in batches (same sums).
        """
        cn = self.cell_nodes()
        Y = np.zeros_like(X)
        shared = mats.ndim == 2
        for c0 in range(0, self.ncells, chunk):
            c1 = min(self.ncells, c0 + chunk)
            Xe = X[cn[c0:c1]]                                   # (nc, ne, N)
            if shared:
                Ye = np.einsum("ij,cjn->cin", mats, Xe)
            else:
                Ye = np.matmul(mats[c0:c1], Xe)
            np.add.at(Y, cn[c0:c1].ravel(), Ye.reshape(-1, X.shape[1]))
        return Y

    def interpolate(self, U):
        """Values at every Gauss point of the nodal field(s) U: (ncells*nq^3, ...)."""
        B = self.basis_at_quad()
        cn = self.cell_nodes()
        U2 = U.reshape(U.shape[0], -1)
        out = np.einsum("ql,cln->cqn", B, U2[cn]).reshape(-1, U2.shape[1])
        return out.reshape((-1,) + U.shape[1:])

    def integrate_against_basis(self, fq):
        """f_j = sum_cells sum_q w_q J N_j(x_q) f(x_q); fq: (ncells*nq^3,)."""
        B = self.basis_at_quad()
        w = self.quad_weights()
        cn = self.cell_nodes()
        fc = fq.reshape(self.ncells, -1) * w[None, :]
        out = np.zeros(self.nnodes)
        np.add.at(out, cn.ravel(), (fc @ B).ravel())
        return out

    def integrate(self, fq):
        """Integral of a field given at every Gauss point."""
        w = self.quad_weights()
        return float(np.sum(fq.reshape(self.ncells, -1) * w[None, :]))
