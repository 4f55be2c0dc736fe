"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Every case uses the same seeded inputs on both sides: the H^E, M^E and M~^-1
products element by element (FP64 to 1e-12 relative), Lanczos bounds, one
residual filter pass, Rayleigh-Ritz and the multipass solver (eigenvalues to
1e-8 Ha, the FP64 bound of the target), plus the FP32 filter against FP64.
Meshes include odd cell counts (colours of unequal size), column counts that
are not multiples of the column tile, and the degenerate cases without
enrichment or without the nonlocal part.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import chfsi as OC  # noqa: E402
from oracle.efe import EFESystem  # noqa: E402
from oracle.fe import Mesh  # noqa: E402
from paper_2607_06848_gb300 import workloads as W  # noqa: E402

T_ENR = 0.33
R_END = 5.0
R0 = R_END * T_ENR / (1 + T_ENR)


def _case(name):
    if name == "dimer":
        w = W.dimer()
        return dict(h=w["h"], ncell=w["ncell"], p=w["p"], atoms=w["atoms"], hproj=w["hproj"], enrich=True, nl=True)
    if name == "ragged":
        atoms = np.array([[5.6, 7.1, 8.2], [7.4, 8.0, 9.3]])
        return dict(h=2.5, ncell=(5, 6, 7), p=3, atoms=atoms, hproj=np.array([[1.1, -0.6], [-1.4, 0.9]]),
                    enrich=True, nl=True)
    if name == "cfe_only":
        return dict(h=2.0, ncell=(5, 4, 6), p=4, atoms=np.array([[5.0, 4.0, 6.0]]), hproj=np.zeros((1, 2)),
                    enrich=False, nl=False)
    if name == "nonlocal_only":
        return dict(h=2.0, ncell=(6, 6, 6), p=2, atoms=np.array([[6.0, 6.1, 5.9]]), hproj=np.array([[1.5, -1.0]]),
                    enrich=False, nl=True)
    if name == "p6_cfe":
        return dict(h=40.0 / 24.0, ncell=(3, 4, 3), p=6, atoms=np.array([[2.5, 3.3, 2.4]]), hproj=np.zeros((1, 2)),
                    enrich=False, nl=False)
    if name == "p6_enriched":
        return dict(h=40.0 / 24.0, ncell=(6, 7, 6), p=6, atoms=np.array([[5.0, 5.9, 5.0]]),
                    hproj=np.array([[0.8, -1.3]]), enrich=True, nl=True)
    if name == "p5_enriched":
        return dict(h=2.0, ncell=(5, 5, 6), p=5, atoms=np.array([[5.0, 5.0, 6.1]]),
                    hproj=np.array([[-0.4, 1.1]]), enrich=True, nl=True)
    if name == "p7_cfe":
        return dict(h=1.5, ncell=(2, 3, 2), p=7, atoms=np.array([[1.5, 2.2, 1.4]]), hproj=np.zeros((1, 2)),
                    enrich=False, nl=False)
    if name == "p1_enriched":
        return dict(h=1.0, ncell=(13, 13, 13), p=1, atoms=np.array([[6.5, 6.4, 6.6]]),
                    hproj=np.array([[0.9, -0.7]]), enrich=True, nl=True)
    if name == "p7_enriched":
        return dict(h=2.0, ncell=(5, 5, 5), p=7, atoms=np.array([[5.0, 5.0, 5.0]]), hproj=np.array([[0.7, -1.1]]),
                    enrich=True, nl=True)
    if name == "p8_cfe":
        return dict(h=2.0, ncell=(2, 2, 2), p=8, atoms=np.array([[2.0, 2.0, 2.0]]), hproj=np.zeros((1, 2)),
                    enrich=False, nl=False)
    if name == "single_atom":
        return dict(h=2.0, ncell=(6, 6, 6), p=4, atoms=np.array([[6.3, 5.8, 6.1]]), hproj=np.array([[-1.2, 0.7]]),
                    enrich=True, nl=True)
    raise KeyError(name)


def _potential(mesh, atoms):
    q = mesh.all_quad_points()
    return -np.sum([3.0 / np.sqrt(0.5 + np.sum((q - a) ** 2, axis=1)) for a in atoms], axis=0)


_CACHE = {}


def _systems(name):
    if name in _CACHE:
        return _CACHE[name]
    from paper_2607_06848_gb300 import EFE
    c = _case(name)
    mesh = Mesh(c["h"], c["ncell"], c["p"])
    enr = dict(alpha=1.2, r0=R0, t=T_ENR) if c["enrich"] else None
    prj = dict(rc=1.0, rtrunc=6.0, h=c["hproj"]) if c["nl"] else None
    o = EFESystem(mesh, c["atoms"], enrich=enr, proj=prj)
    v = _potential(mesh, c["atoms"])
    o.set_potential(v)
    g = EFE(c["h"], c["ncell"], c["p"], c["atoms"], np.full(len(c["atoms"]), 4.0),
            enrich=dict(alpha=1.2, r_end=R_END, t=T_ENR) if c["enrich"] else None,
            psp=dict(rc=1.0, r_trunc=6.0, h=c["hproj"]) if c["nl"] else None)
    g.efe_set_potential(torch.tensor(v, device="cuda"))
    assert g.dims["n_rows"] == o.nn + o.n_enr
    _CACHE[name] = (o, g)
    return o, g


def _rand(o, N, seed):
    X = W.random_block(o.nn + o.n_enr, N, seed)
    X[:o.nn] *= o.mask[:, None]
    return X


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


CASES = ["dimer", "ragged", "cfe_only", "nonlocal_only", "single_atom", "p6_cfe", "p6_enriched", "p5_enriched"]


@pytest.mark.parametrize("name", CASES)
@pytest.mark.parametrize("N", [1, 13, 37])
def test_apply_h_m_minv(name, N):
    o, g = _systems(name)
    X = _rand(o, N, 100 + N)
    Xd = torch.tensor(X, device="cuda")
    Y = torch.empty_like(Xd)
    g.efe_apply_h(Xd, Y)
    assert _rel(Y.cpu().numpy(), o.apply_H(X)) < 1e-12
    # M^ee = A_ee - B^T (M^cc)^-1 B cancels: the finer the FE space resolves the
    # enrichment, the smaller M^ee against A_ee (|A|/|M^ee| ~ 1e2 at p = 4,
    # ~1e4 at p = 6), and M~^-1 multiplies that relative error by the block
    # condition number; the bounds are eps * |A|/|M^ee| * cond with margin.
    canc = 1.0
    if o.n_enr:
        canc = float(np.abs(o.Aee).max() / np.abs(o.Mee).max())
    g.efe_apply_m(Xd, Y)
    assert _rel(Y.cpu().numpy(), o.apply_M(X)) < 1e-14 * max(1.0, canc / 10)
    g.efe_apply_minv(Xd, Y)
    assert _rel(Y.cpu().numpy(), o.apply_Minv_approx(X)) < 1e-13 * max(1.0, canc) * 100


@pytest.mark.parametrize("name", ["dimer", "ragged"])
def test_apply_h_fp32(name):
    o, g = _systems(name)
    X = _rand(o, 13, 7)
    Xd = torch.tensor(X, device="cuda")
    Y = torch.empty_like(Xd)
    g.efe_apply_h(Xd, Y, prec=1)
    # FP32 storage and accumulation: a few ulp of float times the row sums
    assert _rel(Y.cpu().numpy(), o.apply_H(X)) < 2e-5


@pytest.mark.parametrize("name", CASES)
def test_lanczos(name):
    o, g = _systems(name)
    u0 = _rand(o, 1, 5)
    tg = g.efe_lanczos(torch.tensor(u0, device="cuda"), 10)
    to = OC.lanczos_bounds(o, u0, 10)
    assert np.allclose(tg, to, rtol=1e-9), (tg, to)


@pytest.mark.parametrize("name", ["dimer", "ragged", "single_atom"])
def test_filter_pass(name):
    o, g = _systems(name)
    V = _rand(o, 9, 21)
    HV = o.apply_H(V)
    lam = np.sort(np.random.default_rng(3).uniform(-2.0, 1.0, 9))
    bounds = (-2.5, 1.0, 60.0)
    ref = OC.residual_filter(o, V, lam, 12, bounds[1], bounds[2], bounds[0], HV=HV)
    Vd = torch.tensor(V, device="cuda")
    out = torch.empty_like(Vd)
    g.efe_filter(Vd, torch.tensor(HV, device="cuda"), torch.tensor(lam, device="cuda"), 12, bounds, out)
    assert _rel(out.cpu().numpy(), ref) < 1e-10


@pytest.mark.parametrize("name", ["dimer", "ragged", "cfe_only"])
def test_rayleigh_ritz(name):
    o, g = _systems(name)
    X = _rand(o, 8, 31)
    Xd = torch.tensor(X, device="cuda")
    HX = torch.empty_like(Xd)
    eig, res = g.efe_rayleigh_ritz(Xd, HX)
    lam, V, HV = OC.rayleigh_ritz(o, X)
    assert np.allclose(eig, lam, rtol=1e-10, atol=1e-10)
    assert np.allclose(res, OC.residual_norms(o, V, lam, HV), rtol=1e-7, atol=1e-9)
    Vg = Xd.cpu().numpy()
    assert np.allclose(Vg.T @ o.apply_M(Vg), np.eye(8), atol=1e-11)
    # H X returned is H applied to the rotated X
    assert _rel(HX.cpu().numpy(), o.apply_H(Vg)) < 1e-11


@pytest.mark.parametrize("name", ["dimer", "ragged"])
def test_multipass_chfsi_fp64(name):
    o, g = _systems(name)
    N, nconv = 8, 6
    X = _rand(o, N, 41)
    u0 = _rand(o, 1, 42)
    ref = OC.chfsi(o, X, 16, 1e-10, 60, u0, nconv=nconv)
    Xd = torch.tensor(X, device="cuda")
    eig, res, passes, ok = g.efe_chfsi(Xd, 16, u0=torch.tensor(u0, device="cuda"), max_pass=60, tol=1e-10,
                                       nconv=nconv)
    assert ok and res[:nconv].max() < 1e-10
    assert np.max(np.abs(eig[:nconv] - ref["lam"][:nconv])) < 1e-8


@pytest.mark.parametrize("name", ["dimer"])
def test_multipass_chfsi_fp32_vs_fp64(name):
    o, g = _systems(name)
    N, nconv = 8, 6
    X = _rand(o, N, 51)
    u0 = torch.tensor(_rand(o, 1, 52), device="cuda")
    X64 = torch.tensor(X, device="cuda")
    e64, r64, _, ok64 = g.efe_chfsi(X64, 16, u0=u0, max_pass=60, tol=1e-9, nconv=nconv)
    X32 = torch.tensor(X, device="cuda")
    e32, r32, _, _ = g.efe_chfsi(X32, 16, u0=u0, max_pass=60, tol=1e-6, nconv=nconv, prec=1)
    assert ok64
    assert np.max(np.abs(e32[:nconv] - e64[:nconv])) < 1e-6


def test_filter_host_buffers_match_device():
    o, g = _systems("dimer")
    V = _rand(o, 8, 61)
    HV = o.apply_H(V)
    lam = np.linspace(-2, 0.5, 8)
    bounds = (-2.2, 0.5, 50.0)
    out_h = g.efe_filter_host(V, HV, lam, 10, bounds)
    Vd = torch.tensor(V, device="cuda")
    out = torch.empty_like(Vd)
    g.efe_filter(Vd, torch.tensor(HV, device="cuda"), torch.tensor(lam, device="cuda"), 10, bounds, out)
    assert np.array_equal(out_h, out.cpu().numpy())


def test_state_and_argument_errors():
    from paper_2607_06848_gb300 import EFE, EFEError
    c = _case("single_atom")
    g = EFE(c["h"], c["ncell"], c["p"], c["atoms"], [4.0], enrich=dict(alpha=1.2, r_end=R_END, t=T_ENR))
    X = torch.zeros((g.dims["n_rows"], 2), dtype=torch.float64, device="cuda")
    with pytest.raises(EFEError) as e:
        g.efe_apply_h(X, torch.empty_like(X))
    assert e.value.status == 7                  # no potential yet
    with pytest.raises(EFEError) as e:
        g.efe_filter(X, X, torch.zeros(2, dtype=torch.float64, device="cuda"), 5, (1.0, 0.0, 2.0),
                     torch.empty_like(X))
    assert e.value.status in (1, 7)
    g.close()
