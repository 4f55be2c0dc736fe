"""Parity of the learned warm start (through the C ABI) with the FP64 oracle.

Descriptors (double arithmetic, stored float: 1e-6 relative), the network's
forward pass, loss and back-propagated gradient (float arithmetic: the
tolerances below follow from 128-term float dot products, ~sqrt(128) * 2^-24
relative per layer over four layers), the column statistics, one Adam step,
graph-replayed training against the oracle's training loop, the density
correction and the least-squares fit (FP64: 1e-10 of the field's scale, the
transform L^-1 having entries up to ~1e3), and the warm-start density.
Training-set cases span several 32-sample tiles and a ragged tail.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import warmstart as O  # noqa: E402
from oracle.fe import Mesh  # noqa: E402
from oracle.scf import initial_density  # noqa: E402
from paper_2607_06848_gb300 import workloads as W  # noqa: E402

DEV = "cuda"


def _mlp(n=512):
    from paper_2607_06848_gb300 import MLP
    return MLP(n)


def _f32(a):
    return torch.tensor(np.asarray(a, np.float32), device=DEV)


def _case(n, seed):
    rng = np.random.default_rng(seed)
    D = rng.uniform(0.0, 3.0, (n, 32)).astype(np.float32)
    T = rng.standard_normal((n, 8)).astype(np.float32) * np.linspace(0.01, 1.0, 8, dtype=np.float32)
    th = O.set_normalisation(W.mlp_init(seed + 1), D.astype(float), T.astype(float)).astype(np.float32)
    return D, T, th


def test_descriptors_match_oracle():
    w = W.ws_cluster(24, 1003)
    mlp = _mlp()
    xyz = torch.tensor(w["atoms"], device=DEV)
    z = torch.tensor(w["Z"], device=DEV)
    D = torch.empty((24, 32), dtype=torch.float32, device=DEV)
    mlp.efe_descriptors(xyz, z, D)
    Do = O.descriptors(w["atoms"], w["Z"])
    assert np.max(np.abs(D.cpu().numpy() - Do)) <= 1e-6 * np.max(Do)
    assert np.max(Do) > 1.0


def test_forward_matches_oracle():
    D, T, th = _case(200, 3)
    mlp = _mlp()
    C = torch.empty((200, 8), dtype=torch.float32, device=DEV)
    mlp.efe_mlp_forward(_f32(th), _f32(D), C)
    Co = O.predict(th.astype(float), D.astype(float))
    ym = th[O.N_TRAIN + 64:O.N_TRAIN + 72].astype(float)
    ys = th[O.N_TRAIN + 72:O.N_TRAIN + 80].astype(float)
    yo = (Co - ym) / ys                                   # normalised outputs
    err = np.abs(C.cpu().numpy() - Co) / ys
    assert np.max(err) < 2e-5 * (1.0 + np.max(np.abs(yo)))


def test_normalisation_matches_oracle():
    D, T, th = _case(333, 4)
    mlp = _mlp()
    t = _f32(W.mlp_init(0))
    mlp.efe_mlp_normalise(t, _f32(D), _f32(T))
    to = O.set_normalisation(W.mlp_init(0), D.astype(float), T.astype(float))
    tail = t.cpu().numpy()[O.N_TRAIN:]
    assert np.allclose(tail, to[O.N_TRAIN:], rtol=1e-6, atol=1e-7)
    assert np.array_equal(t.cpu().numpy()[:O.N_TRAIN], W.mlp_init(0)[:O.N_TRAIN].astype(np.float32))


@pytest.mark.parametrize("n", [1, 31, 200, 512])
def test_loss_and_gradient_match_oracle(n):
    D, T, th = _case(n, 5 + n)
    mlp = _mlp()
    g = torch.empty(O.N_TRAIN, dtype=torch.float32, device=DEV)
    loss = mlp.efe_mlp_loss_grad(_f32(th), _f32(D), _f32(T), g)
    lo, go = O.loss_and_grad(th.astype(float), D.astype(float), T.astype(float))
    assert abs(loss - lo) < 1e-5 * lo
    gg = g.cpu().numpy()
    for (w, b, m, k) in O.OFFSETS:
        for a, e in ((w, w + m * k), (b, b + m)):
            scale = np.max(np.abs(go[a:e]))
            assert np.max(np.abs(gg[a:e] - go[a:e])) <= 1e-4 * scale + 1e-12, (a, e)
    # fixed-order partial sums: repeated calls give the same bits
    g2 = torch.empty_like(g)
    mlp.efe_mlp_loss_grad(_f32(th), _f32(D), _f32(T), g2)
    assert torch.equal(g, g2)


def test_adam_step_matches_oracle():
    rng = np.random.default_rng(9)
    th = W.mlp_init(2).astype(np.float32)
    m = (rng.standard_normal(O.N_TRAIN) * 1e-2).astype(np.float32)
    v = (rng.uniform(0, 1e-3, O.N_TRAIN)).astype(np.float32)
    g = rng.standard_normal(O.N_TRAIN).astype(np.float32) * 0.1
    mlp = _mlp()
    tt, mm, vv = _f32(th), _f32(m), _f32(v)
    mlp.efe_mlp_adam(tt, mm, vv, _f32(g), 4, lr=2e-3)
    # the kernel's hyperparameters are floats: give the oracle the same rounded values
    f = lambda x: float(np.float32(x))  # noqa: E731
    to, mo, vo = O.adam_step(th.astype(float), m.astype(float), v.astype(float), g.astype(float), 4,
                             lr=f(2e-3), beta1=f(0.9), beta2=f(0.999), eps=f(1e-8))
    assert np.max(np.abs(tt.cpu().numpy()[:O.N_TRAIN] - to[:O.N_TRAIN])) < 1e-6
    # float rounding of the moment updates: a few ulp of the larger operand
    assert np.max(np.abs(mm.cpu().numpy() - mo)) < 4 * 2.0 ** -24 * np.max(np.abs(mo))
    assert np.max(np.abs(vv.cpu().numpy() - vo)) < 4 * 2.0 ** -24 * np.max(np.abs(vo))


def test_graph_training_matches_oracle_and_manual_steps():
    D, T, th = _case(100, 11)
    mlp = _mlp()
    steps = 25
    t1, m1, v1 = _f32(th), torch.zeros(O.N_TRAIN, device=DEV), torch.zeros(O.N_TRAIN, device=DEV)
    hist = torch.empty(steps, dtype=torch.float32, device=DEV)
    mlp.efe_mlp_train(t1, m1, v1, _f32(D), _f32(T), steps, hist, lr=1e-3)
    # the same steps one call at a time give the same bits
    t2, m2, v2 = _f32(th), torch.zeros(O.N_TRAIN, device=DEV), torch.zeros(O.N_TRAIN, device=DEV)
    g = torch.empty(O.N_TRAIN, dtype=torch.float32, device=DEV)
    for s in range(steps):
        mlp.efe_mlp_loss_grad(t2, _f32(D), _f32(T), g)
        mlp.efe_mlp_adam(t2, m2, v2, g, s + 1, lr=1e-3)
    assert torch.equal(t1, t2) and torch.equal(m1, m2)
    to, _, _, ho = O.train(th.astype(float), D.astype(float), T.astype(float), steps, lr=1e-3)
    h = hist.cpu().numpy()
    assert np.allclose(h, ho, rtol=2e-3)
    assert h[-1] < h[0]
    moved = np.linalg.norm(to[:O.N_TRAIN] - th[:O.N_TRAIN])
    assert np.linalg.norm(t1.cpu().numpy()[:O.N_TRAIN] - to[:O.N_TRAIN]) < 2e-2 * moved


def _ctx(w):
    from paper_2607_06848_gb300 import EFE
    return EFE(w["h"], w["ncell"], w["p"], w["atoms"], w["Z"], enrich=dict(alpha=1.2, r_end=5.0, t=0.33),
               psp=dict(rc=1.0, r_trunc=6.0, h=w["hproj"], rloc=0.8))


def test_density_correction_and_fit_match_oracle():
    w = W.ws_cluster(5, 1001)
    m = Mesh(w["h"], w["ncell"], w["p"])
    g = _ctx(w)
    c = np.random.default_rng(3).standard_normal((5, 8)) * 0.05
    dr = torch.empty(g.dims["n_quad"], dtype=torch.float64, device=DEV)
    g.efe_density_correction(torch.tensor(c, device=DEV), dr)
    dro = O.density_correction(m, w["atoms"], c)
    assert np.max(np.abs(dr.cpu().numpy() - dro)) < 1e-10 * np.max(np.abs(dro))
    # fit of the oracle's field plus a smooth non-basis part
    pts = m.all_quad_points()
    tgt = dro + 0.01 * np.exp(-0.1 * np.sum((pts - pts.mean(axis=0)) ** 2, axis=1))
    cf = torch.empty((5, 8), dtype=torch.float64, device=DEV)
    for ridge in (1e-3, 1e-6):
        g.efe_fit_correction(torch.tensor(tgt, device=DEV), cf, ridge=ridge)
        co = O.fit_correction(m, w["atoms"], tgt, ridge=ridge)
        assert np.max(np.abs(cf.cpu().numpy() - co)) < 1e-8 * np.max(np.abs(co)), ridge
    # the difference of two fields, formed inside the call
    base = initial_density(m, w["atoms"], w["Z"])
    g.efe_fit_correction(torch.tensor(tgt + base, device=DEV), cf, base_q=torch.tensor(base, device=DEV))
    co = O.fit_correction(m, w["atoms"], (tgt + base) - base)
    assert np.max(np.abs(cf.cpu().numpy() - co)) < 1e-8 * np.max(np.abs(co))
    g.close()


def test_warm_start_matches_oracle_and_falls_back():
    w = W.ws_cluster(6, 1002)
    m = Mesh(w["h"], w["ncell"], w["p"])
    g = _ctx(w)
    mlp = _mlp()
    th = W.mlp_init(4)
    th[O.N_TRAIN + 32:O.N_TRAIN + 64] = 2.0                        # x_std
    th[O.N_TRAIN + 64:O.N_TRAIN + 72] = np.linspace(-0.03, 0.05, 8)   # y_mean
    th[O.N_TRAIN + 72:O.N_TRAIN + 80] = 0.02                       # y_std
    th32 = th.astype(np.float32)
    rho = torch.empty(g.dims["n_quad"], dtype=torch.float64, device=DEV)
    fb = g.efe_warm_start(mlp, _f32(th32), rho)
    sup = initial_density(m, w["atoms"], w["Z"])
    ro, fbo = O.warm_start_density(m, w["atoms"], w["Z"], th32.astype(float), rho_sup=sup)
    assert not fb and not fbo
    r = rho.cpu().numpy()
    assert np.max(np.abs(r - ro)) < 1e-5 * np.max(ro)
    assert np.max(np.abs(ro - sup)) > 1e-3 * np.max(sup)          # the correction is visible
    assert abs(g.efe_integrate(rho) - 24.0) < 1e-10 and np.all(r >= 0)
    # the same density from explicit coefficients
    c = np.random.default_rng(5).standard_normal((6, 8)) * 0.02
    fb = g.efe_corrected_density(torch.tensor(c, device=DEV), rho)
    ro, fbo = O.corrected_density(m, w["atoms"], w["Z"], c, rho_sup=sup)
    assert not fb and not fbo
    assert np.max(np.abs(rho.cpu().numpy() - ro)) < 1e-12 * np.max(ro)
    # no network: the superposition itself
    fb = g.efe_warm_start(None, None, rho)
    s2 = torch.empty_like(rho)
    g.efe_atomic_density(2.4, s2)
    assert fb and torch.equal(rho, s2)
    # a network whose output is not finite: the superposition again
    bad = th32.copy()
    bad[O.N_TRAIN + 64] = np.nan
    fb = g.efe_warm_start(mlp, _f32(bad), rho)
    assert fb and torch.equal(rho, s2)
    g.close()


def test_learned_start_cuts_scf_iterations():
    """End to end on small clusters: converged FP64 densities of 10 training
    clusters (4-7 atoms) -> targets -> GPU training -> SCF on 2 held-out
    8-atom clusters from the superposition and from the learned density.  The
    learned start must be closer to the converged density, converge in fewer
    iterations, and reach the same energy (1e-6 Ha/atom: both runs stop at
    |dE| < 1e-7 Ha/atom and a density change below 1e-7 N_e)."""
    from paper_2607_06848_gb300 import warmstart as WS
    sizes = [4, 5, 6, 7, 4, 5, 6, 7, 5, 6]
    mlp = _mlp(256)
    Ds, Ts = [], []
    for k, n in enumerate(sizes):
        D, T, rec = WS.training_sample(W.ws_cluster(n, 1000 + k), mlp)
        assert rec["converged"]
        Ds.append(D)
        Ts.append(T)
    theta, hist, _ = WS.train(torch.cat(Ds).contiguous(), torch.cat(Ts).contiguous(), mlp, steps=1500)
    assert hist[-1] < 0.5 * hist[0]
    gains = []
    for k in range(2):
        e = WS.evaluate(W.ws_cluster(8, 2000 + k), mlp, theta)
        s, l = e["superposition"], e["learned"]
        assert s["converged"] and l["converged"] and not l["fallback"]
        assert l["start_error_L2"] < s["start_error_L2"]
        assert abs(l["E"] - s["E"]) / 8 < 1e-6
        gains.append(s["iters"] - l["iters"])
    assert sum(gains) > 0, gains


def test_parameter_file_round_trip_and_rejections(tmp_path):
    mlp = _mlp()
    th = _f32(W.mlp_init(6))
    path = str(tmp_path / "ws.params")
    mlp.efe_mlp_save(th, path)
    back = torch.zeros_like(th)
    mlp.efe_mlp_load(path, back)
    assert torch.equal(th, back)
    raw = open(path, "rb").read()
    assert raw[:8] == b"EFEMLP01" and len(raw) == 12 + 4 * O.N_PARAMS
    from paper_2607_06848_gb300 import EFEError
    for bad in (raw[:100], b"EFEMLP02" + raw[8:]):
        p2 = str(tmp_path / "bad.params")
        open(p2, "wb").write(bad)
        keep = torch.full_like(th, 7.0)
        with pytest.raises(EFEError):
            mlp.efe_mlp_load(p2, keep)
        assert torch.all(keep == 7.0)
    with pytest.raises(EFEError):
        mlp.efe_mlp_load(str(tmp_path / "missing.params"), back)
