"""The allocation-free integral (efe_integrate_noalloc).

Some callers cannot call cudaMalloc while they run (their device memory
belongs to another allocator, or their host must not grow device memory
after start-up); this entry point serves them from a fixed device array.
Checked through the C ABI on two calls in a row (the second must not depend
on what the first left in the array) against the FP64 oracle's quadrature and
against the allocating efe_integrate, with free device memory unchanged
across the calls; on a second context of the same device (which reuses the
cached address of the array); and the rejection of meshes beyond the array's
65,536 cells.  Collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dimer_ctx():
    from paper_2607_06848_gb300 import EFE, workloads as W
    w = W.dimer()
    g = EFE(w["h"], w["ncell"], w["p"], w["atoms"], w["Z"], enrich=dict(alpha=1.2, r_end=5.0, t=0.33),
            psp=dict(rc=1.0, r_trunc=6.0, h=w["hproj"], rloc=0.8))
    return g, w


def test_noalloc_integral_matches_oracle_and_allocating_one():
    from oracle.fe import Mesh
    g, w = _dimer_ctx()
    m = Mesh(w["h"], w["ncell"], w["p"])
    n = g.dims["n_quad"]
    rng = np.random.default_rng(11)
    fields = []
    for k in range(2):
        a = rng.uniform(-1.0, 2.0, n)
        b = rng.uniform(0.5, 1.5, n) if k == 0 else None
        fields.append((a, b, torch.tensor(a, device="cuda"), None if b is None else torch.tensor(b, device="cuda")))
    # a first call outside the measured window: it may load the library's
    # device code lazily (the fixed array is part of it)
    g.efe_integrate_noalloc(fields[0][2], fields[0][3])
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    got = [g.efe_integrate_noalloc(ad, bd) for (_, _, ad, bd) in fields]   # two calls in a row
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0, "device memory changed across the calls"
    for (a, b, ad, bd), v in zip(fields, got):
        ref = m.integrate(a * (1.0 if b is None else b))
        assert abs(v - ref) <= 1e-12 * max(abs(ref), 1.0), (v, ref)
        assert abs(v - g.efe_integrate(ad, bd)) <= 1e-12 * max(abs(ref), 1.0)
    # a second context on the same device: same values through the cached address
    g2, _ = _dimer_ctx()
    for (a, b, ad, bd), v in zip(fields, got):
        assert abs(g2.efe_integrate_noalloc(ad, bd) - v) <= 1e-12 * max(abs(v), 1.0)
    g2.close()
    g.close()


def test_noalloc_rejects_meshes_beyond_the_fixed_array():
    from paper_2607_06848_gb300 import EFE
    from paper_2607_06848_gb300.efe import EFEError
    # 41^3 = 68,921 cells of degree 1, no atoms: past the 65,536-cell array
    g = EFE(1.0, (41, 41, 41), 1, np.zeros((0, 3)), np.zeros(0))
    a = torch.ones(g.dims["n_quad"], dtype=torch.float64, device="cuda")
    with pytest.raises(EFEError) as e:
        g.efe_integrate_noalloc(a)
    assert e.value.status == 1 and "65536" in str(e.value)
    # the allocating entry point still takes it (the box volume)
    assert abs(g.efe_integrate(a) - 41.0 ** 3) < 1e-9 * 41.0 ** 3
    g.close()
