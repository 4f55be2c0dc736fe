"""The allocation-free integral (efe_integrate_noalloc) against efe_integrate.

Some callers cannot call cudaMalloc while they run; this entry point serves
them from a fixed device array.  Checked through the C ABI on two calls in a
row (the second must not depend on what the first left in the array), with
the tolerance of the other integral tests.  Collected last on purpose.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_noalloc_integral_matches_allocating_one():
    from paper_2607_06848_gb300 import EFE, workloads as W
    w = W.dimer()
    g = EFE(w["h"], w["ncell"], w["p"], w["atoms"], w["Z"], enrich=dict(alpha=1.2, r_end=5.0, t=0.33),
            psp=dict(rc=1.0, r_trunc=6.0, h=w["hproj"], rloc=0.8))
    n = g.dims["n_quad"]
    rng = np.random.default_rng(11)
    for k in range(2):
        a = torch.tensor(rng.uniform(-1.0, 2.0, n), device="cuda")
        b = torch.tensor(rng.uniform(0.5, 1.5, n), device="cuda") if k == 0 else None
        ref = g.efe_integrate(a, b)
        got = g.efe_integrate_noalloc(a, b)
        assert abs(got - ref) <= 1e-12 * max(abs(ref), 1.0), (k, got, ref)
    g.close()
