"""Plain steepest descent (no Fourier acceleration) through the C ABI against
the oracle's plain method: links after 1 and 10 steps to 1e-13, convergence,
the single-mode linear contraction (1 - alpha p2(k))^2, and the mixed mode."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1301_3460_gb300 import inputs, lgf

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("L", [(4, 4, 4, 4), (6, 6, 6, 6), (12, 8, 6, 4)])
@pytest.mark.parametrize("steps", [1, 10])
def test_plain_links_after_steps(L, steps):
    U = inputs.rough_gauge_field(L, 0.3, 81)
    ref = orc.fix(L, U, alpha=0.1, tol=0.0, max_iter=steps, accelerate=False)
    with lgf.Lattice(L, accelerate=False) as lat:
        lat.set_links(U)
        r = lat.fix(alpha=0.1, tol=0.0, max_iter=steps)
        Ug = lat.get_links()
    assert r["iters"] == steps
    assert np.max(np.abs(Ug - ref["U"])) < 1e-13
    assert r["F"] == pytest.approx(ref["F"], rel=1e-12)


def test_plain_converges_like_oracle():
    L = (6, 6, 4, 4)
    U = inputs.rough_gauge_field(L, 0.3, 71)
    ref = orc.fix(L, U, alpha=0.1, tol=1e-15, max_iter=20000, accelerate=False)
    with lgf.Lattice(L, accelerate=False) as lat:
        lat.set_links(U)
        r = lat.fix(alpha=0.1, tol=1e-15, max_iter=20000)
    assert r["converged"] and ref["converged"]
    assert abs(r["iters"] - ref["iters"]) <= 1
    assert r["F"] == pytest.approx(ref["F"], rel=1e-12)


def test_plain_single_mode_contraction():
    L = (16, 8, 4, 4)
    V = int(np.prod(L))
    eps = 1e-5
    U = inputs.unit_field(L)
    x = np.arange(V) % L[0]
    c = eps * np.cos(2 * np.pi * x / L[0])
    U[0, :, 0, 0] = np.exp(0.5j * c)
    U[0, :, 1, 1] = np.exp(-0.5j * c)
    p2 = 4 * np.sin(np.pi / L[0]) ** 2
    with lgf.Lattice(L, accelerate=False) as lat:
        lat.set_links(U)
        lat.fix(alpha=0.1, tol=0.0, max_iter=2)
        th = lat.history()[:, 0]
    assert th[1] / th[0] == pytest.approx((1 - 0.1 * p2) ** 2, rel=1e-4)


def test_plain_mixed_matches_fp64_oracle():
    L = (8, 8, 8, 8)
    U = inputs.rough_gauge_field(L, 0.3, 82)
    ref = orc.fix(L, U, alpha=0.1, tol=1e-15, max_iter=20000, accelerate=False)
    with lgf.Lattice(L, mixed=True, accelerate=False) as lat:
        lat.set_links(U)
        r = lat.fix(alpha=0.1, tol=1e-15, max_iter=20000)
        G = lat.get_gauge()
        Um = lat.get_links()
    assert r["converged"] and r["iters_fp32"] > 0
    assert r["F"] == pytest.approx(ref["F"], rel=1e-12)
    np.testing.assert_allclose(orc.gauge_transform(L, U, G), Um, atol=1e-13)
