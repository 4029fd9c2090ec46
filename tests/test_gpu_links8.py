"""Link parametrisation: the 8-real form (u01, u02, u10 and the phases of u00
and u20, the rest rebuilt from unitarity and det = 1 on every load) against the
oracle and to convergence, in FP64 and mixed precision; links the form cannot
hold are refused.  The rebuild divides by n2 = |u01|^2 + |u02|^2, so its rounding
error grows like 1e-16 / n2: along these trajectories n2 comes down to ~2.5e-4
(links rotate toward the singular set |u00| = 1 and away), hence 1e-12 here
against the 12-real form's 1e-13."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1301_3460_gb300 import inputs, lgf

pytestmark = pytest.mark.gpu


def min_n2(U):
    """smallest |u01|^2 + |u02|^2 over the links: the 8-real form's conditioning"""
    return float(np.min(np.abs(U[..., 0, 1]) ** 2 + np.abs(U[..., 0, 2]) ** 2))


@pytest.mark.parametrize("L", [(8, 8, 8, 8), (12, 8, 6, 4)])
def test_links8_matches_oracle(L):
    U = inputs.rough_gauge_field(L, 0.3, 91)
    ref = orc.fix(L, U, alpha=0.08, tol=0.0, max_iter=10)
    assert min_n2(U) > 1e-4 and min_n2(ref["U"]) > 1e-4
    with lgf.Lattice(L, links8=True) as lat:
        lat.set_links(U)
        assert np.max(np.abs(lat.get_links() - U)) < 1e-12  # the round trip
        r = lat.fix(alpha=0.08, tol=0.0, max_iter=10)
        Ug, G = lat.get_links(), lat.get_gauge()
    assert r["iters"] == 10
    err = np.max(np.abs(Ug - ref["U"]))
    print("8-real, %s: max |U - U_oracle| after 10 steps = %.2e" % (L, err))
    assert err < 1e-12
    assert r["F"] == pytest.approx(ref["F"], rel=1e-12)
    np.testing.assert_allclose(orc.gauge_transform(L, U, G), Ug, atol=1e-12)


@pytest.mark.parametrize("mixed", [False, True])
def test_links8_converges(mixed):
    L = (8, 8, 8, 8)
    U = inputs.rough_gauge_field(L, 0.3, 1001)
    ref = orc.fix(L, U, alpha=0.08, tol=1e-15, max_iter=5000)
    with lgf.Lattice(L, mixed=mixed, links8=True) as lat:
        lat.set_links(U)
        r = lat.fix(alpha=0.08, tol=1e-15, max_iter=5000)
        G = lat.get_gauge()
        Ug = lat.get_links()
    assert r["converged"]
    assert r["F"] == pytest.approx(ref["F"], rel=1e-12)
    np.testing.assert_allclose(orc.gauge_transform(L, U, G), Ug, atol=1e-12)


def test_links8_refuses_what_it_cannot_hold():
    L = (4, 4, 4, 4)
    with lgf.Lattice(L, links8=True) as lat:
        with pytest.raises(lgf.LgfError):
            lat.set_links(inputs.unit_field(L))  # |u00| = 1 everywhere
        with pytest.raises(lgf.LgfError):
            lat.set_unit_links()
        lat.set_links(inputs.rough_gauge_field(L, 0.3, 5))
        with pytest.raises(lgf.LgfError):
            lat.wilson_sweeps(6.0, 1)
    with pytest.raises(lgf.LgfError):
        lgf.Lattice(L, links8=True, links18=True)


def test_links8_derivative_matches_links12():
    torch = pytest.importorskip("torch")
    L = (6, 6, 6, 6)
    U = inputs.rough_gauge_field(L, 0.3, 92)
    V = int(np.prod(L))
    G = np.random.default_rng(93).standard_normal((4, V, 3, 3)) + 0j
    out = []
    for l8 in (False, True):
        with lgf.Lattice(L, links8=l8) as lat:
            lat.set_links(U)
            out.append(lat.step_bwd(torch.from_numpy(G).cuda(), 0.08).cpu().numpy())
    assert np.max(np.abs(out[0] - out[1])) < 1e-12
