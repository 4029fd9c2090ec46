"""Link parametrisation: 18-real storage (row 2 kept in memory as the rebuild
from rows 0,1) must give the same numbers as the 12-real storage (row 2 rebuilt
on every load), bit for bit, and therefore the oracle's to 1e-13."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1301_3460_gb300 import inputs, lgf

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("L", [(8, 8, 8, 8), (12, 8, 6, 4)])
def test_links18_equals_links12_and_oracle(L):
    U = inputs.rough_gauge_field(L, 0.3, 91)
    ref = orc.fix(L, U, alpha=0.08, tol=0.0, max_iter=10)
    out = {}
    for l18 in (False, True):
        with lgf.Lattice(L, links18=l18) as lat:
            lat.set_links(U)
            r = lat.fix(alpha=0.08, tol=0.0, max_iter=10)
            out[l18] = (lat.get_links(), lat.get_gauge(), r)
    assert np.max(np.abs(out[True][0] - out[False][0])) == 0.0
    assert np.max(np.abs(out[True][1] - out[False][1])) == 0.0
    assert out[True][2]["F"] == out[False][2]["F"]
    assert np.max(np.abs(out[True][0] - ref["U"])) < 1e-13


@pytest.mark.parametrize("mixed", [False, True])
def test_links18_converges(mixed):
    L = (8, 8, 8, 8)
    U = inputs.rough_gauge_field(L, 0.3, 1001)
    ref = orc.fix(L, U, alpha=0.08, tol=1e-15, max_iter=5000)
    with lgf.Lattice(L, mixed=mixed, links18=True) as lat:
        lat.set_links(U)
        r = lat.fix(alpha=0.08, tol=1e-15, max_iter=5000)
        G = lat.get_gauge()
        Ug = lat.get_links()
    assert r["converged"]
    assert r["F"] == pytest.approx(ref["F"], rel=1e-12)
    np.testing.assert_allclose(orc.gauge_transform(L, U, G), Ug, atol=1e-13)


def test_links18_derivative_matches_links12():
    torch = pytest.importorskip("torch")
    L = (6, 6, 6, 6)
    U = inputs.rough_gauge_field(L, 0.3, 92)
    V = int(np.prod(L))
    G = np.random.default_rng(93).standard_normal((4, V, 3, 3)) + 0j
    out = []
    for l18 in (False, True):
        with lgf.Lattice(L, links18=l18) as lat:
            lat.set_links(U)
            out.append(lat.step_bwd(torch.from_numpy(G).cuda(), 0.08).cpu().numpy())
    assert np.max(np.abs(out[0] - out[1])) == 0.0
