"""The seeded input generator shared by the tests, the oracle comparisons and the
benchmark: its fields are in SU(3), built as stated (a pure gauge at eps = 0,
the gauge-invariant part exp(i eps A) otherwise), Haar-distributed in their gauge
part, and reproducible from the seed."""
import numpy as np
from scipy.linalg import expm

from paper_1301_3460_gb300 import inputs


def dag(m):
    return np.conj(np.swapaxes(m, -1, -2))


def test_generators_are_gell_mann_halves():
    T = inputs.GENERATORS
    for a in range(8):
        assert np.abs(T[a] - dag(T[a])).max() < 1e-15 and abs(np.trace(T[a])) < 1e-15
        for b in range(8):
            assert abs(np.trace(T[a] @ T[b]) - 0.5 * (a == b)) < 1e-15


def test_links_are_su3_and_seeded():
    L = (4, 4, 6, 4)
    U = inputs.rough_gauge_field(L, 0.3, 11)
    M = U.reshape(-1, 3, 3)
    assert np.abs(M @ dag(M) - np.eye(3)).max() < 1e-14
    assert np.abs(np.linalg.det(M) - 1).max() < 1e-14
    assert np.array_equal(U, inputs.rough_gauge_field(L, 0.3, 11))
    assert not np.array_equal(U, inputs.rough_gauge_field(L, 0.3, 12))


def test_eps_zero_is_a_pure_gauge_and_plaquettes_are_trivial():
    """eps = 0: U_mu(x) = h(x) h^dag(x+mu), so every plaquette is the unit matrix."""
    L = (4, 4, 4, 4)
    U = inputs.rough_gauge_field(L, 0.0, 3)
    n = [inputs.neighbour(L, mu) for mu in range(4)]
    for mu in range(4):
        for nu in range(mu + 1, 4):
            P = U[mu] @ U[nu][n[mu]] @ dag(U[mu][n[nu]]) @ dag(U[nu])
            assert np.abs(P - np.eye(3)).max() < 1e-13


def test_field_follows_its_recipe():
    """U_mu(x) = h(x) exp(i eps A_mu(x)) h^dag(x+mu) with h, then w drawn from
    default_rng(seed) in that order and A = sum_a w_a T_a; rebuilt here with
    scipy's matrix exponential, independent of the generator's eigen-decomposition."""
    L = (4, 4, 4, 4)
    V = 256
    eps, seed = 0.3, 21
    U = inputs.rough_gauge_field(L, eps, seed)
    rng = np.random.default_rng(seed)
    h = inputs.haar_su3(rng, V)
    w = rng.standard_normal((4, V, 8))
    A = np.einsum("mva,aij->mvij", w, inputs.GENERATORS)
    for mu in (0, 3):
        nb = inputs.neighbour(L, mu, +1)
        for s in (0, 77, 255):
            want = h[s] @ expm(1j * eps * A[mu, s]) @ dag(h[nb[s]])
            assert np.abs(U[mu, s] - want).max() < 1e-13


def test_gauge_part_is_haar():
    """h(x) is Haar on SU(3): E Tr h = 0, E |Tr h|^2 = 1, E (Tr h)^3 = 1."""
    L = (8, 8, 8, 8)
    U = inputs.rough_gauge_field(L, 0.0, 5)
    # with eps = 0 the link is h(x) h^dag(x+mu); the product of two independent Haar
    # matrices is Haar, so the link traces carry the Haar moments
    t = np.trace(U, axis1=-2, axis2=-1).ravel()
    assert abs(t.mean()) < 0.03
    assert abs(np.mean(np.abs(t) ** 2) - 1) < 0.04
    assert abs(np.mean(t ** 3) - 1) < 0.1
