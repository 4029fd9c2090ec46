"""The GPU input generator (a library of its own, no gauge-fixing arithmetic):
the same distribution as the numpy recipe on another random stream."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1301_3460_gb300 import inputs

pytestmark = pytest.mark.gpu


def dag(m):
    return np.conj(np.swapaxes(m, -1, -2))


def test_cuda_fields_are_su3_seeded_and_pure_gauge_at_eps_zero():
    L = (8, 8, 8, 8)
    U = inputs.rough_gauge_field_cuda(L, 0.3, 5).cpu().numpy()
    M = U.reshape(-1, 3, 3)
    assert np.abs(M @ dag(M) - np.eye(3)).max() < 1e-13
    assert np.abs(np.linalg.det(M) - 1).max() < 1e-13
    assert np.array_equal(U, inputs.rough_gauge_field_cuda(L, 0.3, 5).cpu().numpy())
    P = inputs.rough_gauge_field_cuda(L, 0.0, 6).cpu().numpy()
    assert abs(orc.plaquette(L, P) - 1.0) < 1e-13
    t = np.trace(P, axis1=-2, axis2=-1).ravel()  # h(x) h^dag(x+mu): Haar
    assert abs(np.mean(np.abs(t) ** 2) - 1) < 0.04 and abs(np.mean(t ** 3) - 1) < 0.1


@pytest.mark.parametrize("eps", [0.15, 0.5])
def test_cuda_and_numpy_fields_have_the_same_roughness(eps):
    """The gauge-invariant content (the plaquette) of the two generators agrees
    to its statistical error on 16^4."""
    L = (16, 16, 16, 16)
    pc = orc.plaquette(L, inputs.rough_gauge_field_cuda(L, eps, 7).cpu().numpy())
    pn = orc.plaquette(L, inputs.rough_gauge_field(L, eps, 7))
    assert abs(pc - pn) < 2e-3 * eps ** 2 + 1e-4
