"""Pins of the oracle-side PyTorch reference used for derivatives: its forward
equals the C oracle (itself pinned), and its autograd gradient equals central
finite differences along SU(3)-preserving directions."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import lgf_torch_ref as tref  # noqa: E402
from oracle import oracle as orc  # noqa: E402
from paper_1301_3460_gb300 import inputs  # noqa: E402


@pytest.mark.parametrize("L", [(4, 4, 4, 4), (2, 3, 4, 6)])
def test_forward_equals_c_oracle(L):
    U = inputs.rough_gauge_field(L, 0.4, 3)
    Ut = torch.from_numpy(U)
    for _ in range(3):
        Ut = tref.step(L, Ut, 0.08)
    ref = orc.fix(L, U, alpha=0.08, tol=0.0, max_iter=3)["U"]
    assert np.max(np.abs(Ut.numpy() - ref)) < 1e-13
    D, _ = orc.gluon_pmin(L, ref)
    assert float(tref.gluon_pmin(L, Ut)) == pytest.approx(D, rel=1e-12)


def _direction(L, seed):
    rng = np.random.default_rng(seed)
    X = inputs.random_su3_algebra(rng, (4, int(np.prod(L))))
    return X / np.sqrt(np.sum(np.abs(X) ** 2))


def _exp_i(tX):
    w, v = np.linalg.eigh(tX)
    return (v * np.exp(1j * w)[..., None, :]) @ np.conj(np.swapaxes(v, -1, -2))


def test_autograd_matches_finite_differences():
    L = (4, 4, 4, 4)
    K = 2
    U = inputs.rough_gauge_field(L, 0.3, 5)
    Ut = torch.from_numpy(U).requires_grad_(True)
    D = tref.gluon_after_fixing(L, Ut, K)
    (g,) = torch.autograd.grad(D, Ut)
    g = g.numpy()
    h = 1e-6
    for seed in range(5):
        X = _direction(L, 100 + seed)
        dU = 1j * X @ U
        pred = float(np.real(np.sum(np.conj(g) * dU)))
        Dp = float(tref.gluon_after_fixing(L, torch.from_numpy(_exp_i(h * X) @ U), K))
        Dm = float(tref.gluon_after_fixing(L, torch.from_numpy(_exp_i(-h * X) @ U), K))
        fd = (Dp - Dm) / (2 * h)
        assert pred == pytest.approx(fd, rel=1e-6, abs=1e-12)
