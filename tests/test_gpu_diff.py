"""Derivatives through the C ABI: the step vector-Jacobian product and the gluon
propagator derivative against the oracle-side PyTorch reference, and the
K = 50 unrolled gradient against central finite differences (tolerance 1e-7
relative, FP64)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import lgf_torch_ref as tref  # noqa: E402
from paper_1301_3460_gb300 import autograd as lad  # noqa: E402
from paper_1301_3460_gb300 import inputs, lgf  # noqa: E402

pytestmark = pytest.mark.gpu


def _cot(shape, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


@pytest.mark.parametrize("L", [(4, 4, 4, 4), (6, 4, 8, 4), (8, 8, 8, 8)])
def test_step_vjp_matches_reference(L):
    V = int(np.prod(L))
    U = inputs.rough_gauge_field(L, 0.4, 21)
    G = _cot((4, V, 3, 3), 22)
    Ut = torch.from_numpy(U).requires_grad_(True)
    out = tref.step(L, Ut, 0.08)
    (want,) = torch.autograd.grad(out, Ut, torch.from_numpy(G))
    with lgf.Lattice(L) as lat:
        lat.set_links(U)
        got = lat.step_bwd(torch.from_numpy(G).cuda(), 0.08).cpu().numpy()
    want = want.numpy()
    assert np.max(np.abs(got[..., 2, :])) == 0.0
    assert np.max(np.abs(got - want)) < 1e-12 * np.max(np.abs(want))


def test_gluon_derivative_matches_reference():
    L = (8, 4, 6, 4)
    U = inputs.rough_gauge_field(L, 0.3, 23)
    Ut = torch.from_numpy(U).requires_grad_(True)
    D = tref.gluon_pmin(L, Ut)
    (want,) = torch.autograd.grad(D, Ut)
    with lgf.Lattice(L) as lat:
        lat.set_links(U)
        Dg, _ = lat.gluon_pmin()
        got = lat.gluon_pmin_bwd(1.0).cpu().numpy()
    assert Dg == pytest.approx(float(D), rel=1e-12)
    assert np.max(np.abs(got - want.numpy())) < 1e-12 * np.max(np.abs(want.numpy()))


def test_unrolled_gradient_matches_reference():
    L = (6, 6, 6, 6)
    K = 20
    U = inputs.rough_gauge_field(L, 0.3, 24)
    Ut = torch.from_numpy(U).requires_grad_(True)
    (want,) = torch.autograd.grad(tref.gluon_after_fixing(L, Ut, K), Ut)
    Ud = torch.from_numpy(U).cuda().requires_grad_(True)
    D, lat = lad.gluon_after_fixing(Ud, L, K=K, every=5)
    D.backward()
    got = Ud.grad.cpu().numpy()
    lat.close()
    want = want.numpy()
    assert np.linalg.norm(got - want) < 1e-7 * np.linalg.norm(want)


def _exp_i(tX):
    w, v = np.linalg.eigh(tX)
    return (v * np.exp(1j * w)[..., None, :]) @ np.conj(np.swapaxes(v, -1, -2))


def test_unrolled_gradient_reference_8_K50():
    """The K = 50 unroll with checkpoints every 10 against the oracle-side reference."""
    L = (8, 8, 8, 8)
    K = 50
    U = inputs.rough_gauge_field(L, 0.3, 25)
    Ut = torch.from_numpy(U).requires_grad_(True)
    (want,) = torch.autograd.grad(tref.gluon_after_fixing(L, Ut, K), Ut)
    Ud = torch.from_numpy(U).cuda().requires_grad_(True)
    D, lat = lad.gluon_after_fixing(Ud, L, K=K, every=10)
    D.backward()
    got = Ud.grad.cpu().numpy()
    lat.close()
    want = want.numpy()
    err = np.linalg.norm(got - want) / np.linalg.norm(want)
    print("8^4 K=50: |grad_gpu - grad_ref| / |grad_ref| = %.2e" % err)
    assert err < 1e-7


def test_unrolled_gradient_finite_differences_16():
    """16^4, eps = 0.3 (seed 1602), K = 50 steps with checkpoints every 10, 20
    random su(3) directions (seed 1603).  Central differences at h = 1e-6 carry
    the rounding noise of a 50-step FP64 forward divided by h, about 2e-11 in
    absolute terms (1e-7..1e-4 of the derivative, which ranges over 1e-7..1e-4
    here), so they are checked at 1e-5 relative plus that floor; the 1e-7
    relative check uses the fourth-order central stencil at h = 1e-4 (truncation
    O(h^4), rounding floor about 2e-13)."""
    L = (16, 16, 16, 16)
    K = 50
    U = inputs.rough_gauge_field(L, 0.3, 1602)
    Ud = torch.from_numpy(U).cuda().requires_grad_(True)
    D, lat = lad.gluon_after_fixing(Ud, L, K=K, every=10)
    D.backward()
    g = Ud.grad.cpu().numpy()

    def value(t, X):
        lat.set_links(_exp_i(t * X) @ U)
        lat.fix(0.08, 0.0, K)
        return lat.gluon_pmin()[0]

    rng = np.random.default_rng(1603)
    V = int(np.prod(L))
    w2 = w4 = 0.0
    for _ in range(20):
        X = inputs.random_su3_algebra(rng, (4, V))
        X /= np.sqrt(np.sum(np.abs(X) ** 2))
        pred = float(np.real(np.sum(np.conj(g) * (1j * X @ U))))
        h = 1e-6
        fd2 = (value(h, X) - value(-h, X)) / (2 * h)
        h = 1e-4
        fd4 = (8 * (value(h, X) - value(-h, X)) - (value(2 * h, X) - value(-2 * h, X))) / (12 * h)
        w2 = max(w2, abs(pred - fd2) / abs(fd2))
        w4 = max(w4, abs(pred - fd4) / abs(fd4))
        print("  direction: grad %.6e  fd(h=1e-6) %.6e  fd4(h=1e-4) %.6e" % (pred, fd2, fd4))
        assert abs(pred - fd4) <= 1e-7 * abs(fd4) + 1e-12
        assert abs(pred - fd2) <= 1e-5 * abs(fd2) + 1e-10
    lat.close()
    print("16^4 K=50, 20 directions: worst relative difference to FD: h=1e-6 2nd order %.2e, "
          "h=1e-4 4th order %.2e" % (w2, w4))


@pytest.mark.parametrize("L", [(4, 4, 4, 4), (6, 4, 8, 4)])
def test_step_fwd_matches_oracle(L):
    """lgf_step_fwd (the forward of one step, device pointers) against one oracle step."""
    from oracle import oracle as orc

    U = inputs.rough_gauge_field(L, 0.4, 23)
    ref = orc.fix(L, U, alpha=0.08, tol=0.0, max_iter=1)
    with lgf.Lattice(L) as lat:
        out = lat.step_fwd(torch.from_numpy(U).to("cuda"), 0.08)
        again = lat.step_fwd(out, 0.08)
    assert ref["iters"] == 1
    assert np.max(np.abs(out.cpu().numpy() - ref["U"])) < 1e-13
    ref2 = orc.fix(L, ref["U"], alpha=0.08, tol=0.0, max_iter=1)
    assert np.max(np.abs(again.cpu().numpy() - ref2["U"])) < 1e-13


def test_link_snapshots_round_trip():
    """save_links / load_links (the checkpoints of the unrolled derivative)
    restore the stored links exactly, also into another lattice of the same
    extents and flags, and reset G."""
    L = (6, 4, 8, 4)
    U = inputs.rough_gauge_field(L, 0.4, 31)
    with lgf.Lattice(L) as a, lgf.Lattice(L) as b:
        a.set_links(U)
        snap = a.save_links()
        before = a.get_links()
        a.fix(0.08, 0.0, 3)
        assert np.max(np.abs(a.get_links() - before)) > 1e-3
        a.load_links(snap)
        assert np.array_equal(a.get_links(), before)
        assert np.array_equal(a.get_gauge(), inputs.unit_field(L)[0])
        b.load_links(snap)
        assert np.array_equal(b.get_links(), before)
        r1, r2 = a.fix(0.08, 0.0, 2), b.fix(0.08, 0.0, 2)
        assert np.array_equal(a.get_links(), b.get_links()) and r1["F"] == r2["F"]
