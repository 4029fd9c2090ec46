"""Pins of the FP64 CPU oracle against facts fixed outside the oracle itself:
library transforms and decompositions, closed forms, invariants and brute force.

Every check is chosen so that a plausible slip in the oracle (a dropped term, a
flipped sign or shift direction, a transposed product, a wrong normalisation)
fails at least one of them.  Section references are to arXiv:1301.3460 and to
the steepest-descent method it cites.
"""
import json
import os

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1301_3460_gb300 import inputs

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _grid(L):
    """numpy view order of a scalar field: (Lt, Lz, Ly, Lx)."""
    return tuple(int(v) for v in L[::-1])


def dag(m):
    return np.conj(np.swapaxes(m, -1, -2))


# ---------------------------------------------------------------- transforms


@pytest.mark.parametrize("L", [(4, 4, 4, 4), (2, 3, 4, 6), (6, 4, 3, 2)])
def test_dft_definition_matches_numpy(L):
    rng = np.random.default_rng(1)
    f = rng.standard_normal(np.prod(L)) + 1j * rng.standard_normal(np.prod(L))
    ref = np.fft.fftn(f.reshape(_grid(L))).ravel()
    np.testing.assert_allclose(orc.dft4(L, f, -1), ref, atol=1e-12, rtol=0)
    ref_inv = np.fft.ifftn(f.reshape(_grid(L))).ravel() * np.prod(L)
    np.testing.assert_allclose(orc.dft4(L, f, +1), ref_inv, atol=1e-12, rtol=0)


@pytest.mark.parametrize("L", [(4, 4, 4, 4), (6, 6, 6, 6), (2, 3, 4, 6), (12, 4, 6, 8)])
def test_fft_matches_direct_dft(L):
    rng = np.random.default_rng(2)
    V = int(np.prod(L))
    f = rng.standard_normal(V) + 1j * rng.standard_normal(V)
    for sign in (-1, 1):
        a = orc.fft4(L, f, sign)
        b = orc.dft4(L, f, sign)
        assert np.max(np.abs(a - b)) < 1e-13 * np.sqrt(V) * 10


@pytest.mark.parametrize("L", [(16, 12, 8, 24), (32, 8, 4, 6), (48, 4, 4, 4), (9, 5, 7, 4)])
def test_fft_matches_numpy_and_roundtrip(L):
    rng = np.random.default_rng(3)
    V = int(np.prod(L))
    f = rng.standard_normal(V) + 1j * rng.standard_normal(V)
    F = orc.fft4(L, f, -1)
    ref = np.fft.fftn(f.reshape(_grid(L))).ravel()
    assert np.max(np.abs(F - ref)) < 1e-12 * np.sqrt(V)
    back = orc.fft4(L, F, +1) / V
    assert np.max(np.abs(back - f)) < 1e-13 * 10
    # Parseval
    assert abs(np.sum(np.abs(f) ** 2) - np.sum(np.abs(F) ** 2) / V) < 1e-13 * np.sum(np.abs(f) ** 2)


def test_p2max_closed_form():
    assert orc.p2max((8, 8, 8, 8)) == pytest.approx(16.0, abs=1e-14)
    assert orc.p2max((32, 32, 32, 64)) == pytest.approx(16.0, abs=1e-14)
    # odd extents: 4 sin^2(pi k/L) peaks at k = (L +- 1)/2
    L = (3, 5, 4, 4)
    want = sum(max(4 * np.sin(np.pi * k / n) ** 2 for k in range(n)) for n in L)
    assert orc.p2max(L) == pytest.approx(want, abs=1e-14)


# ---------------------------------------------------------------- Delta, theta, F


def test_unit_field_is_fixed_point():
    L = (4, 4, 4, 6)
    U = inputs.unit_field(L)
    D, th, F = orc.delta(L, U)
    assert np.all(D == 0) and th == 0.0 and F == 1.0
    r = orc.fix(L, U, max_iter=5)
    assert r["iters"] == 0 and r["F"] == 1.0 and r["theta"] == 0.0


def _site(L, c):
    s = 0
    for mu in (3, 2, 1, 0):
        s = s * L[mu] + c[mu]
    return s


def test_delta_single_diagonal_link_closed_form():
    """One non-trivial link U_0(x0) = diag(e^{i phi}, e^{-i phi}, 1):
    Delta(x0) = -(D - D^dag), Delta(x0 + 0) = +(D - D^dag), zero elsewhere;
    theta = 16 sin^2(phi)/(3V); F = 1 - (2 - 2 cos phi)/(12 V)  (the functional of the introduction)."""
    L = (4, 6, 4, 4)
    V = int(np.prod(L))
    phi = 0.7
    U = inputs.unit_field(L)
    x0 = (1, 2, 3, 1)
    s0 = _site(L, x0)
    Dm = np.diag([np.exp(1j * phi), np.exp(-1j * phi), 1.0])
    U[0, s0] = Dm
    D, th, F = orc.delta(L, U)
    ah = Dm - dag(Dm)
    s1 = _site(L, (2, 2, 3, 1))
    np.testing.assert_allclose(D[s0], -ah, atol=1e-15)
    np.testing.assert_allclose(D[s1], ah, atol=1e-15)
    others = np.ones(V, bool)
    others[[s0, s1]] = False
    assert np.all(np.abs(D[others]) == 0)
    assert th == pytest.approx(16 * np.sin(phi) ** 2 / (3 * V), rel=1e-14)
    assert F == pytest.approx(1 - (2 - 2 * np.cos(phi)) / (12 * V), rel=1e-15)


def test_delta_single_offdiagonal_link_direction():
    """A real rotation in the (0,1) block on U_2(x0): Delta is non-zero at x0 and x0 + z only
    (pins the backward shift U_mu(x - mu) and the off-diagonal entries)."""
    L = (4, 4, 6, 4)
    V = int(np.prod(L))
    a = 0.4
    R = np.array([[np.cos(a), np.sin(a), 0], [-np.sin(a), np.cos(a), 0], [0, 0, 1]], np.complex128)
    U = inputs.unit_field(L)
    x0 = (0, 3, 5, 2)
    s0 = _site(L, x0)
    sp = _site(L, (0, 3, 0, 2))  # x0 + z, periodic
    sm = _site(L, (0, 3, 4, 2))  # x0 - z
    U[2, s0] = R
    D, th, F = orc.delta(L, U)
    ah = R - R.T
    np.testing.assert_allclose(D[s0], -ah, atol=1e-15)
    np.testing.assert_allclose(D[sp], ah, atol=1e-15)
    assert np.all(D[sm] == 0)
    assert th == pytest.approx(16 * np.sin(a) ** 2 / (3 * V), rel=1e-14)


def test_delta_is_traceless_antihermitian_and_sums_to_zero():
    L = (6, 4, 8, 4)
    U = inputs.rough_gauge_field(L, 0.4, 77)
    D, th, F = orc.delta(L, U)
    assert np.max(np.abs(D + dag(D))) < 1e-14
    assert np.max(np.abs(np.trace(D, axis1=1, axis2=2))) < 1e-14
    assert np.max(np.abs(D.sum(axis=0))) < 1e-12
    V = D.shape[0]
    assert th == pytest.approx(np.sum(np.abs(D) ** 2) / (3 * V), rel=1e-13)
    assert 0 < th and -1 <= F <= 1


# ---------------------------------------------------------------- Fourier acceleration


def test_accelerate_plane_waves_closed_form():
    """A plane wave of momentum k is an eigenfunction of the accelerator with
    eigenvalue p2max/p2(k); the zero mode is removed."""
    L = (4, 6, 8, 4)
    V = int(np.prod(L))
    c = np.stack(np.meshgrid(*[np.arange(n) for n in L], indexing="ij"), -1)  # (Lx,Ly,Lz,Lt,4)
    c = np.transpose(c, (3, 2, 1, 0, 4)).reshape(V, 4)  # site order s = x + Lx(...)
    D = np.zeros((V, 3, 3), np.complex128)
    want = np.zeros_like(D)
    modes = [((1, 0, 0, 0), (0, 1), 1.0), ((2, 3, 1, 3), (1, 2), 0.5 - 0.25j), ((0, 0, 0, 0), (2, 0), 3.0),
             ((3, 5, 7, 2), (0, 0), -1.0j)]
    p2max = 16.0
    for k, (i, j), amp in modes:
        phase = np.exp(2j * np.pi * np.sum(c * np.array(k) / np.array(L), axis=1))
        D[:, i, j] += amp * phase
        p2 = sum(4 * np.sin(np.pi * k[m] / L[m]) ** 2 for m in range(4))
        if p2 > 0:
            want[:, i, j] += amp * phase * p2max / p2
    for use_dft in (False, True):
        out = orc.accelerate(L, D, use_dft=use_dft)
        np.testing.assert_allclose(out, want, atol=1e-12, rtol=0)


def test_accelerate_fft_equals_dft():
    L = (4, 4, 6, 4)
    U = inputs.rough_gauge_field(L, 0.3, 5)
    D, _, _ = orc.delta(L, U)
    a = orc.accelerate(L, D, use_dft=False)
    b = orc.accelerate(L, D, use_dft=True)
    assert np.max(np.abs(a - b)) < 1e-12


# ---------------------------------------------------------------- reunitarisation


def test_reunit_is_row_gram_schmidt_via_numpy_qr():
    """Row Gram-Schmidt of X is the Q of the LQ decomposition X = L Q with a
    positive diagonal, i.e. (QR of X^dag)^dag; row 2 is Q's third row times conj(det Q)."""
    rng = np.random.default_rng(11)
    X = rng.standard_normal((50, 3, 3)) + 1j * rng.standard_normal((50, 3, 3))
    g = orc.reunit(X)
    q, r = np.linalg.qr(dag(X))
    ph = np.diagonal(r, axis1=1, axis2=2)
    q = q * (ph / np.abs(ph))[:, None, :]  # make diag(R) real positive
    Q = dag(q)
    np.testing.assert_allclose(g[:, :2], Q[:, :2], atol=1e-13)
    det = np.linalg.det(Q)
    np.testing.assert_allclose(g[:, 2], np.conj(det)[:, None] * Q[:, 2], atol=1e-13)
    assert np.max(np.abs(np.linalg.det(g) - 1)) < 1e-14


def test_reunit_fixes_su3():
    h = inputs.random_gauge((2, 2, 2, 2), 3)
    np.testing.assert_allclose(orc.reunit(h), h, atol=2e-15)


# ---------------------------------------------------------------- one update


def test_update_invariants():
    L = (6, 4, 4, 8)
    U0 = inputs.rough_gauge_field(L, 0.5, 13)
    r = orc.fix(L, U0, alpha=0.08, tol=0.0, max_iter=3)
    U, G = r["U"], r["G"]
    uu = np.einsum("msij,mskj->msik", U, U.conj())
    assert np.max(np.abs(uu - np.eye(3))) < 1e-13
    assert np.max(np.abs(np.linalg.det(U) - 1)) < 1e-13
    assert abs(orc.plaquette(L, U) - orc.plaquette(L, U0)) < 1e-13
    np.testing.assert_allclose(orc.gauge_transform(L, U0, G), U, atol=1e-13)
    # the gauge transformation itself is SU(3)
    gg = np.einsum("sij,skj->sik", G, G.conj())
    assert np.max(np.abs(gg - np.eye(3))) < 1e-13


def test_update_direction_by_hand():
    """U_mu(x) <- g(x) U_mu(x) g^dag(x+mu) on a 2^4 lattice, checked link by link with numpy."""
    L = (2, 2, 2, 2)
    V = 16
    U = inputs.rough_gauge_field(L, 0.5, 21)
    g = inputs.random_gauge(L, 22)
    G = inputs.random_gauge(L, 23)
    U2, G2 = orc.update(L, U, G, g)
    for mu in range(4):
        nb = inputs.neighbour(L, mu, +1)
        want = g @ U[mu] @ dag(g[nb])
        np.testing.assert_allclose(U2[mu], want, atol=1e-14)
    np.testing.assert_allclose(G2, g @ G, atol=1e-14)
    assert V == U.shape[1]


# ---------------------------------------------------------------- the iteration


def test_pure_gauge_converges_to_global_maximum():
    """U = h(x) h^dag(x+mu) is a gauge copy of U = 1: the global maximum F = 1 is
    reached and G(x) h(x) is the same matrix at every site (residual global gauge).
    The residual non-constant part of G h scales like sqrt(theta), so the run is
    taken far below the paper's 1e-15 to make that check sharp."""
    L = (6, 6, 4, 4)
    U0 = inputs.pure_gauge_field(L, 31)
    h = inputs.random_gauge(L, 31)  # the same h: random_gauge draws h first from the same seed
    r = orc.fix(L, U0, alpha=0.08, tol=1e-15, max_iter=2000)
    assert r["converged"]
    assert r["F"] == pytest.approx(1.0, abs=1e-14)
    Gh = r["G"] @ h
    assert np.max(np.abs(Gh - Gh[0])) < 100 * np.sqrt(r["theta"])
    r = orc.fix(L, U0, alpha=0.08, tol=1e-26, max_iter=2000)
    assert r["converged"]
    Gh = r["G"] @ h
    assert np.max(np.abs(Gh - Gh[0])) < 1e-10


def test_F_monotone_and_converges():
    L = (8, 8, 8, 8)
    U0 = inputs.rough_gauge_field(L, 0.3, 1001)
    r = orc.fix(L, U0, alpha=0.08, tol=1e-15, max_iter=3000, history=True)
    assert r["converged"] and r["theta"] < 1e-15
    F = r["history"][:, 1]
    assert np.all(np.diff(F) >= -1e-15)
    assert F[-1] > F[0]


def test_linear_regime_contraction_factor():
    """Near the identity every non-zero mode of div A is multiplied by
    (1 - alpha p2max) per step, so theta_1/theta_0 = (1 - 0.08*16)^2 = 0.0784."""
    L = (6, 4, 8, 6)
    U0 = inputs.rough_gauge_field(L, 1e-5, 41, haar=False)
    r = orc.fix(L, U0, alpha=0.08, tol=0.0, max_iter=2, history=True)
    th = r["history"][:, 0]
    assert th[1] / th[0] == pytest.approx(0.0784, rel=2e-3)
    assert th[2] / th[1] == pytest.approx(0.0784, rel=2e-3)


def test_translation_and_axis_swap_covariance():
    L = (6, 6, 4, 4)
    V = int(np.prod(L))
    U0 = inputs.rough_gauge_field(L, 0.4, 51)
    ref = orc.fix(L, U0, tol=0.0, max_iter=3)["U"]
    # translation by (1, 2, 3, 1): field at x moves to x + a
    grid = lambda u: u.reshape((4,) + _grid(L) + (3, 3))  # noqa: E731
    shifts = (1, 3, 2, 1)  # numpy axes order (t, z, y, x) -> shifts for (t=1, z=3, y=2, x=1)
    Ut = np.roll(grid(U0), shifts, axis=(1, 2, 3, 4)).reshape(4, V, 3, 3)
    out = orc.fix(L, Ut, tol=0.0, max_iter=3)["U"]
    want = np.roll(grid(ref), shifts, axis=(1, 2, 3, 4)).reshape(4, V, 3, 3)
    assert np.max(np.abs(out - want)) < 1e-13
    # swap the x and y axes (Lx = Ly): link direction 0 <-> 1 and coordinates swapped
    Us = np.swapaxes(grid(U0), 3, 4)[[1, 0, 2, 3]].reshape(4, V, 3, 3)
    out = orc.fix(L, np.ascontiguousarray(Us), tol=0.0, max_iter=3)["U"]
    want = np.swapaxes(grid(ref), 3, 4)[[1, 0, 2, 3]].reshape(4, V, 3, 3)
    assert np.max(np.abs(out - want)) < 1e-13


def test_direct_dft_and_fft_runs_agree():
    L = (4, 4, 4, 4)
    U0 = inputs.rough_gauge_field(L, 0.3, 61)
    a = orc.fix(L, U0, tol=0.0, max_iter=10)
    b = orc.fix(L, U0, tol=0.0, max_iter=10, use_dft=True)
    assert np.max(np.abs(a["U"] - b["U"])) < 1e-13


# ---------------------------------------------------------------- observables


def test_gluon_propagator_closed_form():
    """A_1(x) = diag(s, -s, 0), s = sin(eps cos(2 pi x/Lx)/2), on U_1 only: D vanishes
    for momenta along y, z, t and equals 2/(8*3*V) * 2|S|^2 along x with
    S = (V/Lx) sum_x exp(-2 pi i x/Lx) s(x)."""
    L = (8, 4, 6, 4)
    V = int(np.prod(L))
    eps = 0.3
    U = inputs.unit_field(L)
    x = np.arange(V) % L[0]
    c = eps * np.cos(2 * np.pi * x / L[0])
    U[1, :, 0, 0] = np.exp(0.5j * c)
    U[1, :, 1, 1] = np.exp(-0.5j * c)
    avg, Dp = orc.gluon_pmin(L, U)
    xs = np.arange(L[0])
    S = (V / L[0]) * np.sum(np.exp(-2j * np.pi * xs / L[0]) * np.sin(eps * np.cos(2 * np.pi * xs / L[0]) / 2))
    want = 2.0 / (8 * 3 * V) * 2 * abs(S) ** 2
    assert Dp[0] == pytest.approx(want, rel=1e-13)
    assert np.all(np.abs(Dp[1:]) < 1e-25)
    assert avg == pytest.approx(want / 4, rel=1e-13)


def test_paper_parameters_fixture():
    with open(os.path.join(GOLD, "paper_parameters.json")) as f:
        p = json.load(f)
    assert p["alpha"] == 0.08 and p["theta_tol"] == 1e-15 and p["L"] == [32, 32, 32, 32]
    # (1 - alpha p2max)^2 at the paper's alpha on any even lattice
    assert (1 - p["alpha"] * orc.p2max(p["L"])) ** 2 == pytest.approx(p["linear_theta_ratio"], rel=1e-12)


def test_plain_sd_single_mode_contraction():
    """Plain steepest descent (no Fourier acceleration) contracts a single
    momentum mode k of div A by (1 - alpha p2(k)) per step: theta_1/theta_0 =
    (1 - alpha p2(k))^2 in the linear regime, where the accelerated method gives
    (1 - alpha p2max)^2 for every k.  A_0(x) = eps cos(2 pi x/Lx) T_3 has div A
    in the modes +-(1,0,0,0)."""
    L = (8, 6, 4, 4)
    V = int(np.prod(L))
    eps = 1e-5
    U = inputs.unit_field(L)
    x = np.arange(V) % L[0]
    c = eps * np.cos(2 * np.pi * x / L[0])
    U[0, :, 0, 0] = np.exp(0.5j * c)
    U[0, :, 1, 1] = np.exp(-0.5j * c)
    p2 = 4 * np.sin(np.pi / L[0]) ** 2
    for alpha in (0.08, 0.05):
        r = orc.fix(L, U, alpha=alpha, tol=0.0, max_iter=2, history=True, accelerate=False)
        th = r["history"][:, 0]
        assert th[1] / th[0] == pytest.approx((1 - alpha * p2) ** 2, rel=1e-4)
        assert th[2] / th[1] == pytest.approx((1 - alpha * p2) ** 2, rel=1e-4)
    r = orc.fix(L, U, alpha=0.08, tol=0.0, max_iter=1, history=True, accelerate=True)
    th = r["history"][:, 0]
    assert th[1] / th[0] == pytest.approx((1 - 0.08 * 16) ** 2, rel=1e-4)


def test_plain_sd_converges_and_keeps_invariants():
    L = (6, 6, 4, 4)
    U0 = inputs.rough_gauge_field(L, 0.3, 71)
    r = orc.fix(L, U0, alpha=0.1, tol=1e-15, max_iter=20000, history=True, accelerate=False)
    assert r["converged"]
    assert np.all(np.diff(r["history"][:, 1]) >= -1e-15)
    assert abs(orc.plaquette(L, r["U"]) - orc.plaquette(L, U0)) < 1e-13
    ra = orc.fix(L, U0, alpha=0.08, tol=1e-15, max_iter=20000, accelerate=True)
    assert ra["iters"] < r["iters"]


def test_delta_is_the_gradient_of_F():
    """Delta is the gradient of the functional (the steepest-descent direction):
    rotating one site by g = exp(t X), X traceless anti-Hermitian, changes
    F_U[g] = 1/(12 V) sum Re Tr[g(x) U_mu(x) g^dag(x+mu)] at the rate
    dF/dt = -Tr[X Delta(x0)] / (24 V).  Central differences of the oracle's F
    against that formula pin Delta's sign, normalisation and site convention."""
    from scipy.linalg import expm

    L = (4, 4, 6, 4)
    V = int(np.prod(L))
    U = inputs.rough_gauge_field(L, 0.4, 77)
    D, _, F0 = orc.delta(L, U)
    rng = np.random.default_rng(5)
    for x0 in (0, 17, V - 1):
        X = 1j * inputs.random_su3_algebra(rng, (1,))[0]  # traceless anti-Hermitian
        assert abs(np.trace(X)) < 1e-14 and np.abs(X + dag(X)).max() < 1e-14
        h = 1e-5
        vals = []
        for t in (h, -h):
            G = np.zeros((V, 3, 3), complex)
            G[:] = np.eye(3)
            G[x0] = expm(t * X)
            _, _, F = orc.delta(L, orc.gauge_transform(L, U, G))
            vals.append(F)
        fd = (vals[0] - vals[1]) / (2 * h)
        want = -np.real(np.trace(X @ D[x0])) / (24 * V)
        assert abs(fd - want) < 1e-9 * max(1.0, abs(want)) + 1e-12
        assert abs(want) > 1e-6


def test_fixed_point_is_a_local_maximum():
    """Landau gauge is a maximum of the functional F_U[g] (the display equation of
    the introduction): after a run to theta < 1e-15, gauge rotations
    g(x) = exp(t X(x)) with random traceless anti-Hermitian X at every site,
    applied here with numpy to the oracle's output links, leave F unchanged at
    first order (the gradient is of order sqrt(theta)) and lower it at second
    order along every direction tried.  On the unfixed input the first-order
    change is large, so the check has teeth; a run converging to a saddle or a
    minimum would fail the second-order check."""
    from scipy.linalg import expm

    L = (4, 4, 4, 6)
    V = int(np.prod(L))
    grid = _grid(L)
    U0 = inputs.rough_gauge_field(L, 0.3, 91)
    r = orc.fix(L, U0, alpha=0.08, tol=1e-15, max_iter=3000)
    assert r["converged"]

    def F_of(U):
        return np.real(np.trace(U, axis1=-2, axis2=-1)).sum() / (12 * V)

    def rotated(U, g):
        gg = g.reshape(grid + (3, 3))
        out = np.empty_like(U)
        for mu in range(4):
            gn = np.roll(gg, -1, axis=3 - mu).reshape(V, 3, 3)  # g(x + mu)
            out[mu] = g @ U[mu] @ dag(gn)
        return out

    rng = np.random.default_rng(17)
    h = 1e-3
    for U, fixed in ((r["U"], True), (U0, False)):
        U = np.asarray(U).reshape(4, V, 3, 3)
        F0 = F_of(U)
        for _ in range(3):
            X = 1j * inputs.random_su3_algebra(rng, (V,))
            Fp, Fm = F_of(rotated(U, expm(h * X))), F_of(rotated(U, expm(-h * X)))
            first = (Fp - Fm) / (2 * h)
            second = (Fp + Fm - 2 * F0) / h**2
            if fixed:
                assert abs(first) < 2e-8
                assert second < -0.05
            else:
                assert abs(first) > 5e-5
