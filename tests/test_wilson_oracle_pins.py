"""Pins of the Wilson-action configuration generator in the oracle
(oracle/lgf_wilson_oracle.c): the kind of input the paper gauge-fixes (its
32^4 runs use Wilson-action configurations at three couplings).

Each check is fixed by something outside the oracle: published generator
vectors, closed forms of the SU(2) heat-bath density, an exact conservation
law of overrelaxation, the Haar measure of SU(3) at beta = 0, and the strong-
and weak-coupling expansions of the plaquette.
"""
import json
import os

import numpy as np
import pytest
from scipy import integrate
from scipy.special import iv

from oracle import oracle
from paper_1301_3460_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answers():
    with open(os.path.join(GOLDEN, "philox_kat.json")) as f:
        kat = json.load(f)
    for v in kat["vectors"]:
        got = oracle.philox4x32([int(x, 16) for x in v["ctr"]], [int(x, 16) for x in v["key"]])
        assert [int(x) for x in got] == [int(x, 16) for x in v["out"]]


@pytest.mark.parametrize("b", [0.0, 0.3, 1.5, 1.7, 5.0, 12.0])
def test_su2_sampler_density(b):
    """y0 has density sqrt(1 - y0^2) exp(b y0) on [-1, 1] (Haar measure of SU(2)
    times the local Boltzmann weight); the direction (y1, y2, y3) is isotropic.
    b < 1.6 exercises Creutz's method, b >= 1.6 Kennedy-Pendleton."""
    n = 40000
    y = oracle.su2_samples(b, 17, n)
    assert np.abs((y ** 2).sum(1) - 1).max() < 1e-14
    w = lambda t, k: t ** k * np.sqrt(1 - t * t) * np.exp(b * t)
    z = integrate.quad(w, -1, 1, args=(0,))[0]
    m1 = integrate.quad(w, -1, 1, args=(1,))[0] / z
    m2 = integrate.quad(w, -1, 1, args=(2,))[0] / z
    if b > 0:  # closed form of the first moment
        assert abs(m1 - iv(2, b) / iv(1, b)) < 1e-10
    se = lambda a: 5 * a.std() / np.sqrt(n) + 1e-12
    y0 = y[:, 0]
    assert abs(y0.mean() - m1) < se(y0)
    assert abs((y0 ** 2).mean() - m2) < se(y0 ** 2)
    for k in (1, 2, 3):  # isotropy: odd moments vanish, each axis carries a third of 1 - y0^2
        assert abs(y[:, k].mean()) < se(y[:, k])
        assert abs((y[:, k] ** 2).mean() - (1 - m2) / 3) < se(y[:, k] ** 2)


def test_overrelaxation_conserves_action():
    """Overrelaxation maps each link to another with the same local action
    Re Tr(U A), so the plaquette of the whole field is unchanged while the links
    move; a wrong staple (orientation, a missing term) breaks the equality."""
    L = (4, 4, 4, 6)
    U = inputs.rough_gauge_field(L, 0.5, seed=3)
    U2 = oracle.wilson_sweeps(L, U, 5.7, 11, 2, mode=1)
    assert np.abs(U2 - U).max() > 0.1
    assert abs(oracle.wilson_plaquette(L, U2) - oracle.wilson_plaquette(L, U)) < 1e-13
    # the plaquette here and the gauge-fixing oracle's are independent loops
    assert abs(oracle.wilson_plaquette(L, U) - oracle.plaquette(L, U)) < 1e-14


def test_heatbath_keeps_su3():
    L = (4, 4, 4, 4)
    U = oracle.wilson_sweeps(L, inputs.rough_gauge_field(L, 0.3, seed=5), 6.0, 2, 3)
    M = U.reshape(-1, 3, 3)
    eye = np.eye(3)
    assert np.abs(M @ np.conj(np.transpose(M, (0, 2, 1))) - eye).max() < 1e-14
    assert np.abs(np.linalg.det(M) - 1).max() < 1e-14


def test_beta_zero_is_haar():
    """At beta = 0 the chain samples the Haar measure of SU(3): E Tr U = 0,
    E |Tr U|^2 = 1, E (Tr U)^3 = 1 (the last is 0 for U(3))."""
    L = (4, 4, 4, 4)
    U = oracle.wilson_sweeps(L, inputs.unit_field(L), 0.0, 5, 4)
    tr = []
    for n in range(10):
        U = oracle.wilson_sweeps(L, U, 0.0, 5, 1, first_sweep=4 + n)
        tr.append(np.trace(U, axis1=-2, axis2=-1).ravel())
    tr = np.concatenate(tr)
    assert abs(tr.mean()) < 0.05
    assert abs(np.mean(np.abs(tr) ** 2) - 1) < 0.06
    assert abs(np.mean(tr ** 3) - 1) < 0.15


def _plaquette_chain(L, beta, n_therm, n_meas, seed=9):
    U = oracle.wilson_sweeps(L, inputs.unit_field(L), beta, seed, n_therm)
    ps = []
    for n in range(n_meas):
        U = oracle.wilson_sweeps(L, U, beta, seed, 1, first_sweep=n_therm + n)
        U = oracle.wilson_sweeps(L, U, beta, seed, 2, mode=1)
        ps.append(oracle.wilson_plaquette(L, U))
    return np.mean(ps)


def test_strong_coupling_expansion():
    """<Re Tr U_P / 3> = beta/18 + beta^2/216 + O(beta^4) for SU(3) with the
    action beta sum (1 - Re Tr U_P / 3) (single-plaquette Haar integrals:
    E (Re Tr U)^2 = 1/2, E (Re Tr U)^3 = 1/4, the beta^3 term cancels).  A
    wrong normalisation of the heat-bath parameter (beta instead of 2 beta/3
    per unit k, say) moves it by more than 0.02; dropping the second-order
    term by 0.0046."""
    beta = 1.0
    p = _plaquette_chain((4, 4, 4, 4), beta, 10, 100)
    assert abs(p - (beta / 18 + beta ** 2 / 216)) < 0.003


def test_weak_coupling_expansion():
    """1 - <Re Tr U_P / 3> = 2/beta + 1.2208/beta^2 + O(beta^-3) for SU(3): the
    first coefficient is equipartition (24 V non-gauge quadratic modes over 6 V
    plaquettes), the second the published two-loop value."""
    beta = 30.0
    p = _plaquette_chain((4, 4, 4, 4), beta, 30, 60)
    assert abs(p - (1 - 2 / beta - 1.2208 / beta ** 2)) < 0.001


def test_single_link_update_matches_sweep():
    """Link (mu = 0, even site) is the first kind a sweep updates, so its update
    on the starting field is what the sweep leaves there; the single-link entry
    leaves its input untouched."""
    L = (4, 4, 4, 4)
    U = inputs.rough_gauge_field(L, 0.4, seed=8)
    U1 = oracle.wilson_sweeps(L, U, 5.7, 4, 1, first_sweep=3)
    before = U.copy()
    for s in (0, 2, 5, 255 - 3):  # even sites: parity of x+y+z+t
        c = np.unravel_index(s, L[::-1])[::-1]
        if sum(c) % 2:
            continue
        assert np.abs(oracle.wilson_link(L, U, s, 0, 5.7, 4, 3) - U1[0, s]).max() < 1e-15
    assert np.array_equal(U, before)


def test_single_link_heat_bath_samples_the_local_boltzmann_weight():
    """With every other link held fixed, repeated heat-bath updates of one link
    form a Markov chain whose stationary law is exp((beta/3) Re Tr(U A)) dU (Haar
    measure dU, A the sum of the six staples).  The chain's averages of Re Tr(UA),
    Im Tr(UA) and (Re Tr(UA))^2 must equal those of Haar-random SU(3) matrices
    reweighted by that factor.  A rotation applied on the wrong side, a staple of
    the wrong orientation or a wrong subgroup projection samples another law.
    The staple sum is written out here from the plaquettes that contain the
    link, and checked by overrelaxation, which keeps Re Tr(UA) exactly."""
    L = (4, 4, 4, 4)
    V = int(np.prod(L))
    grid = tuple(L[::-1])
    U = inputs.rough_gauge_field(L, 0.7, seed=8).reshape(4, V, 3, 3).copy()
    site, mu, beta = 37, 2, 2.0

    def dag(m):
        return np.conj(np.swapaxes(m, -1, -2))

    def shift(s, nu, k):
        t, z, y, x = np.unravel_index(s, grid)
        c = [x, y, z, t]
        c[nu] = (c[nu] + k) % L[nu]
        return int(np.ravel_multi_index((c[3], c[2], c[1], c[0]), grid))

    # Re Tr of the plaquettes through U_mu(x) = Re Tr(U_mu(x) A)
    A = np.zeros((3, 3), complex)
    xp = shift(site, mu, 1)
    for nu in range(4):
        if nu == mu:
            continue
        A += U[nu, xp] @ dag(U[mu, shift(site, nu, 1)]) @ dag(U[nu, site])
        xm = shift(site, nu, -1)
        A += dag(U[nu, shift(xp, nu, -1)]) @ dag(U[mu, xm]) @ U[nu, xm]
    u_or = oracle.wilson_link(L, U, site, mu, beta, 5, 0, mode=1)
    assert abs(np.trace(u_or @ A).real - np.trace(U[mu, site] @ A).real) < 1e-12
    assert np.abs(u_or - U[mu, site]).max() > 0.1

    n = 20000
    tr = np.empty(n, complex)
    for k in range(n):
        U[mu, site] = oracle.wilson_link(L, U, site, mu, beta, 11, k)
        tr[k] = np.trace(U[mu, site] @ A)
    H = inputs.haar_su3(np.random.default_rng(3), 400000)
    th = np.einsum("nij,ji->n", H, A)
    lw = beta / 3 * th.real
    w = np.exp(lw - lw.max())
    errs = []
    for chain, haar in ((tr.real, th.real), (tr.imag, th.imag), (tr.real ** 2, th.real ** 2)):
        want = (w * haar).sum() / w.sum()
        err_w = np.sqrt((w * w * (haar - want) ** 2).sum()) / w.sum()
        batches = chain.reshape(100, -1).mean(1)  # batch means absorb the chain's autocorrelation
        err_c = batches.std() / np.sqrt(len(batches))
        errs.append(np.hypot(err_w, err_c))
        assert abs(chain.mean() - want) < 5 * errs[-1]
    # the check has teeth at this resolution: beta off by 10% moves <Re Tr(UA)> by
    # many standard errors
    w2 = np.exp(0.9 * lw - (0.9 * lw).max())
    assert abs((w2 * th.real).sum() / w2.sum() - tr.real.mean()) > 10 * errs[0]
