"""Wilson-action configuration generation on the GPU (heat bath and
overrelaxation of the stored links) through the C ABI, against the oracle's
generator: links after whole sweeps element by element (up to 32^4), the
plaquette, and the pipeline generate -> fix."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1301_3460_gb300 import inputs, lgf

pytestmark = pytest.mark.gpu


def oracle_chain(L, U, beta, seed, first, n_hb, n_or):
    for i in range(n_hb):
        U = orc.wilson_sweeps(L, U, beta, seed, 1, mode=0, first_sweep=first + i)
        U = orc.wilson_sweeps(L, U, beta, seed, n_or, mode=1)
    return U


@pytest.mark.parametrize("L", [(4, 4, 4, 4), (4, 6, 8, 4)])
@pytest.mark.parametrize("links18", [False, True])
def test_sweeps_match_oracle(L, links18):
    """Two rounds of one heat-bath and two overrelaxation sweeps at beta = 5.7
    (mostly Kennedy-Pendleton draws); 12- and 18-real link storage."""
    U = inputs.rough_gauge_field(L, 0.5, 21)
    ref = oracle_chain(L, U, 5.7, 123, 5, 2, 2)
    with lgf.Lattice(L, links18=links18) as lat:
        lat.set_links(U)
        lat.wilson_sweeps(5.7, 123, first_sweep=5, n_heatbath=2, n_overrelax=2)
        Ug = lat.get_links()
        P = lat.plaquette()
    assert np.max(np.abs(Ug - ref)) < 1e-12
    assert abs(P - orc.wilson_plaquette(L, ref)) < 1e-13


@pytest.mark.parametrize("L", [(4, 4, 4, 4), (4, 6, 8, 4)])
@pytest.mark.parametrize("beta", [0.0, 0.8])
def test_strong_coupling_sweep_matches_oracle(L, beta):
    """At strong coupling (Creutz draws) one heat-bath sweep, element by element.
    The SU(2) frame V = (r, s)/k is ill-conditioned where the projected staple k
    is small, which there it often is: rounding differences grow by about 10^2
    per sweep, so chains are compared through their statistics instead
    (test_strong_coupling_chain)."""
    U = inputs.rough_gauge_field(L, 0.5, 21)
    ref = orc.wilson_sweeps(L, U, beta, 123, 1, mode=0, first_sweep=5)
    with lgf.Lattice(L) as lat:
        lat.set_links(U)
        lat.wilson_sweeps(beta, 123, first_sweep=5, n_heatbath=1)
        Ug = lat.get_links()
    assert np.max(np.abs(Ug - ref)) < 1e-11


def test_strong_coupling_chain():
    """<Re Tr U_P / 3> = beta/18 + beta^2/216 + O(beta^4) (the oracle's pin)."""
    L = (8, 8, 8, 8)
    beta = 1.0
    with lgf.Lattice(L, track_gauge=False) as lat:
        lat.set_unit_links()
        lat.wilson_sweeps(beta, 8, first_sweep=0, n_heatbath=20, n_overrelax=2)
        ps = []
        for n in range(100):
            lat.wilson_sweeps(beta, 8, first_sweep=20 + n, n_heatbath=1, n_overrelax=2)
            ps.append(lat.plaquette())
    assert abs(np.mean(ps) - (beta / 18 + beta ** 2 / 216)) < 0.0015


def test_overrelaxation_only_and_mixed_context():
    L = (6, 4, 4, 6)
    U = inputs.rough_gauge_field(L, 0.4, 22)
    ref = orc.wilson_sweeps(L, U, 6.0, 1, 3, mode=1)
    with lgf.Lattice(L, mixed=True) as lat:
        lat.set_links(U)
        lat.wilson_sweeps(6.0, 1, n_heatbath=0, n_overrelax=3)
        Ug = lat.get_links()
        assert lat.plaquette() == pytest.approx(orc.wilson_plaquette(L, U), abs=1e-13)
    assert np.max(np.abs(Ug - ref)) < 1e-12


def test_cold_start_and_split_calls():
    L = (4, 4, 6, 4)
    with lgf.Lattice(L) as lat:
        lat.set_unit_links()
        assert lat.plaquette() == 1.0
        assert np.array_equal(lat.get_links(), inputs.unit_field(L))
        lat.wilson_sweeps(6.0, 77, first_sweep=0, n_heatbath=3, n_overrelax=1)
        whole = lat.get_links()
        lat.set_unit_links()
        lat.wilson_sweeps(6.0, 77, first_sweep=0, n_heatbath=1, n_overrelax=1)
        lat.wilson_sweeps(6.0, 77, first_sweep=1, n_heatbath=2, n_overrelax=1)
        split = lat.get_links()
    assert np.array_equal(whole, split)
    ref = oracle_chain(L, inputs.unit_field(L), 6.0, 77, 0, 3, 1)
    assert np.max(np.abs(whole - ref)) < 1e-12


@pytest.mark.parametrize("L", [(4, 4, 4, 4), (8, 6, 4, 12), (16, 16, 16, 16)])
def test_plaquette_matches_oracle(L):
    U = inputs.rough_gauge_field(L, 0.6, 23)
    with lgf.Lattice(L) as lat:
        lat.set_links(U)
        p1, p2 = lat.plaquette(), lat.plaquette()
    assert p1 == p2
    assert abs(p1 - orc.wilson_plaquette(L, U)) < 1e-13


def test_argument_and_state_errors():
    with lgf.Lattice((4, 4, 4, 4)) as lat:
        with pytest.raises(lgf.LgfError):
            lat.wilson_sweeps(6.0, 1)  # no links stored yet
        lat.set_unit_links()
        with pytest.raises(lgf.LgfError):
            lat.wilson_sweeps(-1.0, 1)
        with pytest.raises(lgf.LgfError):
            lat.wilson_sweeps(6.0, 1, first_sweep=-1)


def test_generate_then_fix_matches_oracle():
    """The device-made configuration goes straight into the fixing loop; the
    oracle makes the same configuration and fixes it."""
    L = (8, 8, 8, 8)
    ref_U = oracle_chain(L, inputs.unit_field(L), 6.0, 5, 0, 4, 1)
    ref = orc.fix(L, ref_U, alpha=0.08, tol=1e-15, max_iter=2000)
    with lgf.Lattice(L) as lat:
        lat.set_unit_links()
        lat.wilson_sweeps(6.0, 5, n_heatbath=4, n_overrelax=1)
        assert np.max(np.abs(lat.get_links() - ref_U)) < 1e-12
        r = lat.fix(alpha=0.08, tol=1e-15, max_iter=2000)
        Ug, G = lat.get_links(), lat.get_gauge()
    assert r["converged"] and ref["converged"]
    assert abs(r["iters"] - ref["iters"]) <= 1
    assert r["F"] == pytest.approx(ref["F"], rel=1e-12)
    assert np.max(np.abs(orc.gauge_transform(L, ref_U, G) - Ug)) < 1e-11


def test_full_size_sweeps():
    """32^4 (the size of the paper's runs), in the launch configuration the
    benchmark times: two heat-bath sweeps and one overrelaxation sweep from a
    cold start, every link against the oracle's sweeps (about 6 s each on one
    host core)."""
    L = (32, 32, 32, 32)
    beta, seed = 6.0, 99
    U = inputs.unit_field(L)
    with lgf.Lattice(L, track_gauge=False) as lat:
        lat.set_unit_links()
        for n in range(2):
            lat.wilson_sweeps(beta, seed, first_sweep=n, n_heatbath=1)
            U = orc.wilson_sweeps(L, U, beta, seed, 1, mode=0, first_sweep=n)
            assert np.max(np.abs(lat.get_links() - U)) < 1e-12
        lat.wilson_sweeps(beta, seed, n_heatbath=0, n_overrelax=1)
        U = orc.wilson_sweeps(L, U, beta, seed, 1, mode=1)
        assert np.max(np.abs(lat.get_links() - U)) < 1e-12
        assert abs(lat.plaquette() - orc.wilson_plaquette(L, U)) < 1e-13


def test_beta6_plaquette():
    """Thermalised at beta = 6.0 on 16^4 the plaquette sits at the published
    large-volume value 0.5937 (a statistical check of the whole chain)."""
    L = (16, 16, 16, 16)
    with lgf.Lattice(L, track_gauge=False) as lat:
        lat.set_unit_links()
        lat.wilson_sweeps(6.0, 2024, first_sweep=0, n_heatbath=150, n_overrelax=4)
        ps = []
        for n in range(40):
            lat.wilson_sweeps(6.0, 2024, first_sweep=150 + n, n_heatbath=1, n_overrelax=4)
            ps.append(lat.plaquette())
    assert abs(np.mean(ps) - 0.5937) < 0.001


def test_fp32_generator():
    """The FP32-staple generator: links stay in SU(3) to FP64 rounding,
    overrelaxation keeps the action to FP32 rounding of the staples, and the
    chain has the Wilson action's plaquette at strong coupling (beta/18 +
    beta^2/216) and at beta = 6.0 (0.5937 on 16^4)."""
    L = (6, 6, 4, 8)
    U = inputs.rough_gauge_field(L, 0.5, 41)
    with lgf.Lattice(L, track_gauge=False) as lat:
        lat.set_generator_precision(32)
        lat.set_links(U)
        p0 = lat.plaquette()
        lat.wilson_sweeps(6.0, 3, n_heatbath=0, n_overrelax=2)
        assert abs(lat.plaquette() - p0) < 1e-5
        Ug = lat.get_links()
        assert np.max(np.abs(Ug - U)) > 0.1
        lat.wilson_sweeps(6.0, 3, n_heatbath=3, n_overrelax=1)
        M = lat.get_links().reshape(-1, 3, 3)
        assert np.abs(M @ np.conj(np.transpose(M, (0, 2, 1))) - np.eye(3)).max() < 1e-13
        with pytest.raises(lgf.LgfError):
            lat.set_generator_precision(16)
    for L, beta, n_therm, n_meas, want, tol in (((8, 8, 8, 8), 1.0, 20, 100, 1.0 / 18 + 1.0 / 216, 0.0015),
                                                  ((16, 16, 16, 16), 6.0, 150, 40, 0.5937, 0.001)):
        with lgf.Lattice(L, track_gauge=False) as lat:
            lat.set_generator_precision(32)
            lat.set_unit_links()
            lat.wilson_sweeps(beta, 99, first_sweep=0, n_heatbath=n_therm, n_overrelax=4 if beta > 3 else 2)
            ps = []
            for n in range(n_meas):
                lat.wilson_sweeps(beta, 99, first_sweep=n_therm + n, n_heatbath=1, n_overrelax=4 if beta > 3 else 2)
                ps.append(lat.plaquette())
        assert abs(np.mean(ps) - want) < tol
