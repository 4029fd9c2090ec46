"""Mixed precision: FP32 Delta/FFT/update until theta < 1e-6, then an FP64
finish from links rebuilt in FP64 as G U_in G^dag.  Checked against the FP64
oracle (and the FP64 GPU path at full size): theta < 1e-15, F within 1e-12
relative, links exactly on the gauge orbit of the input; the link difference
to the FP64 result is reported."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1301_3460_gb300 import inputs
from paper_1301_3460_gb300 import lgf

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("L,seed", [((16, 16, 16, 16), 1601), ((24, 24, 24, 24), 2401), ((8, 8, 8, 8), 1001)])
def test_mixed_matches_fp64_oracle(L, seed):
    U = inputs.rough_gauge_field(L, 0.3, seed)
    ref = orc.fix(L, U, alpha=0.08, tol=1e-15, max_iter=5000)
    with lgf.Lattice(L, mixed=True) as lat:
        lat.set_links(U)
        r = lat.fix(alpha=0.08, tol=1e-15, max_iter=5000)
        Um = lat.get_links()
        G = lat.get_gauge()
        hist = lat.history()
    assert ref["converged"] and r["converged"] and r["theta"] < 1e-15
    assert r["iters_fp32"] > 0 and r["iters_fp64"] > 0
    assert r["F"] == pytest.approx(ref["F"], rel=1e-12)
    # exactly on the input's gauge orbit (FP64 rounding only)
    np.testing.assert_allclose(orc.gauge_transform(L, U, G), Um, atol=1e-13)
    assert abs(orc.plaquette(L, Um) - orc.plaquette(L, U)) < 1e-13
    uu = np.einsum("msij,mskj->msik", Um, Um.conj())
    assert np.max(np.abs(uu - np.eye(3))) < 1e-13
    err = float(np.max(np.abs(Um - ref["U"])))
    print("mixed %s: iters %d (+%d fp64) vs oracle %d; max|U_mixed - U_fp64| = %.2e; dF/F = %.2e" % (
        L, r["iters_fp32"], r["iters_fp64"], ref["iters"], err, abs(r["F"] / ref["F"] - 1)))
    # the FP32 phase ends below the switch threshold
    assert hist[r["iters_fp32"] - 1, 0] >= 1e-6


def test_mixed_benchmark_lattice_against_oracle(bench_lattice, bench_lattice_fixed):
    """32^4 benchmark lattice in mixed precision (FP32 until theta < 1e-6) against
    the oracle's FP64 fix: theta < 1e-15, F to 1e-12 relative, links exactly on the
    input's gauge orbit; their distance to the FP64 links is the residual global
    rotation left by the FP32 phase (reading 12), a few 1e-7."""
    L, U = bench_lattice
    ref = bench_lattice_fixed
    with lgf.Lattice(L, mixed=True) as lat:
        lat.set_links(U)
        r = lat.fix(alpha=0.08, tol=1e-15, max_iter=5000)
        Um = lat.get_links()
        G = lat.get_gauge()
    assert ref["converged"] and r["converged"] and r["theta"] < 1e-15
    assert r["iters_fp32"] > 0 and r["iters_fp64"] > 0
    assert r["F"] == pytest.approx(ref["F"], rel=1e-12)
    assert np.max(np.abs(orc.gauge_transform(L, U, G) - Um)) < 1e-12
    err = float(np.max(np.abs(Um - ref["U"])))
    print("32^4 mixed: %d + %d iters vs oracle %d; max|U_mixed - U_oracle| = %.2e" % (
        r["iters_fp32"], r["iters_fp64"], ref["iters"], err))
    assert err < 1e-4


def test_mixed_full_size_against_fp64_gpu():
    """48^4 (radix-3 FFT lengths): the mixed result against the FP64 GPU path."""
    L = (48, 48, 48, 48)
    U = inputs.rough_gauge_field(L, 0.3, 4801)
    with lgf.Lattice(L) as lat:
        lat.set_links(U)
        r64 = lat.fix(alpha=0.08, tol=1e-15, max_iter=5000)
        U64 = lat.get_links()
    with lgf.Lattice(L, mixed=True) as lat:
        lat.set_links(U)
        rm = lat.fix(alpha=0.08, tol=1e-15, max_iter=5000)
        Um = lat.get_links()
    assert r64["converged"] and rm["converged"]
    assert rm["F"] == pytest.approx(r64["F"], rel=1e-12)
    err = float(np.max(np.abs(Um - U64)))
    print("48^4: fp64 %d iters, mixed %d+%d iters, max|dU| = %.2e" % (r64["iters"], rm["iters_fp32"],
                                                                     rm["iters_fp64"], err))
    assert err < 1e-4


@pytest.mark.parametrize("fused", [True, False])
@pytest.mark.parametrize("autotune", [False, True])
@pytest.mark.parametrize("L,seed", [((8, 8, 8, 8), 1001), ((16, 16, 16, 16), 1601), ((8, 8, 32, 32), 3301),
                                    ((12, 6, 24, 48), 3302)])
def test_fp32_phase_follows_the_fp64_iteration(L, seed, autotune, fused):
    """The FP32 phase is the FP64 iteration to FP32 rounding: theta_n of its first
    eight updates matches the oracle's to 1e-5 relative (measured 5e-8 to 1.3e-7:
    a few FP32 roundings) and the links after them (re-projected in FP64) to 1e-4
    (measured 1.2e-6 to 2.3e-6), with the default launch shapes and with the
    autotuned ones, with the update fused with Delta and in the two-kernel form,
    on radix-2 and radix-3 extents (two lanes per line at 24, 32 and 48).  A
    wrong mode anywhere in the FP32 Delta, transforms, accelerator or update
    shows at O(1)."""
    U = inputs.rough_gauge_field(L, 0.3, seed)
    ref = orc.fix(L, U, alpha=0.08, tol=0.0, max_iter=8, history=True)
    with lgf.Lattice(L, mixed=True) as lat:
        lat.set_fp32_update(fused)
        lat.set_switch_tol(0.0)
        lat.set_links(U)
        if autotune:
            lat.autotune()
            lat.set_links(U)
        r = lat.fix(alpha=0.08, tol=1e-15, max_iter=8)
        hist = lat.history()
        Um = lat.get_links()
    assert r["iters"] == 8 and r["iters_fp64"] == 0
    th64, th32 = ref["history"][:8, 0], hist[:8, 0]
    rel = np.abs(th32 / th64 - 1)
    print("%s autotune=%s: theta_0..7 max rel diff %.2e, links %.2e" % (L, autotune, rel.max(),
                                                                        np.abs(Um - ref["U"]).max()))
    assert rel.max() < 1e-5
    assert np.max(np.abs(Um - ref["U"])) < 1e-4


@pytest.mark.parametrize("L,seed", [((16, 16, 16, 16), 1601), ((24, 12, 8, 6), 2402)])
def test_fp32_update_forms_reach_the_same_maximum(L, seed):
    """The fused and the two-kernel FP32 update both reach theta < 1e-15 on the
    input's orbit with the oracle's F (the FP32 phases differ by FP32 rounding
    only; the FP64 finish removes it)."""
    U = inputs.rough_gauge_field(L, 0.3, seed)
    ref = orc.fix(L, U, alpha=0.08, tol=1e-15, max_iter=5000)
    with lgf.Lattice(L, mixed=True) as lat:
        for fused in (True, False):
            lat.set_fp32_update(fused)
            lat.set_links(U)
            r = lat.fix(alpha=0.08, tol=1e-15, max_iter=5000)
            assert r["converged"] and r["theta"] < 1e-15 and r["iters_fp32"] > 0
            assert r["F"] == pytest.approx(ref["F"], rel=1e-12)
            np.testing.assert_allclose(orc.gauge_transform(L, U, lat.get_gauge()), lat.get_links(), atol=1e-13)
        assert lat._lib.lgf_set_fp32_update(lat._h, 3) == lgf.LGF_ERR_ARG


def test_mixed_max_iter_in_fp32_phase_keeps_progress():
    L = (8, 8, 8, 8)
    U = inputs.rough_gauge_field(L, 0.3, 5)
    with lgf.Lattice(L, mixed=True) as lat:
        lat.set_links(U)
        r = lat.fix(alpha=0.08, tol=1e-15, max_iter=3)
        Um = lat.get_links()
        G = lat.get_gauge()
    assert r["status"] == lgf.LGF_ERR_NOT_CONVERGED and r["iters"] == 3 and r["iters_fp64"] == 0
    np.testing.assert_allclose(orc.gauge_transform(L, U, G), Um, atol=1e-13)
    _, th0, F0 = orc.delta(L, U)
    _, th3, F3 = orc.delta(L, Um)
    assert F3 > F0


@pytest.mark.parametrize("switch", [1e-13, 0.0])
@pytest.mark.parametrize("L,seed", [((16, 16, 16, 16), 1601), ((8, 8, 8, 8), 1001)])
def test_deep_fp32_phase(L, seed, switch):
    """A deep FP32 phase: to theta < 1e-13, or (switch_tol = 0) until FP32
    stops improving theta (50 iterations without a new smallest value near its
    floor); then the FP64 finish.  The result is the FP64 oracle's maximum all
    the same."""
    U = inputs.rough_gauge_field(L, 0.3, seed)
    ref = orc.fix(L, U, alpha=0.08, tol=1e-15, max_iter=5000)
    with lgf.Lattice(L, mixed=True) as lat:
        lat.set_links(U)
        r6 = lat.fix(alpha=0.08, tol=1e-15, max_iter=5000)
        lat.set_switch_tol(switch)
        lat.set_links(U)
        r = lat.fix(alpha=0.08, tol=1e-15, max_iter=5000)
        hist = lat.history()
        Um, G = lat.get_links(), lat.get_gauge()
    assert r["converged"] and r["theta"] < 1e-15
    assert r["iters_fp32"] > r6["iters_fp32"] and r["iters_fp64"] <= r6["iters_fp64"]
    assert r["iters_fp32"] < 5000
    th32 = hist[: r["iters_fp32"], 0]
    assert th32.min() < 1e-9  # far below the default switch
    assert r["F"] == pytest.approx(ref["F"], rel=1e-12)
    np.testing.assert_allclose(orc.gauge_transform(L, U, G), Um, atol=1e-13)
    with pytest.raises(lgf.LgfError):
        lat2 = lgf.Lattice(L, mixed=True)
        try:
            lat2.set_switch_tol(-1.0)
        finally:
            lat2.close()


def test_fp32_refresh_keeps_the_fp32_links_on_the_orbit():
    """Rebuilding the FP32 links from the input and G during the FP32 phase
    (every 5 updates here) leaves much less for the FP64 finish to remove: theta
    right after the switch drops, and the result is the oracle's either way."""
    L, seed = (16, 16, 16, 16), 1601
    U = inputs.rough_gauge_field(L, 0.3, seed)
    ref = orc.fix(L, U, alpha=0.08, tol=1e-15, max_iter=5000)
    after = {}
    with lgf.Lattice(L, mixed=True) as lat:
        lat.set_switch_tol(1e-13)
        for every in (0, 5):
            lat.set_fp32_refresh(every)
            lat.set_links(U)
            r = lat.fix(alpha=0.08, tol=1e-15, max_iter=5000)
            assert r["converged"]
            assert r["F"] == pytest.approx(ref["F"], rel=1e-12)
            after[every] = lat.history()[r["iters_fp32"], 0]
            np.testing.assert_allclose(orc.gauge_transform(L, U, lat.get_gauge()), lat.get_links(), atol=1e-13)
        with pytest.raises(lgf.LgfError):
            lat.set_fp32_refresh(-1)
    print("theta after the switch: no refresh %.3e, every 5: %.3e" % (after[0], after[5]))
    assert after[5] < 0.2 * after[0]
