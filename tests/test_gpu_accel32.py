"""FP64 iterations with the accelerator's transforms in FP32
(lgf_set_accel_precision(32)): Delta, theta, F, the Gram-Schmidt of g and the
update stay FP64, the FFT, multiplier and inverse FFT run in the FP32 phase's
kernels.  The accelerator preconditions the step (its output vanishes exactly
where Delta does), so the fix must stop at the same FP64 theta < 1e-15 on the
same maximum: F to 1e-12 of the oracle's, the links exactly on the input's gauge
orbit and in SU(3) to 1e-13, the iteration count within two of the oracle's.
The links differ from the oracle's by the residual global rotation that the
changed trajectory leaves (a few 1e-7, as in the mixed mode; bound 1e-4)."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1301_3460_gb300 import inputs
from paper_1301_3460_gb300 import lgf

pytestmark = pytest.mark.gpu

CASES = [((8, 8, 8, 8), 1001), ((16, 16, 16, 16), 1601), ((12, 8, 6, 24), 1203), ((8, 4, 48, 6), 1204)]


def _check_fixed(L, U, r, Um, G, ref):
    assert ref["converged"] and r["converged"] and r["theta"] < 1e-15
    assert r["F"] == pytest.approx(ref["F"], rel=1e-12)
    np.testing.assert_allclose(orc.gauge_transform(L, U, G), Um, atol=1e-13)
    uu = np.einsum("msij,mskj->msik", Um, Um.conj())
    assert np.max(np.abs(uu - np.eye(3))) < 1e-13
    assert abs(orc.plaquette(L, Um) - orc.plaquette(L, U)) < 1e-13
    err = float(np.max(np.abs(Um - ref["U"])))
    assert err < 1e-4
    return err


@pytest.mark.parametrize("L,seed", CASES)
def test_fp64_fix_with_fp32_accelerator(L, seed):
    """The whole fix in FP64 iterations (switch_tol above theta: no FP32 phase)."""
    U = inputs.rough_gauge_field(L, 0.3, seed)
    ref = orc.fix(L, U, alpha=0.08, tol=1e-15, max_iter=5000)
    with lgf.Lattice(L, mixed=True) as lat:
        lat.set_switch_tol(1e300)
        lat.set_accel_precision(32)
        lat.set_links(U)
        r = lat.fix(alpha=0.08, tol=1e-15, max_iter=5000)
        Um = lat.get_links()
        G = lat.get_gauge()
    assert r["iters_fp32"] == 0
    assert abs(r["iters"] - ref["iters"]) <= 2
    err = _check_fixed(L, U, r, Um, G, ref)
    print("%s: %d iters (oracle %d), max|U - U_oracle| = %.2e" % (L, r["iters"], ref["iters"], err))


@pytest.mark.parametrize("L,seed", CASES[:3])
def test_mixed_fix_with_fp32_accelerator(L, seed):
    """FP32 phase to theta < 1e-6, then FP64 iterations with the FP32 accelerator."""
    U = inputs.rough_gauge_field(L, 0.3, seed)
    ref = orc.fix(L, U, alpha=0.08, tol=1e-15, max_iter=5000)
    with lgf.Lattice(L, mixed=True) as lat:
        lat.set_accel_precision(32)
        lat.set_links(U)
        r = lat.fix(alpha=0.08, tol=1e-15, max_iter=5000)
        Um = lat.get_links()
        G = lat.get_gauge()
    assert r["iters_fp32"] > 0 and r["iters_fp64"] > 0
    _check_fixed(L, U, r, Um, G, ref)


def test_first_steps_follow_the_oracle():
    """Each step with the FP32 accelerator is the oracle's step up to FP32 rounding
    of Delta~: g differs by ~alpha/2 times the transforms' rounding (a few 1e-7 of
    |Delta~|, see the FP32 stage tests), and the differences add up over the steps:
    links within 1e-6 after one step and 1e-5 after ten (measured 1.3e-6 on 8^4),
    theta_n within 1e-5 relative, and exactly on the orbit."""
    L = (8, 8, 8, 8)
    U = inputs.rough_gauge_field(L, 0.3, 1001)
    with lgf.Lattice(L, mixed=True) as lat:
        lat.set_switch_tol(1e300)
        lat.set_accel_precision(32)
        for n, tol in ((1, 1e-6), (10, 1e-5)):
            ref = orc.fix(L, U, alpha=0.08, tol=0.0, max_iter=n, history=True)
            lat.set_links(U)
            r = lat.fix(alpha=0.08, tol=0.0, max_iter=n)
            Um = lat.get_links()
            G = lat.get_gauge()
            hist = lat.history()
            assert r["iters"] == n
            assert np.max(np.abs(Um - ref["U"])) < tol
            np.testing.assert_allclose(orc.gauge_transform(L, U, G), Um, atol=1e-13)
            th_ref = np.asarray(ref["history"])[:n, 0]
            assert np.max(np.abs(hist[:n, 0] / th_ref - 1)) < 1e-5


def test_benchmark_lattice_with_fp32_accelerator(bench_lattice, bench_lattice_fixed):
    """32^4, eps = 0.3, seed 3202: FP64 iterations with the FP32 accelerator, and the
    mixed mode with it, against the oracle's FP64 fix."""
    L, U = bench_lattice
    ref = bench_lattice_fixed
    with lgf.Lattice(L, mixed=True) as lat:
        lat.set_accel_precision(32)
        for switch in (1e300, 1e-6):
            lat.set_switch_tol(switch)
            lat.set_links(U)
            r = lat.fix(alpha=0.08, tol=1e-15, max_iter=5000)
            Um = lat.get_links()
            G = lat.get_gauge()
            assert ref["converged"] and r["converged"] and r["theta"] < 1e-15
            assert r["F"] == pytest.approx(ref["F"], rel=1e-12)
            assert np.max(np.abs(orc.gauge_transform(L, U, G) - Um)) < 1e-12
            assert np.max(np.abs(Um - ref["U"])) < 1e-4
            if switch > 1:
                assert r["iters_fp32"] == 0 and abs(r["iters"] - ref["iters"]) <= 2


def test_batch_with_fp32_accelerator():
    Ls = [((8, 8, 8, 8), 0.3, 101), ((12, 12, 8, 8), 0.15, 103), ((8, 8, 8, 12), 0.4, 105)]
    U = [inputs.rough_gauge_field(L, e, s) for L, e, s in Ls]
    refs = [orc.fix(L, u, alpha=0.08, tol=1e-15, max_iter=5000) for (L, _, _), u in zip(Ls, U)]
    with lgf.Batch([L for L, _, _ in Ls], mixed=True) as b:
        b.set_accel_precision(32)
        for i, u in enumerate(U):
            b.set_links(i, u)
        r = b.fix(alpha=0.08, tol=1e-15, max_iter=5000)
        links = [b.get_links(i) for i in range(len(U))]
        gauges = [b.get_gauge(i) for i in range(len(U))]
    assert r["rc"] == lgf.LGF_OK
    for i, ((L, _, _), u, ref) in enumerate(zip(Ls, U, refs)):
        assert r["theta"][i] < 1e-15
        assert r["F"][i] == pytest.approx(ref["F"], rel=1e-12)
        np.testing.assert_allclose(orc.gauge_transform(L, u, gauges[i]), links[i], atol=1e-13)


def test_accel_precision_state_and_args():
    L = (8, 8, 8, 8)
    U = inputs.rough_gauge_field(L, 0.3, 1001)
    with lgf.Lattice(L) as lat:  # FP64 context: no FP32 kernels prepared
        with pytest.raises(lgf.LgfError) as e:
            lat.set_accel_precision(32)
        assert e.value.status == lgf.LGF_ERR_STATE
    with lgf.Lattice(L, mixed=True) as lat:
        with pytest.raises(lgf.LgfError) as e:
            lat.set_accel_precision(16)
        assert e.value.status == lgf.LGF_ERR_ARG
        lat.set_links(U)
        lat.set_accel_precision(32)
        ms = lat.time_kernels(0.08, n_iter=3, precision=64)
        assert all(v > 0 for v in ms.values())
        lat.set_accel_precision(64)  # back to every step in FP64: the oracle's links to 1e-13
        lat.set_switch_tol(1e300)
        lat.set_links(U)  # the timed iterations updated the stored links
        r = lat.fix(alpha=0.08, tol=0.0, max_iter=3)
        ref = orc.fix(L, U, alpha=0.08, tol=0.0, max_iter=3)
        assert r["iters"] == 3
        assert np.max(np.abs(lat.get_links() - ref["U"])) < 1e-13
