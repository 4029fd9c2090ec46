"""The FP32 phase's g builder and update in one persistent launch
(lgf_set_fp32_update(ctx, 2), the default of mixed contexts): blocks take xy-planes from a queue, and each
update waits for the g of the three planes it reads.  Every site is computed by
the same functions from the same inputs as in the two-kernel form, so fixes must
agree bit for bit with form 0 (links, G, theta/F history, iteration counts), on
grids with more items than resident blocks, across repeated fixes of one context
(the per-plane flags carry an epoch), with the FP32-link refresh, and reach the
oracle's F."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1301_3460_gb300 import inputs
from paper_1301_3460_gb300 import lgf

pytestmark = pytest.mark.gpu


def _fix(lat, U, switch=1e-6):
    lat.set_switch_tol(switch)
    lat.set_links(U)
    r = lat.fix(alpha=0.08, tol=1e-15, max_iter=5000)
    return r, lat.get_links(), lat.get_gauge(), lat.history()


@pytest.mark.parametrize("L", [(8, 8, 8, 8), (12, 8, 6, 24), (8, 4, 48, 6), (32, 32, 32, 32)])
def test_persistent_form_is_bit_identical(L):
    U = inputs.rough_gauge_field(L, 0.3, 3101)
    with lgf.Lattice(L, mixed=True) as lat:
        lat.set_fp32_update(0)
        r0, U0, G0, h0 = _fix(lat, U)
        lat.set_fp32_update(2)
        for rep in range(2):  # a second fix in the same context: the flags' epochs carry over
            r, Un, Gn, hn = _fix(lat, U)
            assert (r["iters"], r["iters_fp32"], r["F"], r["theta"]) == (r0["iters"], r0["iters_fp32"], r0["F"],
                                                                          r0["theta"]), rep
            assert np.array_equal(Un, U0) and np.array_equal(Gn, G0) and np.array_equal(hn, h0), rep


def test_persistent_form_deep_phase_against_oracle():
    """Switch 1e-13 (FP32 refreshes every 25 updates) on 16^4: bit-identical to the
    two-kernel form, and the oracle's F on the input's orbit."""
    L = (16, 16, 16, 16)
    U = inputs.rough_gauge_field(L, 0.3, 1601)
    ref = orc.fix(L, U, alpha=0.08, tol=1e-15, max_iter=5000)
    with lgf.Lattice(L, mixed=True) as lat:
        lat.set_fp32_update(0)
        r0, U0, G0, _ = _fix(lat, U, switch=1e-13)
        lat.set_fp32_update(2)
        r, Un, Gn, _ = _fix(lat, U, switch=1e-13)
    assert r["iters_fp32"] > 25 and r["converged"] and r["theta"] < 1e-15
    assert np.array_equal(Un, U0) and np.array_equal(Gn, G0)
    assert r["F"] == pytest.approx(ref["F"], rel=1e-12)
    np.testing.assert_allclose(orc.gauge_transform(L, U, Gn), Un, atol=1e-13)


def test_persistent_form_with_fp32_accelerator_and_args():
    L = (8, 8, 8, 8)
    U = inputs.rough_gauge_field(L, 0.3, 1001)
    ref = orc.fix(L, U, alpha=0.08, tol=1e-15, max_iter=5000)
    with lgf.Lattice(L, mixed=True) as lat:
        lat.set_fp32_update(2)
        lat.set_accel_precision(32)
        r, Un, Gn, _ = _fix(lat, U)
        assert r["converged"] and r["F"] == pytest.approx(ref["F"], rel=1e-12)
        np.testing.assert_allclose(orc.gauge_transform(L, U, Gn), Un, atol=1e-13)
        lat.set_links(U)
        ms = lat.time_kernels(0.08, n_iter=3, precision=32)
        assert ms["xyifft_g"] > 0 and ms["update"] >= 0
    with lgf.Lattice(L) as lat:
        with pytest.raises(lgf.LgfError) as e:
            lat.set_fp32_update(2)
        assert e.value.status == lgf.LGF_ERR_STATE
