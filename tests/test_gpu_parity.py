"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances: the FP64 path must match the oracle to 1e-13 max-abs on links after
steps 1 and 10 and reach theta < 1e-15 with F within 1e-12 relative; the
stage checks use the same 1e-13 scale (relative to the size of the field
where the field is not O(1)).
"""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1301_3460_gb300 import inputs
from paper_1301_3460_gb300 import lgf

pytestmark = pytest.mark.gpu

SHAPES = [(4, 4, 4, 4), (6, 6, 6, 6), (8, 8, 8, 8), (12, 8, 6, 4), (16, 12, 8, 24), (8, 16, 32, 4)]


def dag(m):
    return np.conj(np.swapaxes(m, -1, -2))


def field(L, eps=0.4, seed=7):
    return inputs.rough_gauge_field(L, eps, seed)


@pytest.mark.parametrize("L", SHAPES)
def test_delta_theta_F(L):
    U = field(L)
    with lgf.Lattice(L) as lat:
        lat.set_links(U)
        D, th, F = lat.delta()
    Do, tho, Fo = orc.delta(L, U)
    assert np.max(np.abs(D - Do)) < 1e-13
    assert th == pytest.approx(tho, rel=1e-12)
    assert F == pytest.approx(Fo, rel=1e-12, abs=1e-15)


@pytest.mark.parametrize("L", SHAPES)
def test_accelerate(L):
    U = field(L, seed=8)
    Do, _, _ = orc.delta(L, U)
    want = orc.accelerate(L, Do)
    with lgf.Lattice(L) as lat:
        got = lat.accelerate(Do)
    assert np.max(np.abs(got - want)) < 1e-13 * max(1.0, np.max(np.abs(want)))


@pytest.mark.parametrize("L", SHAPES[:4])
def test_build_g(L):
    U = field(L, seed=9)
    Do, _, _ = orc.delta(L, U)
    Dt = orc.accelerate(L, Do)
    want = orc.build_g(L, Dt, 0.08)
    with lgf.Lattice(L) as lat:
        got = lat.build_g(Dt, 0.08)
    assert np.max(np.abs(got - want)) < 1e-13


@pytest.mark.parametrize("L", SHAPES)
@pytest.mark.parametrize("steps", [1, 10])
def test_links_after_steps(L, steps):
    U = field(L, eps=0.3, seed=11)
    ref = orc.fix(L, U, alpha=0.08, tol=0.0, max_iter=steps)
    with lgf.Lattice(L) as lat:
        lat.set_links(U)
        r = lat.fix(alpha=0.08, tol=0.0, max_iter=steps)
        Ug = lat.get_links()
        Gg = lat.get_gauge()
    assert r["iters"] == steps and r["status"] == lgf.LGF_ERR_NOT_CONVERGED
    assert np.max(np.abs(Ug - ref["U"])) < 1e-13
    assert np.max(np.abs(Gg - ref["G"])) < 1e-13
    assert r["F"] == pytest.approx(ref["F"], rel=1e-12)
    assert r["theta"] == pytest.approx(ref["theta"], rel=1e-10)


def test_small_lattice_converges_like_oracle():
    """8^4, eps = 0.3, seed 1001, alpha = 0.08, theta < 1e-15."""
    L = (8, 8, 8, 8)
    U = inputs.rough_gauge_field(L, 0.3, 1001)
    ref = orc.fix(L, U, alpha=0.08, tol=1e-15, max_iter=5000, history=True)
    with lgf.Lattice(L) as lat:
        lat.set_links(U)
        r = lat.fix(alpha=0.08, tol=1e-15, max_iter=5000)
        Ug = lat.get_links()
        Gg = lat.get_gauge()
        hist = lat.history()
    assert ref["converged"] and r["converged"]
    assert r["theta"] < 1e-15
    # the stop test may fall on the other side of tol only when theta_n is within 1e-10 of it
    th_ref = ref["history"][:, 0]
    if r["iters"] != ref["iters"]:
        n = min(r["iters"], ref["iters"])
        assert abs(r["iters"] - ref["iters"]) == 1 and abs(th_ref[n] / 1e-15 - 1) < 1e-10
    assert r["F"] == pytest.approx(ref["F"], rel=1e-12)
    assert np.max(np.abs(Ug - ref["U"])) < 1e-11
    np.testing.assert_allclose(orc.gauge_transform(L, U, Gg), Ug, atol=1e-13)
    assert hist.shape[0] == r["iters"] + 1
    assert np.all(np.diff(hist[:, 1]) >= -1e-15)
    np.testing.assert_allclose(hist[:, 0], th_ref[: hist.shape[0]], rtol=1e-9, atol=1e-24)


def test_pure_gauge_reaches_F_one():
    L = (8, 8, 4, 6)
    U = inputs.pure_gauge_field(L, 31)
    with lgf.Lattice(L) as lat:
        lat.set_links(U)
        r = lat.fix(alpha=0.08, tol=1e-15, max_iter=3000)
    assert r["converged"] and r["F"] == pytest.approx(1.0, abs=1e-14)


def test_linear_regime_contraction():
    L = (8, 6, 8, 4)
    U = inputs.rough_gauge_field(L, 1e-5, 41, haar=False)
    with lgf.Lattice(L) as lat:
        lat.set_links(U)
        lat.fix(alpha=0.08, tol=0.0, max_iter=2)
        th = lat.history()[:, 0]
    assert th[1] / th[0] == pytest.approx(0.0784, rel=2e-3)


def test_device_pointers_match_host():
    torch = pytest.importorskip("torch")
    L = (8, 8, 6, 4)
    U = field(L, seed=5)
    with lgf.Lattice(L) as lat:
        lat.set_links(U)
        lat.fix(tol=0.0, max_iter=3)
        host = lat.get_links()
    Ud = torch.from_numpy(U).cuda()
    with lgf.Lattice(L, stream=torch.cuda.current_stream()) as lat:
        lat.set_links(Ud)
        lat.fix(tol=0.0, max_iter=3)
        dev = lat.get_links(device="cuda").cpu().numpy()
    assert np.max(np.abs(dev - host)) == 0.0


def test_status_codes():
    with pytest.raises(lgf.LgfError) as e:
        lgf.Lattice((5, 4, 4, 4))
    assert e.value.status == lgf.LGF_ERR_UNSUPPORTED_DIMS
    L = (4, 4, 4, 4)
    with lgf.Lattice(L) as lat:
        with pytest.raises(lgf.LgfError) as e:
            lat.fix()
        assert e.value.status == lgf.LGF_ERR_STATE
        U = field(L)
        bad = U.copy()
        bad[2, 17] *= 1.001
        with pytest.raises(lgf.LgfError) as e:
            lat.set_links(bad)
        assert e.value.status == lgf.LGF_ERR_NOT_SU3
        bad = U.copy()
        bad[1, 3, 0, 0] = np.nan
        with pytest.raises(lgf.LgfError) as e:
            lat.set_links(bad)
        assert e.value.status == lgf.LGF_ERR_NOT_SU3
        lat.set_links(U)
        r = lat.fix(max_iter=2)
        assert r["status"] == lgf.LGF_ERR_NOT_CONVERGED and r["iters"] == 2 and r["theta"] > 1e-15
        r = lat.fix(max_iter=0)
        assert r["iters"] == 0
        with pytest.raises(lgf.LgfError) as e:
            lat.fix(alpha=-1.0)
        assert e.value.status == lgf.LGF_ERR_ARG


def test_full_size_one_step():
    """32^4, eps = 0.3 (the benchmark workload): one step against the oracle."""
    L = (32, 32, 32, 32)
    U = inputs.rough_gauge_field(L, 0.3, 3202)
    ref = orc.fix(L, U, alpha=0.08, tol=0.0, max_iter=1)
    with lgf.Lattice(L) as lat:
        lat.set_links(U)
        r = lat.fix(alpha=0.08, tol=0.0, max_iter=1)
        Ug = lat.get_links()
    assert np.max(np.abs(Ug - ref["U"])) < 1e-13
    assert r["F"] == pytest.approx(ref["F"], rel=1e-12)


def test_full_size_ten_steps(bench_lattice):
    """32^4 benchmark lattice: links and G after 10 steps against the oracle (1e-13)."""
    L, U = bench_lattice
    ref = orc.fix(L, U, alpha=0.08, tol=0.0, max_iter=10)
    with lgf.Lattice(L) as lat:
        lat.set_links(U)
        r = lat.fix(alpha=0.08, tol=0.0, max_iter=10)
        assert r["iters"] == 10
        assert np.max(np.abs(lat.get_links() - ref["U"])) < 1e-13
        assert np.max(np.abs(lat.get_gauge() - ref["G"])) < 1e-13
    assert r["F"] == pytest.approx(ref["F"], rel=1e-12)


def test_full_size_converges_like_oracle(bench_lattice, bench_lattice_fixed):
    """32^4 benchmark lattice run to theta < 1e-15 in both: the iteration count
    (one apart only when theta_n is within 1e-10 of tol), F to 1e-12 relative,
    links to 1e-11, and the GPU's G relating its links to the input."""
    L, U = bench_lattice
    ref = bench_lattice_fixed
    with lgf.Lattice(L) as lat:
        lat.set_links(U)
        r = lat.fix(alpha=0.08, tol=1e-15, max_iter=500)
        Ug = lat.get_links()
        Gg = lat.get_gauge()
    assert ref["converged"] and r["converged"] and r["theta"] < 1e-15
    if r["iters"] != ref["iters"]:
        n = min(r["iters"], ref["iters"])
        assert abs(r["iters"] - ref["iters"]) == 1 and abs(ref["history"][n, 0] / 1e-15 - 1) < 1e-10
    assert r["F"] == pytest.approx(ref["F"], rel=1e-12)
    assert np.max(np.abs(Ug - ref["U"])) < 1e-11
    assert np.max(np.abs(orc.gauge_transform(L, U, Gg) - Ug)) < 1e-12


def test_contexts_of_different_sizes_coexist():
    """Creating a context for a small lattice must not break a live one with larger planes."""
    Lb, Ls = (16, 16, 16, 16), (4, 4, 4, 4)
    U = field(Lb, seed=3)
    big = lgf.Lattice(Lb)
    small = lgf.Lattice(Ls)
    try:
        big.set_links(U)
        r = big.fix(tol=0.0, max_iter=1)
        ref = orc.fix(Lb, U, tol=0.0, max_iter=1)
        assert r["iters"] == 1
        assert np.max(np.abs(big.get_links() - ref["U"])) < 1e-13
        small.set_links(field(Ls))
        assert small.fix(tol=0.0, max_iter=1)["iters"] == 1
    finally:
        big.close()
        small.close()


@pytest.mark.parametrize("mixed", [False, True])
def test_device_loop_cap_reports_timeout(mixed):
    """Host-side fault injection: a device loop stopped by its body-run cap before
    its stop condition is reported as LGF_ERR_TIMEOUT, and the context stays usable."""
    L = (8, 8, 8, 8)
    U = field(L, seed=13)
    with lgf.Lattice(L, mixed=mixed) as lat:
        lat.set_links(U)
        lat.set_loop_bound(3)
        r = lat.fix(tol=1e-15, max_iter=1000, check=False)
        assert r["status"] == lgf.LGF_ERR_TIMEOUT
        lat.set_loop_bound(0)
        lat.set_links(U)
        r = lat.fix(tol=1e-15, max_iter=1000)
        assert r["converged"]


def test_pinned_host_buffers_match_pageable():
    """Pinned host arrays are read and written in place by the kernels; pageable
    ones go through a device staging copy.  Both give the same bytes."""
    torch = pytest.importorskip("torch")
    L = (8, 8, 6, 4)
    U = field(L, seed=6)
    with lgf.Lattice(L) as lat:
        lat.set_links(U)
        lat.fix(tol=0.0, max_iter=3)
        pageable = lat.get_links()
        Gp = lat.get_gauge()
        pin_in = torch.from_numpy(U).pin_memory()
        lat.set_links(pin_in)
        lat.fix(tol=0.0, max_iter=3)
        out = torch.empty((4, lat.V, 3, 3), dtype=torch.complex128).pin_memory()
        assert lat._lib.lgf_get_links(lat._h, lgf.ctypes.c_void_p(out.data_ptr()), 0) == 0
        gout = torch.empty((lat.V, 3, 3), dtype=torch.complex128).pin_memory()
        assert lat._lib.lgf_get_gauge(lat._h, lgf.ctypes.c_void_p(gout.data_ptr()), 0) == 0
    assert np.max(np.abs(out.numpy() - pageable)) == 0.0
    assert np.max(np.abs(gout.numpy() - Gp)) == 0.0


# every FFT length the kernels take, along each axis, on thin lattices the oracle runs in
# seconds; the last four are the largest planes and pencils the FP64 tiles hold
# (Ly (Lx + 1) = 3096 and 3120 of at most 3520, Lt (3 Lz + 2) = 27840 and 24832 of
# at most 28160)
LONG_AXES = [(128, 4, 4, 4), (4, 96, 4, 4), (4, 4, 64, 4), (4, 4, 4, 128), (48, 6, 4, 4), (4, 4, 24, 48),
             (16, 4, 96, 4), (128, 24, 4, 4), (64, 48, 4, 4), (4, 4, 96, 96), (4, 4, 64, 128)]


@pytest.mark.parametrize("L", LONG_AXES)
def test_long_axes_links_after_steps(L):
    U = field(L, eps=0.3, seed=12)
    ref = orc.fix(L, U, alpha=0.08, tol=0.0, max_iter=3)
    with lgf.Lattice(L) as lat:
        lat.set_links(U)
        r = lat.fix(alpha=0.08, tol=0.0, max_iter=3)
        Ug, Gg = lat.get_links(), lat.get_gauge()
    assert r["iters"] == 3
    assert np.max(np.abs(Ug - ref["U"])) < 1e-13
    assert np.max(np.abs(Gg - ref["G"])) < 1e-13
    assert r["F"] == pytest.approx(ref["F"], rel=1e-12)


def test_over_the_plane_limits_is_refused():
    for L in [(128, 32, 4, 4), (64, 64, 4, 4), (96, 48, 4, 4), (4, 4, 128, 128), (4, 4, 96, 128)]:
        with pytest.raises(lgf.LgfError) as e:
            lgf.Lattice(L)
        assert e.value.status == lgf.LGF_ERR_UNSUPPORTED_DIMS


def test_degenerate_stops():
    """max_iter = 0 measures and stops; a tolerance above theta stops at once; a
    field already in Landau gauge (U = 1) stops with theta = 0 and F = 1."""
    L = (8, 8, 8, 8)
    U = field(L, eps=0.3, seed=13)
    _, th0, f0 = orc.delta(L, U)
    with lgf.Lattice(L) as lat:
        lat.set_links(U)
        r = lat.fix(alpha=0.08, tol=1e-15, max_iter=0)
        assert r["iters"] == 0 and r["status"] == lgf.LGF_ERR_NOT_CONVERGED
        assert r["theta"] == pytest.approx(th0, rel=1e-12) and r["F"] == pytest.approx(f0, rel=1e-12)
        assert np.array_equal(lat.get_links(), lat.get_links())
        np.testing.assert_allclose(lat.get_links(), U, atol=1e-15)
        r = lat.fix(alpha=0.08, tol=10 * th0, max_iter=100)
        assert r["iters"] == 0 and r["converged"]
        lat.set_links(inputs.unit_field(L))
        r = lat.fix(alpha=0.08, tol=1e-15, max_iter=100)
        assert r["iters"] == 0 and r["converged"] and r["theta"] == 0.0 and r["F"] == pytest.approx(1.0, abs=1e-15)
