"""The persistent z,t kernel with TMA-staged pencils (lgf_set_shape zt_form = 1)
against the oracle: the accelerator in FP64 (1e-13 of the field's size) and with
the FP32 phase's kernels (5e-6, the FP32 rounding bound of the FP32 stage tests),
FP64 links and G after three steps (1e-13), and a mixed fix (F to 1e-12, links on
the input's gauge orbit).  Shapes cover short lines, radix 3, ragged extents,
lines of 48 and 64 split over lanes, every pencil width the form takes, several
pencils per block (grids smaller than the pencil count) and both FFT kernel
variants (lines up to 32, general)."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1301_3460_gb300 import inputs
from paper_1301_3460_gb300 import lgf

pytestmark = pytest.mark.gpu

SHAPES = [(8, 8, 8, 8), (12, 8, 6, 4), (16, 12, 8, 24), (8, 16, 32, 4), (8, 4, 48, 6), (4, 6, 8, 64)]


def widths(L, precision):
    lo = 1 if precision == 64 else 2
    return [w for w in (1, 2, 4, 8) if w >= lo and L[0] % w == 0]


def field(L, eps=0.4, seed=31):
    return inputs.rough_gauge_field(L, eps, seed)


@pytest.mark.parametrize("L", SHAPES)
def test_accelerate_tma_fp64(L):
    U = field(L)
    Do, _, _ = orc.delta(L, U)
    want = orc.accelerate(L, Do)
    scale = max(1.0, float(np.max(np.abs(want))))
    with lgf.Lattice(L) as lat:
        for xw in widths(L, 64):
            for nt in (64, 128):
                lat.set_shape(64, nt_xy=128, nt_zt=nt, xw=xw, zt_form=1)
                sh = lat.get_shape(64)
                assert sh["zt_form"] == 1 and sh["xw"] == xw and sh["zt_grid"] > 0
                got = lat.accelerate(Do)
                assert np.max(np.abs(got - want)) < 1e-13 * scale, (xw, nt)


@pytest.mark.parametrize("L", SHAPES)
def test_accelerate_tma_fp32(L):
    U = field(L, seed=32)
    Do, _, _ = orc.delta(L, U)
    want = orc.accelerate(L, Do)
    scale = float(np.max(np.abs(want)))
    with lgf.Lattice(L, mixed=True) as lat:
        for xw in widths(L, 32):
            for nt in (128, 256):
                lat.set_shape(32, nt_xy=128, nt_zt=nt, xw=xw, zt_form=1)
                got = lat.accelerate(Do, precision=32)
                assert np.max(np.abs(got - want)) < 5e-6 * scale, (xw, nt)


def test_tma_grid_smaller_than_pencil_count():
    """32^4: more pencils than resident blocks, so each block loads, transforms and
    stores several pencils through both buffers."""
    L = (32, 32, 32, 32)
    U = field(L, seed=33)
    Do, _, _ = orc.delta(L, U)
    want = orc.accelerate(L, Do)
    with lgf.Lattice(L, mixed=True) as lat:
        lat.set_shape(64, nt_xy=128, nt_zt=128, xw=4, zt_form=1)
        lat.set_shape(32, nt_xy=128, nt_zt=256, xw=4, zt_form=1)
        units64 = (32 // 4) * 32 * 4
        assert lat.get_shape(64)["zt_grid"] < units64 and lat.get_shape(32)["zt_grid"] < units64
        got64 = lat.accelerate(Do)
        got32 = lat.accelerate(Do, precision=32)
    scale = float(np.max(np.abs(want)))
    assert np.max(np.abs(got64 - want)) < 1e-13 * max(1.0, scale)
    assert np.max(np.abs(got32 - want)) < 5e-6 * scale


@pytest.mark.parametrize("L", [(8, 8, 8, 8), (12, 8, 6, 4), (8, 4, 48, 6)])
def test_steps_tma_fp64(L):
    U = field(L, eps=0.3, seed=34)
    ref = orc.fix(L, U, alpha=0.08, tol=0.0, max_iter=3)
    with lgf.Lattice(L) as lat:
        lat.set_shape(64, nt_xy=128, nt_zt=128, xw=2 if L[0] % 2 == 0 else 1, zt_form=1)
        lat.set_links(U)
        r = lat.fix(alpha=0.08, tol=0.0, max_iter=3)
        got = lat.get_links()
        G = lat.get_gauge()
    assert r["iters"] == 3
    assert np.max(np.abs(got - ref["U"])) < 1e-13
    assert np.max(np.abs(G - ref["G"])) < 1e-13


@pytest.mark.parametrize("L,seed", [((8, 8, 8, 8), 1001), ((16, 16, 16, 16), 1601)])
def test_mixed_fix_tma(L, seed):
    U = inputs.rough_gauge_field(L, 0.3, seed)
    ref = orc.fix(L, U, alpha=0.08, tol=1e-15, max_iter=5000)
    with lgf.Lattice(L, mixed=True) as lat:
        lat.set_shape(64, nt_xy=128, nt_zt=128, xw=4, zt_form=1)
        lat.set_shape(32, nt_xy=128, nt_zt=256, xw=4, zt_form=1)
        lat.set_links(U)
        r = lat.fix(alpha=0.08, tol=1e-15, max_iter=5000)
        Um = lat.get_links()
        G = lat.get_gauge()
    assert ref["converged"] and r["converged"] and r["theta"] < 1e-15
    assert r["iters_fp32"] > 0 and r["iters_fp64"] > 0
    assert r["F"] == pytest.approx(ref["F"], rel=1e-12)
    np.testing.assert_allclose(orc.gauge_transform(L, U, G), Um, atol=1e-13)


def test_tma_shape_refusals():
    L = (8, 8, 8, 8)
    with lgf.Lattice(L, mixed=True) as lat:
        # an FP32 pencil one column wide has 8-byte box rows (tensor copies need 16)
        with pytest.raises(lgf.LgfError) as e:
            lat.set_shape(32, nt_xy=128, nt_zt=128, xw=1, zt_form=1)
        assert e.value.status == lgf.LGF_ERR_ARG
        for bad in (dict(zt_form=2), dict(xw=3), dict(nt_zt=100)):
            kw = dict(nt_xy=128, nt_zt=128, xw=2, zt_form=1)
            kw.update(bad)
            with pytest.raises(lgf.LgfError):
                lat.set_shape(64, **kw)
    with lgf.Lattice(L) as lat:
        with pytest.raises(lgf.LgfError) as e:
            lat.set_shape(32, nt_xy=128, nt_zt=128, xw=2, zt_form=1)
        assert e.value.status == lgf.LGF_ERR_STATE
    # 64 x 96 pencils in FP64: the tiled kernel takes them, two buffers and the tile
    # of the TMA form do not fit in shared memory
    with lgf.Lattice((4, 4, 64, 96)) as lat:
        with pytest.raises(lgf.LgfError) as e:
            lat.set_shape(64, nt_xy=128, nt_zt=128, xw=1, zt_form=1)
        assert e.value.status == lgf.LGF_ERR_ARG
