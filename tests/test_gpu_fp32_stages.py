"""The FP32 phase's kernels stage by stage against the FP64 oracle, element by
element (through lgf_delta32, lgf_accelerate32, lgf_build_g32).

Tolerances from the FP32 arithmetic (unit roundoff u = 2^-24 ~ 6e-8): the links
rounded to FP32 and the eight anti-Hermitian parts summed into Delta give ~16 u
of its size, a forward and an inverse transform along an axis of length L add
~2 log2(L) u, the multiplier one u; the Gram-Schmidt runs in FP64 and g is
rounded to FP32 (rows 0,1: u; row 2 rebuilt in FP32: ~3 u).  The bound for
Delta, Delta~ and g is therefore a few u times the logarithm of the extents,
relative to the field's largest entry (measured on 8^4: 1.6e-7, 2.4e-7, 1.5e-7);
the tests allow 5e-6 (g: absolute; theta 5e-6 and F 1e-6 relative).
"""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1301_3460_gb300 import inputs
from paper_1301_3460_gb300 import lgf

pytestmark = pytest.mark.gpu

# short lines (the FP32 kernels for lines <= 32), radix 3, ragged extents, and
# the general kernels (a 48- and a 64-point axis)
SHAPES = [(8, 8, 8, 8), (12, 8, 6, 4), (16, 12, 8, 24), (8, 16, 32, 4), (48, 8, 4, 6), (4, 6, 64, 8)]


def field(L, eps=0.4, seed=7):
    return inputs.rough_gauge_field(L, eps, seed)


@pytest.mark.parametrize("L", SHAPES)
@pytest.mark.parametrize("fused", [False, True])
def test_delta32(L, fused):
    U = field(L, seed=21)
    Do, tho, Fo = orc.delta(L, U)
    with lgf.Lattice(L, mixed=True) as lat:
        lat.set_fp32_update(fused)
        lat.set_links(U)
        D, th, F = lat.delta(precision=32)
        # the FP64 stage of the same context is unaffected by the FP32 one
        D64, _, _ = lat.delta()
    scale = np.max(np.abs(Do))
    assert np.max(np.abs(D - Do)) < 5e-6 * scale
    assert th == pytest.approx(tho, rel=5e-6)
    assert F == pytest.approx(Fo, rel=1e-6)
    assert np.max(np.abs(D64 - Do)) < 1e-13


@pytest.mark.parametrize("L", SHAPES)
def test_accelerate32(L):
    U = field(L, seed=22)
    Do, _, _ = orc.delta(L, U)
    want = orc.accelerate(L, Do)
    with lgf.Lattice(L, mixed=True) as lat:
        got = lat.accelerate(Do, precision=32)
    assert np.max(np.abs(got - want)) < 5e-6 * np.max(np.abs(want))


@pytest.mark.parametrize("L", SHAPES)
@pytest.mark.parametrize("alpha", [0.08, 0.3])
def test_build_g32(L, alpha):
    U = field(L, seed=23)
    Do, _, _ = orc.delta(L, U)
    Dt = orc.accelerate(L, Do)
    want = orc.build_g(L, Dt, alpha)
    with lgf.Lattice(L, mixed=True) as lat:
        got = lat.build_g(Dt, alpha, precision=32)
    assert np.max(np.abs(got - want)) < 5e-6
    # unitary and of unit determinant to FP32 rounding
    eye = np.eye(3)
    assert np.max(np.abs(got @ np.conj(np.swapaxes(got, -1, -2)) - eye)) < 2e-6
    assert np.max(np.abs(np.linalg.det(got) - 1)) < 2e-6


def test_fp32_stages_need_a_mixed_context():
    L = (4, 4, 4, 4)
    U = field(L)
    with lgf.Lattice(L) as lat:
        lat.set_links(U)
        D = np.zeros((lat.V, 3, 3), dtype=np.complex128)
        for call in (lambda: lat.delta(precision=32), lambda: lat.accelerate(D, precision=32),
                     lambda: lat.build_g(D, 0.08, precision=32)):
            with pytest.raises(lgf.LgfError) as e:
                call()
            assert e.value.status == lgf.LGF_ERR_STATE
        with pytest.raises(ValueError):
            lat.delta(precision=16)
    with lgf.Lattice(L, mixed=True) as lat:  # no links yet
        with pytest.raises(lgf.LgfError) as e:
            lat.delta(precision=32)
        assert e.value.status == lgf.LGF_ERR_STATE
