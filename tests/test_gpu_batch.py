"""Batched ensembles: lattices of different extents and uneven convergence fixed
by one graph launch; each result must equal what the FP64 oracle gives for that
lattice alone (mixed mode: to the mixed-precision tolerances), and each lattice
retires on its own."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1301_3460_gb300 import inputs
from paper_1301_3460_gb300 import lgf

pytestmark = pytest.mark.gpu

ENSEMBLE = [((8, 8, 8, 8), 0.3, 101), ((8, 8, 8, 8), 0.5, 102), ((12, 12, 8, 8), 0.15, 103),
            ((16, 16, 16, 16), 0.3, 104), ((8, 8, 8, 12), 0.4, 105), ((12, 12, 8, 8), 0.3, 106)]


def _fields():
    return [inputs.rough_gauge_field(L, e, s) for L, e, s in ENSEMBLE]


@pytest.mark.parametrize("mixed", [False, True])
def test_batch_against_oracle(mixed):
    U = _fields()
    refs = [orc.fix(L, u, alpha=0.08, tol=1e-15, max_iter=5000) for (L, _, _), u in zip(ENSEMBLE, U)]
    with lgf.Batch([L for L, _, _ in ENSEMBLE], mixed=mixed) as b:
        for i, u in enumerate(U):
            b.set_links(i, u)
        r = b.fix(alpha=0.08, tol=1e-15, max_iter=5000)
        links = [b.get_links(i) for i in range(len(U))]
        gauges = [b.get_gauge(i) for i in range(len(U))]
    assert r["rc"] == lgf.LGF_OK and all(s == lgf.LGF_OK for s in r["status"])
    for i, ((L, _, _), u, ref) in enumerate(zip(ENSEMBLE, U, refs)):
        assert r["theta"][i] < 1e-15
        assert r["F"][i] == pytest.approx(ref["F"], rel=1e-12)
        np.testing.assert_allclose(orc.gauge_transform(L, u, gauges[i]), links[i], atol=1e-13)
        if not mixed:
            assert abs(r["iters"][i] - ref["iters"]) <= 1
            assert np.max(np.abs(links[i] - ref["U"])) < 1e-11
        else:
            assert r["iters_fp32"][i] > 0
            assert np.max(np.abs(links[i] - ref["U"])) < 1e-4
    t = np.array(r["t_retire_ms"])
    assert np.all(t > 0)


def test_batch_retires_converged_lattices_first():
    """A lattice already in Landau gauge (U = 1) retires at once, before the others."""
    dims = [(8, 8, 8, 8), (16, 16, 16, 16), (8, 8, 8, 8)]
    U = [inputs.unit_field(dims[0]), inputs.rough_gauge_field(dims[1], 0.3, 7), inputs.rough_gauge_field(dims[2], 0.3, 8)]
    with lgf.Batch(dims, mixed=True) as b:
        for i, u in enumerate(U):
            b.set_links(i, u)
        r = b.fix(tol=1e-15, max_iter=5000)
    assert r["iters"][0] == 0 and r["F"][0] == 1.0
    assert r["t_retire_ms"][0] < r["t_retire_ms"][1]
    assert all(s == lgf.LGF_OK for s in r["status"])


def test_batch_max_iter_status():
    dims = [(8, 8, 8, 8), (8, 8, 8, 8)]
    with lgf.Batch(dims, mixed=False) as b:
        b.set_links(0, inputs.rough_gauge_field(dims[0], 0.3, 9))
        b.set_links(1, inputs.unit_field(dims[1]))
        r = b.fix(tol=1e-15, max_iter=3)
    assert r["rc"] == lgf.LGF_ERR_NOT_CONVERGED
    assert r["status"] == [lgf.LGF_ERR_NOT_CONVERGED, lgf.LGF_OK] and r["iters"] == [3, 0]


def test_autotune_keeps_results():
    L = (16, 12, 8, 24)
    U = inputs.rough_gauge_field(L, 0.3, 12)
    ref = orc.fix(L, U, alpha=0.08, tol=0.0, max_iter=10)
    with lgf.Lattice(L, mixed=True) as lat:
        lat.set_links(U)
        lat.autotune()
        lat.set_links(U)
        lat.fix(tol=0.0, max_iter=10)
        Um = lat.get_links()
    with lgf.Lattice(L) as lat:
        lat.set_links(U)
        lat.autotune()
        lat.set_links(U)
        lat.fix(tol=0.0, max_iter=10)
        U64 = lat.get_links()
    assert np.max(np.abs(U64 - ref["U"])) < 1e-13
    # mixed: 10 steps in the FP32 phase, then the links are re-projected in FP64
    assert np.max(np.abs(Um - ref["U"])) < 1e-4


def test_cuda_generator_is_su3():
    pytest.importorskip("torch")
    L = (8, 8, 4, 4)
    U = inputs.rough_gauge_field_cuda(L, 0.3, 3).cpu().numpy()
    uu = np.einsum("msij,mskj->msik", U, U.conj())
    assert np.max(np.abs(uu - np.eye(3))) < 1e-12
    assert np.max(np.abs(np.linalg.det(U) - 1)) < 1e-12
    with lgf.Lattice(L) as lat:
        lat.set_links(U)
        assert lat.fix(tol=1e-15, max_iter=3000)["converged"]


def test_full_ensemble():
    """The benchmark's ensemble at full size (32 x 16^4, 16 x 24^4, 8 x 32^3x64,
    2 x 48^3x96, eps uniform in [0.15, 0.5], mixed precision, one graph launch):
    every lattice converges; a 16^4 and a 24^4 member agree with the FP64 oracle;
    the 32^3x64 members' links are the gauge transform of their inputs by G."""
    torch = pytest.importorskip("torch")
    sizes = ((32, (16, 16, 16, 16)), (16, (24, 24, 24, 24)), (8, (32, 32, 32, 64)), (2, (48, 48, 48, 96)))
    dims = [d for n, d in sizes for _ in range(n)]
    eps = np.random.default_rng(5000).uniform(0.15, 0.5, size=len(dims))
    dev = [inputs.rough_gauge_field_cuda(d, float(e), 5000 + i) for i, (d, e) in enumerate(zip(dims, eps))]
    with lgf.Batch(dims, mixed=True) as b:
        for i, u in enumerate(dev):
            b.set_links(i, u)
        r = b.fix(alpha=0.08, tol=1e-15, max_iter=20000)
        assert all(s == lgf.LGF_OK for s in r["status"]) and r["rc"] == lgf.LGF_OK
        assert max(r["theta"]) < 1e-15
        for i in (0, 32):
            L, U = dims[i], dev[i].cpu().numpy()
            ref = orc.fix(L, U, alpha=0.08, tol=1e-15, max_iter=5000)
            assert r["F"][i] == pytest.approx(ref["F"], rel=1e-12)
            np.testing.assert_allclose(orc.gauge_transform(L, U, b.get_gauge(i)), b.get_links(i), atol=1e-13)
        for i in (48, 55):
            L = dims[i]
            np.testing.assert_allclose(orc.gauge_transform(L, dev[i].cpu().numpy(), b.get_gauge(i)),
                                       b.get_links(i), atol=1e-13)
    del dev
    torch.cuda.empty_cache()
