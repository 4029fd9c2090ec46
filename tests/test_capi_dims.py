"""lgf_create's checks of its arguments, on the CPU: the extents and the tile
limits that include/lgf.h documents are the ones the library applies, and
argument errors are status codes.  Without a GPU an accepted lattice fails
later, with LGF_ERR_CUDA; the test is skipped where a GPU would let it allocate."""
import ctypes
import itertools

import pytest

from paper_1301_3460_gb300 import lgf

LENGTHS = (4, 6, 8, 12, 16, 24, 32, 48, 64, 96, 128)


def create(dims, flags=lgf.LGF_FP64):
    lib = lgf.load()
    d = (ctypes.c_int * 4)(*dims)
    h = ctypes.c_void_p()
    st = lib.lgf_create(d, flags, ctypes.byref(h))
    if st == lgf.LGF_OK:
        lib.lgf_destroy(h)
    return st


@pytest.fixture(scope="module", autouse=True)
def no_gpu():
    if create((4, 4, 4, 4)) != lgf.LGF_ERR_CUDA:
        pytest.skip("a usable GPU is present: accepted lattices would be allocated")


def documented_ok(L):
    """The header's rule: every extent in LENGTHS, Ly*(Lx + 1) <= 3520,
    Lt*(3 Lz + 2) <= 28160, and 24 V within a signed 32-bit offset."""
    Lx, Ly, Lz, Lt = L
    V = Lx * Ly * Lz * Lt
    return Ly * (Lx + 1) <= 3520 and Lt * (3 * Lz + 2) <= 28160 and 24 * V <= 2**31 - 1


def test_every_supported_extent_combination():
    bad = []
    for L in itertools.product(LENGTHS, repeat=4):
        want = lgf.LGF_ERR_CUDA if documented_ok(L) else lgf.LGF_ERR_UNSUPPORTED_DIMS
        for flags in (lgf.LGF_FP64, lgf.LGF_MIXED):
            st = create(L, flags)
            if st != want:
                bad.append((L, flags, st))
    assert not bad, bad[:10]


@pytest.mark.parametrize("L", [(10, 8, 8, 8), (8, 8, 8, 0), (8, -4, 8, 8), (256, 4, 4, 4), (8, 8, 2, 8),
                               (8, 8, 8, 20)])
def test_unsupported_lengths(L):
    assert create(L) == lgf.LGF_ERR_UNSUPPORTED_DIMS


def test_argument_errors():
    lib = lgf.load()
    h = ctypes.c_void_p()
    d = (ctypes.c_int * 4)(8, 8, 8, 8)
    assert lib.lgf_create(None, 0, ctypes.byref(h)) == lgf.LGF_ERR_ARG
    assert lib.lgf_create(d, 0, None) == lgf.LGF_ERR_ARG
    assert create((8, 8, 8, 8), 1 << 10) == lgf.LGF_ERR_ARG
    assert create((8, 8, 8, 8), lgf.LGF_LINKS18 | lgf.LGF_LINKS8) == lgf.LGF_ERR_ARG
    # calls on a null context are argument errors, not crashes
    assert lib.lgf_fix(None, 0.08, 1e-15, 10, None, None, None) == lgf.LGF_ERR_ARG
    assert lib.lgf_set_links(None, None, 0) == lgf.LGF_ERR_ARG
    assert lib.lgf_get_links(None, None, 0) == lgf.LGF_ERR_ARG
    lib.lgf_destroy(None)


def test_noalloc_limits():
    """lgf_accelerate_noalloc takes the extents of lgf_create up to V = 65536
    sites; larger lattices are refused before any CUDA call."""
    lib = lgf.load()
    buf = (ctypes.c_double * 2)()
    bad = []
    for L in itertools.product(LENGTHS, repeat=4):
        V = L[0] * L[1] * L[2] * L[3]
        if V > 4 * 65536:
            continue
        want = lgf.LGF_ERR_CUDA if (documented_ok(L) and V <= 65536) else lgf.LGF_ERR_UNSUPPORTED_DIMS
        st = lib.lgf_accelerate_noalloc((ctypes.c_int * 4)(*L), buf, buf, None)
        if st != want:
            bad.append((L, st))
    assert not bad, bad[:10]
    assert lib.lgf_accelerate_noalloc(None, buf, buf, None) == lgf.LGF_ERR_ARG


def test_batch_create_checks_every_member():
    lib = lgf.load()
    h = ctypes.c_void_p()

    def batch(dims_list, flags=lgf.LGF_MIXED):
        flat = (ctypes.c_int * (4 * len(dims_list)))(*[v for d in dims_list for v in d])
        return lib.lgf_batch_create(len(dims_list), flat, flags, ctypes.byref(h))

    # members are created in order and the first failure is returned: without a
    # GPU an accepted member fails with LGF_ERR_CUDA, so refused extents go first
    assert batch([(8, 8, 8, 8), (16, 16, 16, 16)]) == lgf.LGF_ERR_CUDA
    assert batch([(10, 16, 16, 16), (8, 8, 8, 8)]) == lgf.LGF_ERR_UNSUPPORTED_DIMS
    assert batch([(128, 128, 8, 8), (8, 8, 8, 8)]) == lgf.LGF_ERR_UNSUPPORTED_DIMS
    assert batch([(8, 8, 8, 8)], flags=1 << 10) == lgf.LGF_ERR_ARG
    assert lib.lgf_batch_create(0, (ctypes.c_int * 4)(8, 8, 8, 8), 0, ctypes.byref(h)) == lgf.LGF_ERR_ARG
