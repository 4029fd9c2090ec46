"""lgf_accelerate_noalloc, the accelerator for callers that cannot let a library
allocate device memory (all of their GPU memory belongs to their own allocator:
a framework's caching pool, or a runtime with one fixed arena).  Checked through
the C ABI against the oracle's accelerator and against lgf_accelerate, on two
calls in a row that share the library's static scratch.

Kept in a file that pytest collects last, so that a run stopping at the first
failure has already run every other test."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1301_3460_gb300 import inputs
from paper_1301_3460_gb300 import lgf

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("L", [(8, 8, 8, 8), (12, 8, 6, 4), (16, 16, 16, 16)])
def test_noalloc_matches_oracle_and_accelerate_twice(L):
    torch = pytest.importorskip("torch")
    V = int(np.prod(L))
    D = [orc.delta(L, inputs.rough_gauge_field(L, 0.4, seed))[0] for seed in (21, 22)]
    with lgf.Lattice(L) as lat:
        want = [lat.accelerate(x) for x in D]
    stream = torch.cuda.current_stream()
    for x, w in zip(D, want):  # two calls in a row share the static scratch
        ref = orc.accelerate(L, x)
        din = torch.from_numpy(x).cuda()
        out = torch.zeros((V, 3, 3), dtype=torch.complex128, device="cuda")
        lgf.lgf_accelerate_noalloc(L, din, out, stream)
        got = out.cpu().numpy()
        scale = max(1.0, np.max(np.abs(ref)))
        assert np.max(np.abs(got - ref)) < 1e-13 * scale
        assert np.max(np.abs(got - w)) < 1e-13 * scale


def test_noalloc_allocates_no_device_memory():
    torch = pytest.importorskip("torch")
    Ls = [(8, 8, 8, 8), (16, 8, 12, 4)]
    bufs = []
    for L in Ls:
        V = int(np.prod(L))
        x = orc.delta(L, inputs.rough_gauge_field(L, 0.3, 31))[0]
        bufs.append((L, torch.from_numpy(x).cuda(), torch.empty((V, 3, 3), dtype=torch.complex128, device="cuda")))
    # warm-up on every extent: the first-call set-up, and the CUDA runtime loading
    # kernel code lazily at a kernel's first launch
    for L, din, out in bufs:
        lgf.lgf_accelerate_noalloc(L, din, out)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(2):
        for L, din, out in bufs:  # alternating extents
            lgf.lgf_accelerate_noalloc(L, din, out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_rejects_lattices_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    L = (32, 16, 16, 16)  # 131072 sites > 65536
    V = int(np.prod(L))
    x = torch.zeros((V, 3, 3), dtype=torch.complex128, device="cuda")
    with pytest.raises(lgf.LgfError) as e:
        lgf.lgf_accelerate_noalloc(L, x, x.clone())
    assert e.value.status == lgf.LGF_ERR_UNSUPPORTED_DIMS


def test_noalloc_refuses_other_dtypes_before_the_library():
    torch = pytest.importorskip("torch")
    L = (8, 8, 8, 8)
    V = int(np.prod(L))
    good = torch.zeros((V, 3, 3), dtype=torch.complex128, device="cuda")
    for bad in (torch.zeros((V, 3, 3), dtype=torch.complex64, device="cuda"),
                torch.zeros((V, 3, 3), dtype=torch.float64, device="cuda")):
        with pytest.raises(TypeError):
            lgf.lgf_accelerate_noalloc(L, bad, good)
        with pytest.raises(TypeError):
            lgf.lgf_accelerate_noalloc(L, good, bad)
    with pytest.raises(ValueError):
        lgf.lgf_accelerate_noalloc(L, good[:-1], good)
