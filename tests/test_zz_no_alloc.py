"""lgf_accelerate_noalloc (the entry point for callers whose device memory is
all owned by their own allocator) against lgf_accelerate, through the C ABI.

Kept in a file that pytest collects last, so that a run stopping at the first
failure has already run every other test."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1301_3460_gb300 import inputs
from paper_1301_3460_gb300 import lgf

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("L", [(8, 8, 8, 8), (12, 8, 6, 4), (16, 16, 16, 16)])
def test_noalloc_matches_accelerate_twice(L):
    torch = pytest.importorskip("torch")
    V = int(np.prod(L))
    D = [orc.delta(L, inputs.rough_gauge_field(L, 0.4, seed))[0] for seed in (21, 22)]
    with lgf.Lattice(L) as lat:
        want = [lat.accelerate(x) for x in D]
    stream = torch.cuda.current_stream()
    for x, w in zip(D, want):  # two calls in a row share the static scratch
        din = torch.from_numpy(x).cuda()
        out = torch.zeros((V, 3, 3), dtype=torch.complex128, device="cuda")
        lgf.lgf_accelerate_noalloc(L, din, out, stream)
        got = out.cpu().numpy()
        assert np.max(np.abs(got - w)) < 1e-13 * max(1.0, np.max(np.abs(w)))


def test_noalloc_rejects_lattices_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    L = (32, 16, 16, 16)  # 131072 sites > 65536
    V = int(np.prod(L))
    x = torch.zeros((V, 3, 3), dtype=torch.complex128, device="cuda")
    with pytest.raises(lgf.LgfError) as e:
        lgf.lgf_accelerate_noalloc(L, x, x.clone())
    assert e.value.status == lgf.LGF_ERR_UNSUPPORTED_DIMS
