"""The integer-pipe float/double conversions used by the FP32 phase's g builder,
bit for bit against the hardware conversions (torch's CUDA casts)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _edge_doubles():
    """Binary64 patterns at the edges of the binary32 rounding: ties to even with
    an even and an odd kept fraction, one unit either side of a tie, carries out
    of the fraction into the exponent, the largest binade (overflow to infinity),
    the exponent limits of binary32 normals and subnormals, zeros, infinities, NaN."""
    out = []
    for sign in (0, 1):
        for E in (1, 500, 873, 874, 896, 897, 898, 1000, 1023, 1100, 1149, 1150, 1151, 1152, 2046):
            for m23 in (0, 1, 2, 0x3FFFFE, 0x3FFFFF, 0x7FFFFE, 0x7FFFFF, 0x555555, 0x2AAAAA):
                for rest in (0, 1, 0x0FFFFFFF, 0x10000000, 0x10000001, 0x1FFFFFFF):
                    frac = (m23 << 29) | rest
                    out.append((sign << 63) | (E << 52) | frac)
        out += [(sign << 63), (sign << 63) | (0x7FF << 52), (sign << 63) | (0x7FF << 52) | 1,
                (sign << 63) | 1, (sign << 63) | ((1 << 52) - 1)]
    return np.array(out, dtype=np.uint64)


def _edge_floats():
    out = []
    for sign in (0, 1):
        for e in (0, 1, 2, 126, 127, 128, 253, 254, 255):
            for m in (0, 1, 2, 7, 8, 0x3FFFFF, 0x400000, 0x7FFFFF):
                out.append((sign << 31) | (e << 23) | m)
    return np.array(out, dtype=np.uint32)


def test_conversions_match_hardware():
    import torch

    from paper_1301_3460_gb300 import lgf

    rng = np.random.default_rng(20240611)
    n_rand = 1 << 22
    # random binary64 patterns over every exponent, and values in the range the
    # g builder sees (|x| <= 1, many binades below 1)
    d_bits = np.concatenate([
        rng.integers(0, np.iinfo(np.uint64).max, size=n_rand, dtype=np.uint64, endpoint=True),
        rng.uniform(-1.0, 1.0, size=n_rand).view(np.uint64),
        (rng.uniform(-1.0, 1.0, size=n_rand) * np.exp2(-rng.integers(0, 140, size=n_rand))).view(np.uint64),
        _edge_doubles(),
    ])
    f_bits = np.concatenate([
        rng.integers(0, np.iinfo(np.uint32).max, size=d_bits.size - _edge_floats().size, dtype=np.uint32,
                     endpoint=True),
        _edge_floats(),
    ])
    assert f_bits.size == d_bits.size
    d_in = torch.from_numpy(d_bits.view(np.float64)).cuda()
    f_in = torch.from_numpy(f_bits.view(np.float32)).cuda()
    f_out, d_out = lgf.check_conversions(d_in, f_in)
    torch.cuda.synchronize()
    f_ref = d_in.to(torch.float32)
    d_ref = f_in.to(torch.float64)
    # compare encodings; a NaN result must be a NaN on both sides
    fo, fr = f_out.view(torch.int32), f_ref.view(torch.int32)
    bad_f = (fo != fr) & ~(torch.isnan(f_out) & torch.isnan(f_ref))
    do, dr = d_out.view(torch.int64), d_ref.view(torch.int64)
    bad_d = (do != dr) & ~(torch.isnan(d_out) & torch.isnan(d_ref))
    nf, nd = int(bad_f.sum()), int(bad_d.sum())
    if nf:
        i = int(torch.nonzero(bad_f)[0])
        pytest.fail("double->float differs on %d of %d, first %r -> %r (hardware %r)"
                    % (nf, d_in.numel(), float(d_in[i]), float(f_out[i]), float(f_ref[i])))
    if nd:
        i = int(torch.nonzero(bad_d)[0])
        pytest.fail("float->double differs on %d of %d, first %r -> %r (hardware %r)"
                    % (nd, f_in.numel(), float(f_in[i]), float(d_out[i]), float(d_ref[i])))


def test_conversions_argument_errors():
    import torch

    from paper_1301_3460_gb300 import lgf

    with pytest.raises(TypeError):
        lgf.check_conversions(torch.zeros(4, dtype=torch.float32, device="cuda"),
                              torch.zeros(4, dtype=torch.float32, device="cuda"))
    with pytest.raises(TypeError):
        lgf.check_conversions(torch.zeros(4, dtype=torch.float64, device="cuda"),
                              torch.zeros(3, dtype=torch.float32, device="cuda"))
    f_out, d_out = lgf.check_conversions(torch.zeros(0, dtype=torch.float64, device="cuda"),
                                         torch.zeros(0, dtype=torch.float32, device="cuda"))
    assert f_out.numel() == 0 and d_out.numel() == 0
