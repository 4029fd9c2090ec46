"""The t-slab decomposition of one lattice over several ranks (paper_1301_3460_gb300
/slabs.py), on CPU with the gloo backend, world size 2: the halo planes are the
neighbouring slabs' boundary planes; the Delta stencil and the update computed
slab by slab with those halos equal the oracle's on the whole lattice; and the
accelerator run as x,y,z transforms on t-slabs, a transpose to z-slabs, the t
transform with the multiplier, and the transpose back equals the accelerator of
the whole field and the single-rank run of the same steps."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

L = (6, 4, 4, 8)  # Lx, Ly, Lz, Lt; Lz and Lt divisible by the world size


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def multiplier(dims):
    """p2max / p2(k) on [Lt, Lz, Ly, Lx], zero mode 0 (the accelerator before 1/V)."""
    Lx, Ly, Lz, Lt = dims
    s2 = [4 * np.sin(np.pi * np.arange(n) / n) ** 2 for n in (Lx, Ly, Lz, Lt)]
    p2 = s2[3][:, None, None, None] + s2[2][None, :, None, None] + s2[1][None, None, :, None] + s2[0][None, None, None, :]
    p2max = sum(v.max() for v in s2)
    return np.where(p2 > 0, p2max / np.where(p2 > 0, p2, 1.0), 0.0)


def fields(seed=5):
    Lx, Ly, Lz, Lt = L
    rng = np.random.default_rng(seed)
    return rng.standard_normal((4, Lt, Lz, Ly, Lx)) + 1j * rng.standard_normal((4, Lt, Lz, Ly, Lx))


def accelerate_slabs(sl, local, rank, M, group=None):
    """The accelerator on t-slabs: x,y,z transforms, t_to_z, t transform, multiplier,
    inverse t transform, z_to_t, inverse x,y,z transforms (numpy normalisation:
    the inverse transforms divide by the length)."""
    f = torch.fft.fftn(local, dim=(2, 3, 4))
    z = sl.t_to_z(f, group)
    z = torch.fft.fft(z, dim=1)
    z0, z1 = sl.z_range(rank)
    z = z * torch.from_numpy(M[:, z0:z1])[None]
    z = torch.fft.ifft(z, dim=1)
    f = sl.z_to_t(z, group)
    return torch.fft.ifftn(f, dim=(2, 3, 4))


def site_array(U, dims):
    """[4, V, 3, 3] -> [4, Lt, Lz, Ly, Lx, 3, 3]"""
    Lx, Ly, Lz, Lt = dims
    return U.reshape(4, Lt, Lz, Ly, Lx, 3, 3)


def dag(m):
    return np.conj(np.swapaxes(m, -1, -2))


def row2(m):
    """rows 0,1 kept, row 2 rebuilt as conj(row0 x row1) (the 12-real form)"""
    out = m.copy()
    out[..., 2, :] = np.conj(np.cross(m[..., 0, :], m[..., 1, :]))
    return out


def _worker(rank, world, port, out):
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    from oracle import oracle as orc
    from paper_1301_3460_gb300 import inputs
    from paper_1301_3460_gb300.slabs import TSlabs

    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    sl = TSlabs(L, world)
    t0, t1 = sl.t_range(rank)
    Lx, Ly, Lz, Lt = L
    res = {}

    # halo planes of a field
    G = fields()
    prev, nxt = sl.halo_planes(torch.from_numpy(G[:, t0:t1].copy()), rank)
    res["halo"] = max(np.abs(prev.numpy() - G[:, (t0 - 1) % Lt]).max(), np.abs(nxt.numpy() - G[:, t1 % Lt]).max())

    # accelerator through the transposes
    M = multiplier(L)
    got = accelerate_slabs(sl, torch.from_numpy(G[:, t0:t1].copy()), rank, M).numpy()
    want = np.fft.ifftn(M[None] * np.fft.fftn(G, axes=(1, 2, 3, 4)), axes=(1, 2, 3, 4))[:, t0:t1]
    res["accelerate"] = np.abs(got - want).max() / np.abs(want).max()

    # Delta with the previous slab's t-links as halo
    U = inputs.rough_gauge_field(L, 0.4, 61)
    Us = site_array(U, L)
    loc = Us[:, t0:t1]  # [4, nt, Lz, Ly, Lx, 3, 3]
    ut = torch.from_numpy(np.ascontiguousarray(loc[3].reshape(loc.shape[1:4] + (Lx, 9)).transpose(4, 0, 1, 2, 3)))
    prev_t, _ = sl.halo_planes(ut, rank)
    prev_t = prev_t.numpy().transpose(1, 2, 3, 0).reshape(Lz, Ly, Lx, 3, 3)
    Mx = np.zeros(loc.shape[1:], complex)
    for mu, ax in ((0, 3), (1, 2), (2, 1)):  # x, y, z inside the slab (axes of [nt, Lz, Ly, Lx])
        Mx += np.roll(loc[mu], 1, axis=ax) - loc[mu]
    Mx += np.concatenate([prev_t[None], loc[3][:-1]], axis=0) - loc[3]
    A = Mx - dag(Mx)
    D = A - np.trace(A, axis1=-2, axis2=-1)[..., None, None] / 3 * np.eye(3)
    Dref = orc.delta(L, U)[0].reshape(Lt, Lz, Ly, Lx, 3, 3)[t0:t1]
    res["delta"] = np.abs(D - Dref).max()

    # the update with the next slab's g as halo
    Dt = orc.accelerate(L, orc.delta(L, U)[0])
    g = orc.build_g(L, Dt, 0.08).reshape(Lt, Lz, Ly, Lx, 3, 3)
    gl = g[t0:t1]
    gt = torch.from_numpy(np.ascontiguousarray(gl.reshape(gl.shape[:4] + (9,)).transpose(4, 0, 1, 2, 3)))
    _, next_g = sl.halo_planes(gt, rank)
    next_g = next_g.numpy().transpose(1, 2, 3, 0).reshape(Lz, Ly, Lx, 3, 3)
    Unew = np.empty_like(loc)
    for mu, ax in ((0, 3), (1, 2), (2, 1)):
        Unew[mu] = row2(gl @ loc[mu] @ dag(np.roll(gl, -1, axis=ax)))
    gnext = np.concatenate([gl[1:], next_g[None]], axis=0)
    Unew[3] = row2(gl @ loc[3] @ dag(gnext))
    G1 = np.zeros((Lt * Lz * Ly * Lx, 3, 3), complex)
    G1[:, 0, 0] = G1[:, 1, 1] = G1[:, 2, 2] = 1
    Uref, _ = orc.update(L, U, G1, g.reshape(-1, 3, 3))
    res["update"] = np.abs(Unew - site_array(Uref, L)[:, t0:t1]).max()

    out[rank] = res
    dist.barrier()
    dist.destroy_process_group()


def test_slab_decomposition_two_gloo_ranks():
    from oracle import oracle as orc

    orc.build()
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        assert res[r]["halo"] == 0.0
        assert res[r]["accelerate"] < 1e-13
        assert res[r]["delta"] < 1e-13
        assert res[r]["update"] < 1e-13


def test_single_rank_matches_the_slabs():
    """The same steps with one rank (no exchange) give the whole-field accelerator."""
    from paper_1301_3460_gb300.slabs import TSlabs

    G = fields(9)
    M = multiplier(L)
    got = accelerate_slabs(TSlabs(L, 1), torch.from_numpy(G), 0, M).numpy()
    want = np.fft.ifftn(M[None] * np.fft.fftn(G, axes=(1, 2, 3, 4)), axes=(1, 2, 3, 4))
    assert np.abs(got - want).max() / np.abs(want).max() < 1e-13


def test_slab_extents_must_divide():
    from paper_1301_3460_gb300.slabs import TSlabs

    with pytest.raises(ValueError):
        TSlabs((4, 4, 6, 8), 4)
