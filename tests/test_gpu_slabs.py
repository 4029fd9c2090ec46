"""One lattice over several ranks on the GPU: the lgf_slab_* entry points and the
slab driver (paper_1301_3460_gb300.slabs), against the oracle's whole-lattice
iteration at the single-GPU tolerances (links and G to 1e-13 after 1 and 10
steps; a whole fix: iteration count, F to 1e-12 relative, links to 1e-11).

The ranks run as slabs of one process on one GPU (LocalExchange: device copies
in place of the messages), and as two processes sharing the GPU over a gloo
group (DistExchange with the exchanges staged through host memory); in both,
every exchange happens on the host between kernel launches, and no kernel waits
on another rank's.
"""
import os
import tempfile

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1301_3460_gb300 import inputs, lgf
from paper_1301_3460_gb300.slabs import DistExchange, LocalExchange, Slab, fix_slabs

pytestmark = pytest.mark.gpu

# ranks dividing Lt and Lz; a 48-point z axis and a 64-point t axis run the
# lines split over lanes
CASES = [((8, 8, 8, 8), 1), ((8, 8, 8, 8), 2), ((8, 8, 8, 8), 4), ((12, 8, 8, 16), 2), ((12, 8, 8, 16), 4),
         ((8, 8, 16, 4), 2), ((8, 8, 48, 64), 2)]


def split(U, N):
    import torch

    Vs = U.shape[1] // N
    return [torch.from_numpy(np.ascontiguousarray(U[:, r * Vs:(r + 1) * Vs])).cuda() for r in range(N)]


def run_local(L, N, U, tol, max_iter):
    import torch

    slabs = [Slab(L, N, r) for r in range(N)]
    try:
        for s, u in zip(slabs, split(U, N)):
            s.set_links(u)
        r = fix_slabs(LocalExchange(slabs), alpha=0.08, tol=tol, max_iter=max_iter)
        Ug = torch.cat([s.get_links() for s in slabs], dim=1).cpu().numpy()
        Gg = torch.cat([s.get_gauge() for s in slabs], dim=0).cpu().numpy()
    finally:
        for s in slabs:
            s.close()
    return r, Ug, Gg


@pytest.mark.parametrize("L,N", CASES)
@pytest.mark.parametrize("steps", [1, 10])
def test_slabs_steps_match_oracle(L, N, steps):
    U = inputs.rough_gauge_field(L, 0.3, 31)
    ref = orc.fix(L, U, alpha=0.08, tol=0.0, max_iter=steps)
    r, Ug, Gg = run_local(L, N, U, 0.0, steps)
    assert r["iters"] == steps
    assert np.max(np.abs(Ug - ref["U"])) < 1e-13
    assert np.max(np.abs(Gg - ref["G"])) < 1e-13
    assert r["F"] == pytest.approx(ref["F"], rel=1e-12)
    assert r["theta"] == pytest.approx(ref["theta"], rel=1e-10)


@pytest.mark.parametrize("L,N", [((8, 8, 8, 8), 2), ((12, 8, 8, 16), 4)])
def test_slabs_fix_like_oracle(L, N):
    U = inputs.rough_gauge_field(L, 0.3, 32)
    ref = orc.fix(L, U, alpha=0.08, tol=1e-15, max_iter=500, history=True)
    r, Ug, _ = run_local(L, N, U, 1e-15, 500)
    assert ref["converged"] and r["converged"] and r["theta"] < 1e-15
    if r["iters"] != ref["iters"]:
        n = min(r["iters"], ref["iters"])
        assert abs(r["iters"] - ref["iters"]) == 1 and abs(ref["history"][n, 0] / 1e-15 - 1) < 1e-10
    assert r["F"] == pytest.approx(ref["F"], rel=1e-12)
    assert np.max(np.abs(Ug - ref["U"])) < 1e-11


def _dist_worker(rank, world, port, L, steps, outdir):
    import datetime

    import torch
    import torch.distributed as dist

    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=120))
    try:
        torch.cuda.set_device(0)
        U = inputs.rough_gauge_field(L, 0.3, 33)
        slab = Slab(L, world, rank)
        try:
            slab.set_links(split(U, world)[rank])
            r = fix_slabs(DistExchange(slab, staged=True), alpha=0.08, tol=0.0, max_iter=steps)
            np.save(os.path.join(outdir, "U%d.npy" % rank), slab.get_links().cpu().numpy())
            np.save(os.path.join(outdir, "G%d.npy" % rank), slab.get_gauge().cpu().numpy())
            np.save(os.path.join(outdir, "r%d.npy" % rank), np.array([r["iters"], r["theta"], r["F"]]))
        finally:
            slab.close()
    finally:
        dist.destroy_process_group()


def test_slabs_over_a_process_group():
    import socket

    import torch.multiprocessing as mp

    L, world, steps = (8, 8, 8, 8), 2, 10
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    with tempfile.TemporaryDirectory() as d:
        mp.start_processes(_dist_worker, args=(world, port, L, steps, d), nprocs=world, join=True,
                           start_method="spawn")
        Ug = np.concatenate([np.load(os.path.join(d, "U%d.npy" % r)) for r in range(world)], axis=1)
        Gg = np.concatenate([np.load(os.path.join(d, "G%d.npy" % r)) for r in range(world)], axis=0)
        res = [np.load(os.path.join(d, "r%d.npy" % r)) for r in range(world)]
    U = inputs.rough_gauge_field(L, 0.3, 33)
    ref = orc.fix(L, U, alpha=0.08, tol=0.0, max_iter=steps)
    assert all(int(x[0]) == steps for x in res)
    assert np.max(np.abs(Ug - ref["U"])) < 1e-13
    assert np.max(np.abs(Gg - ref["G"])) < 1e-13
    assert res[0][2] == pytest.approx(ref["F"], rel=1e-12) and res[1][2] == res[0][2]


def test_slab_errors():
    import torch

    with pytest.raises(lgf.LgfError) as e:
        Slab((8, 8, 8, 12), 8, 0)  # Lt not a multiple of the ranks
    assert e.value.status == lgf.LGF_ERR_UNSUPPORTED_DIMS
    with pytest.raises(lgf.LgfError) as e:
        Slab((8, 8, 8, 8), 2, 2)  # no such rank
    assert e.value.status == lgf.LGF_ERR_ARG
    s = Slab((8, 8, 8, 8), 2, 1)
    try:
        with pytest.raises(lgf.LgfError) as e:
            s.delta()
        assert e.value.status == lgf.LGF_ERR_STATE
        bad = torch.zeros((4, s.V, 3, 3), dtype=torch.complex128, device="cuda")
        with pytest.raises(lgf.LgfError) as e:
            s.set_links(bad)
        assert e.value.status == lgf.LGF_ERR_NOT_SU3
        with pytest.raises(TypeError):
            s.set_links(bad.to(torch.complex64))
    finally:
        s.close()
