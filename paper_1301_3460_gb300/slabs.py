"""One lattice over several processes: the t-slab decomposition of the
Fourier-accelerated iteration (the single-lattice analogue of the paper's MPI
code, whose 4D FFT is distributed by transposes).  This module holds only the
data movement; every step of the method stays in the per-rank kernels.

Rank r of N holds the sites with t in [r Lt/N, (r+1) Lt/N) in the library's
site order, a field of C components as a tensor [C, nt, Lz, Ly, Lx] (x fastest,
nt = Lt/N).  One iteration needs two kinds of exchange:

  halo planes   the Delta stencil reads the t-link entering x from x - t (the
                previous slab's last plane) and the update reads g(x + t) (the
                next slab's first plane): halo_planes() returns both neighbouring
                planes of a field, one send and one receive per direction.
  transposes    x, y and z lie inside a slab, so the x,y,z transforms and the
                x,y inverse run on the local planes; the t transform needs whole
                t-lines, so the fields go from t-slabs to z-slabs ([C, Lt, nz, Ly,
                Lx], z in [r Lz/N, (r+1) Lz/N)) by one all-to-all (t_to_z), are
                transformed along t, multiplied by the accelerator and
                transformed back, and return by a second all-to-all (z_to_t).

Per iteration and rank, with V the lattice volume: the halo moves 2 planes
(the packed anti-Hermitian parts of the entering t-links and g, 64 + 144 B per
site of a plane in FP64) and the transposes move 2 x 64 B x V/N (four packed
complex FP64 fields), of which (N-1)/N leaves the rank.  Any torch.distributed
process group works (NCCL on GPUs, gloo on CPUs); no multicast.
"""
from __future__ import annotations

import torch


class TSlabs:
    """t-slab decomposition of an Lx x Ly x Lz x Lt lattice over `world` ranks."""

    def __init__(self, dims, world: int):
        self.dims = tuple(int(v) for v in dims)
        Lx, Ly, Lz, Lt = self.dims
        if world < 1 or Lt % world or Lz % world:
            raise ValueError("Lt and Lz must be multiples of the number of ranks (%s, %d)" % (self.dims, world))
        self.world = world
        self.nt = Lt // world
        self.nz = Lz // world

    def t_range(self, rank: int):
        return rank * self.nt, (rank + 1) * self.nt

    def z_range(self, rank: int):
        return rank * self.nz, (rank + 1) * self.nz

    def local_shape(self, C: int):
        Lx, Ly, Lz, _ = self.dims
        return (C, self.nt, Lz, Ly, Lx)

    def halo_planes(self, field: torch.Tensor, rank: int, group=None):
        """(prev, next): plane t0 - 1 and plane t0 + nt of `field` [C, nt, Lz, Ly,
        Lx] (periodic in t), from the neighbouring ranks."""
        import torch.distributed as dist

        if self.world == 1:
            return field[:, -1].clone(), field[:, 0].clone()
        first = field[:, 0].contiguous()
        last = field[:, -1].contiguous()
        prev = torch.empty_like(first)
        nxt = torch.empty_like(first)
        up, down = (rank + 1) % self.world, (rank - 1) % self.world
        # tag 1: a slab's last plane going up (the next rank's prev halo);
        # tag 2: its first plane going down (the previous rank's next halo)
        ops = [dist.P2POp(dist.isend, last, up, group, tag=1), dist.P2POp(dist.irecv, prev, down, group, tag=1),
               dist.P2POp(dist.isend, first, down, group, tag=2), dist.P2POp(dist.irecv, nxt, up, group, tag=2)]
        for req in dist.batch_isend_irecv(ops):
            req.wait()
        return prev, nxt

    def t_to_z(self, field: torch.Tensor, group=None) -> torch.Tensor:
        """[C, nt, Lz, Ly, Lx] on t-slabs -> [C, Lt, nz, Ly, Lx] on z-slabs."""
        import torch.distributed as dist

        C = field.shape[0]
        N, nt, nz = self.world, self.nt, self.nz
        Lx, Ly, Lz, Lt = self.dims
        # send block j: this slab's z-range of rank j
        send = field.reshape(C, nt, N, nz, Ly, Lx).permute(2, 0, 1, 3, 4, 5).contiguous()
        recv = torch.empty_like(send)  # block i: rank i's t-range of this rank's z-range
        if N == 1:
            recv.copy_(send)
        else:
            dist.all_to_all_single(recv, send, group=group)
        return recv.permute(1, 0, 2, 3, 4, 5).reshape(C, Lt, nz, Ly, Lx)

    def z_to_t(self, field: torch.Tensor, group=None) -> torch.Tensor:
        """[C, Lt, nz, Ly, Lx] on z-slabs -> [C, nt, Lz, Ly, Lx] on t-slabs."""
        import torch.distributed as dist

        C = field.shape[0]
        N, nt, nz = self.world, self.nt, self.nz
        Lx, Ly, Lz, Lt = self.dims
        # send block i: rank i's t-range of this z-slab
        send = field.reshape(C, N, nt, nz, Ly, Lx).permute(1, 0, 2, 3, 4, 5).contiguous()
        recv = torch.empty_like(send)  # block j: rank j's z-range of this t-slab
        if N == 1:
            recv.copy_(send)
        else:
            dist.all_to_all_single(recv, send, group=group)
        return recv.permute(1, 2, 0, 3, 4, 5).reshape(C, nt, Lz, Ly, Lx)


# ---------------------------------------------------------------- GPU ranks

class _DeviceBuffer:
    """A library-owned device buffer seen as a flat float64 array (pairs of re, im)."""

    def __init__(self, ptr: int, nbytes: int):
        self.__cuda_array_interface__ = {"shape": (nbytes // 8,), "typestr": "<f8", "data": (ptr, False),
                                         "version": 3}


class Slab:
    """One rank's t-slab on the current GPU (the library's lgf_slab_* entry
    points).  Links and G are complex128 CUDA tensors of the slab's sites,
    [4, V_slab, 3, 3] and [V_slab, 3, 3]."""

    def __init__(self, dims, nranks: int, rank: int, stream=None):
        import ctypes

        from . import lgf

        self._lgf = lgf
        self._lib = lib = lgf.load()
        self.dims = tuple(int(v) for v in dims)
        self.nranks, self.rank = int(nranks), int(rank)
        arr = (ctypes.c_int * 4)(*self.dims)
        h = ctypes.c_void_p()
        lgf._check(lib.lgf_slab_create(arr, self.nranks, self.rank, ctypes.byref(h)), "lgf_slab_create")
        self._h = h
        self.layout = TSlabs(self.dims, self.nranks)
        Lx, Ly, Lz, _ = self.dims
        self.V = Lx * Ly * Lz * self.layout.nt
        self._stream = stream
        if stream is not None:
            raw = getattr(stream, "cuda_stream", stream)
            lgf._check(lib.lgf_slab_set_stream(h, ctypes.c_void_p(raw or 0)), "lgf_slab_set_stream")
        self._bufs = {}

    def close(self):
        if getattr(self, "_h", None):
            self._bufs.clear()
            self._lib.lgf_slab_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def _call(self, name, *args):
        self._lgf._check(getattr(self._lib, name)(self._h, *args), name)

    def buffer(self, which: int):
        """Flat complex128 tensor over the slab's buffer `which` (LGF_SLAB_*);
        valid while the slab lives."""
        import ctypes

        import torch

        if which not in self._bufs:
            p, n = ctypes.c_void_p(), ctypes.c_size_t()
            self._call("lgf_slab_buffer", int(which), ctypes.byref(p), ctypes.byref(n))
            flat = torch.as_tensor(_DeviceBuffer(p.value, n.value), device="cuda")
            self._bufs[which] = torch.view_as_complex(flat.view(-1, 2))
        return self._bufs[which]

    def set_links(self, U):
        import ctypes

        import torch

        if not (isinstance(U, torch.Tensor) and U.is_cuda and U.dtype == torch.complex128
                and tuple(U.shape) == (4, self.V, 3, 3)):
            raise TypeError("set_links takes a complex128 CUDA tensor (4, %d, 3, 3)" % self.V)
        U = U.contiguous()
        self._call("lgf_slab_set_links", ctypes.c_void_p(U.data_ptr()))

    def get_links(self):
        import ctypes

        import torch

        out = torch.empty((4, self.V, 3, 3), dtype=torch.complex128, device="cuda")
        self._call("lgf_slab_get_links", ctypes.c_void_p(out.data_ptr()))
        return out

    def get_gauge(self):
        import ctypes

        import torch

        out = torch.empty((self.V, 3, 3), dtype=torch.complex128, device="cuda")
        self._call("lgf_slab_get_gauge", ctypes.c_void_p(out.data_ptr()))
        return out

    def pack_halo(self, which: int):
        self._call("lgf_slab_pack_halo", int(which))

    def delta(self):
        import ctypes

        th, F = ctypes.c_double(), ctypes.c_double()
        self._call("lgf_slab_delta", ctypes.byref(th), ctypes.byref(F))
        return th.value, F.value

    def accelerate(self):
        self._call("lgf_slab_accelerate")

    def build_g(self, alpha: float):
        import ctypes

        self._call("lgf_slab_build_g", ctypes.c_double(float(alpha)))

    def update(self):
        self._call("lgf_slab_update")


class LocalExchange:
    """The exchanges of ranks held as several slabs of one process (one GPU):
    device copies in place of the messages."""

    def __init__(self, slabs):
        self.slabs = list(slabs)
        self.N = len(self.slabs)

    def halo_ah(self):  # a slab's last plane goes up
        from .lgf import LGF_SLAB_AH_RECV, LGF_SLAB_AH_SEND

        for r, s in enumerate(self.slabs):
            self.slabs[(r + 1) % self.N].buffer(LGF_SLAB_AH_RECV).copy_(s.buffer(LGF_SLAB_AH_SEND))

    def halo_g(self):  # a slab's first plane goes down
        from .lgf import LGF_SLAB_G_RECV, LGF_SLAB_G_SEND

        for r, s in enumerate(self.slabs):
            self.slabs[(r - 1) % self.N].buffer(LGF_SLAB_G_RECV).copy_(s.buffer(LGF_SLAB_G_SEND))

    def all_to_all(self, src: int, dst: int):  # block i of rank r's src -> block r of rank i's dst
        for r in range(self.N):
            out = self.slabs[r].buffer(dst).view(self.N, -1)
            for i in range(self.N):
                out[i].copy_(self.slabs[i].buffer(src).view(self.N, -1)[r])

    def mean(self, values):
        n = len(values)
        return tuple(sum(v[k] for v in values) / n for k in range(len(values[0])))


class DistExchange:
    """The exchanges of one slab per process over a torch.distributed group:
    NCCL on device buffers, or (staged=True, for gloo) through host copies."""

    def __init__(self, slab: Slab, group=None, staged: bool = False):
        import torch.distributed as dist

        self.slabs = [slab]
        self.group = group
        self.staged = staged
        self.N = dist.get_world_size(group)
        self.rank = dist.get_rank(group)

    def _t(self, x):  # what goes on the wire: real views, on the host if staged
        import torch

        x = torch.view_as_real(x)
        return x.cpu() if self.staged else x

    def _sendrecv(self, send, recv, to, frm, tag):
        import torch
        import torch.distributed as dist

        if self.N == 1:
            recv.copy_(send)
            return
        s, r = self._t(send), (torch.empty_like(self._t(recv)))
        reqs = dist.batch_isend_irecv([dist.P2POp(dist.isend, s, to, self.group, tag=tag),
                                       dist.P2POp(dist.irecv, r, frm, self.group, tag=tag)])
        for q in reqs:
            q.wait()
        recv.copy_(torch.view_as_complex(r.to(recv.device)))

    def halo_ah(self):
        from .lgf import LGF_SLAB_AH_RECV, LGF_SLAB_AH_SEND

        s = self.slabs[0]
        self._sendrecv(s.buffer(LGF_SLAB_AH_SEND), s.buffer(LGF_SLAB_AH_RECV), (self.rank + 1) % self.N,
                       (self.rank - 1) % self.N, 1)

    def halo_g(self):
        from .lgf import LGF_SLAB_G_RECV, LGF_SLAB_G_SEND

        s = self.slabs[0]
        self._sendrecv(s.buffer(LGF_SLAB_G_SEND), s.buffer(LGF_SLAB_G_RECV), (self.rank - 1) % self.N,
                       (self.rank + 1) % self.N, 2)

    def all_to_all(self, src: int, dst: int):
        import torch
        import torch.distributed as dist

        s = self.slabs[0]
        a, b = s.buffer(src), s.buffer(dst)
        if self.N == 1:
            b.copy_(a)
            return
        sa = self._t(a)
        rb = torch.empty_like(sa)
        dist.all_to_all_single(rb, sa, group=self.group)
        b.copy_(torch.view_as_complex(rb.to(b.device)))

    def mean(self, values):
        import torch
        import torch.distributed as dist

        t = torch.tensor(values[0], dtype=torch.float64, device="cpu" if self.staged else "cuda")
        dist.all_reduce(t, group=self.group)
        return tuple(float(v) / self.N for v in t.tolist())


def fix_slabs(exchange, alpha: float = 0.08, tol: float = 1e-15, max_iter: int = 100000) -> dict:
    """The Fourier-accelerated iteration of one lattice over the slabs of
    `exchange` (LocalExchange: all ranks in this process; DistExchange: this
    process's rank), stopping when theta of the current links is below tol or
    after max_iter updates, like lgf_fix."""
    from .lgf import LGF_SLAB_A, LGF_SLAB_AH_SEND, LGF_SLAB_B, LGF_SLAB_G_SEND

    slabs = exchange.slabs
    n = 0
    while True:
        for s in slabs:
            s.pack_halo(LGF_SLAB_AH_SEND)
        exchange.halo_ah()
        theta, F = exchange.mean([s.delta() for s in slabs])
        if not (theta == theta):
            raise FloatingPointError("theta is NaN after %d updates" % n)
        if theta < tol or n >= max_iter:
            break
        exchange.all_to_all(LGF_SLAB_A, LGF_SLAB_B)
        for s in slabs:
            s.accelerate()
        exchange.all_to_all(LGF_SLAB_B, LGF_SLAB_A)
        for s in slabs:
            s.build_g(alpha)
            s.pack_halo(LGF_SLAB_G_SEND)
        exchange.halo_g()
        for s in slabs:
            s.update()
        n += 1
    return dict(iters=n, theta=theta, F=F, converged=theta < tol)
