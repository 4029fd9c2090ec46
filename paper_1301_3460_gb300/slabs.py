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
