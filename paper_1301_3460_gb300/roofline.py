"""Algorithmic bytes and floating-point operations of the iteration kernels.

Per lattice site and per launch, counting each unique array element once
(neighbour re-reads served by caches are not counted) and flops as real
multiplies/adds (an FMA is 2), with the FFT at the conventional 5 N log2 N per
complex transform of length N.

FP64 path, per site (V sites per launch):
  delta_xyfft   reads the packed anti-Hermitian parts of the four links (4 x 4
                complex) and their Re Tr sum, writes the four packed Delta
                fields: 256 + 8 + 64 B.  Flops: Delta as 16 complex differences
                (64), theta and F (21), x,y FFT of 4 fields (4 x 5 log2(Lx Ly)).
  zt_fft_accel  reads the multiplier table and reads/writes the 4 fields: 8 + 64 + 64 B
                (FP32: the multiplier is computed from per-axis tables, 32 + 32 B).
                Flops: forward and inverse z,t FFT of 4 fields
                (2 x 4 x 5 log2(Lz Lt)) + scale (8).
  xyifft_g      reads the 4 fields, writes g (full 3x3): 64 + 144 B.  Flops:
                inverse x,y FFT (4 x 5 log2(Lx Ly)) + Gram-Schmidt and row 2 (134).
  update        reads links, g, G; writes links, G, the packed anti-Hermitian
                parts and Re Tr: 384 + 144 + 96 + 384 + 96 + 256 + 8 B.  Flops:
                per link row-2 rebuild (42), two 2x3 by 3x3 complex products
                (2 x 132), row 2 of the result (42), packing (12), Re Tr (2);
                G: rebuild (42) + one product (132).
FP32 kernels move half the bytes of every array they keep in FP32 (links, G, g,
fields, packed parts, multiplier); their flop counts are the same.  The FP32
phase's other form fuses Delta into the update (fused32=True):
  delta_xyfft   the forward x,y FFT alone: reads and writes the 4 fields (32 + 32 B).
  update        reads links, g, G; writes links, G and Delta: 192 + 72 + 48 + 192 +
                48 + 32 B (the neighbours' links and g that it also reads are other
                sites' data, counted once).  Flops: the four links leaving the site
                as above, the four entering it recomputed for their anti-Hermitian
                parts (4 x (42 + 2 x 132 + 42 + 12)), G, Delta (64), theta and F (21).

FP64 iterations with the accelerator's transforms in FP32 (accel32=True): the
update as in FP64; the other three kernels move FP32 fields:
  delta_xyfft   reads the FP64 packed parts and Re Tr, writes the four FP32 fields:
                256 + 8 + 32 B (flops as in FP64).
  zt_fft_accel  the FP32 phase's kernel: 32 + 32 B.
  xyifft_g      reads the FP32 fields, writes the FP64 g: 32 + 144 B.

Wilson-action generation (k_wilson, one launch per direction and checkerboard
parity), per link updated, with full 3x3 complex products of 198 flops (27
complex multiplies, 18 complex adds) and 216 when accumulated into a sum:
  staples   6 products + 6 accumulated products               2484
  W = U A   one product                                          198
  subgroups 3 x (projection 20, R 56, rotation of two rows of U
            and of W 168)                                        732
  reunit    Gram-Schmidt of two rows and the row-2 rebuild       100
  total                                                         3514
The sampler's transcendental functions (heat bath) are not counted.  Bytes: a
launch reads about the whole link field (7/8 of it) and writes V/2 links, far
below what the FP64 pipe takes to do the arithmetic: the kernel is ALU-bound.
"""
from __future__ import annotations

import math

KERNELS = ("delta_xyfft", "zt_fft_accel", "xyifft_g", "update")


def per_site(dims, precision: int = 64, fused32: bool = False, accel32: bool = False) -> dict:
    Lx, Ly, Lz, Lt = (int(v) for v in dims)
    w = 1.0 if precision == 64 else 0.5
    lxy = math.log2(Lx * Ly)
    lzt = math.log2(Lz * Lt)
    if precision == 32 and fused32:
        return {
            "delta_xyfft": dict(bytes=(64 + 64) * w, flops=4 * 5 * lxy),
            "zt_fft_accel": dict(bytes=(64 + 64) * w, flops=2 * 4 * 5 * lzt + 8),
            "xyifft_g": dict(bytes=(64 + 144) * w, flops=4 * 5 * lxy + 134),
            "update": dict(bytes=(384 + 144 + 96 + 384 + 96 + 64) * w,
                           flops=4 * (42 + 2 * 132 + 42 + 12 + 2) + 4 * (42 + 2 * 132 + 42 + 12) + 42 + 132
                           + 64 + 21),
        }
    if precision == 64 and accel32:
        return {
            "delta_xyfft": dict(bytes=256 + 8 + 32, flops=64 + 21 + 4 * 5 * lxy),
            "zt_fft_accel": dict(bytes=32 + 32, flops=2 * 4 * 5 * lzt + 8),
            "xyifft_g": dict(bytes=32 + 144, flops=4 * 5 * lxy + 134),
            "update": dict(bytes=384 + 144 + 96 + 384 + 96 + 256 + 8,
                           flops=4 * (42 + 2 * 132 + 42 + 12 + 2) + 42 + 132),
        }
    return {
        "delta_xyfft": dict(bytes=(256 + 8 + 64) * w, flops=64 + 21 + 4 * 5 * lxy),
        "zt_fft_accel": dict(bytes=(64 + 64) * w + (8 if precision == 64 else 0), flops=2 * 4 * 5 * lzt + 8),
        "xyifft_g": dict(bytes=(64 + 144) * w, flops=4 * 5 * lxy + 134),
        "update": dict(bytes=(384 + 144 + 96 + 384 + 96 + 256 + 8) * w,
                       flops=4 * (42 + 2 * 132 + 42 + 12 + 2) + 42 + 132),
    }


def per_iteration(dims, precision: int = 64, fused32: bool = False) -> dict:
    V = 1
    for v in dims:
        V *= int(v)
    ps = per_site(dims, precision, fused32)
    return dict(bytes=V * sum(k["bytes"] for k in ps.values()), flops=V * sum(k["flops"] for k in ps.values()))


WILSON_FLOPS_PER_LINK = 3514
