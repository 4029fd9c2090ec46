"""Oracle-side reference for derivatives: the Fourier-accelerated step and the
gluon propagator written with plain PyTorch CPU operations in complex128, so
that torch's autograd supplies a reference gradient.

TEST INFRASTRUCTURE ONLY (like the C oracle): it shares no code with the CUDA
path.  Each operation follows the same readings of arXiv:1301.3460 as the C
oracle (lgf_oracle.c): the functional of the introduction, steepest descent
with Fourier acceleration, Delta = (M - M^dag) - trace/3, p2max/p2 with the zero
mode removed, first-order exponential and row Gram-Schmidt, 12-real links
(row 2 rebuilt as conj(row0 x row1)).  Links are tensors (4, V, 3, 3);
site s = x + Lx*(y + Ly*(z + Lz*t)).
"""
from __future__ import annotations

import math

import torch


def _shift_index(L, mu, d):
    V = L[0] * L[1] * L[2] * L[3]
    s = torch.arange(V)
    c = []
    r = s
    for v in L:
        c.append(r % v)
        r = r // v
    c[mu] = (c[mu] + d) % L[mu]
    out = torch.zeros(V, dtype=torch.long)
    for nu in (3, 2, 1, 0):
        out = out * L[nu] + c[nu]
    return out


def rebuild(U):
    """Full matrices from rows 0,1: row 2 = conj(row0 x row1)."""
    r0, r1 = U[..., 0, :], U[..., 1, :]
    r2 = torch.conj(torch.linalg.cross(r0, r1, dim=-1))
    return torch.stack([r0, r1, r2], dim=-2)


def dag(m):
    return torch.conj(m.transpose(-1, -2))


def delta(L, U):
    """Delta(x) = T(M - M^dag), M = sum_mu [U_mu(x-mu) - U_mu(x)]."""
    Uf = rebuild(U)
    M = 0
    for mu in range(4):
        M = M + Uf[mu][_shift_index(L, mu, -1)] - Uf[mu]
    D = M - dag(M)
    tr = torch.diagonal(D, dim1=-2, dim2=-1).sum(-1) / 3
    return D - tr[:, None, None] * torch.eye(3, dtype=D.dtype)


def multiplier(L):
    """p2max / (p2(k) V) on the momentum grid (numpy order t,z,y,x), zero mode 0."""
    ks = [torch.arange(n, dtype=torch.float64) for n in L]
    s2 = [4 * torch.sin(math.pi * k / n) ** 2 for k, n in zip(ks, L)]
    p2 = s2[3][:, None, None, None] + s2[2][None, :, None, None] + s2[1][None, None, :, None] + s2[0][None, None, None, :]
    p2max = sum(float(v.max()) for v in s2)
    V = L[0] * L[1] * L[2] * L[3]
    m = torch.where(p2 > 0, p2max / p2.clamp(min=1e-300) / V, torch.zeros_like(p2))
    return m


def accelerate(L, D):
    grid = D.reshape(L[3], L[2], L[1], L[0], 3, 3)
    f = torch.fft.fftn(grid, dim=(0, 1, 2, 3))
    f = f * multiplier(L)[..., None, None]
    return torch.fft.ifftn(f, dim=(0, 1, 2, 3), norm="forward").reshape(-1, 3, 3)


def reunit(X):
    x0, x1 = X[..., 0, :], X[..., 1, :]
    r0 = x0 / torch.sqrt((x0.conj() * x0).real.sum(-1, keepdim=True))
    ip = (r0.conj() * x1).sum(-1, keepdim=True)
    v = x1 - ip * r0
    r1 = v / torch.sqrt((v.conj() * v).real.sum(-1, keepdim=True))
    r2 = torch.conj(torch.linalg.cross(r0, r1, dim=-1))
    return torch.stack([r0, r1, r2], dim=-2)


def step(L, U, alpha=0.08):
    """One step; returns the full new links (row 2 rebuilt)."""
    Dt = accelerate(L, delta(L, U))
    g = reunit(torch.eye(3, dtype=Dt.dtype) + 0.5 * alpha * Dt)
    Uf = rebuild(U)
    out = []
    for mu in range(4):
        out.append(g @ Uf[mu] @ dag(g[_shift_index(L, mu, +1)]))
    return rebuild(torch.stack(out))


def gluon_pmin(L, U):
    """Mean over the four momenta with one k_mu = 1 of
    D(p) = 2/((N_c^2-1)(N_d-1)V) sum_mu Tr[A~_mu(p) A~_mu(p)^dag]."""
    Uf = rebuild(U)
    A = (Uf - dag(Uf)) / 2j
    tr = torch.diagonal(A, dim1=-2, dim2=-1).sum(-1) / 3
    A = A - tr[..., None, None] * torch.eye(3, dtype=A.dtype)
    V = L[0] * L[1] * L[2] * L[3]
    s = torch.arange(V)
    coords = []
    r = s
    for v in L:
        coords.append(r % v)
        r = r // v
    D = 0
    for nu in range(4):
        ph = torch.exp(-2j * math.pi * coords[nu].to(torch.float64) / L[nu])
        At = (ph[None, :, None, None] * A).sum(1)  # (4, 3, 3)
        D = D + 2.0 / (8 * 3 * V) * (At.conj() * At).real.sum() / 4
    return D


def gluon_after_fixing(L, U0, K, alpha=0.08):
    U = U0
    for _ in range(K):
        U = step(L, U, alpha)
    return gluon_pmin(L, U)
