"""ctypes front end of the plain FP64 CPU oracle (``lgf_oracle.c`` for gauge
fixing, ``lgf_wilson_oracle.c`` for the Wilson-action configurations it is
applied to).

TEST INFRASTRUCTURE ONLY: the tests, the smoke entry point and the benchmark's
CPU-baseline leg are the only callers.  The CUDA library never imports this
module and this module never imports the CUDA library.

Arrays are numpy complex128, C-contiguous:
  links          (4, V, 3, 3)   mu-major, site index s = x + Lx*(y + Ly*(z + Lz*t))
  matrix fields  (V, 3, 3)
  scalar fields  (V,)
Every function follows the step of arXiv:1301.3460 (Landau gauge fixing by
Fourier-accelerated steepest descent) named in its docstring; the readings of
the steps the paper leaves implicit are listed in the header of the C file.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lgf_oracle.c")
_SRC_W = os.path.join(_HERE, "lgf_wilson_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liblgf_oracle.so")
_lock = threading.Lock()
_lib = None

_dbl_p = ctypes.POINTER(ctypes.c_double)
_int_p = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (ISO C11, no fast-math, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    stale = not os.path.exists(_LIB) or any(os.path.getmtime(_LIB) < os.path.getmtime(p) for p in (_SRC, _SRC_W))
    if force or stale:
        tmp = _LIB + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, _SRC_W, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            v = ctypes.c_void_p
            lib.orc_delta.argtypes = [_int_p, v, v, _dbl_p, _dbl_p]
            lib.orc_fft4.argtypes = [_int_p, v, ctypes.c_int]
            lib.orc_dft4.argtypes = [_int_p, v, v, ctypes.c_int]
            lib.orc_p2max.argtypes = [_int_p]
            lib.orc_p2max.restype = ctypes.c_double
            lib.orc_accelerate.argtypes = [_int_p, v, v, ctypes.c_int]
            lib.orc_reunit.argtypes = [v, v]
            lib.orc_build_g.argtypes = [_int_p, v, ctypes.c_double, v]
            lib.orc_update.argtypes = [_int_p, v, v, v]
            lib.orc_gauge_transform.argtypes = [_int_p, v, v, v]
            lib.orc_fix.argtypes = [_int_p, v, v, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                    ctypes.c_int, _int_p, _dbl_p, _dbl_p, _dbl_p]
            lib.orc_fix.restype = ctypes.c_int
            lib.orc_fix_sd.argtypes = [_int_p, v, v, ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_int, _int_p, _dbl_p, _dbl_p, _dbl_p]
            lib.orc_fix_sd.restype = ctypes.c_int
            lib.orc_plaquette.argtypes = [_int_p, v]
            lib.orc_plaquette.restype = ctypes.c_double
            lib.orc_gluon_pmin.argtypes = [_int_p, v, _dbl_p]
            lib.orc_gluon_pmin.restype = ctypes.c_double
            u64, u32 = ctypes.c_uint64, ctypes.c_uint32
            lib.orc_wilson_sweep.argtypes = [_int_p, v, ctypes.c_double, u64, u32, ctypes.c_int]
            lib.orc_wilson_plaquette.argtypes = [_int_p, v]
            lib.orc_wilson_plaquette.restype = ctypes.c_double
            lib.orc_wilson_link.argtypes = [_int_p, v, ctypes.c_long, ctypes.c_int, ctypes.c_double, u64, u32,
                                             ctypes.c_int, v]
            lib.orc_philox4x32.argtypes = [v, v, v]
            lib.orc_su2_samples.argtypes = [ctypes.c_double, u64, ctypes.c_int, _dbl_p]
            lib.orc_threads.restype = ctypes.c_int
            lib.orc_set_threads.argtypes = [ctypes.c_int]
            _lib = lib
    return _lib


def _dims(L):
    L = [int(v) for v in L]
    assert len(L) == 4 and all(v >= 1 for v in L)
    return (ctypes.c_int * 4)(*L), int(np.prod(L))


def _c(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.complex128)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def threads() -> int:
    """OpenMP threads the oracle uses."""
    return int(_load().orc_threads())


def set_threads(n: int) -> None:
    _load().orc_set_threads(int(n))


def delta(L, U):
    """Delta(x) = (M - M^dag) - Tr(M - M^dag)/3, M = sum_mu [U_mu(x-mu) - U_mu(x)];
    theta = Tr(Delta Delta^dag) summed / (N_c V); F = Re Tr U summed / (N_d N_c V)
    (the functional of the introduction at g = 1).  Returns (Delta, theta, F)."""
    d, V = _dims(L)
    U = _c(U, (4, V, 3, 3))
    D = np.empty((V, 3, 3), np.complex128)
    th, f = ctypes.c_double(), ctypes.c_double()
    _load().orc_delta(d, _ptr(U), _ptr(D), ctypes.byref(th), ctypes.byref(f))
    return D, th.value, f.value


def fft4(L, f, sign):
    """Unnormalised 4D FFT (recursive mixed radix) of a scalar field; sign -1 forward."""
    d, V = _dims(L)
    out = _c(f, (V,)).copy()
    _load().orc_fft4(d, _ptr(out), int(sign))
    return out


def dft4(L, f, sign):
    """Unnormalised 4D DFT by its O(V^2) definition."""
    d, V = _dims(L)
    f = _c(f, (V,))
    out = np.empty(V, np.complex128)
    _load().orc_dft4(d, _ptr(f), _ptr(out), int(sign))
    return out


def p2max(L) -> float:
    """max over lattice momenta of p2(k) = sum_mu 4 sin^2(pi k_mu/L_mu)."""
    d, _ = _dims(L)
    return float(_load().orc_p2max(d))


def accelerate(L, D, use_dft=False):
    """Fourier acceleration of every entry: IDFT[p2max/p2(k) DFT[D](k)]/V, k = 0 removed."""
    d, V = _dims(L)
    D = _c(D, (V, 3, 3))
    out = np.empty((V, 3, 3), np.complex128)
    _load().orc_accelerate(d, _ptr(D), _ptr(out), int(bool(use_dft)))
    return out


def reunit(X):
    """Row Gram-Schmidt projection of each 3x3 matrix onto SU(3)."""
    X = _c(X)
    flat = X.reshape(-1, 3, 3)
    out = np.empty_like(flat)
    lib = _load()
    for i in range(flat.shape[0]):
        lib.orc_reunit(_ptr(flat[i]), _ptr(out[i]))
    return out.reshape(X.shape)


def build_g(L, Dt, alpha):
    """g(x) = reunit(1 + (alpha/2) Dt(x))."""
    d, V = _dims(L)
    Dt = _c(Dt, (V, 3, 3))
    g = np.empty((V, 3, 3), np.complex128)
    _load().orc_build_g(d, _ptr(Dt), float(alpha), _ptr(g))
    return g


def update(L, U, G, g):
    """U_mu(x) <- g(x) U_mu(x) g^dag(x+mu), G(x) <- g(x) G(x), row 2 recomputed.
    Returns new (U, G) (inputs untouched); G may be None."""
    d, V = _dims(L)
    U = _c(U, (4, V, 3, 3)).copy()
    g = _c(g, (V, 3, 3))
    Gc = None if G is None else _c(G, (V, 3, 3)).copy()
    _load().orc_update(d, _ptr(U), None if Gc is None else _ptr(Gc), _ptr(g))
    return U, Gc


def gauge_transform(L, U, G):
    """U'_mu(x) = G(x) U_mu(x) G^dag(x+mu)."""
    d, V = _dims(L)
    U = _c(U, (4, V, 3, 3))
    G = _c(G, (V, 3, 3))
    out = np.empty_like(U)
    _load().orc_gauge_transform(d, _ptr(U), _ptr(G), _ptr(out))
    return out


def fix(L, U, alpha=0.08, tol=1e-15, max_iter=1000, use_dft=False, track_gauge=True, history=False,
        accelerate=True):
    """Fourier-accelerated (accelerate=True) or plain steepest descent to
    theta < tol or max_iter updates.  Returns a dict with U, G (or None), iters,
    F, theta, converged, history."""
    d, V = _dims(L)
    U = _c(U, (4, V, 3, 3)).copy()
    G = None
    if track_gauge:
        G = np.zeros((V, 3, 3), np.complex128)
        G[:, 0, 0] = G[:, 1, 1] = G[:, 2, 2] = 1.0
    hist = np.zeros(2 * (int(max_iter) + 1), np.float64) if history else None
    it, f, th = ctypes.c_int(), ctypes.c_double(), ctypes.c_double()
    rc = _load().orc_fix_sd(d, _ptr(U), None if G is None else _ptr(G), float(alpha), float(tol), int(max_iter),
                            int(bool(use_dft)), int(bool(accelerate)), ctypes.byref(it), ctypes.byref(f),
                            ctypes.byref(th), None if hist is None else hist.ctypes.data_as(_dbl_p))
    out = dict(U=U, G=G, iters=it.value, F=f.value, theta=th.value, converged=(rc == 0))
    if hist is not None:
        out["history"] = hist[: 2 * (it.value + 1)].reshape(-1, 2)
    return out


def plaquette(L, U) -> float:
    """Average plaquette Re Tr / 3 over the six planes: a gauge-invariant check quantity."""
    d, V = _dims(L)
    U = _c(U, (4, V, 3, 3))
    return float(_load().orc_plaquette(d, _ptr(U)))


def gluon_pmin(L, U):
    """Gluon propagator D(p) at the four momenta with one k_mu = 1; returns (average, D[4])."""
    d, V = _dims(L)
    U = _c(U, (4, V, 3, 3))
    Dp = (ctypes.c_double * 4)()
    avg = _load().orc_gluon_pmin(d, _ptr(U), Dp)
    return float(avg), np.array(list(Dp))


def wilson_sweeps(L, U, beta, seed, sweeps, mode=0, first_sweep=0):
    """Sweeps of the Wilson-action Monte Carlo (configurations of the kind the
    paper fixes): SU(2)-subgroup heat bath (mode 0) or overrelaxation (mode 1) of
    every link, mu = 0..3, even then odd sites (lgf_wilson_oracle.c).  Heat-bath
    sweep n draws random numbers with sweep counter first_sweep + n.  Returns new
    links (input untouched)."""
    d, V = _dims(L)
    U = _c(U, (4, V, 3, 3)).copy()
    for n in range(int(sweeps)):
        _load().orc_wilson_sweep(d, _ptr(U), float(beta), int(seed), int(first_sweep + n), int(mode))
    return U


def wilson_link(L, U, site, mu, beta, seed, sweep, mode=0):
    """The update of one link U_mu(site) given all other links, as inside a
    sweep; returns the new 3x3 link (U is not modified)."""
    d, V = _dims(L)
    U = _c(U, (4, V, 3, 3))
    out = np.empty((3, 3), np.complex128)
    _load().orc_wilson_link(d, _ptr(U), int(site), int(mu), float(beta), int(seed), int(sweep), int(mode), _ptr(out))
    return out


def wilson_plaquette(L, U) -> float:
    """Mean of Re Tr U_P / 3 over all plaquettes (independent loop of this file)."""
    d, V = _dims(L)
    U = _c(U, (4, V, 3, 3))
    return float(_load().orc_wilson_plaquette(d, _ptr(U)))


def philox4x32(ctr, key):
    """Philox4x32-10 of a 4-word counter and 2-word key (Salmon et al., SC'11)."""
    c = np.array(ctr, np.uint32)
    k = np.array(key, np.uint32)
    out = np.empty(4, np.uint32)
    _load().orc_philox4x32(c.ctypes.data_as(ctypes.c_void_p), k.ctypes.data_as(ctypes.c_void_p),
                           out.ctypes.data_as(ctypes.c_void_p))
    return out


def su2_samples(b, seed, n):
    """n draws y = (y0, y1, y2, y3) of the SU(2) heat-bath sampler for parameter b."""
    y = np.empty((int(n), 4), np.float64)
    _load().orc_su2_samples(float(b), int(seed), int(n), y.ctypes.data_as(_dbl_p))
    return y
