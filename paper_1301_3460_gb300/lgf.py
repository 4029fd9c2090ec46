"""Python binding of the CUDA gauge-fixing library (liblgf.so, C ABI in include/lgf.h).

Argument marshalling only: every step of the method runs in the library's CUDA
kernels.  There is no CPU fallback; if the library or a CUDA device is missing
the calls raise.

Arrays follow the C ABI: links complex128 (4, V, 3, 3), gauge transformations
and matrix fields complex128 (V, 3, 3), site s = x + Lx*(y + Ly*(z + Lz*t)).
Each may be a numpy array (host) or a contiguous torch complex128 CUDA tensor
(device; then the copy stays on the device).
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

LGF_OK = 0
LGF_ERR_ARG = 1
LGF_ERR_CUDA = 2
LGF_ERR_NOT_SU3 = 3
LGF_ERR_UNSUPPORTED_DIMS = 4
LGF_ERR_NOT_CONVERGED = 5
LGF_ERR_NAN = 6
LGF_ERR_TIMEOUT = 7
LGF_ERR_STATE = 8
LGF_SLAB_A, LGF_SLAB_B, LGF_SLAB_AH_SEND, LGF_SLAB_AH_RECV, LGF_SLAB_G_SEND, LGF_SLAB_G_RECV = range(6)

LGF_FP64 = 0
LGF_MIXED = 1
LGF_NO_GAUGE = 2
LGF_PLAIN_SD = 4
LGF_LINKS18 = 8
LGF_LINKS8 = 16

_lock = threading.Lock()
_lib = None


class LgfError(RuntimeError):
    def __init__(self, status: int, call: str):
        self.status = status
        lib = _lib
        msg = lib.lgf_strerror(status).decode() if lib else str(status)
        detail = lib.lgf_last_error().decode() if (lib and status == LGF_ERR_CUDA) else ""
        super().__init__("%s failed: %s (status %d)%s" % (call, msg, status, (": " + detail) if detail else ""))


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load liblgf.so (building it in-tree with nvcc if absent or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if build_if_missing and not _build.up_to_date():
            _build.build()
        if not os.path.exists(path):
            raise RuntimeError("liblgf.so is not built (%s); run paper_1301_3460_gb300/build.py" % path)
        lib = ctypes.CDLL(path)
        P = ctypes.c_void_p
        I = ctypes.c_int
        D = ctypes.c_double
        IP = ctypes.POINTER(ctypes.c_int)
        DP = ctypes.POINTER(ctypes.c_double)
        sig = {
            "lgf_create": ([ctypes.POINTER(ctypes.c_int), I, ctypes.POINTER(P)], I),
            "lgf_set_stream": ([P, P], I),
            "lgf_set_links": ([P, P, I], I),
            "lgf_fix": ([P, D, D, I, IP, DP, DP], I),
            "lgf_get_links": ([P, P, I], I),
            "lgf_get_gauge": ([P, P, I], I),
            "lgf_get_history": ([P, DP, I, IP], I),
            "lgf_get_stats": ([P, IP, IP], I),
            "lgf_set_switch_tol": ([P, D], I),
            "lgf_set_fp32_refresh": ([P, I], I),
            "lgf_set_fp32_update": ([P, I], I),
            "lgf_set_accel_precision": ([P, I], I),
            "lgf_batch_set_accel_precision": ([P, I], I),
            "lgf_batch_set_fp32_update": ([P, I], I),
            "lgf_set_loop_bound": ([P, I], I),
            "lgf_delta": ([P, P, I, DP, DP], I),
            "lgf_accelerate": ([P, P, P, I], I),
            "lgf_build_g": ([P, P, D, P, I], I),
            "lgf_delta32": ([P, P, I, DP, DP], I),
            "lgf_accelerate32": ([P, P, P, I], I),
            "lgf_build_g32": ([P, P, D, P, I], I),
            "lgf_time_kernels": ([P, D, I, I, DP], I),
            "lgf_accelerate_noalloc": ([ctypes.POINTER(ctypes.c_int), P, P, P], I),
            "lgf_autotune": ([P], I),
            "lgf_set_shape": ([P, I, I, I, I, I], I),
            "lgf_get_shape": ([P, I, ctypes.POINTER(ctypes.c_int)], I),
            "lgf_probe_fma": ([I, I, DP, DP], I),
            "lgf_check_conversions": ([P, P, P, P, I], I),
            "lgf_step_fwd": ([P, D, P, P], I),
            "lgf_step_bwd": ([P, D, P, P], I),
            "lgf_gluon_pmin": ([P, DP, DP], I),
            "lgf_gluon_pmin_bwd": ([P, D, P], I),
            "lgf_set_unit_links": ([P], I),
            "lgf_links_state_bytes": ([P], ctypes.c_size_t),
            "lgf_save_links": ([P, P], I),
            "lgf_load_links": ([P, P], I),
            "lgf_wilson_sweeps": ([P, D, ctypes.c_ulonglong, I, I, I], I),
            "lgf_plaquette": ([P, DP], I),
            "lgf_set_generator_precision": ([P, I], I),
            "lgf_batch_create": ([I, ctypes.POINTER(ctypes.c_int), I, ctypes.POINTER(P)], I),
            "lgf_batch_set_stream": ([P, P], I),
            "lgf_batch_set_links": ([P, I, P, I], I),
            "lgf_batch_set_switch_tol": ([P, D], I),
            "lgf_batch_fix": ([P, D, D, I, IP, DP, DP, IP, DP], I),
            "lgf_batch_get_links": ([P, I, P, I], I),
            "lgf_batch_get_gauge": ([P, I, P, I], I),
            "lgf_batch_get_stats": ([P, I, IP, IP], I),
            "lgf_batch_destroy": ([P], None),
            "lgf_destroy": ([P], None),
            "lgf_slab_create": ([ctypes.POINTER(ctypes.c_int), I, I, ctypes.POINTER(P)], I),
            "lgf_slab_destroy": ([P], None),
            "lgf_slab_set_stream": ([P, P], I),
            "lgf_slab_set_links": ([P, P], I),
            "lgf_slab_get_links": ([P, P], I),
            "lgf_slab_get_gauge": ([P, P], I),
            "lgf_slab_buffer": ([P, I, ctypes.POINTER(P), ctypes.POINTER(ctypes.c_size_t)], I),
            "lgf_slab_pack_halo": ([P, I], I),
            "lgf_slab_delta": ([P, DP, DP], I),
            "lgf_slab_accelerate": ([P], I),
            "lgf_slab_build_g": ([P, D], I),
            "lgf_slab_update": ([P], I),
            "lgf_strerror": ([I], ctypes.c_char_p),
            "lgf_last_error": ([], ctypes.c_char_p),
        }
        for name, (args, res) in sig.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = res
        _lib = lib
        return lib


def _check(status: int, call: str):
    if status != LGF_OK:
        raise LgfError(status, call)


def _is_torch(a) -> bool:
    return type(a).__module__.startswith("torch")


def _in_ptr(a, shape):
    """(pointer, on_device, keepalive) of an input array."""
    if _is_torch(a):
        import torch

        assert a.dtype == torch.complex128 and tuple(a.shape) == tuple(shape), (a.dtype, a.shape, shape)
        if not a.is_cuda:
            a = a.numpy()
        else:
            assert a.is_contiguous()
            return ctypes.c_void_p(a.data_ptr()), 1, a
    a = np.ascontiguousarray(a, dtype=np.complex128).reshape(shape)
    return a.ctypes.data_as(ctypes.c_void_p), 0, a


def _out(like, shape, device):
    if device is not None:
        import torch

        t = torch.empty(shape, dtype=torch.complex128, device=device)
        return t, ctypes.c_void_p(t.data_ptr()), 1
    a = np.empty(shape, np.complex128)
    return a, a.ctypes.data_as(ctypes.c_void_p), 0


class Lattice:
    """One gauge field on the GPU and its gauge-fixing state (an lgf_ctx)."""

    def __init__(self, dims, mixed: bool = False, track_gauge: bool = True, stream=None, accelerate: bool = True,
                 links18: bool = False, links8: bool = False):
        lib = load()
        self.dims = tuple(int(v) for v in dims)
        self.V = int(np.prod(self.dims))
        flags = (LGF_MIXED if mixed else LGF_FP64) | (0 if track_gauge else LGF_NO_GAUGE)
        if not accelerate:
            flags |= LGF_PLAIN_SD
        if links18:
            flags |= LGF_LINKS18
        if links8:
            flags |= LGF_LINKS8
        arr = (ctypes.c_int * 4)(*self.dims)
        h = ctypes.c_void_p()
        _check(lib.lgf_create(arr, flags, ctypes.byref(h)), "lgf_create")
        self._h = h
        self._lib = lib
        self.mixed = mixed
        self._stream = None
        if stream is not None:
            self.set_stream(stream)

    # -- lifetime
    def close(self):
        if getattr(self, "_h", None):
            self._lib.lgf_destroy(self._h)
            self._h = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- calls
    def set_stream(self, stream):
        """stream: a torch.cuda.Stream, a raw cudaStream_t integer, or None (legacy default)."""
        raw = getattr(stream, "cuda_stream", stream)
        _check(self._lib.lgf_set_stream(self._h, ctypes.c_void_p(raw or 0)), "lgf_set_stream")
        self._stream = stream  # the context launches on it: keep the object alive as long as the context

    def set_loop_bound(self, n: int):
        """Fault injection: cap each device loop at n body runs (0: no cap)."""
        _check(self._lib.lgf_set_loop_bound(self._h, int(n)), "lgf_set_loop_bound")

    def set_switch_tol(self, tol: float):
        _check(self._lib.lgf_set_switch_tol(self._h, float(tol)), "lgf_set_switch_tol")

    def set_fp32_refresh(self, every: int):
        _check(self._lib.lgf_set_fp32_refresh(self._h, int(every)), "lgf_set_fp32_refresh")

    def set_fp32_update(self, form):
        """FP32 phase: the two-kernel update (False or 0), the update fused with
        Delta (True or 1), or the g builder and update in one persistent launch (2,
        the default)."""
        _check(self._lib.lgf_set_fp32_update(self._h, int(form)), "lgf_set_fp32_update")

    def set_accel_precision(self, bits: int):
        """Mixed contexts: the accelerator's transforms of the FP64 iterations in
        FP64 (64, the default) or FP32 (32; Delta, theta, F, g and the update stay FP64)."""
        _check(self._lib.lgf_set_accel_precision(self._h, int(bits)), "lgf_set_accel_precision")

    def set_links(self, U):
        p, dev, keep = _in_ptr(U, (4, self.V, 3, 3))
        _check(self._lib.lgf_set_links(self._h, p, dev), "lgf_set_links")
        del keep

    def fix(self, alpha: float = 0.08, tol: float = 1e-15, max_iter: int = 100000, check: bool = True) -> dict:
        it = ctypes.c_int()
        F = ctypes.c_double()
        th = ctypes.c_double()
        st = self._lib.lgf_fix(self._h, float(alpha), float(tol), int(max_iter), ctypes.byref(it), ctypes.byref(F),
                               ctypes.byref(th))
        if check and st not in (LGF_OK, LGF_ERR_NOT_CONVERGED):
            raise LgfError(st, "lgf_fix")
        a, b = ctypes.c_int(), ctypes.c_int()
        self._lib.lgf_get_stats(self._h, ctypes.byref(a), ctypes.byref(b))
        return dict(status=st, iters=it.value, F=F.value, theta=th.value, converged=(st == LGF_OK),
                    iters_fp32=a.value, iters_fp64=b.value)

    def get_links(self, device=None):
        out, p, dev = _out(None, (4, self.V, 3, 3), device)
        _check(self._lib.lgf_get_links(self._h, p, dev), "lgf_get_links")
        return out

    def get_gauge(self, device=None):
        out, p, dev = _out(None, (self.V, 3, 3), device)
        _check(self._lib.lgf_get_gauge(self._h, p, dev), "lgf_get_gauge")
        return out

    def history(self, n_max: int = 1 << 16) -> np.ndarray:
        buf = np.zeros(2 * n_max, np.float64)
        w = ctypes.c_int()
        _check(self._lib.lgf_get_history(self._h, buf.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), n_max,
                                         ctypes.byref(w)), "lgf_get_history")
        return buf[: 2 * w.value].reshape(-1, 2)

    def delta(self, device=None, precision: int = 64):
        """Delta, theta and F of the stored links; precision 32: as the FP32
        phase of a mixed context computes them (lgf_delta32)."""
        fn, name = self._stage_fn("lgf_delta", precision)
        out, p, dev = _out(None, (self.V, 3, 3), device)
        th, F = ctypes.c_double(), ctypes.c_double()
        _check(fn(self._h, p, dev, ctypes.byref(th), ctypes.byref(F)), name)
        return out, th.value, F.value

    def accelerate(self, D, precision: int = 64):
        """Delta~ of D; precision 32: with the FP32 phase's kernels (lgf_accelerate32)."""
        fn, name = self._stage_fn("lgf_accelerate", precision)
        p, dev_in, keep = _in_ptr(D, (self.V, 3, 3))
        out, q, dev = _out(None, (self.V, 3, 3), keep.device if dev_in else None)
        _check(fn(self._h, p, q, dev), name)
        del keep
        return out

    def build_g(self, Dt, alpha: float, precision: int = 64):
        """g = reunit(1 + alpha/2 Dt); precision 32: with the FP32 phase's kernels (lgf_build_g32)."""
        fn, name = self._stage_fn("lgf_build_g", precision)
        p, dev_in, keep = _in_ptr(Dt, (self.V, 3, 3))
        out, q, dev = _out(None, (self.V, 3, 3), keep.device if dev_in else None)
        _check(fn(self._h, p, float(alpha), q, dev), name)
        del keep
        return out

    def _stage_fn(self, base: str, precision: int):
        if precision not in (64, 32):
            raise ValueError("precision must be 64 or 32")
        name = base if precision == 64 else base + "32"
        return getattr(self._lib, name), name


def lgf_accelerate_noalloc(dims, Delta_in, Dt_out, stream=None) -> None:
    """Context-free Fourier acceleration into a caller-provided output, with the
    library's static device scratch (no device allocation by the call).
    Delta_in and Dt_out: contiguous torch complex128 CUDA tensors (V, 3, 3)."""
    import torch

    lib = load()
    V = int(np.prod([int(v) for v in dims]))
    # the kernels read and write V*9 complex128 values on the current device: refuse
    # anything else here, before a pointer reaches the library
    for name, t in (("Delta_in", Delta_in), ("Dt_out", Dt_out)):
        if not _is_torch(t) or not t.is_cuda:
            raise TypeError("%s must be a torch CUDA tensor" % name)
        if t.dtype != torch.complex128:
            raise TypeError("%s must be complex128, got %s" % (name, t.dtype))
        if tuple(t.shape) != (V, 3, 3) or not t.is_contiguous():
            raise ValueError("%s must be a contiguous (%d, 3, 3) tensor, got %s" % (name, V, tuple(t.shape)))
        if t.device.index != torch.cuda.current_device():
            raise ValueError("%s is on %s, not on the current device cuda:%d"
                             % (name, t.device, torch.cuda.current_device()))
    raw = getattr(stream, "cuda_stream", stream) or 0
    arr = (ctypes.c_int * 4)(*[int(v) for v in dims])
    _check(lib.lgf_accelerate_noalloc(arr, ctypes.c_void_p(Delta_in.data_ptr()), ctypes.c_void_p(Dt_out.data_ptr()),
                                      ctypes.c_void_p(raw)), "lgf_accelerate_noalloc")


KERNELS = ("delta_xyfft", "zt_fft_accel", "xyifft_g", "update")


def _time_kernels(self, alpha: float = 0.08, n_iter: int = 5, precision: int = 64) -> dict:
    """Mean per-launch time (ms) of the four iteration kernels, launched one by one."""
    ms = (ctypes.c_double * 4)()
    _check(self._lib.lgf_time_kernels(self._h, float(alpha), int(n_iter), int(precision), ms), "lgf_time_kernels")
    return dict(zip(KERNELS, list(ms)))


Lattice.time_kernels = _time_kernels


def _autotune(self) -> None:
    """Pick the FFT kernels' launch shapes for this lattice by timing (needs links)."""
    _check(self._lib.lgf_autotune(self._h), "lgf_autotune")


Lattice.autotune = _autotune


def _set_shape(self, precision: int = 64, nt_xy: int = 128, nt_zt: int = 128, xw: int = 4, zt_form: int = 0) -> None:
    """Launch shape of one precision's FFT kernels (zt_form 1: the persistent z,t
    kernel with TMA-staged pencils); raises LgfError (LGF_ERR_ARG) for a shape the
    kernels cannot run."""
    _check(self._lib.lgf_set_shape(self._h, int(precision), int(nt_xy), int(nt_zt), int(xw), int(zt_form)),
           "lgf_set_shape")


def _get_shape(self, precision: int = 64) -> dict:
    out = (ctypes.c_int * 5)()
    _check(self._lib.lgf_get_shape(self._h, int(precision), out), "lgf_get_shape")
    return dict(zip(("nt_xy", "nt_zt", "xw", "zt_form", "zt_grid"), list(out)))


Lattice.set_shape = _set_shape
Lattice.get_shape = _get_shape


def probe_fma(precision: int = 64, n_iter: int = 100000) -> dict:
    """FMA rate (GFLOP/s, an FMA counted as two flops) of the current GPU in FP64 or FP32."""
    lib = load()
    gf, ms = ctypes.c_double(), ctypes.c_double()
    _check(lib.lgf_probe_fma(int(precision), int(n_iter), ctypes.byref(gf), ctypes.byref(ms)), "lgf_probe_fma")
    return dict(gflops=gf.value, ms=ms.value, precision=precision, n_iter=n_iter)


def check_conversions(d_in, f_in):
    """The integer-pipe float/double conversions of the FP32 phase's g builder,
    applied to d_in (float64 CUDA tensor) and f_in (float32 CUDA tensor, same
    length): returns (d_in rounded to float32, f_in widened to float64)."""
    import torch

    if not (_is_torch(d_in) and _is_torch(f_in) and d_in.is_cuda and f_in.is_cuda):
        raise TypeError("check_conversions takes CUDA tensors")
    if d_in.dtype != torch.float64 or f_in.dtype != torch.float32 or d_in.numel() != f_in.numel():
        raise TypeError("check_conversions takes a float64 and a float32 tensor of the same length")
    d_in, f_in = d_in.contiguous(), f_in.contiguous()
    f_out = torch.empty_like(f_in)
    d_out = torch.empty_like(d_in)
    with torch.cuda.device(d_in.device):
        _check(load().lgf_check_conversions(d_in.data_ptr(), f_out.data_ptr(), f_in.data_ptr(), d_out.data_ptr(),
                                            int(d_in.numel())), "lgf_check_conversions")
    return f_out, d_out


def _step_fwd(self, U_in, alpha: float = 0.08):
    """One Fourier-accelerated step of U_in (contiguous complex128 CUDA tensor
    (4, V, 3, 3)); returns the new links (the context then holds them)."""
    import torch

    assert _is_torch(U_in) and U_in.is_cuda and U_in.dtype == torch.complex128
    U_in = U_in.contiguous()
    U_out = torch.empty_like(U_in)
    _check(self._lib.lgf_step_fwd(self._h, float(alpha), ctypes.c_void_p(U_in.data_ptr()),
                                  ctypes.c_void_p(U_out.data_ptr())), "lgf_step_fwd")
    return U_out


def _step_bwd(self, g_out, alpha: float = 0.08):
    """Cotangent of the stored links (the step's input) from the cotangent g_out of
    the step's output; both contiguous complex128 CUDA tensors (4, V, 3, 3)."""
    import torch

    assert _is_torch(g_out) and g_out.is_cuda and g_out.dtype == torch.complex128
    g_out = g_out.contiguous()
    g_in = torch.empty_like(g_out)
    _check(self._lib.lgf_step_bwd(self._h, float(alpha), ctypes.c_void_p(g_out.data_ptr()),
                                  ctypes.c_void_p(g_in.data_ptr())), "lgf_step_bwd")
    return g_in


def _gluon_pmin(self):
    """(mean, [D(p) for the four momenta with one k_mu = 1]) of the stored links."""
    D = ctypes.c_double()
    Dp = (ctypes.c_double * 4)()
    _check(self._lib.lgf_gluon_pmin(self._h, ctypes.byref(D), Dp), "lgf_gluon_pmin")
    return D.value, list(Dp)


def _gluon_pmin_bwd(self, gD: float = 1.0, device="cuda"):
    import torch

    g = torch.empty((4, self.V, 3, 3), dtype=torch.complex128, device=device)
    _check(self._lib.lgf_gluon_pmin_bwd(self._h, float(gD), ctypes.c_void_p(g.data_ptr())), "lgf_gluon_pmin_bwd")
    return g


Lattice.step_fwd = _step_fwd
Lattice.step_bwd = _step_bwd
Lattice.gluon_pmin = _gluon_pmin
Lattice.gluon_pmin_bwd = _gluon_pmin_bwd


class Batch:
    """An ensemble of lattices (possibly of different extents) fixed by one graph launch."""

    def __init__(self, dims_list, mixed: bool = True, stream=None):
        lib = load()
        self.dims = [tuple(int(v) for v in d) for d in dims_list]
        self.n = len(self.dims)
        self.V = [int(np.prod(d)) for d in self.dims]
        arr = (ctypes.c_int * (4 * self.n))(*[v for d in self.dims for v in d])
        h = ctypes.c_void_p()
        flags = LGF_MIXED if mixed else LGF_FP64
        _check(lib.lgf_batch_create(self.n, arr, flags, ctypes.byref(h)), "lgf_batch_create")
        self._h, self._lib = h, lib
        if stream is not None:
            raw = getattr(stream, "cuda_stream", stream)
            _check(lib.lgf_batch_set_stream(h, ctypes.c_void_p(raw or 0)), "lgf_batch_set_stream")
            self._stream = stream

    def close(self):
        if getattr(self, "_h", None):
            self._lib.lgf_batch_destroy(self._h)
            self._h = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_switch_tol(self, tol: float):
        _check(self._lib.lgf_batch_set_switch_tol(self._h, float(tol)), "lgf_batch_set_switch_tol")

    def set_accel_precision(self, bits: int):
        _check(self._lib.lgf_batch_set_accel_precision(self._h, int(bits)), "lgf_batch_set_accel_precision")

    def set_fp32_update(self, form: int):
        _check(self._lib.lgf_batch_set_fp32_update(self._h, int(form)), "lgf_batch_set_fp32_update")

    def set_links(self, i: int, U):
        p, dev, keep = _in_ptr(U, (4, self.V[i], 3, 3))
        _check(self._lib.lgf_batch_set_links(self._h, int(i), p, dev), "lgf_batch_set_links")
        del keep

    def fix(self, alpha: float = 0.08, tol: float = 1e-15, max_iter: int = 100000) -> dict:
        n = self.n
        it = (ctypes.c_int * n)()
        F = (ctypes.c_double * n)()
        th = (ctypes.c_double * n)()
        st = (ctypes.c_int * n)()
        tr = (ctypes.c_double * n)()
        rc = self._lib.lgf_batch_fix(self._h, float(alpha), float(tol), int(max_iter), it, F, th, st, tr)
        if rc not in (LGF_OK, LGF_ERR_NOT_CONVERGED):
            raise LgfError(rc, "lgf_batch_fix")
        a, b = ctypes.c_int(), ctypes.c_int()
        i32, i64 = [], []
        for i in range(n):
            self._lib.lgf_batch_get_stats(self._h, i, ctypes.byref(a), ctypes.byref(b))
            i32.append(a.value)
            i64.append(b.value)
        return dict(status=list(st), iters=list(it), F=list(F), theta=list(th), t_retire_ms=list(tr),
                    iters_fp32=i32, iters_fp64=i64, rc=rc)

    def get_links(self, i: int, device=None):
        out, p, dev = _out(None, (4, self.V[i], 3, 3), device)
        _check(self._lib.lgf_batch_get_links(self._h, int(i), p, dev), "lgf_batch_get_links")
        return out

    def get_gauge(self, i: int, device=None):
        out, p, dev = _out(None, (self.V[i], 3, 3), device)
        _check(self._lib.lgf_batch_get_gauge(self._h, int(i), p, dev), "lgf_batch_get_gauge")
        return out


def fix(U, dims, alpha: float = 0.08, tol: float = 1e-15, max_iter: int = 100000, mixed: bool = False):
    """One-shot convenience: gauge-fix U and return (links, G, info)."""
    with Lattice(dims, mixed=mixed) as lat:
        lat.set_links(U)
        info = lat.fix(alpha, tol, max_iter)
        return lat.get_links(), lat.get_gauge(), info


def _set_unit_links(self):
    """Store U_mu(x) = 1 (cold start) and reset G."""
    _check(self._lib.lgf_set_unit_links(self._h), "lgf_set_unit_links")


def _wilson_sweeps(self, beta: float, seed: int, first_sweep: int = 0, n_heatbath: int = 1, n_overrelax: int = 0):
    """Wilson-action Monte Carlo of the stored links on the GPU: n_heatbath times,
    one heat-bath sweep (random-number sweep counter first_sweep + i) followed by
    n_overrelax overrelaxation sweeps.  Resets G."""
    _check(self._lib.lgf_wilson_sweeps(self._h, float(beta), int(seed) & 0xFFFFFFFFFFFFFFFF, int(first_sweep),
                                       int(n_heatbath), int(n_overrelax)), "lgf_wilson_sweeps")


def _plaquette(self) -> float:
    """Mean Re Tr U_P / 3 over all plaquettes of the stored links."""
    P = ctypes.c_double()
    _check(self._lib.lgf_plaquette(self._h, ctypes.byref(P)), "lgf_plaquette")
    return P.value


def _set_generator_precision(self, bits: int):
    """64 (default) or 32: arithmetic of the Wilson generator's staples, draws and
    rotations (with 32 the links stay FP64 in memory, re-orthonormalised in FP64)."""
    _check(self._lib.lgf_set_generator_precision(self._h, int(bits)), "lgf_set_generator_precision")


Lattice.set_generator_precision = _set_generator_precision
Lattice.set_unit_links = _set_unit_links
Lattice.wilson_sweeps = _wilson_sweeps
Lattice.plaquette = _plaquette


def _save_links(self, out=None):
    """Snapshot of the stored links in the library's layout: a uint8 CUDA tensor
    (reused when `out` is given)."""
    import torch

    n = int(self._lib.lgf_links_state_bytes(self._h))
    if out is None:
        out = torch.empty(n, dtype=torch.uint8, device="cuda")
    assert out.is_cuda and out.numel() == n and out.is_contiguous()
    _check(self._lib.lgf_save_links(self._h, ctypes.c_void_p(out.data_ptr())), "lgf_save_links")
    return out


def _load_links(self, snap):
    """Store a snapshot made by save_links of a lattice with the same extents and flags."""
    n = int(self._lib.lgf_links_state_bytes(self._h))
    assert snap.is_cuda and snap.numel() * snap.element_size() == n and snap.is_contiguous()
    _check(self._lib.lgf_load_links(self._h, ctypes.c_void_p(snap.data_ptr())), "lgf_load_links")


Lattice.save_links = _save_links
Lattice.load_links = _load_links
