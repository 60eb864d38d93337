"""Python binding of libpd, the sm_103a peridynamic stiffness library.

The functions below carry the names of the C entry points declared in
``include/pd.h`` and only marshal arguments (torch CUDA tensors -> device
pointers, the current torch stream -> cudaStream_t); every step of the
computation runs in the library's CUDA kernels.  There is no CPU fallback:
importing works without a GPU (so the exported symbols can be checked), but
every call needs the compiled library and a CUDA device and raises otherwise.

``Grid`` is a small convenience wrapper around the same calls.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpd.so")

PD_OK, PD_ERR_INVALID, PD_ERR_CUDA, PD_ERR_OOM, PD_ERR_NOT_CONVERGED, PD_ERR_TIMEOUT, PD_ERR_STATE = range(7)
PD_F32 = 0x1
PD_F64 = 0x2
PD_METHOD_AUTO = 0x00
PD_METHOD_STENCIL = 0x10
PD_METHOD_FFT = 0x20
PD_PROJECT = 0x100
PD_IGNORE_BROKEN = 0x200
PD_NO_TMA = 0x400
PD_ACCURATE = 0x800
PD_PAIR_FORM = 0x1000
PD_CG_F64 = 0x1
PD_CG_MIXED = 0x2
PD_CG_GRAPH = 0x10
PD_SC_NONE = 0
PD_SC_VOLUME = 1
PD_ADR_F64 = 0x1
PD_ADR_MIXED = 0x2
PD_PLANE_STRESS = 0
PD_PLANE_STRAIN = 1

_STATUS = {0: "PD_OK", 1: "PD_ERR_INVALID", 2: "PD_ERR_CUDA", 3: "PD_ERR_OOM", 4: "PD_ERR_NOT_CONVERGED",
           5: "PD_ERR_TIMEOUT", 6: "PD_ERR_STATE"}


class PDError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_STATUS.get(code, code)}: {msg}")
        self.code = code


class pd_grid_info(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("M", ctypes.c_int), ("nnb", ctypes.c_int), ("mask_words", ctypes.c_int),
                ("n", ctypes.c_int64 * 3), ("N", ctypes.c_int64), ("h", ctypes.c_double),
                ("delta", ctypes.c_double), ("alpha", ctypes.c_double), ("n_broken_nodes", ctypes.c_int64),
                ("device_error", ctypes.c_int32), ("auto_method", ctypes.c_int32 * 2),
                ("stencil_tile_rows", ctypes.c_int32)]


class pd_cg_stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("outer", ctypes.c_int), ("f64_matvecs", ctypes.c_int),
                ("rel_residual", ctypes.c_double), ("seconds", ctypes.c_double), ("persistent", ctypes.c_int)]


class pd_step_stats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int64), ("newly_broken", ctypes.c_int64), ("broken_total", ctypes.c_int64)]


# name -> (restype, argtypes); mirrors include/pd.h
_VP, _I, _U32, _D, _I64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint32, ctypes.c_double, ctypes.c_int64
SIGNATURES = {
    "pd_create_grid": (_I, [_I, ctypes.POINTER(_I64), _D, _D, _VP, ctypes.POINTER(_VP)]),
    "pd_set_material": (_I, [_VP, _D, _D, _D, _D, _VP]),
    "pd_set_surface_correction": (_I, [_VP, _I]),
    "pd_matvec": (_I, [_VP, _VP, _VP, _U32, _VP]),
    "pd_matvec_batch": (_I, [_VP, _I64, _VP, _VP, _U32, _VP]),
    "pd_matvec_batch_host": (_I, [_VP, _I64, _VP, _VP, _U32, _VP]),
    "pd_matvec_rows": (_I, [_VP, _I64, _I64, _I64, _VP, _I64, _I64, _VP, _U32, _VP]),
    "pd_cg_solve": (_I, [_VP, _VP, _VP, _D, _I, _U32, ctypes.POINTER(pd_cg_stats), _VP]),
    "pd_adr_solve": (_I, [_VP, _VP, _VP, _D, _I, _U32, ctypes.POINTER(pd_cg_stats), _VP]),
    "pd_step": (_I, [_VP, _VP, _VP, _VP, _I, _D, _VP, _VP, ctypes.c_int32, ctypes.POINTER(pd_step_stats), _VP]),
    "pd_step_noalloc": (_I, [_VP, _VP, _VP, _VP, _I, _D, _VP, _VP, ctypes.c_int32, ctypes.POINTER(pd_step_stats),
                             _VP]),
    "pd_step_adjoint": (_I, [_VP, _VP, _VP, _VP, _I, _D, _VP, _VP, _VP, ctypes.c_int32, _VP, _VP, _VP, _VP, _VP]),
    "pd_batch_create": (_I, [_VP, _I, ctypes.POINTER(_VP)]),
    "pd_batch_cg_solve": (_I, [_VP, _VP, _VP, _D, _I, ctypes.POINTER(pd_cg_stats), _VP]),
    "pd_batch_destroy": (_I, [_VP]),
    "pd_break_bonds": (_I, [_VP, _VP, _U32, ctypes.POINTER(_I64), _VP]),
    "pd_break_segment": (_I, [_VP, ctypes.POINTER(_I64), _I64, ctypes.POINTER(_I64), _VP]),
    "pd_set_method": (_I, [_VP, _U32]),
    "pd_set_stencil_tile_rows": (_I, [_VP, _I]),
    "pd_autotune": (_I, [_VP, _U32, _VP, _VP]),
    "pd_autotune_cached": (_I, [_VP, _U32, ctypes.c_char_p, ctypes.POINTER(_I), _VP, _VP]),
    "pd_get_info": (_I, [_VP, ctypes.POINTER(pd_grid_info)]),
    "pd_get_offsets": (_I, [_VP, _VP, _I]),
    "pd_get_coefficients": (_I, [_VP, _VP, _I]),
    "pd_get_bond_mask": (_I, [_VP, _VP, _VP]),
    "pd_set_bond_mask": (_I, [_VP, _VP, _VP]),
    "pd_grad_modulus": (_I, [_VP, _VP, _VP, _D, _VP, _VP]),
    "pd_destroy": (_I, [_VP]),
    "pd_critical_stretch": (_I, [_D, _D, _D, _I, ctypes.POINTER(_D)]),
    "pd_check_wait_timeout": (_I, [_VP, _I64, _VP]),
    "pd_probe_fma_rate": (_I, [_U32, ctypes.POINTER(_D), _VP]),
    "pd_stable_dt": (_I, [_VP, ctypes.POINTER(_D)]),
    "pd_last_error": (ctypes.c_char_p, []),
}

_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Loads libpd.so (raises if it has not been built: there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise ImportError(f"libpd.so is not built ({path}); run __graft_entry__.build()")
        L = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(rc: int):
    if rc != PD_OK:
        raise PDError(rc, load_library().pd_last_error().decode())


def _stream(stream=None):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _dptr(t, dtype=None):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"expected {dtype}, got {t.dtype}")
    return ctypes.c_void_p(t.data_ptr())


def _dtype_flag(t):
    import torch
    if t.dtype == torch.float32:
        return PD_F32
    if t.dtype == torch.float64:
        return PD_F64
    raise ValueError("vectors must be float32 or float64")


# ------------------------------------------------------------------ the C entry points

def pd_create_grid(dim: int, n: Sequence[int], h: float, delta: float, constrained=None) -> ctypes.c_void_p:
    arr = (ctypes.c_int64 * 3)(*(list(int(v) for v in n) + [1] * (3 - len(n))))
    cons = None
    if constrained is not None:
        c = np.ascontiguousarray(constrained, dtype=np.uint8)
        cons = c.ctypes.data_as(ctypes.c_void_p)
    out = ctypes.c_void_p()
    _check(load_library().pd_create_grid(dim, arr, float(h), float(delta), cons, ctypes.byref(out)))
    return out


def pd_set_material(g, E=1.0, rho=1.0, thickness=1.0, s0=0.0, E_field=None):
    import torch
    _check(load_library().pd_set_material(g, float(E), float(rho), float(thickness), float(s0),
                                          _dptr(E_field, torch.float64)))


def pd_check_wait_timeout(g, spins: int, stream=None):
    """Bounded device wait on a flag nothing sets: raises PDError(PD_ERR_TIMEOUT)."""
    _check(load_library().pd_check_wait_timeout(g, int(spins), _stream(stream)))


def pd_stable_dt(g) -> float:
    """Largest stable Verlet step of the grid (see pd.h)."""
    out = ctypes.c_double(0.0)
    _check(load_library().pd_stable_dt(g, ctypes.byref(out)))
    return out.value


def pd_probe_fma_rate(flags: int, stream=None) -> float:
    """Measured FMA throughput of the current device in FLOP/s (PD_F32 or PD_F64)."""
    out = ctypes.c_double(0.0)
    _check(load_library().pd_probe_fma_rate(int(flags), ctypes.byref(out), _stream(stream)))
    return out.value


def pd_critical_stretch(G0: float, E: float, delta: float, mode: int = PD_PLANE_STRESS) -> float:
    """Critical bond stretch from the energy release rate (host only)."""
    out = ctypes.c_double(0.0)
    _check(load_library().pd_critical_stretch(float(G0), float(E), float(delta), int(mode), ctypes.byref(out)))
    return out.value


def pd_set_surface_correction(g, mode: int):
    _check(load_library().pd_set_surface_correction(g, int(mode)))


def pd_matvec(g, u, out, flags: int, stream=None):
    _check(load_library().pd_matvec(g, _dptr(u), _dptr(out), int(flags), _stream(stream)))


def pd_matvec_batch(g, batch: int, u, out, flags: int, stream=None):
    _check(load_library().pd_matvec_batch(g, int(batch), _dptr(u), _dptr(out), int(flags), _stream(stream)))


def pd_matvec_rows(g, batch: int, row0: int, rows: int, u_ext, ext_row0: int, ext_rows: int, out, flags: int,
                   stream=None):
    _check(load_library().pd_matvec_rows(g, int(batch), int(row0), int(rows), _dptr(u_ext), int(ext_row0),
                                         int(ext_rows), _dptr(out), int(flags), _stream(stream)))


def _hptr(t):
    if t.is_cuda:
        raise ValueError("expected a host (CPU) tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def pd_matvec_batch_host(g, batch: int, u_host, out_host, flags: int, stream=None):
    """K u for `batch` fields in HOST memory (pinned for full bandwidth), copies overlapped
    with the product; ordered on `stream` (out_host is complete after it synchronises)."""
    _check(load_library().pd_matvec_batch_host(g, int(batch), _hptr(u_host), _hptr(out_host), int(flags),
                                               _stream(stream)))


def pd_adr_solve(g, b, u, rtol: float, max_iter: int, stream=None, allow_not_converged=False, mode=PD_ADR_F64):
    import torch
    st = pd_cg_stats()
    rc = load_library().pd_adr_solve(g, _dptr(b, torch.float64), _dptr(u, torch.float64), float(rtol), int(max_iter),
                                     int(mode), ctypes.byref(st), _stream(stream))
    if not (allow_not_converged and rc == PD_ERR_NOT_CONVERGED):
        _check(rc)
    return st


def pd_cg_solve(g, b, u, rtol: float, max_iter: int, mode: int, stream=None, allow_not_converged=False):
    import torch
    st = pd_cg_stats()
    rc = load_library().pd_cg_solve(g, _dptr(b, torch.float64), _dptr(u, torch.float64), float(rtol),
                                    int(max_iter), int(mode), ctypes.byref(st), _stream(stream))
    if not (allow_not_converged and rc == PD_ERR_NOT_CONVERGED):
        _check(rc)
    return st


def pd_step(g, u, v, b, nsteps: int, dt: float, v_prescribed=None, break_step=None, step_base: int = 0,
            stream=None):
    import torch
    st = pd_step_stats()
    _check(load_library().pd_step(g, _dptr(u, torch.float64), _dptr(v, torch.float64), _dptr(b, torch.float64),
                                  int(nsteps), float(dt), _dptr(v_prescribed, torch.float64),
                                  _dptr(break_step, torch.int32), int(step_base), ctypes.byref(st),
                                  _stream(stream)))
    return st


def pd_step_noalloc(g, u, v, b, nsteps: int, dt: float, v_prescribed=None, break_step=None, step_base: int = 0,
                    stream=None):
    """pd_step without device allocation (fixed internal scratch; dim * N <= 524288)."""
    import torch
    st = pd_step_stats()
    _check(load_library().pd_step_noalloc(g, _dptr(u, torch.float64), _dptr(v, torch.float64),
                                          _dptr(b, torch.float64), int(nsteps), float(dt),
                                          _dptr(v_prescribed, torch.float64), _dptr(break_step, torch.int32),
                                          int(step_base), ctypes.byref(st), _stream(stream)))
    return st


def pd_step_adjoint(g, u_start, v_start, b, nsteps: int, dt: float, v_prescribed, mask0, break_step,
                    step_base: int, ubar, vbar, abar, grad_E=None, stream=None):
    import torch
    f64 = torch.float64
    _check(load_library().pd_step_adjoint(g, _dptr(u_start, f64), _dptr(v_start, f64), _dptr(b, f64), int(nsteps),
                                          float(dt), _dptr(v_prescribed, f64), _dptr(mask0, torch.int32),
                                          _dptr(break_step, torch.int32), int(step_base), _dptr(ubar, f64),
                                          _dptr(vbar, f64), _dptr(abar, f64), _dptr(grad_E, f64), _stream(stream)))


def pd_batch_create(grids) -> ctypes.c_void_p:
    arr = (ctypes.c_void_p * len(grids))(*[getattr(g, "handle", g) for g in grids])
    out = ctypes.c_void_p()
    _check(load_library().pd_batch_create(arr, len(grids), ctypes.byref(out)))
    return out


def pd_batch_cg_solve(bt, bs, us, rtol: float, max_iter: int, stream=None, allow_not_converged=False):
    """bs, us: lists of float64 CUDA tensors [2, ny_i, nx_i]; returns per-plate pd_cg_stats."""
    import torch
    n = len(bs)
    bp = (ctypes.c_void_p * n)(*[_dptr(b, torch.float64).value for b in bs])
    up = (ctypes.c_void_p * n)(*[_dptr(u, torch.float64).value for u in us])
    st = (pd_cg_stats * n)()
    rc = load_library().pd_batch_cg_solve(bt, bp, up, float(rtol), int(max_iter), st, _stream(stream))
    if not (allow_not_converged and rc == PD_ERR_NOT_CONVERGED):
        _check(rc)
    return list(st)


def pd_batch_destroy(bt):
    if bt is not None and bt.value:
        _check(load_library().pd_batch_destroy(bt))


def pd_break_bonds(g, u, stream=None) -> int:
    n = ctypes.c_int64(0)
    _check(load_library().pd_break_bonds(g, _dptr(u), _dtype_flag(u), ctypes.byref(n), _stream(stream)))
    return int(n.value)


def pd_break_segment(g, seg, den: int, stream=None) -> int:
    s = (ctypes.c_int64 * 4)(*[int(v) for v in seg])
    n = ctypes.c_int64(0)
    _check(load_library().pd_break_segment(g, s, int(den), ctypes.byref(n), _stream(stream)))
    return int(n.value)


def pd_set_method(g, method: int):
    _check(load_library().pd_set_method(g, int(method)))


def pd_autotune(g, flags: int = PD_F32 | PD_F64, stream=None):
    t = (ctypes.c_double * 4)()
    _check(load_library().pd_autotune(g, int(flags), t, _stream(stream)))
    return {"stencil_f32_ms": t[0], "fft_f32_ms": t[1], "stencil_f64_ms": t[2], "fft_f64_ms": t[3]}


def pd_autotune_cached(g, cache_path: str, flags: int = PD_F32 | PD_F64, stream=None):
    """pd_autotune through a JSON cache file; returns (times, from_cache)."""
    t = (ctypes.c_double * 4)()
    hit = ctypes.c_int(0)
    _check(load_library().pd_autotune_cached(g, int(flags), os.fsencode(cache_path), ctypes.byref(hit), t,
                                             _stream(stream)))
    return ({"stencil_f32_ms": t[0], "fft_f32_ms": t[1], "stencil_f64_ms": t[2], "fft_f64_ms": t[3]},
            bool(hit.value))


def pd_set_stencil_tile_rows(g, rows: int):
    _check(load_library().pd_set_stencil_tile_rows(g, int(rows)))


def pd_get_info(g) -> pd_grid_info:
    info = pd_grid_info()
    _check(load_library().pd_get_info(g, ctypes.byref(info)))
    return info


def pd_get_offsets(g) -> np.ndarray:
    info = pd_get_info(g)
    buf = np.zeros((info.nnb, 3), dtype=np.int32)
    _check(load_library().pd_get_offsets(g, buf.ctypes.data_as(ctypes.c_void_p), info.nnb))
    return buf


def pd_get_coefficients(g) -> np.ndarray:
    """Bond blocks at the grid's modulus, [nnb][3] (2D) or [nnb][6] (3D), offset order."""
    info = pd_get_info(g)
    buf = np.zeros((info.nnb, 3 if info.dim == 2 else 6), dtype=np.float64)
    _check(load_library().pd_get_coefficients(g, buf.ctypes.data_as(ctypes.c_void_p), info.nnb))
    return buf


def pd_get_bond_mask(g, mask, stream=None):
    import torch
    _check(load_library().pd_get_bond_mask(g, _dptr(mask, torch.int32), _stream(stream)))


def pd_set_bond_mask(g, mask, stream=None):
    import torch
    _check(load_library().pd_set_bond_mask(g, _dptr(mask, torch.int32), _stream(stream)))


def pd_grad_modulus(g, u, lam, scale: float, grad, stream=None):
    import torch
    _check(load_library().pd_grad_modulus(g, _dptr(u, torch.float64), _dptr(lam, torch.float64), float(scale),
                                          _dptr(grad, torch.float64), _stream(stream)))


def pd_destroy(g):
    if g is not None and g.value:
        _check(load_library().pd_destroy(g))


def pd_last_error() -> str:
    return load_library().pd_last_error().decode()


# ------------------------------------------------------------------ convenience wrapper

class Grid:
    """Owns one pd_grid.  Vectors are torch CUDA tensors shaped [dim, (nz,) ny, nx]."""

    def __init__(self, dim: int, n: Sequence[int], h: float, M: int, constrained=None, E=1.0, rho=1.0,
                 thickness=1.0, s0=0.0, E_field=None, surface_correction: int = PD_SC_NONE):
        # M: delta / h (an integer in the paper's examples, any real >= 1 here)
        self.dim, self.n, self.h, self.m = dim, tuple(int(v) for v in n), float(h), float(M)
        self.handle = pd_create_grid(dim, self.n, h, self.m * h, constrained)
        self.set_material(E, rho, thickness, s0, E_field)
        if surface_correction:
            pd_set_surface_correction(self.handle, surface_correction)
        info = pd_get_info(self.handle)
        self.M = info.M   # the kernels' radius, ceil(delta / h)
        self.nnb, self.mask_words, self.alpha = info.nnb, info.mask_words, info.alpha

    @property
    def shape(self):
        return (self.dim,) + tuple(reversed(self.n))

    @property
    def N(self):
        return int(np.prod(self.n))

    def set_surface_correction(self, mode: int):
        """PD_SC_VOLUME: scale the bonds of incomplete horizons (volume method); PD_SC_NONE: off."""
        pd_set_surface_correction(self.handle, mode)

    def set_material(self, E=1.0, rho=1.0, thickness=1.0, s0=0.0, E_field=None):
        pd_set_material(self.handle, E, rho, thickness, s0, E_field)
        self.E, self.rho, self.thickness, self.s0 = float(E), float(rho), float(thickness), float(s0)
        self.alpha = pd_get_info(self.handle).alpha

    def matvec(self, u, out=None, flags: int = 0, stream=None):
        import torch
        if out is None:
            out = torch.empty_like(u)
        batch = u.numel() // (self.dim * self.N)
        if batch == 1:
            pd_matvec(self.handle, u, out, flags | _dtype_flag(u), stream)
        else:
            pd_matvec_batch(self.handle, batch, u, out, flags | _dtype_flag(u), stream)
        return out

    def adr_solve(self, b, u=None, rtol=1e-8, max_iter=1000000, mode=PD_ADR_F64, stream=None):
        """The paper's ADR/CDEI static solver (Algorithm 1): FP64, or FP32 operator with FP64 refresh."""
        import torch
        if u is None:
            u = torch.zeros_like(b)
        st = pd_adr_solve(self.handle, b, u, rtol, max_iter, stream, mode=mode)
        return u, st

    def cg_solve(self, b, u=None, rtol=1e-8, max_iter=100000, mode=PD_CG_MIXED, stream=None):
        import torch
        if u is None:
            u = torch.zeros_like(b)
        st = pd_cg_solve(self.handle, b, u, rtol, max_iter, mode, stream)
        return u, st

    def stable_dt(self) -> float:
        return pd_stable_dt(self.handle)

    def step(self, u, v, b=None, nsteps=1, dt=1e-3, v_prescribed=None, break_step=None, step_base=0, stream=None):
        return pd_step(self.handle, u, v, b, nsteps, dt, v_prescribed, break_step, step_base, stream)

    def break_bonds(self, u, stream=None) -> int:
        return pd_break_bonds(self.handle, u, stream)

    def break_segment(self, seg, den, stream=None) -> int:
        return pd_break_segment(self.handle, seg, den, stream)

    def prefer_method(self, method: int):
        pd_set_method(self.handle, method)

    def set_stencil_tile_rows(self, rows: int):
        pd_set_stencil_tile_rows(self.handle, rows)

    def autotune(self, flags: int = PD_F32 | PD_F64, stream=None):
        return pd_autotune(self.handle, flags, stream)

    def offsets(self) -> np.ndarray:
        return pd_get_offsets(self.handle)

    def bond_mask(self):
        import torch
        m = torch.empty((self.mask_words, self.N), dtype=torch.int32, device="cuda")
        pd_get_bond_mask(self.handle, m)
        return m

    def set_bond_mask(self, mask):
        pd_set_bond_mask(self.handle, mask.contiguous())

    def info(self) -> pd_grid_info:
        return pd_get_info(self.handle)

    def grad_modulus(self, u, lam, scale=-0.5, grad=None):
        import torch
        if grad is None:
            grad = torch.zeros(tuple(reversed(self.n)), dtype=torch.float64, device=u.device)
        pd_grad_modulus(self.handle, u, lam, scale, grad)
        return grad

    def close(self):
        if getattr(self, "handle", None) is not None:
            pd_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
