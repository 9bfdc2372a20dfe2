"""Thin ctypes binding of the C ABI in include/sem.h (libsemgb.so).

Argument marshalling only: every computation runs in the CUDA library.  The
functions keep the C names (sem_setup, sem_apply_condensed, ...); device
vectors are torch CUDA float64 tensors, host vectors NumPy float64 arrays.
Streams default to torch's current stream on the tensors' device.

If the library has not been built, loading fails loudly: there is no CPU or
Python fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# SEM_LIB selects another build of the library (the debug build of build.py)
LIB_PATH = os.environ.get("SEM_LIB") or os.path.join(_HERE, "libsemgb.so")

SEM_OK, SEM_EINVAL, SEM_ENOMEM, SEM_ECUDA, SEM_ENOCONV, SEM_EBREAKDOWN, SEM_ENOTSUP = range(7)
SPACE_NODAL, SPACE_TRANSFORMED = 0, 1
PREC_FP64, PREC_MIXED = 0, 1
# sem_transform_skeleton kinds
SOLUTION_TO_T, SOLUTION_FROM_T, LOAD_TO_T, LOAD_FROM_T = 0, 1, 2, 3


class SemError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{message} (status {status})")
        self.status = status


class sem_opts(ctypes.Structure):
    _fields_ = [("rtol", ctypes.c_double), ("maxit", ctypes.c_int), ("precision", ctypes.c_int),
                ("check_every", ctypes.c_int), ("inner_rtol", ctypes.c_double), ("max_refine", ctypes.c_int),
                ("mixed_scheme", ctypes.c_int), ("reliable_delta", ctypes.c_double), ("deterministic", ctypes.c_int),
                ("onepass_step", ctypes.c_int)]


class sem_info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("refinements", ctypes.c_int), ("rel_res", ctypes.c_double),
                ("t_solve_s", ctypes.c_double)]


_lib = None
_D = ctypes.POINTER(ctypes.c_double)
_P = ctypes.c_void_p


def lib():
    """Loads libsemgb.so (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_1601_08179_gb300.build`")
    L = ctypes.CDLL(LIB_PATH)
    sig = {
        "sem_default_opts": (None, [ctypes.POINTER(sem_opts)]),
        "sem_setup": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     _D, _D, _D, ctypes.c_double, ctypes.POINTER(sem_opts)]),
        "sem_set_lambda": (ctypes.c_int, [_P, ctypes.c_double]),
        "sem_set_opts": (ctypes.c_int, [_P, ctypes.POINTER(sem_opts)]),
        "sem_skeleton_size": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_longlong)]),
        "sem_grid_size": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_longlong)]),
        "sem_node_coords": (ctypes.c_int, [_P, _D, _D, _D]),
        "sem_get_basis": (ctypes.c_int, [_P, _D, _D, _D, _D]),
        "sem_apply_condensed": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, _P]),
        "sem_condense_rhs": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, _P]),
        "sem_apply_condensed_f32": (ctypes.c_int, [_P, _P, _P, _P]),
        "sem_condense_rhs_noalloc": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, _P]),
        "sem_precond_diag": (ctypes.c_int, [_P, _P, _P]),
        "sem_recover_interior": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, _P, _P]),
        "sem_solve": (ctypes.c_int, [_P, _P, _P, _P, ctypes.POINTER(sem_info), _P]),
        "sem_solve_host": (ctypes.c_int, [_P, _D, _D, ctypes.POINTER(sem_info), _P]),
        "sem_transform_skeleton": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, _P]),
        "sem_pack_skeleton": (ctypes.c_int, [_P, _P, _P, _P]),
        "sem_unpack_skeleton": (ctypes.c_int, [_P, _P, _P, _P]),
        "sem_refine_history": (ctypes.c_int, [_P, _D, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
        "sem_solve_adjoint": (ctypes.c_int, [_P, _P, _P, ctypes.POINTER(sem_info), _P]),
        "sem_autotune": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
        "sem_set_operator_kernel": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
        "sem_check_vector": (ctypes.c_int, [_P, _P, ctypes.c_int]),
        "sem_debug_oob": (ctypes.c_int, [ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)]),
        "sem_debug_limit_skeleton": (ctypes.c_int, [_P, ctypes.c_longlong]),
        "sem_debug_cg_step_timeout": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
        "sem_get_operator_kernel": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                                   ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
        "sem_batch_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, ctypes.POINTER(_P), ctypes.POINTER(_P),
                                            ctypes.POINTER(_P)]),
        "sem_batch_solve": (ctypes.c_int, [_P, ctypes.POINTER(sem_info), _P]),
        "sem_batch_destroy": (None, [_P]),
        "sem_solve_batch": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, ctypes.POINTER(_P), ctypes.POINTER(_P),
                                           ctypes.POINTER(sem_info), _P]),
        "sem_gradients": (ctypes.c_int, [_P, _P, _P, _P, _P, _D, _D, _D, _D, _P]),
        "sem_apply_condensed_variant": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, _P]),
        "sem_diag_nodal": (ctypes.c_int, [_P, _P, _P]),
        "sem_solve_variant": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, _P, _P, ctypes.POINTER(sem_info), _P]),
        "sem_profile_enable": (ctypes.c_int, [_P, ctypes.c_int]),
        "sem_profile_read": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong),
                                            ctypes.c_int]),
        "sem_launch_count": (ctypes.c_longlong, []),
        "sem_destroy": (None, [_P]),
        "sem_status_string": (ctypes.c_char_p, [ctypes.c_int]),
        "sem_last_error": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def exported_symbols():
    """Names of the entry points the binding expects the library to export."""
    return ["sem_default_opts", "sem_setup", "sem_set_lambda", "sem_set_opts", "sem_skeleton_size",
            "sem_grid_size", "sem_node_coords", "sem_get_basis", "sem_apply_condensed", "sem_condense_rhs",
            "sem_condense_rhs_noalloc", "sem_apply_condensed_f32",
            "sem_precond_diag", "sem_recover_interior", "sem_solve", "sem_solve_host",
            "sem_transform_skeleton", "sem_pack_skeleton", "sem_unpack_skeleton", "sem_refine_history",
            "sem_solve_adjoint", "sem_gradients", "sem_autotune", "sem_set_operator_kernel",
            "sem_get_operator_kernel", "sem_check_vector", "sem_debug_oob", "sem_debug_limit_skeleton",
            "sem_debug_cg_step_timeout",
            "sem_batch_create", "sem_batch_solve",
            "sem_batch_destroy", "sem_solve_batch",
            "sem_apply_condensed_variant", "sem_diag_nodal", "sem_solve_variant",
            "sem_profile_enable",
            "sem_profile_read", "sem_launch_count",
            "sem_destroy", "sem_status_string", "sem_last_error"]


def _check(status: int, allow=()):
    if status == SEM_OK or status in allow:
        return status
    msg = lib().sem_last_error().decode() or lib().sem_status_string(status).decode()
    raise SemError(status, msg)


def _dptr(t, n=None, name="tensor"):
    """Device pointer of a contiguous CUDA float64 torch tensor."""
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA torch tensor")
    if t.dtype != torch.float64 or not t.is_contiguous():
        raise TypeError(f"{name} must be contiguous float64")
    if n is not None and t.numel() != n:
        raise ValueError(f"{name} has {t.numel()} entries, expected {n}")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream, ref=None):
    import torch
    if stream is None:
        dev = ref.device if ref is not None else None
        stream = torch.cuda.current_stream(dev)
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _host(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_D)


def default_opts(**kw) -> sem_opts:
    o = sem_opts()
    lib().sem_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


@dataclass
class SemContext:
    """Handle returned by sem_setup (owns the C context)."""
    handle: ctypes.c_void_p
    p: int
    m: tuple
    nb: int
    n_nodes: int
    grid_shape: tuple

    def __del__(self):
        try:
            if self.handle:
                lib().sem_destroy(self.handle)
                self.handle = None
        except Exception:
            pass


def sem_setup(p, hx, hy, hz, lam, opts: sem_opts | None = None) -> SemContext:
    hx, phx = _host(hx)
    hy, phy = _host(hy)
    hz, phz = _host(hz)
    h = ctypes.c_void_p()
    _check(lib().sem_setup(ctypes.byref(h), int(p), len(hx), len(hy), len(hz), phx, phy, phz, float(lam),
                           ctypes.byref(opts) if opts is not None else None))
    nb, nn = ctypes.c_longlong(), ctypes.c_longlong()
    lib().sem_skeleton_size(h, ctypes.byref(nb))
    lib().sem_grid_size(h, ctypes.byref(nn))
    shape = (len(hz) * p + 1, len(hy) * p + 1, len(hx) * p + 1)
    return SemContext(h, int(p), (len(hx), len(hy), len(hz)), nb.value, nn.value, shape)


def sem_set_lambda(ctx: SemContext, lam: float):
    _check(lib().sem_set_lambda(ctx.handle, float(lam)))


def sem_set_opts(ctx: SemContext, opts: sem_opts | None):
    _check(lib().sem_set_opts(ctx.handle, ctypes.byref(opts) if opts is not None else None))


def sem_node_coords(ctx: SemContext):
    nz, ny, nx = ctx.grid_shape
    x, y, z = np.empty(nx), np.empty(ny), np.empty(nz)
    _check(lib().sem_node_coords(ctx.handle, x.ctypes.data_as(_D), y.ctypes.data_as(_D), z.ctypes.data_as(_D)))
    return x, y, z


def sem_get_basis(ctx: SemContext):
    p, n = ctx.p, ctx.p - 1
    gx, gw, lam, V = np.empty(p + 1), np.empty(p + 1), np.empty(n), np.empty(n * n)
    _check(lib().sem_get_basis(ctx.handle, gx.ctypes.data_as(_D), gw.ctypes.data_as(_D), lam.ctypes.data_as(_D),
                               V.ctypes.data_as(_D)))
    return gx, gw, lam, V.reshape(n, n)


def sem_apply_condensed(ctx: SemContext, uB, vB, space=SPACE_TRANSFORMED, stream=None):
    _check(lib().sem_apply_condensed(ctx.handle, _dptr(uB, ctx.nb, "uB"), _dptr(vB, ctx.nb, "vB"), int(space),
                                     _stream(stream, uB)))


def _fptr(t, n, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous CUDA float32 tensor")
    if t.numel() != n:
        raise ValueError(f"{name} has {t.numel()} entries, expected {n}")
    return ctypes.c_void_p(t.data_ptr())


def sem_apply_condensed_f32(ctx: SemContext, uB, vB, stream=None):
    """FP32 transformed-space operator (float32 tensors of length N_B)."""
    _check(lib().sem_apply_condensed_f32(ctx.handle, _fptr(uB, ctx.nb, "uB"), _fptr(vB, ctx.nb, "vB"),
                                         _stream(stream, uB)))


def sem_condense_rhs(ctx: SemContext, f, fB, space=SPACE_TRANSFORMED, stream=None):
    _check(lib().sem_condense_rhs(ctx.handle, _dptr(f, ctx.n_nodes, "f"), _dptr(fB, ctx.nb, "fB"), int(space),
                                  _stream(stream, f)))


def sem_condense_rhs_noalloc(ctx: SemContext, f, fB, space=SPACE_TRANSFORMED, stream=None):
    """sem_condense_rhs for callers that cannot allocate device memory during
    the call (it uses the library's fixed scratch array; see include/sem.h)."""
    _check(lib().sem_condense_rhs_noalloc(ctx.handle, _dptr(f, ctx.n_nodes, "f"), _dptr(fB, ctx.nb, "fB"),
                                          int(space), _stream(stream, f)))


def sem_precond_diag(ctx: SemContext, diag, stream=None):
    _check(lib().sem_precond_diag(ctx.handle, _dptr(diag, ctx.nb, "diag"), _stream(stream, diag)))


def sem_recover_interior(ctx: SemContext, f, uB, u, space=SPACE_TRANSFORMED, stream=None):
    _check(lib().sem_recover_interior(ctx.handle, _dptr(f, ctx.n_nodes, "f"), _dptr(uB, ctx.nb, "uB"), int(space),
                                      _dptr(u, ctx.n_nodes, "u"), _stream(stream, f)))


def sem_solve(ctx: SemContext, f, u, u0=None, stream=None, check=True) -> dict:
    info = sem_info()
    st = lib().sem_solve(ctx.handle, _dptr(f, ctx.n_nodes, "f"), _dptr(u, ctx.n_nodes, "u"),
                         _dptr(u0, ctx.nb, "u0") if u0 is not None else None, ctypes.byref(info),
                         _stream(stream, f))
    if check:
        _check(st)
    return dict(status=st, iters=info.iters, refinements=info.refinements, rel_res=info.rel_res,
                t_solve_s=info.t_solve_s)


def sem_solve_host(ctx: SemContext, f_host: np.ndarray, u_host: np.ndarray, stream=None, check=True) -> dict:
    if f_host.dtype != np.float64 or not f_host.flags.c_contiguous or f_host.size != ctx.n_nodes:
        raise TypeError("f_host must be a contiguous float64 array of the grid size")
    if u_host.dtype != np.float64 or not u_host.flags.c_contiguous or u_host.size != ctx.n_nodes:
        raise TypeError("u_host must be a contiguous float64 array of the grid size")
    info = sem_info()
    st = lib().sem_solve_host(ctx.handle, f_host.ctypes.data_as(_D), u_host.ctypes.data_as(_D), ctypes.byref(info),
                              _stream(stream))
    if check:
        _check(st)
    return dict(status=st, iters=info.iters, refinements=info.refinements, rel_res=info.rel_res,
                t_solve_s=info.t_solve_s)


def sem_transform_skeleton(ctx: SemContext, inp, out, kind: int, stream=None):
    _check(lib().sem_transform_skeleton(ctx.handle, _dptr(inp, ctx.nb, "in"), _dptr(out, ctx.nb, "out"), int(kind),
                                        _stream(stream, inp)))


def sem_pack_skeleton(ctx: SemContext, u_full, uB, stream=None):
    _check(lib().sem_pack_skeleton(ctx.handle, _dptr(u_full, ctx.n_nodes, "u_full"), _dptr(uB, ctx.nb, "uB"),
                                   _stream(stream, u_full)))


def sem_unpack_skeleton(ctx: SemContext, uB, u_full, stream=None):
    _check(lib().sem_unpack_skeleton(ctx.handle, _dptr(uB, ctx.nb, "uB"), _dptr(u_full, ctx.n_nodes, "u_full"),
                                     _stream(stream, uB)))


def sem_solve_adjoint(ctx: SemContext, g, w, stream=None, check=True) -> dict:
    """w = A^-1 g (g a nodal load, e.g. dJ/du)."""
    info = sem_info()
    st = lib().sem_solve_adjoint(ctx.handle, _dptr(g, ctx.n_nodes, "g"), _dptr(w, ctx.n_nodes, "w"),
                                 ctypes.byref(info), _stream(stream, g))
    if check:
        _check(st)
    return dict(status=st, iters=info.iters, refinements=info.refinements, rel_res=info.rel_res,
                t_solve_s=info.t_solve_s)


def sem_gradients(ctx: SemContext, w, u, f, df, stream=None):
    """Returns (dlambda, dhx, dhy, dhz); writes df (device) in place."""
    mx, my, mz = ctx.m
    dl = ctypes.c_double()
    dhx, dhy, dhz = np.empty(mx), np.empty(my), np.empty(mz)
    _check(lib().sem_gradients(ctx.handle, _dptr(w, ctx.n_nodes, "w"), _dptr(u, ctx.n_nodes, "u"),
                               _dptr(f, ctx.n_nodes, "f"), _dptr(df, ctx.n_nodes, "df"), ctypes.byref(dl),
                               dhx.ctypes.data_as(_D), dhy.ctypes.data_as(_D), dhz.ctypes.data_as(_D),
                               _stream(stream, w)))
    return dl.value, dhx, dhy, dhz


KERNEL_AUTO, KERNEL_CTA_TILE, KERNEL_WARP, KERNEL_PLANE, KERNEL_ELEMENT, KERNEL_SLAB, KERNEL_ROW = 0, 1, 2, 3, 4, 5, 6
KERNEL_PENCIL = 7
KERNEL_NAMES = {KERNEL_CTA_TILE: "cta_tile", KERNEL_WARP: "warp", KERNEL_PLANE: "plane", KERNEL_ELEMENT: "element",
                KERNEL_SLAB: "slab", KERNEL_ROW: "row", KERNEL_PENCIL: "pencil"}


def sem_set_operator_kernel(ctx: SemContext, precision: int, kind: int, epb: int = 0, ks: int = 0):
    """Selects the operator kernel variant of one precision (PREC_FP64 or PREC_MIXED)."""
    _check(lib().sem_set_operator_kernel(ctx.handle, int(precision), int(kind), int(epb), int(ks)))


def sem_get_operator_kernel(ctx: SemContext, precision: int):
    """(kind, epb, ks) of the operator kernel in use for one precision."""
    k, e, s = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(lib().sem_get_operator_kernel(ctx.handle, int(precision), ctypes.byref(k), ctypes.byref(e),
                                         ctypes.byref(s)))
    return k.value, e.value, s.value


def sem_check_vector(ctx: SemContext, ptr: int, elem_bytes: int) -> int:
    """Status of the check every entry point makes of a vector address (no
    launch): SEM_OK for device memory of the context's device (or managed
    memory) aligned to elem_bytes, else SEM_EINVAL."""
    return lib().sem_check_vector(ctx.handle, ctypes.c_void_p(ptr), int(elem_bytes))


def sem_debug_oob():
    """(status, count, first) of the debug build's bounds record since the last
    call (status SEM_ENOTSUP in a release build); clears the record."""
    n, f = ctypes.c_longlong(), ctypes.c_longlong()
    st = lib().sem_debug_oob(ctypes.byref(n), ctypes.byref(f))
    return st, n.value, f.value


def sem_debug_limit_skeleton(ctx: SemContext, bound: int) -> int:
    """Lowers the bound of the debug build's offset checks (status)."""
    return lib().sem_debug_limit_skeleton(ctx.handle, int(bound))


def sem_debug_cg_step_timeout(ctx: SemContext):
    """(status, bar_fail, done) of one one-pass CG step whose grid barrier
    never completes (debug build; SEM_ENOTSUP in a release build)."""
    bf, dn = ctypes.c_int(), ctypes.c_int()
    st = lib().sem_debug_cg_step_timeout(ctx.handle, ctypes.byref(bf), ctypes.byref(dn))
    return st, bf.value, dn.value


def sem_autotune(ctx: SemContext):
    """Returns (ms per application with the built-in config, with the chosen one)."""
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(lib().sem_autotune(ctx.handle, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


class SemBatch:
    """Handle of sem_batch_create (one captured graph over many contexts)."""

    def __init__(self, ctxs, fs, us):
        n = len(ctxs)
        if not (n == len(fs) == len(us)) or n == 0:
            raise ValueError("need equally many contexts, loads and outputs")
        self.ctxs, self.fs, self.us = list(ctxs), list(fs), list(us)   # keep them alive
        C = (_P * n)(*[c.handle for c in ctxs])
        F = (_P * n)(*[_dptr(f, c.n_nodes, "f") for f, c in zip(fs, ctxs)])
        U = (_P * n)(*[_dptr(u, c.n_nodes, "u") for u, c in zip(us, ctxs)])
        self.handle = ctypes.c_void_p()
        _check(lib().sem_batch_create(C, n, F, U, ctypes.byref(self.handle)))

    def solve(self, stream=None, check=True):
        n = len(self.ctxs)
        infos = (sem_info * n)()
        st = lib().sem_batch_solve(self.handle, infos, _stream(stream, self.fs[0]))
        if check:
            _check(st)
        return st, [dict(iters=i.iters, refinements=i.refinements, rel_res=i.rel_res, t_solve_s=i.t_solve_s)
                    for i in infos]

    def __del__(self):
        try:
            if self.handle:
                lib().sem_batch_destroy(self.handle)
                self.handle = None
        except Exception:
            pass


OP_TPT, OP_TPC, OP_MMC = 0, 1, 2
PC_NONE, PC_DIAG, PC_BLOCK = 0, 1, 2


def sem_apply_condensed_variant(ctx: SemContext, op: int, uB, vB, stream=None):
    """vB = Hhat uB on the nodal skeleton with the paper's operator variant op
    (OP_TPT, OP_TPC, OP_MMC)."""
    _check(lib().sem_apply_condensed_variant(ctx.handle, int(op), _dptr(uB, ctx.nb, "uB"), _dptr(vB, ctx.nb, "vB"),
                                             _stream(stream, uB)))


def sem_diag_nodal(ctx: SemContext, diag, stream=None):
    """Assembled diagonal of the nodal condensed operator."""
    _check(lib().sem_diag_nodal(ctx.handle, _dptr(diag, ctx.nb, "diag"), _stream(stream, diag)))


def sem_solve_variant(ctx: SemContext, op: int, pc: int, f, u, stream=None, check=True) -> dict:
    """CG on the nodal condensed system with operator op and preconditioner pc
    (PC_NONE, PC_DIAG, PC_BLOCK), then interior recovery into u."""
    info = sem_info()
    st = lib().sem_solve_variant(ctx.handle, int(op), int(pc), _dptr(f, ctx.n_nodes, "f"), _dptr(u, ctx.n_nodes, "u"),
                                 ctypes.byref(info), _stream(stream, f))
    if check:
        _check(st)
    return dict(status=st, iters=info.iters, rel_res=info.rel_res, t_solve_s=info.t_solve_s)


def sem_refine_history(ctx: SemContext):
    """Relative FP64 residuals of the last mixed-precision solve, per refinement step."""
    buf = np.empty(256)
    cnt = ctypes.c_int()
    _check(lib().sem_refine_history(ctx.handle, buf.ctypes.data_as(_D), len(buf), ctypes.byref(cnt)))
    return buf[:min(cnt.value, len(buf))].copy()


def sem_profile_enable(ctx: SemContext, enable: bool = True):
    _check(lib().sem_profile_enable(ctx.handle, 1 if enable else 0))


def sem_profile_read(ctx: SemContext, reset: bool = False):
    """(summed device milliseconds, number of timed operator launches)."""
    ms, cnt = ctypes.c_double(), ctypes.c_longlong()
    _check(lib().sem_profile_read(ctx.handle, ctypes.byref(ms), ctypes.byref(cnt), 1 if reset else 0))
    return ms.value, cnt.value


def sem_launch_count() -> int:
    return int(lib().sem_launch_count())
