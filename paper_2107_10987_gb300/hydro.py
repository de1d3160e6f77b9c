"""Thin Python binding of the C ABI in include/hydro.h (argument marshalling only).

Every function has the name of the C entry point it calls and takes torch CUDA
tensors (float64, contiguous) for device buffers; the stream defaults to
torch's current stream.  No step of the hydro method runs here: all of it runs
in the CUDA library, and loading fails loudly when that library is missing.
"""
from __future__ import annotations

import ctypes as C
import os

import torch

from . import _build

HYDRO_OK, HYDRO_EINVAL, HYDRO_ECUDA, HYDRO_ENOMEM, HYDRO_EUNSUP, HYDRO_ERANGE = 0, -1, -2, -3, -4, -5
HYDRO_STATIC_MAX_SUB = 192
HYDRO_ST_NONPHYS, HYDRO_ST_TIMEOUT = 0x1, 0x2
HYDRO_PREC_FP64, HYDRO_PREC_MIXED = 0, 1
HYDRO_BC_PERIODIC, HYDRO_BC_OUTFLOW = 0, 1
HYDRO_DECOMP_AUTO, HYDRO_DECOMP_ROWS, HYDRO_DECOMP_PLANES = 0, 1, 2

EXPORTS = ("hydro_create", "hydro_set_mode", "hydro_step", "hydro_update", "hydro_dt", "hydro_fill_ghosts_uniform",
           "hydro_conserved_sums", "hydro_status", "hydro_strerror", "hydro_last_cuda_error", "hydro_destroy",
           "hydro_step_static", "hydro_rk3_step", "hydro_rk3_graph_create", "hydro_rk3_graph_launch",
           "hydro_rk3_graph_state", "hydro_rk3_graph_destroy", "hydro_gate_data", "hydro_mlp_forward",
           "hydro_mlp_work_bytes", "hydro_mlp_loss_grad", "hydro_mlp_adam", "hydro_set_indicator",
           "hydro_fill_ghosts_amr", "hydro_flux_correct_amr", "hydro_autotune_step", "hydro_selftest_wait",
           "hydro_set_launch", "hydro_get_launch", "hydro_selftest_arith")
HYDRO_ST_MESH = 0x4
HYDRO_GATE_NPARAM, HYDRO_GATE_NIN = 2849, 54


class HydroError(RuntimeError):
    def __init__(self, code: int, where: str):
        lib = _lib()
        msg = lib.hydro_strerror(code).decode()
        if code == HYDRO_ECUDA:
            msg += ": " + lib.hydro_last_cuda_error().decode()
        super().__init__(f"{where} failed ({code}): {msg}")
        self.code = code


class Layout(C.Structure):
    _fields_ = [("N", C.c_int), ("ghost", C.c_int), ("n_species", C.c_int)]


class Mode(C.Structure):
    _fields_ = [("precision", C.c_int), ("cfl", C.c_double), ("de_eta1", C.c_double), ("de_eta2", C.c_double),
                ("flux_points", C.c_int), ("contact", C.c_int), ("spin", C.c_int)]


class Batch(C.Structure):
    _fields_ = [("n_sub", C.c_int), ("U", C.c_void_p), ("origin", C.c_void_p), ("h", C.c_void_p), ("g", C.c_void_p)]


class RK3Desc(C.Structure):
    _fields_ = [("a", Batch), ("U_b", C.c_void_p), ("nbx", C.c_int), ("nby", C.c_int), ("nbz", C.c_int),
                ("bc", C.c_int), ("dUdt", C.c_void_p), ("amax", C.c_void_p), ("dt", C.c_void_p), ("cfl", C.c_double),
                ("amr", C.c_void_p), ("face_flux", C.c_void_p), ("fused", C.c_int)]


_L = None


def library_path() -> str:
    return _build.LIB


def _lib(load: bool = True):
    """Load the CUDA library.  It must have been built (``build()``); there is
    no fallback."""
    global _L
    if _L is None and load:
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library {path} is missing: run __graft_entry__.build() first")
        L = C.CDLL(path)
        vp, dp, ip = C.c_void_p, C.c_double, C.c_int
        L.hydro_create.argtypes = [C.POINTER(Layout), dp, dp, C.POINTER(vp)]
        L.hydro_set_mode.argtypes = [vp, C.POINTER(Mode)]
        L.hydro_step.argtypes = [vp, C.POINTER(Batch), dp, vp, vp, vp, vp]
        L.hydro_update.argtypes = [vp, C.POINTER(Batch), vp, vp, dp, vp, ip, vp, vp]
        L.hydro_dt.argtypes = [vp, vp, vp, ip, dp, vp, vp]
        L.hydro_fill_ghosts_uniform.argtypes = [vp, C.POINTER(Batch), ip, ip, ip, ip, vp]
        L.hydro_conserved_sums.argtypes = [vp, C.POINTER(Batch), vp, vp]
        L.hydro_status.argtypes = [vp, C.POINTER(C.c_uint32)]
        L.hydro_scatter_interior.argtypes = [vp, C.POINTER(Batch), vp, vp]
        L.hydro_gather_interior.argtypes = [vp, C.POINTER(Batch), vp, vp]
        L.hydro_strerror.argtypes = [ip]
        L.hydro_strerror.restype = C.c_char_p
        L.hydro_last_cuda_error.argtypes = []
        L.hydro_last_cuda_error.restype = C.c_char_p
        L.hydro_step_static.argtypes = [vp, C.POINTER(Batch), dp, vp, vp, vp, vp]
        L.hydro_destroy.argtypes = [vp]
        L.hydro_destroy.restype = None
        L.hydro_rk3_step.argtypes = [vp, C.POINTER(RK3Desc), ip, vp]
        L.hydro_rk3_graph_create.argtypes = [vp, C.POINTER(RK3Desc), C.POINTER(vp)]
        L.hydro_rk3_graph_launch.argtypes = [vp, vp]
        L.hydro_rk3_graph_state.argtypes = [vp]
        L.hydro_rk3_graph_destroy.argtypes = [vp]
        L.hydro_selftest_wait.argtypes = [vp, dp, vp]
        L.hydro_selftest_arith.argtypes = [vp, vp, ip, vp, vp]
        L.hydro_gate_data.argtypes = [vp, C.POINTER(Batch), vp, vp, vp]
        L.hydro_mlp_forward.argtypes = [vp, vp, ip, vp, vp]
        L.hydro_mlp_work_bytes.argtypes = [ip]
        L.hydro_mlp_work_bytes.restype = C.c_size_t
        L.hydro_mlp_loss_grad.argtypes = [vp, vp, vp, ip, C.c_float, C.c_float, vp, vp, vp, C.c_size_t, vp]
        L.hydro_mlp_adam.argtypes = [vp, vp, vp, vp, ip, C.c_float, vp]
        L.hydro_set_indicator.argtypes = [vp, vp, dp, vp]
        L.hydro_fill_ghosts_amr.argtypes = [vp, C.POINTER(Batch), vp, vp]
        L.hydro_autotune_step.argtypes = [vp, C.POINTER(Batch), vp, vp, C.POINTER(C.c_int), vp]
        L.hydro_set_launch.argtypes = [vp, ip, ip]
        L.hydro_get_launch.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int)]
        L.hydro_flux_correct_amr.argtypes = [vp, C.POINTER(Batch), vp, vp, vp, vp]
        for name in EXPORTS:
            if name not in ("hydro_strerror", "hydro_last_cuda_error", "hydro_destroy", "hydro_rk3_graph_destroy",
                            "hydro_mlp_work_bytes"):
                getattr(L, name).restype = C.c_int
        _L = L
    return _L


def _check(rc: int, where: str):
    if rc != HYDRO_OK:
        raise HydroError(rc, where)


def _ptr(t) -> int | None:
    if t is None:
        return None
    if isinstance(t, int):
        return t
    assert t.is_cuda and t.dtype == torch.float64 and t.is_contiguous(), "expects contiguous float64 CUDA tensors"
    return t.data_ptr()


def _stream(stream) -> int:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def make_batch(U, origin, h, g=None) -> Batch:
    """A batch descriptor; it keeps references to the tensors whose device
    pointers it holds, so they stay allocated as long as the descriptor."""
    n = U.shape[0]
    b = Batch(n, _ptr(U), _ptr(origin), _ptr(h), _ptr(g))
    b._keep = (U, origin, h, g)
    return b


class Context:
    """Owns one hydro_ctx_t (a context per stream)."""

    def __init__(self, gamma: float = 5.0 / 3.0, omega: float = 0.0, N: int = 8, ghost: int = 3, n_species: int = 1):
        self.ptr = hydro_create(Layout(N, ghost, n_species), gamma, omega)
        self.gamma, self.omega, self.N = gamma, omega, N

    def close(self):
        if self.ptr:
            hydro_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- entry points (same names as the C ABI) ---------------------------------
def hydro_create(layout: Layout, gamma: float, omega: float) -> int:
    out = C.c_void_p()
    _check(_lib().hydro_create(C.byref(layout), gamma, omega, C.byref(out)), "hydro_create")
    return out.value


def hydro_set_mode(ctx, precision=HYDRO_PREC_FP64, cfl=0.4, de_eta1=1e-3, de_eta2=0.1, flux_points=9, contact=0,
                   spin=0):
    _check(_lib().hydro_set_mode(_cp(ctx), C.byref(Mode(precision, cfl, de_eta1, de_eta2, flux_points, contact,
                                                        spin))),
           "hydro_set_mode")


def _cp(ctx):
    return ctx.ptr if isinstance(ctx, Context) else ctx


def hydro_step(ctx, batch: Batch, dt: float, dUdt, amax, face_flux=None, stream=None):
    _check(_lib().hydro_step(_cp(ctx), C.byref(batch), float(dt), _ptr(dUdt), _ptr(amax), _ptr(face_flux),
                             _stream(stream)), "hydro_step")


def hydro_update(ctx, batch: Batch, U0, dUdt, dt: float = 0.0, dt_dev=None, stage: int = 0, U_out=None,
                 stream=None):
    _check(_lib().hydro_update(_cp(ctx), C.byref(batch), _ptr(U0), _ptr(dUdt), float(dt), _ptr(dt_dev), int(stage),
                               _ptr(U_out), _stream(stream)), "hydro_update")


def hydro_dt(ctx, amax, h, n_sub: int, cfl: float, dt_out, stream=None):
    _check(_lib().hydro_dt(_cp(ctx), _ptr(amax), _ptr(h), int(n_sub), float(cfl), _ptr(dt_out), _stream(stream)),
           "hydro_dt")


def hydro_fill_ghosts_uniform(ctx, batch: Batch, nbx: int, nby: int, nbz: int, bc: int, stream=None):
    _check(_lib().hydro_fill_ghosts_uniform(_cp(ctx), C.byref(batch), nbx, nby, nbz, bc, _stream(stream)),
           "hydro_fill_ghosts_uniform")


def _ptr_device_or_pinned(t) -> int:
    """A contiguous float64 tensor on the GPU or in page-locked host memory."""
    if isinstance(t, int):
        return t
    assert t.dtype == torch.float64 and t.is_contiguous(), "expects a contiguous float64 tensor"
    assert t.is_cuda or t.is_pinned(), "expects a CUDA tensor or a pinned host tensor"
    return t.data_ptr()


def hydro_scatter_interior(ctx, batch: Batch, interior, stream=None):
    """interior: [n_sub][F][N][N][N] float64 tensor (CUDA, or pinned host memory
    read directly by the kernel) -> the batch's interior cells."""
    _check(_lib().hydro_scatter_interior(_cp(ctx), C.byref(batch), _ptr_device_or_pinned(interior),
                                         _stream(stream)), "hydro_scatter_interior")


def hydro_gather_interior(ctx, batch: Batch, interior, stream=None):
    """The batch's interior cells -> interior [n_sub][F][N][N][N] float64 tensor
    (CUDA, or pinned host memory written directly by the kernel)."""
    _check(_lib().hydro_gather_interior(_cp(ctx), C.byref(batch), _ptr_device_or_pinned(interior),
                                        _stream(stream)), "hydro_gather_interior")


def hydro_conserved_sums(ctx, batch: Batch, sums, stream=None):
    _check(_lib().hydro_conserved_sums(_cp(ctx), C.byref(batch), _ptr(sums), _stream(stream)), "hydro_conserved_sums")


def hydro_status(ctx) -> int:
    v = C.c_uint32()
    _check(_lib().hydro_status(_cp(ctx), C.byref(v)), "hydro_status")
    return v.value


def hydro_strerror(code: int) -> str:
    return _lib().hydro_strerror(code).decode()


def hydro_destroy(ctx):
    _lib().hydro_destroy(_cp(ctx))


def hydro_last_cuda_error() -> str:
    return _lib().hydro_last_cuda_error().decode()


def hydro_step_static(ctx, batch: Batch, dt: float, dUdt, amax, status=None, stream=None):
    """Allocation-free hydro_step (fixed scratch; at most HYDRO_STATIC_MAX_SUB sub-grids).
    status: optional int32/uint32 CUDA tensor of one element receiving this call's bits."""
    sp = None
    if status is not None:
        assert status.is_cuda and status.numel() >= 1 and status.element_size() == 4
        sp = status.data_ptr()
    _check(_lib().hydro_step_static(_cp(ctx), C.byref(batch), float(dt), _ptr(dUdt), _ptr(amax), sp,
                                    _stream(stream)), "hydro_step_static")


def make_rk3_desc(Ua, Ub, origin, h, nb, bc, dUdt, amax, dt, cfl=0.4, g=None, mesh=None, face_flux=None,
                  fused=False) -> RK3Desc:
    """Descriptor of one RK3 time step: of a uniform mesh of nb = (nbx, nby, nbz)
    sub-grids, or (mesh: an amr.AMRMesh, face_flux its work buffer) of an
    adaptive mesh.  fused: the whole step as one persistent launch (uniform
    mesh, mixed precision)."""
    nb = nb or (0, 0, 0)
    d = RK3Desc(make_batch(Ua, origin, h, g), _ptr(Ub), nb[0], nb[1], nb[2], bc, _ptr(dUdt), _ptr(amax), _ptr(dt),
                float(cfl), C.addressof(mesh.desc) if mesh is not None else None, _ptr(face_flux),
                1 if fused else 0)
    d._keep = (Ua, Ub, origin, h, g, dUdt, amax, dt, mesh, face_flux)
    return d


def hydro_selftest_wait(ctx, seconds: float = 0.01, stream=None):
    _check(_lib().hydro_selftest_wait(_cp(ctx), float(seconds), _stream(stream)), "hydro_selftest_wait")


def hydro_selftest_arith(x, y, out, stream=None):
    """The FP64 kernels' integer-pipe halving and MC slope on device float64
    tensors x, y (n values) into out (2n values)."""
    n = x.numel()
    if y.numel() != n or out.numel() != 2 * n:
        raise ValueError("x, y: n values; out: 2n values")
    _check(_lib().hydro_selftest_arith(_ptr(x), _ptr(y), n, _ptr(out), _stream(stream)), "hydro_selftest_arith")


def hydro_rk3_step(ctx, desc: RK3Desc, parity: int, stream=None):
    _check(_lib().hydro_rk3_step(_cp(ctx), C.byref(desc), int(parity), _stream(stream)),
           "hydro_rk3_step")


def hydro_rk3_graph_create(ctx, desc: RK3Desc) -> int:
    out = C.c_void_p()
    _check(_lib().hydro_rk3_graph_create(_cp(ctx), C.byref(desc), C.byref(out)), "hydro_rk3_graph_create")
    return out.value


def hydro_rk3_graph_launch(graph: int, stream=None):
    _check(_lib().hydro_rk3_graph_launch(graph, _stream(stream)), "hydro_rk3_graph_launch")


def hydro_rk3_graph_state(graph: int) -> int:
    return _lib().hydro_rk3_graph_state(graph)


def hydro_rk3_graph_destroy(graph: int):
    _lib().hydro_rk3_graph_destroy(graph)


def _fptr(t) -> int | None:
    if t is None:
        return None
    assert t.is_cuda and t.is_contiguous(), "expects contiguous CUDA tensors"
    return t.data_ptr()


def hydro_gate_data(ctx, batch: Batch, X=None, y=None, stream=None):
    """X: float32 [n_sub*512][54] CUDA tensor, y: uint8 [n_sub*512] (either may be None)."""
    assert X is None or X.dtype == torch.float32
    assert y is None or y.dtype == torch.uint8
    _check(_lib().hydro_gate_data(_cp(ctx), C.byref(batch), _fptr(X), _fptr(y), _stream(stream)), "hydro_gate_data")


def hydro_mlp_forward(params, X, out, stream=None):
    _check(_lib().hydro_mlp_forward(_fptr(params), _fptr(X), X.shape[0], _fptr(out), _stream(stream)),
           "hydro_mlp_forward")


def hydro_mlp_work_bytes(n: int) -> int:
    return int(_lib().hydro_mlp_work_bytes(int(n)))


def hydro_mlp_loss_grad(params, X, y, grad, loss=None, w1=1.0, w0=1.0, work=None, stream=None):
    n = X.shape[0]
    if work is None:
        work = torch.empty(hydro_mlp_work_bytes(n) // 4 + 1, dtype=torch.float32, device=X.device)
    _check(_lib().hydro_mlp_loss_grad(_fptr(params), _fptr(X), _fptr(y), n, float(w1), float(w0), _fptr(grad),
                                      _fptr(loss), _fptr(work), work.numel() * work.element_size(), _stream(stream)),
           "hydro_mlp_loss_grad")


def hydro_mlp_adam(params, m, v, grad, t: int, lr: float, stream=None):
    _check(_lib().hydro_mlp_adam(_fptr(params), _fptr(m), _fptr(v), _fptr(grad), int(t), float(lr), _stream(stream)),
           "hydro_mlp_adam")


def hydro_set_indicator(ctx, params=None, threshold: float = 0.5, stream=None):
    _check(_lib().hydro_set_indicator(_cp(ctx), _fptr(params), float(threshold), _stream(stream)),
           "hydro_set_indicator")


def hydro_fill_ghosts_amr(ctx, batch: Batch, mesh, stream=None):
    """mesh: an amr.AMRMesh (its .desc is the hydro_amr_t)."""
    _check(_lib().hydro_fill_ghosts_amr(_cp(ctx), C.byref(batch), C.addressof(mesh.desc), _stream(stream)),
           "hydro_fill_ghosts_amr")


def hydro_flux_correct_amr(ctx, batch: Batch, mesh, face_flux, dUdt, stream=None):
    _check(_lib().hydro_flux_correct_amr(_cp(ctx), C.byref(batch), C.addressof(mesh.desc), _ptr(face_flux),
                                         _ptr(dUdt), _stream(stream)), "hydro_flux_correct_amr")


def hydro_autotune_step(ctx, batch: Batch, dUdt, amax, stream=None) -> int:
    """Pick and keep the fastest decomposition and persistent grid for this batch;
    returns the grid (hydro_get_launch gives both)."""
    out = C.c_int()
    _check(_lib().hydro_autotune_step(_cp(ctx), C.byref(batch), _ptr(dUdt), _ptr(amax), C.byref(out),
                                      _stream(stream)), "hydro_autotune_step")
    return out.value


def hydro_set_launch(ctx, decomposition=HYDRO_DECOMP_AUTO, ctas=0):
    """Fix the step's decomposition (HYDRO_DECOMP_*) and persistent CTAs (0: default)."""
    _check(_lib().hydro_set_launch(_cp(ctx), int(decomposition), int(ctas)), "hydro_set_launch")


def hydro_get_launch(ctx):
    """(decomposition, ctas) of the context's next step."""
    d, n = C.c_int(), C.c_int()
    _check(_lib().hydro_get_launch(_cp(ctx), C.byref(d), C.byref(n)), "hydro_get_launch")
    return d.value, n.value
