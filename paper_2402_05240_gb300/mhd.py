"""Thin ctypes binding of libmhd.so (include/mhd_api.h).

Every function here marshals arguments and calls the C ABI of the same name;
all numerical work runs in the library's CUDA kernels.  Importing this module
raises if the library has not been built: there is no CPU fallback.

State tensors are torch float64 CUDA tensors of shape [8, nz, ny, nx]
(fields rho, mx, my, mz, E, Bx, By, Bz; face fields on upper faces).
"""
from __future__ import annotations

import ctypes
import os
import weakref

import numpy as np
import torch

from . import build as _build

MHD_OK = 0
MHD_ERR_ARG = -1
MHD_ERR_CUDA = -2
MHD_ERR_OOM = -3
MHD_ERR_NONFINITE = -4
MHD_ERR_DT = -5
MHD_ERR_TOO_LARGE = -6

RECON = {"pcm": 0, "plmc": 1, "ppmc": 2, "plm_prim": 3}
PRECISION = {"fp64": 0, "fp32_bulk": 1, "fp64_df": 2}
BC = {"periodic": 0, "outflow": 1, "halo": 2}


class mhd_config(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double),
                ("gamma", ctypes.c_double), ("cfl", ctypes.c_double),
                ("recon", ctypes.c_int), ("precision", ctypes.c_int),
                ("rho_floor", ctypes.c_double), ("p_floor", ctypes.c_double),
                ("bc", ctypes.c_int * 3)]


def _load_library():
    path = _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"libmhd.so not built ({path}); run paper_2402_05240_gb300.build.build() "
                           "or __graft_entry__.build() first")
    lib = ctypes.CDLL(path)
    vp, dp, ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int
    sig = {
        "mhd_workspace_bytes": (ip, [ctypes.POINTER(mhd_config), ctypes.POINTER(ctypes.c_size_t)]),
        "mhd_init": (ip, [ctypes.POINTER(vp), ctypes.POINTER(mhd_config), vp]),
        "mhd_destroy": (None, [vp]),
        "mhd_dt": (ip, [vp, vp, dp]),
        "mhd_step": (ip, [vp, vp, ctypes.c_double, dp]),
        "mhd_floor_count": (ip, [vp, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)]),
        "mhd_run": (ip, [vp, vp, ip, vp]),
        "mhd_run_host": (ip, [vp, vp, ip, dp]),
        "mhd_evolve": (ip, [vp, vp, ctypes.c_double, ip, dp, ctypes.POINTER(ip)]),
        "mhd_step_sub": (ip, [vp, vp, ctypes.POINTER(ip), ctypes.POINTER(ip), ctypes.c_double, vp]),
        "mhd_dt_sub": (ip, [vp, vp, ctypes.POINTER(ip), ctypes.POINTER(ip), dp]),
        "mhd_adjoint_step": (ip, [vp, vp, ctypes.c_double, vp, vp]),
        "mhd_adjoint_step_cfl": (ip, [vp, vp, vp, vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
        "mhd_diagnostics": (ip, [vp, vp, dp, dp]),
        "mhd_status": (ip, [vp, ctypes.POINTER(ctypes.c_longlong)]),
        "mhd_strerror": (ctypes.c_char_p, [ip]),
        "mhd_stage_primitives": (ip, [vp, vp, vp]),
        "mhd_stage_fluxes": (ip, [vp, vp, ip, vp]),
        "mhd_stage_edges": (ip, [vp, vp, vp, vp]),
        "mhd_stage_recon": (ip, [vp, vp, ip, ip, vp, vp]),
        "mhd_profile_enable": (ip, [vp, ip]),
        "mhd_profile_read": (ip, [vp, dp, ctypes.POINTER(ctypes.c_longlong)]),
        "mhd_stage_name": (ctypes.c_char_p, [ip]),
        "mhd_diagnostics_static": (ip, [ctypes.POINTER(mhd_config), vp, vp, dp, dp]),
        "mhd_adjoint_workspace_bytes": (ip, [ctypes.POINTER(mhd_config), ctypes.POINTER(ctypes.c_size_t)]),
        "mhd_stage_recon_vjp": (ip, [vp, vp, ip, ip, vp, vp, vp]),
        "mhd_stage_hlld_vjp": (ip, [ip, ctypes.c_double, ip, vp, vp, vp, vp, vp, vp, vp, vp, vp]),
        "mhd_host_alloc": (ip, [ctypes.c_size_t, ctypes.POINTER(vp)]),
        "mhd_host_free": (ip, [vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


LIB = _load_library()


class MHDError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__(f"{where}: {LIB.mhd_strerror(code).decode()} ({code})")


def _check(code, where):
    if code != MHD_OK:
        raise MHDError(code, where)


# Cells and device of every live context (recorded by mhd_init, dropped by
# mhd_destroy).  The library takes raw pointers and cannot see buffer sizes,
# so the binding checks each buffer against its context before the call.
_CTX = {}


def _ptr(t: torch.Tensor, numel: int | None = None, name: str = "tensor", cuda: bool = True,
         device: int | None = None):
    """Address of a float64 contiguous tensor with at least ``numel``
    elements, on the GPU ``device`` (any GPU if None) or, with cuda=False, in
    host memory.  Raises TypeError / ValueError otherwise."""
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name}: torch.Tensor expected, got {type(t).__name__}")
    if t.dtype != torch.float64:
        raise TypeError(f"{name}: float64 expected, got {t.dtype}")
    if t.is_cuda != cuda:
        raise ValueError(f"{name}: {'CUDA' if cuda else 'host'} tensor expected, got one on {t.device}")
    if cuda and device is not None and t.device.index != device:
        raise ValueError(f"{name}: on {t.device}, the context lives on cuda:{device}")
    if not t.is_contiguous():
        raise ValueError(f"{name}: contiguous tensor expected")
    if numel is not None and t.numel() < numel:
        raise ValueError(f"{name}: {t.numel()} elements, at least {numel} needed")
    return ctypes.c_void_p(t.data_ptr())


def _cells(ctx):
    """(cells, device) of a context made by mhd_init, else (None, None)."""
    v = ctx.value if isinstance(ctx, ctypes.c_void_p) else ctx
    return _CTX.get(v, (None, None))


def _field(ctx, t, fields: int, name: str):
    """_ptr for a [fields][N] array of the context's grid."""
    n, dev = _cells(ctx)
    return _ptr(t, None if n is None else fields * n, name, device=dev)


# ---- C ABI, same names --------------------------------------------------
def mhd_workspace_bytes(cfg: mhd_config) -> int:
    b = ctypes.c_size_t(0)
    _check(LIB.mhd_workspace_bytes(ctypes.byref(cfg), ctypes.byref(b)), "mhd_workspace_bytes")
    return b.value


def mhd_init(cfg: mhd_config, stream=None):
    ctx = ctypes.c_void_p(0)
    s = ctypes.c_void_p(stream if stream is not None else torch.cuda.current_stream().cuda_stream)
    _check(LIB.mhd_init(ctypes.byref(ctx), ctypes.byref(cfg), s), "mhd_init")
    _CTX[ctx.value] = (cfg.nx * cfg.ny * cfg.nz, torch.cuda.current_device())
    return ctx


def mhd_destroy(ctx):
    _CTX.pop(ctx.value if isinstance(ctx, ctypes.c_void_p) else ctx, None)
    LIB.mhd_destroy(ctx)


def mhd_dt(ctx, U: torch.Tensor) -> float:
    v = ctypes.c_double(0)
    _check(LIB.mhd_dt(ctx, _field(ctx, U, 8, "U"), ctypes.byref(v)), "mhd_dt")
    return v.value


def mhd_step(ctx, U: torch.Tensor, dt: float, want_next_dt: bool = False):
    """One step at dt in place; with want_next_dt, returns the CFL dt of the new state (synchronises)."""
    if not want_next_dt:
        _check(LIB.mhd_step(ctx, _field(ctx, U, 8, "U"), float(dt), None), "mhd_step")
        return None
    v = ctypes.c_double(0)
    _check(LIB.mhd_step(ctx, _field(ctx, U, 8, "U"), float(dt), ctypes.byref(v)), "mhd_step")
    return v.value


def mhd_floor_count(ctx):
    """(density, pressure) floor triggers since the last call; resets them."""
    a, b = ctypes.c_longlong(0), ctypes.c_longlong(0)
    _check(LIB.mhd_floor_count(ctx, ctypes.byref(a), ctypes.byref(b)), "mhd_floor_count")
    return a.value, b.value


def mhd_run(ctx, U: torch.Tensor, nsteps: int, dt_log: torch.Tensor | None = None):
    p = ctypes.c_void_p(0)
    if dt_log is not None:
        p = _ptr(dt_log, max(int(nsteps), 0), "dt_log", device=_cells(ctx)[1])
    _check(LIB.mhd_run(ctx, _field(ctx, U, 8, "U"), int(nsteps), p), "mhd_run")


def mhd_evolve(ctx, U: torch.Tensor, t_end: float, max_steps: int = 1 << 30):
    """Advance U in place to t_end; returns (time reached, steps taken)."""
    t = ctypes.c_double(0)
    n = ctypes.c_int(0)
    _check(LIB.mhd_evolve(ctx, _field(ctx, U, 8, "U"), float(t_end), int(max_steps), ctypes.byref(t),
                          ctypes.byref(n)), "mhd_evolve")
    return t.value, n.value


def _sub_dims(Ug):
    """gn = (gnx, gny, gnz) of a [8, gnz, gny, gnx] state."""
    if not isinstance(Ug, torch.Tensor) or Ug.dim() != 4 or Ug.shape[0] != 8:
        raise ValueError("Ug: a [8, gnz, gny, gnx] tensor expected")
    return (ctypes.c_int * 3)(Ug.shape[3], Ug.shape[2], Ug.shape[1])


def mhd_step_sub(ctx, Ug: torch.Tensor, offset, dt: float, Ug_out: torch.Tensor):
    """One step of a subdomain: Ug is [8, gnz, gny, gnx] holding it at
    offset (ox, oy, oz) with its halo; its new interior goes to Ug_out."""
    gn = _sub_dims(Ug)
    if not isinstance(Ug_out, torch.Tensor) or Ug_out.shape != Ug.shape:
        raise ValueError("Ug_out: same shape as Ug expected")
    off = (ctypes.c_int * 3)(*[int(o) for o in offset])
    dev = _cells(ctx)[1]
    _check(LIB.mhd_step_sub(ctx, _ptr(Ug, name="Ug", device=dev), gn, off, float(dt),
                            _ptr(Ug_out, name="Ug_out", device=dev)), "mhd_step_sub")


def mhd_dt_sub(ctx, Ug: torch.Tensor, offset) -> float:
    gn = _sub_dims(Ug)
    off = (ctypes.c_int * 3)(*[int(o) for o in offset])
    v = ctypes.c_double(0)
    _check(LIB.mhd_dt_sub(ctx, _ptr(Ug, name="Ug", device=_cells(ctx)[1]), gn, off, ctypes.byref(v)), "mhd_dt_sub")
    return v.value


def mhd_run_host(ctx, U_host: torch.Tensor, nsteps: int) -> float:
    n = _cells(ctx)[0]
    p = _ptr(U_host, None if n is None else 8 * n, "U_host", cuda=False)
    t = ctypes.c_double(0)
    _check(LIB.mhd_run_host(ctx, p, int(nsteps), ctypes.byref(t)), "mhd_run_host")
    return t.value


def host_buffer(*shape) -> torch.Tensor:
    """A float64 host tensor of the given shape in page-locked, huge-page
    backed memory from mhd_host_alloc (the buffer for mhd_run_host that
    keeps the copies at the link rate); freed when the last tensor viewing
    it is gone."""
    numel = 1
    for s in shape:
        numel *= int(s)
    if numel < 1:
        raise ValueError("host_buffer: empty shape")
    p = ctypes.c_void_p()
    _check(LIB.mhd_host_alloc(numel * 8, ctypes.byref(p)), "mhd_host_alloc")
    raw = (ctypes.c_double * numel).from_address(p.value)
    arr = np.frombuffer(raw, dtype=np.float64)
    weakref.finalize(arr, LIB.mhd_host_free, ctypes.c_void_p(p.value))
    return torch.from_numpy(arr).view(*shape)


def mhd_adjoint_step(ctx, U_n: torch.Tensor, dt: float, gU_np1: torch.Tensor, gU_n: torch.Tensor):
    _check(LIB.mhd_adjoint_step(ctx, _field(ctx, U_n, 8, "U_n"), float(dt), _field(ctx, gU_np1, 8, "gU_np1"),
                                _field(ctx, gU_n, 8, "gU_n")), "mhd_adjoint_step")


def mhd_adjoint_step_cfl(ctx, U_n: torch.Tensor, gU_np1: torch.Tensor, gU_n: torch.Tensor):
    """Returns (dt, g_dt)."""
    dt, gdt = ctypes.c_double(0), ctypes.c_double(0)
    _check(LIB.mhd_adjoint_step_cfl(ctx, _field(ctx, U_n, 8, "U_n"), _field(ctx, gU_np1, 8, "gU_np1"),
                                    _field(ctx, gU_n, 8, "gU_n"), ctypes.byref(dt), ctypes.byref(gdt)),
           "mhd_adjoint_step_cfl")
    return dt.value, gdt.value


def mhd_diagnostics(ctx, U: torch.Tensor):
    m = ctypes.c_double(0)
    tot = (ctypes.c_double * 8)()
    _check(LIB.mhd_diagnostics(ctx, _field(ctx, U, 8, "U"), ctypes.byref(m), tot), "mhd_diagnostics")
    return m.value, list(tot)


def mhd_diagnostics_static(cfg: mhd_config, U: torch.Tensor, stream=None):
    """mhd_diagnostics without a context or any device allocation (static
    device scratch, grids up to 512^3); for callers that cannot allocate."""
    m = ctypes.c_double(0)
    tot = (ctypes.c_double * 8)()
    s = ctypes.c_void_p(stream if stream is not None else torch.cuda.current_stream().cuda_stream)
    p = _ptr(U, 8 * cfg.nx * cfg.ny * cfg.nz, "U")
    _check(LIB.mhd_diagnostics_static(ctypes.byref(cfg), p, s, ctypes.byref(m), tot), "mhd_diagnostics_static")
    return m.value, list(tot)


def mhd_status(ctx):
    """Returns (status code, (rho floor triggers, pressure floor triggers))."""
    cnt = (ctypes.c_longlong * 2)()
    code = LIB.mhd_status(ctx, cnt)
    return code, (cnt[0], cnt[1])


def mhd_stage_primitives(ctx, U, W):
    _check(LIB.mhd_stage_primitives(ctx, _field(ctx, U, 8, "U"), _field(ctx, W, 8, "W")), "mhd_stage_primitives")


def mhd_stage_fluxes(ctx, U, recon: int, F):
    _check(LIB.mhd_stage_fluxes(ctx, _field(ctx, U, 8, "U"), int(recon), _field(ctx, F, 21, "F")),
           "mhd_stage_fluxes")


def mhd_stage_edges(ctx, U, F, E):
    _check(LIB.mhd_stage_edges(ctx, _field(ctx, U, 8, "U"), _field(ctx, F, 21, "F"), _field(ctx, E, 3, "E")),
           "mhd_stage_edges")


def mhd_stage_recon(ctx, U, axis: int, recon: int, WL, WR):
    _check(LIB.mhd_stage_recon(ctx, _field(ctx, U, 8, "U"), int(axis), int(recon), _field(ctx, WL, 7, "WL"),
                               _field(ctx, WR, 7, "WR")), "mhd_stage_recon")


def mhd_adjoint_workspace_bytes(cfg: mhd_config) -> int:
    b = ctypes.c_size_t(0)
    _check(LIB.mhd_adjoint_workspace_bytes(ctypes.byref(cfg), ctypes.byref(b)), "mhd_adjoint_workspace_bytes")
    return b.value


def mhd_stage_recon_vjp(ctx, U, axis: int, recon: int, gWL, gWR, gU):
    _check(LIB.mhd_stage_recon_vjp(ctx, _field(ctx, U, 8, "U"), int(axis), int(recon), _field(ctx, gWL, 7, "gWL"),
                                   _field(ctx, gWR, 7, "gWR"), _field(ctx, gU, 8, "gU")), "mhd_stage_recon_vjp")


def mhd_stage_hlld_vjp(gamma, precision: int, wl, wr, bn, gf, gwl, gwr, gbn, f, stream=None):
    s = ctypes.c_void_p(stream if stream is not None else torch.cuda.current_stream().cuda_stream)
    n = bn.numel()
    faces = {k: _ptr(t, 7 * n, k) for k, t in (("wl", wl), ("wr", wr), ("gf", gf), ("gwl", gwl), ("gwr", gwr),
                                                ("f", f))}
    _check(LIB.mhd_stage_hlld_vjp(int(n), float(gamma), int(precision), faces["wl"], faces["wr"], _ptr(bn, n, "bn"),
                                  faces["gf"], faces["gwl"], faces["gwr"], _ptr(gbn, n, "gbn"), faces["f"], s),
           "mhd_stage_hlld_vjp")


MHD_NUM_STAGES = 10


def mhd_profile_enable(ctx, on: bool):
    _check(LIB.mhd_profile_enable(ctx, 1 if on else 0), "mhd_profile_enable")


def mhd_profile_read(ctx):
    """{stage name: (device ms, launches)} since the last enable/read."""
    ms = (ctypes.c_double * MHD_NUM_STAGES)()
    n = (ctypes.c_longlong * MHD_NUM_STAGES)()
    _check(LIB.mhd_profile_read(ctx, ms, n), "mhd_profile_read")
    return {LIB.mhd_stage_name(i).decode(): (ms[i], n[i]) for i in range(MHD_NUM_STAGES)}


# ---- convenience ------------------------------------------------------
class Sim:
    """Owns one library context for a grid and a configuration."""

    def __init__(self, nx, ny, nz, lx=1.0, ly=1.0, lz=1.0, gamma=5.0 / 3.0, cfl=0.4, recon="plmc",
                 precision="fp64", rho_floor=1e-20, p_floor=1e-20, stream=None, bc=("periodic",) * 3):
        self.shape = (nz, ny, nx)
        bcs = (ctypes.c_int * 3)(*[BC[b] if isinstance(b, str) else int(b) for b in bc])
        self.cfg = mhd_config(nx, ny, nz, lx / nx, ly / ny, lz / nz, gamma, cfl,
                              RECON[recon] if isinstance(recon, str) else recon,
                              PRECISION[precision] if isinstance(precision, str) else precision,
                              rho_floor, p_floor, bcs)
        self.ctx = mhd_init(self.cfg, stream)

    def close(self):
        if self.ctx is not None:
            mhd_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def N(self):
        nz, ny, nx = self.shape
        return nx * ny * nz

    def dt(self, U):
        return mhd_dt(self.ctx, U)

    def step(self, U, dt, want_next_dt=False):
        return mhd_step(self.ctx, U, dt, want_next_dt)

    def floor_count(self):
        return mhd_floor_count(self.ctx)

    def run(self, U, nsteps, dt_log=None):
        mhd_run(self.ctx, U, nsteps, dt_log)

    def evolve(self, U, t_end, max_steps=1 << 30):
        return mhd_evolve(self.ctx, U, t_end, max_steps)

    def status(self):
        code, counts = mhd_status(self.ctx)
        _check(code, "mhd_status")
        return counts

    def diagnostics(self, U):
        return mhd_diagnostics(self.ctx, U)

    def primitives(self, U):
        W = torch.empty_like(U)
        mhd_stage_primitives(self.ctx, U, W)
        return W

    def fluxes(self, U, recon=None):
        r = self.cfg.recon if recon is None else (RECON[recon] if isinstance(recon, str) else recon)
        F = torch.empty((3, 7) + self.shape, dtype=torch.float64, device=U.device)
        mhd_stage_fluxes(self.ctx, U, r, F)
        return F

    def edges(self, U, F):
        E = torch.empty((3,) + self.shape, dtype=torch.float64, device=U.device)
        mhd_stage_edges(self.ctx, U, F.contiguous(), E)
        return E

    def adjoint_step(self, U_n, dt, gU_np1):
        """gU_n = (dU^{n+1}/dU^n)^T gU_np1 for one step at fixed dt."""
        gU = torch.empty_like(gU_np1)
        mhd_adjoint_step(self.ctx, U_n, dt, gU_np1.contiguous(), gU)
        return gU

    def adjoint_step_cfl(self, U_n, gU_np1):
        """(gU_n, dt, g_dt) for one step at the CFL dt of U_n, the dt's own
        dependence on U_n included."""
        gU = torch.empty_like(gU_np1)
        dt, gdt = mhd_adjoint_step_cfl(self.ctx, U_n, gU_np1.contiguous(), gU)
        return gU, dt, gdt

    def recon_vjp(self, U, axis, gWL, gWR, recon=None):
        r = self.cfg.recon if recon is None else (RECON[recon] if isinstance(recon, str) else recon)
        gU = torch.empty_like(U)
        mhd_stage_recon_vjp(self.ctx, U, axis, r, gWL.contiguous(), gWR.contiguous(), gU)
        return gU

    def recon(self, U, axis, recon=None):
        r = self.cfg.recon if recon is None else (RECON[recon] if isinstance(recon, str) else recon)
        WL = torch.empty((7,) + self.shape, dtype=torch.float64, device=U.device)
        WR = torch.empty_like(WL)
        mhd_stage_recon(self.ctx, U, axis, r, WL, WR)
        return WL, WR
