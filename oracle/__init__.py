"""CPU oracle of the VL+CT ideal-MHD step (TEST INFRASTRUCTURE ONLY).

A plain, slow FP64 C++ implementation (``mhd_oracle.cpp``) of what the CUDA
path computes, loaded through ctypes.  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may import
this package.  It shares no code with ``paper_2402_05240_gb300``; the only
module both sides use is the seeded input generator
``paper_2402_05240_gb300.inputs``, which holds none of the method's arithmetic.

Functions without an independent pin are marked "parity unpinned" in their
docstring; every other function is pinned by a ``tests/test_oracle_*.py`` test.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mhd_oracle.cpp")
_LIB = os.path.join(_HERE, "_build", "libmhd_oracle.so")
_lock = threading.Lock()
_lib = None

RECON = {"pcm": 0, "plmc": 1, "ppmc": 2, "plm_prim": 3}


def build(force: bool = False) -> str:
    """Compile the oracle shared library with g++ (-O2, no fast-math, no FMA
    contraction, OpenMP over cells)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["g++", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC",
               "-o", tmp, _SRC]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class Params(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int * 3), ("d", ctypes.c_double * 3), ("gamma", ctypes.c_double),
                ("rho_floor", ctypes.c_double), ("p_floor", ctypes.c_double), ("recon", ctypes.c_int)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.POINTER(Params)
            dp = ctypes.POINTER(ctypes.c_double)
            lib.oracle_dt.restype = ctypes.c_double
            lib.oracle_dt.argtypes = [P, dp, ctypes.c_double]
            lib.oracle_set_threads.restype = ctypes.c_int
            lib.oracle_set_threads.argtypes = [ctypes.c_int]
            ip3 = ctypes.POINTER(ctypes.c_int)
            lib.oracle_dt_box.restype = ctypes.c_double
            lib.oracle_dt_box.argtypes = [P, dp, ctypes.c_double, ip3, ip3]
            lib.oracle_fast_speed.restype = ctypes.c_double
            lib.oracle_fast_speed.argtypes = [ctypes.c_double] * 6
            lib.oracle_hlld.argtypes = [ctypes.c_double, dp, dp, ctypes.c_double, dp]
            lib.oracle_hlld_detail.restype = ctypes.c_int
            lib.oracle_hlld_detail.argtypes = [ctypes.c_double, dp, dp, ctypes.c_double, dp, dp, dp, dp]
            lib.oracle_eigen.argtypes = [ctypes.c_double, dp, ctypes.c_double, dp, dp, dp]
            lib.oracle_primitives.argtypes = [P, dp, dp]
            lib.oracle_recon.argtypes = [P, dp, ctypes.c_int, ctypes.c_int, dp, dp]
            lib.oracle_fluxes.argtypes = [P, dp, ctypes.c_int, dp]
            lib.oracle_edges.argtypes = [P, dp, dp, dp]
            lib.oracle_update.argtypes = [P, dp, dp, dp, ctypes.c_double, dp]
            lib.oracle_step.argtypes = [P, dp, ctypes.c_double, ctypes.POINTER(ctypes.c_longlong)]
            lib.oracle_step_jvp.argtypes = [P, dp, dp, ctypes.c_double]
            lib.oracle_step_cfl_jvp.argtypes = [P, dp, dp, ctypes.c_double, dp]
            lib.oracle_dt_jvp.restype = ctypes.c_double
            lib.oracle_dt_jvp.argtypes = [P, dp, dp, ctypes.c_double, dp]
            lib.oracle_diagnostics.argtypes = [P, dp, dp, dp]
            lib.oracle_hlld_jvp.argtypes = [ctypes.c_double, dp, dp, ctypes.c_double, dp, dp, ctypes.c_double, dp, dp]
            lib.oracle_recon_jvp.argtypes = [P, dp, dp, ctypes.c_int, ctypes.c_int, dp, dp, dp, dp]
            _lib = lib
    return _lib


GHOST = 10  # ghost depth of the outflow oracle: more than one step's dependency radius (5 cells)


class OutflowOracle:
    """The step on a grid with outflow (zero-gradient) boundaries on some axes
    (Sec. 3.1.4: the Riemann problems): U^n is padded with GHOST ghost cells
    on both sides of each outflow axis, every ghost cell a copy of the nearest
    interior cell (all 8 fields, face fields included), the periodic oracle
    step runs on the padded grid and the interior is kept -- ghost cells
    filled once per step.  dt is Eq. dt over the interior cells of the padded
    state.  ``bc``: per axis x, y, z, "periodic" or "outflow"."""

    def __init__(self, nx, ny, nz, bc, gamma=5.0 / 3.0, recon="plmc", rho_floor=1e-20, p_floor=1e-20,
                 lx=1.0, ly=1.0, lz=1.0):
        self.shape = (nz, ny, nx)
        self.g = [GHOST if b == "outflow" else 0 for b in bc]  # x, y, z
        gx, gy, gz = self.g
        self.inner = Oracle(nx + 2 * gx, ny + 2 * gy, nz + 2 * gz, dx=lx / nx, dy=ly / ny, dz=lz / nz,
                            gamma=gamma, recon=recon, rho_floor=rho_floor, p_floor=p_floor)
        self.lo = (ctypes.c_int * 3)(gx, gy, gz)
        self.hi = (ctypes.c_int * 3)(gx + nx, gy + ny, gz + nz)

    def pad(self, U):
        gx, gy, gz = self.g
        U = np.ascontiguousarray(U, np.float64)
        assert U.shape == (8,) + self.shape
        return np.ascontiguousarray(np.pad(U, ((0, 0), (gz, gz), (gy, gy), (gx, gx)), mode="edge"))

    def unpad(self, V):
        gx, gy, gz = self.g
        nz, ny, nx = self.shape
        return np.ascontiguousarray(V[:, gz:gz + nz, gy:gy + ny, gx:gx + nx])

    def dt(self, U, cfl):
        P = self.pad(U)
        return self.inner.lib.oracle_dt_box(ctypes.byref(self.inner.p), _ptr(P), cfl, self.lo, self.hi)

    def step(self, U, dt):
        return self.unpad(self.inner.step(self.pad(U), dt))

    def run(self, U, nsteps, cfl=None, dts=None):
        V = np.ascontiguousarray(U, np.float64).copy()
        used = []
        for s in range(nsteps):
            dt = dts[s] if dts is not None else self.dt(V, cfl)
            V = self.step(V, dt)
            used.append(dt)
        return V, used


def set_threads(n: int) -> int:
    """Threads of the oracle's OpenMP loops (n <= 0: unchanged); returns the previous count."""
    return int(_load().oracle_set_threads(int(n)))


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class Oracle:
    """Oracle bound to one grid.  ``U`` arrays are float64 ``[8, nz, ny, nx]``."""

    def __init__(self, nx, ny, nz, dx=None, dy=None, dz=None, gamma=5.0 / 3.0, recon="plmc",
                 rho_floor=1e-20, p_floor=1e-20, lx=1.0, ly=1.0, lz=1.0):
        self.lib = _load()
        self.shape = (nz, ny, nx)
        self.N = nx * ny * nz
        self.p = Params()
        self.p.n[:] = [nx, ny, nz]
        self.p.d[:] = [dx if dx else lx / nx, dy if dy else ly / ny, dz if dz else lz / nz]
        self.p.gamma = gamma
        self.p.rho_floor = rho_floor
        self.p.p_floor = p_floor
        self.p.recon = RECON[recon] if isinstance(recon, str) else int(recon)
        self.floor_counts = (ctypes.c_longlong * 2)(0, 0)

    @property
    def gamma(self):
        return self.p.gamma

    def _chk(self, U):
        U = np.ascontiguousarray(U, np.float64)
        assert U.shape == (8,) + self.shape, U.shape
        return U

    def primitives(self, U):
        """(rho, vx, vy, vz, P, Bcc_x, Bcc_y, Bcc_z) per cell, shape [8, nz, ny, nx]."""
        U = self._chk(U)
        W = np.empty_like(U)
        self.lib.oracle_primitives(ctypes.byref(self.p), _ptr(U), _ptr(W))
        return W

    def dt(self, U, cfl):
        U = self._chk(U)
        return self.lib.oracle_dt(ctypes.byref(self.p), _ptr(U), cfl)

    def recon(self, U, axis, recon=None):
        """(WL, WR): WL[:, c] = W_{L, c+1/2}, WR[:, c] = W_{R, c-1/2} along ``axis``,
        in the solver frame (rho, v_n, v_t1, v_t2, P, B_t1, B_t2)."""
        U = self._chk(U)
        r = self.p.recon if recon is None else (RECON[recon] if isinstance(recon, str) else recon)
        WL = np.empty((7,) + self.shape)
        WR = np.empty((7,) + self.shape)
        self.lib.oracle_recon(ctypes.byref(self.p), _ptr(U), axis, r, _ptr(WL), _ptr(WR))
        return WL, WR

    def fluxes(self, U, recon=None):
        """F[3, 7, nz, ny, nx]: flux through the upper face of each cell per axis,
        solver frame (rho, m_n, m_t1, m_t2, E, B_t1, B_t2)."""
        U = self._chk(U)
        r = self.p.recon if recon is None else (RECON[recon] if isinstance(recon, str) else recon)
        F = np.empty((3, 7) + self.shape)
        self.lib.oracle_fluxes(ctypes.byref(self.p), _ptr(U), r, _ptr(F))
        return F

    def edges(self, U, F):
        """E[3, nz, ny, nx]: edge electric field E_a of each cell at p + e_b/2 + e_c/2."""
        U = self._chk(U)
        F = np.ascontiguousarray(F, np.float64)
        E = np.empty((3,) + self.shape)
        self.lib.oracle_edges(ctypes.byref(self.p), _ptr(U), _ptr(F), _ptr(E))
        return E

    def update(self, U0, F, E, h):
        U0 = self._chk(U0)
        F = np.ascontiguousarray(F, np.float64)
        E = np.ascontiguousarray(E, np.float64)
        out = np.empty_like(U0)
        self.lib.oracle_update(ctypes.byref(self.p), _ptr(U0), _ptr(F), _ptr(E), h, _ptr(out))
        return out

    def step(self, U, dt):
        """One VL+CT step at fixed dt; returns the new state (input untouched)."""
        V = self._chk(U).copy()
        self.lib.oracle_step(ctypes.byref(self.p), _ptr(V), dt, self.floor_counts)
        return V

    def run(self, U, nsteps, cfl=None, dts=None):
        """``nsteps`` steps with dt = CFL min (Step 1) or the given dts; returns (U, dts)."""
        V = self._chk(U).copy()
        used = []
        for s in range(nsteps):
            dt = dts[s] if dts is not None else self.dt(V, cfl)
            self.lib.oracle_step(ctypes.byref(self.p), _ptr(V), dt, self.floor_counts)
            used.append(dt)
        return V, used

    def step_jvp(self, U, dU, dt):
        """(U^{n+1}, J dU) for one step at fixed dt (forward-mode dual numbers)."""
        V = self._chk(U).copy()
        dV = self._chk(dU).copy()
        self.lib.oracle_step_jvp(ctypes.byref(self.p), _ptr(V), _ptr(dV), dt)
        return V, dV

    def dt_jvp(self, U, dU, cfl):
        """(dt, d dt) of Eq. dt and its derivative along dU."""
        d = ctypes.c_double(0)
        dt = self.lib.oracle_dt_jvp(ctypes.byref(self.p), _ptr(self._chk(U)), _ptr(self._chk(dU)), cfl, ctypes.byref(d))
        return dt, d.value

    def step_cfl_jvp(self, U, dU, cfl):
        """(U^{n+1}, J dU, dt) for one step at the CFL dt of U, the dt's
        dependence on U differentiated too."""
        V = self._chk(U).copy()
        dV = self._chk(dU).copy()
        dt = ctypes.c_double(0)
        self.lib.oracle_step_cfl_jvp(ctypes.byref(self.p), _ptr(V), _ptr(dV), cfl, ctypes.byref(dt))
        return V, dV, dt.value

    def recon_jvp(self, U, dU, axis, recon=None):
        """(WL, WR, dWL, dWR) of U -> (W_L, W_R) along ``axis`` and its derivative along dU."""
        U = self._chk(U)
        dU = self._chk(dU)
        r = self.p.recon if recon is None else (RECON[recon] if isinstance(recon, str) else recon)
        out = [np.empty((7,) + self.shape) for _ in range(4)]
        self.lib.oracle_recon_jvp(ctypes.byref(self.p), _ptr(U), _ptr(dU), axis, r, *[_ptr(x) for x in out])
        return tuple(out)

    def diagnostics(self, U):
        U = self._chk(U)
        m = ctypes.c_double(0)
        tot = np.zeros(8)
        self.lib.oracle_diagnostics(ctypes.byref(self.p), _ptr(U), ctypes.byref(m), _ptr(tot))
        return m.value, tot


def hlld(gamma, wl, wr, bn):
    lib = _load()
    wl = np.ascontiguousarray(wl, np.float64)
    wr = np.ascontiguousarray(wr, np.float64)
    f = np.zeros(7)
    lib.oracle_hlld(gamma, _ptr(wl), _ptr(wr), bn, _ptr(f))
    return f


def hlld_detail(gamma, wl, wr, bn):
    """(flux, speeds[5], states[6,7], physical fluxes[2,7], star_formed)."""
    lib = _load()
    wl = np.ascontiguousarray(wl, np.float64)
    wr = np.ascontiguousarray(wr, np.float64)
    f = np.zeros(7)
    sp = np.full(5, np.nan)
    st = np.full((6, 7), np.nan)
    fl = np.zeros((2, 7))
    star = lib.oracle_hlld_detail(gamma, _ptr(wl), _ptr(wr), bn, _ptr(f), _ptr(sp), _ptr(st), _ptr(fl))
    return f, sp, st, fl, bool(star)


def hlld_jvp(gamma, wl, wr, bn, dwl, dwr, dbn):
    """(flux, J (dwl, dwr, dbn)) of the HLLD flux (forward-mode dual numbers)."""
    lib = _load()
    args = [np.ascontiguousarray(x, np.float64) for x in (wl, wr, dwl, dwr)]
    f = np.zeros(7)
    df = np.zeros(7)
    lib.oracle_hlld_jvp(gamma, _ptr(args[0]), _ptr(args[1]), float(bn), _ptr(args[2]), _ptr(args[3]), float(dbn),
                        _ptr(f), _ptr(df))
    return f, df


def eigen(gamma, w, bn):
    """(lambda[7], R[7,7], L[7,7]) of the primitive system in the solver frame."""
    lib = _load()
    w = np.ascontiguousarray(w, np.float64)
    lam = np.zeros(7)
    R = np.zeros((7, 7))
    L = np.zeros((7, 7))
    lib.oracle_eigen(gamma, _ptr(w), bn, _ptr(lam), _ptr(R), _ptr(L))
    return lam, R, L


def fast_speed(gamma, rho, p, bl, bt1, bt2):
    return _load().oracle_fast_speed(gamma, rho, p, bl, bt1, bt2)
