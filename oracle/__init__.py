"""FP64 CPU oracle of the UGKS step (test infrastructure only).

The oracle is the plain C program ``ugks_oracle.c`` in this folder, compiled
with gcc (OpenMP over cells and faces) and called through ctypes.  It is the
independent reference that the CUDA path is checked against: it shares no code
with the CUDA library, and the product path never imports it.  Only tests/,
``__graft_entry__.smoke()`` and the CPU-baseline leg of bench.py may use it.

All arrays are numpy float64 / int64.  The distribution is stored as
``f[r, cell, k]`` with r = 0 for h and r = 1 for b (present when K_xi > 0).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sysconfig
from typing import Optional, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ugks_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None

LIMITERS = {"none": 0, "venkatakrishnan": 1, "barth_jespersen": 2}
MODELS = {"bgk": 0, "shakhov": 1}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into oracle/_build/liboracle.so."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=gnu11", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _BCStruct(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int32), ("rho", ctypes.c_double), ("u", ctypes.c_double * 3),
                ("T", ctypes.c_double)]


class _MeshStruct(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("n_cells", ctypes.c_int64), ("n_faces", ctypes.c_int64),
                ("vol", ctypes.c_void_p), ("xc", ctypes.c_void_p), ("own", ctypes.c_void_p),
                ("nei", ctypes.c_void_p), ("area", ctypes.c_void_p), ("nrm", ctypes.c_void_p),
                ("xf", ctypes.c_void_p), ("shift", ctypes.c_void_p), ("n_bc", ctypes.c_int32),
                ("bc", ctypes.c_void_p)]


class _ParamsStruct(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int32), ("model", ctypes.c_int32), ("Pr", ctypes.c_double),
                ("omega", ctypes.c_double), ("mu_ref", ctypes.c_double), ("cfl", ctypes.c_double),
                ("dt_override", ctypes.c_double), ("limiter", ctypes.c_int32),
                ("venkat_K", ctypes.c_double), ("shock_tau_fix", ctypes.c_int32),
                ("block_v", ctypes.c_int32), ("p_v", ctypes.c_int32)]


def load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        lib.orc_run.restype = ctypes.c_int
        lib.orc_run.argtypes = [P, ctypes.c_int64, P, P, P, P, P, ctypes.c_int32, P, P, P]
        lib.orc_surface.argtypes = [P, P, ctypes.c_double, P, P, P, P]
        lib.orc_moments13.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int64, ctypes.c_int64, P, P, P, P, P]
        lib.orc_chapman_enskog.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int64, ctypes.c_int64, P, P, P]
        lib.orc_surface.restype = ctypes.c_int64
        lib.orc_time_step.restype = ctypes.c_double
        lib.orc_time_step.argtypes = [P, ctypes.c_int64, P, P, ctypes.c_double]
        lib.orc_time_coefficients.argtypes = [ctypes.c_double, ctypes.c_double, P]
        lib.orc_micro_slope.argtypes = [ctypes.c_int, ctypes.c_int, P, P, P]
        lib.orc_time_slope.argtypes = [ctypes.c_int, ctypes.c_int, P, P, P]
        lib.orc_interface_W0.argtypes = [ctypes.c_int, ctypes.c_int, P, P, P, P]
        lib.orc_heat_flux.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int64, P, P, P, P, P, P]
        lib.orc_reduced_equilibrium.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, P, P, P, P]
        lib.orc_initial_f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int64, ctypes.c_int64, P, P, P]
        lib.orc_limiter_phi.restype = ctypes.c_double
        lib.orc_limiter_phi.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_double]
        lib.orc_num_threads.restype = ctypes.c_int
        lib.orc_set_threads.restype = ctypes.c_int
        lib.orc_set_threads.argtypes = [ctypes.c_int]
        _lib = lib
    return _lib


def _p(a: np.ndarray) -> int:
    return a.ctypes.data


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


class _Packed:
    """Keeps the numpy buffers alive while the C structs point into them."""

    def __init__(self, mesh):
        self.vol = _f64(mesh.cell_volume)
        self.xc = _f64(mesh.cell_centroid)
        self.own = np.ascontiguousarray(mesh.face_owner, dtype=np.int64)
        self.nei = np.ascontiguousarray(mesh.face_neighbor, dtype=np.int64)
        self.area = _f64(mesh.face_area)
        self.nrm = _f64(mesh.face_normal)
        self.xf = _f64(mesh.face_centroid)
        self.shift = _f64(mesh.face_shift)
        nbc = max(1, len(mesh.bc))
        self.bcs = (_BCStruct * nbc)()
        for i, b in enumerate(mesh.bc):
            self.bcs[i].type = b.type
            self.bcs[i].rho = b.rho
            for d in range(3):
                self.bcs[i].u[d] = b.u[d]
            self.bcs[i].T = b.T
        self.s = _MeshStruct(mesh.dim, mesh.n_cells, mesh.n_faces, _p(self.vol), _p(self.xc), _p(self.own),
                             _p(self.nei), _p(self.area), _p(self.nrm), _p(self.xf), _p(self.shift),
                             len(mesh.bc), ctypes.addressof(self.bcs))


def _params(gas, block_v: int = 0, p_v: int = 0, dt: Optional[float] = None) -> _ParamsStruct:
    return _ParamsStruct(int(gas.K), MODELS[gas.model], float(gas.Pr), float(gas.omega), float(gas.mu_ref),
                         float(gas.cfl), float(gas.dt if dt is None else dt), LIMITERS[gas.limiter],
                         float(gas.venkat_K), int(bool(gas.shock_tau_fix)), int(block_v), int(p_v))


def n_reduced(dim: int, K: int) -> int:
    return 2 if K + 3 - dim > 0 else 1


def initial_f(mesh, vgrid, W: np.ndarray, K: int) -> np.ndarray:
    """Discrete reduced Maxwellians of W (reading R18): f[r, cell, k]."""
    lib = load()
    nr = n_reduced(mesh.dim, K)
    f = np.zeros((nr, mesh.n_cells, vgrid.n_v))
    u = _f64(vgrid.u)
    W = _f64(W)
    lib.orc_initial_f(mesh.dim, K, mesh.n_cells, vgrid.n_v, _p(u), _p(W), _p(f))
    return f


def time_step(mesh, vgrid, cfl: float) -> float:
    lib = load()
    pk = _Packed(mesh)
    u = _f64(vgrid.u)
    w = _f64(vgrid.weight)
    return float(lib.orc_time_step(ctypes.addressof(pk.s), vgrid.n_v, _p(u), _p(w), float(cfl)))


def run(mesh, vgrid, gas, W: np.ndarray, f: np.ndarray, nsteps: int, block_v: int = 0, p_v: int = 0,
        dt: Optional[float] = None, face_flux: bool = False):
    """Advance (W, f) by nsteps UGKS steps.  Returns (W, f, dt, diag) where diag
    has one row per step: residual per conservative variable, then the largest
    |wall mass flux|; with face_flux=True also the last step's macro fluxes
    F[face, 5] (time-integrated, Eq. 28)."""
    lib = load()
    pk = _Packed(mesh)
    prm = _params(gas, block_v, p_v, dt)
    u = _f64(vgrid.u)
    w = _f64(vgrid.weight)
    W = _f64(W).copy()
    f = _f64(f).copy()
    assert f.shape == (n_reduced(mesh.dim, gas.K), mesh.n_cells, vgrid.n_v)
    diag = np.zeros((max(nsteps, 1), mesh.dim + 3))
    F = np.zeros((mesh.n_faces, 5))
    dt_out = ctypes.c_double(0.0)
    rc = lib.orc_run(ctypes.addressof(pk.s), vgrid.n_v, _p(u), _p(w), ctypes.addressof(prm), _p(W), _p(f),
                     int(nsteps), ctypes.addressof(dt_out), _p(diag), _p(F))
    if rc != 0:
        raise RuntimeError("oracle step failed (non-physical state or unsupported mesh)")
    if face_flux:
        return W, f, dt_out.value, diag[:nsteps], F
    return W, f, dt_out.value, diag[:nsteps]


def surface(mesh, F: np.ndarray, dt: float, freestream=None):
    """Surface quantities of the diffuse-wall faces from their time-integrated
    fluxes F (reading R20): (faces, vals[:, p_w, tau_w[dim], q_w], coef[:, C_p,
    C_t, C_h] or None)."""
    lib = load()
    pk = _Packed(mesh)
    F = _f64(F)
    nwall = int(np.sum([(mesh.bc[-j - 1].type == 1) for j in mesh.face_neighbor if j < 0]))
    faces = np.zeros(max(nwall, 1), dtype=np.int64)
    vals = np.zeros((max(nwall, 1), mesh.dim + 2))
    coef = np.zeros((max(nwall, 1), 3))
    fs = None if freestream is None else _f64(freestream)
    n = lib.orc_surface(ctypes.addressof(pk.s), _p(F), float(dt), _p(fs) if fs is not None else None, _p(faces),
                        _p(vals), _p(coef))
    assert n == nwall
    return faces[:n], vals[:n], (coef[:n] if fs is not None else None)


def limiter_phi(kind: str, d2: float, dmax: float, dmin: float, eps2: float = 0.0) -> float:
    """The oracle's limiter value for one face increment d2 of a cell whose
    stencil spans [dmin, dmax] around the cell value (reading R1)."""
    return float(load().orc_limiter_phi(LIMITERS[kind], float(d2), float(dmax), float(dmin), float(eps2)))


def time_coefficients(dt: float, tau: float) -> np.ndarray:
    lib = load()
    G = np.zeros(5)
    lib.orc_time_coefficients(float(dt), float(tau), _p(G))
    return G


def interface_W0(dim: int, K: int, Wl, Wr, n) -> np.ndarray:
    lib = load()
    Wl, Wr, n = _f64(Wl), _f64(Wr), _f64(n)
    W0 = np.zeros(dim + 2)
    lib.orc_interface_W0(dim, K, _p(Wl), _p(Wr), _p(n), _p(W0))
    return W0


def micro_slope(dim: int, K: int, W0, dW) -> np.ndarray:
    lib = load()
    W0, dW = _f64(W0), _f64(dW)
    a = np.zeros(dim + 2)
    lib.orc_micro_slope(dim, K, _p(W0), _p(dW), _p(a))
    return a


def time_slope(dim: int, K: int, W0, a) -> np.ndarray:
    lib = load()
    W0, a = _f64(W0), _f64(a)
    A = np.zeros(dim + 2)
    lib.orc_time_slope(dim, K, _p(W0), _p(a), _p(A))
    return A


def heat_flux(dim: int, K: int, vgrid, h, b, W) -> np.ndarray:
    lib = load()
    u, w, h, W = _f64(vgrid.u), _f64(vgrid.weight), _f64(h), _f64(W)
    bp = _p(_f64(b)) if b is not None else None
    bb = _f64(b) if b is not None else None
    q = np.zeros(3)
    lib.orc_heat_flux(dim, K, vgrid.n_v, _p(u), _p(w), _p(h), _p(bb) if bb is not None else None, _p(W), _p(q))
    del bp
    return q[:dim]


def reduced_equilibrium(dim: int, K: int, Pr: float, rho: float, U, lam: float, q, u) -> np.ndarray:
    """{H, B, H+, B+} at one velocity u (Eq. 16-19)."""
    lib = load()
    prim = _f64([rho] + list(U)[:dim] + [lam])
    q = _f64(list(q)[:dim] + [0.0] * (3 - dim))
    u = _f64(u)
    out = np.zeros(4)
    lib.orc_reduced_equilibrium(dim, K, float(Pr), _p(prim), _p(q), _p(u), _p(out))
    return out


def n13(dim: int) -> int:
    """Entries of the thirteen-moment fields per cell: rho, U, T, sigma, q."""
    return 2 * dim + 2 + dim * (dim + 1) // 2


def moments13(dim: int, K: int, vgrid, W: np.ndarray, f: np.ndarray) -> np.ndarray:
    """Thirteen-moment fields [cell, n13(dim)] of (W, f) (reading R21)."""
    lib = load()
    W, f = _f64(W), _f64(f)
    nc = W.shape[0]
    out = np.zeros((nc, n13(dim)))
    lib.orc_moments13(dim, K, nc, vgrid.n_v, _p(_f64(vgrid.u)), _p(_f64(vgrid.weight)), _p(W), _p(f), _p(out))
    return out


def chapman_enskog(dim: int, K: int, vgrid, fields: np.ndarray) -> np.ndarray:
    """Chapman-Enskog distribution f[r, cell, k] of thirteen-moment fields (reading R21)."""
    lib = load()
    fields = _f64(fields)
    nc = fields.shape[0]
    f = np.zeros((n_reduced(dim, K), nc, vgrid.n_v))
    lib.orc_chapman_enskog(dim, K, nc, vgrid.n_v, _p(_f64(vgrid.u)), _p(fields), _p(f))
    return f


def num_threads() -> int:
    return int(load().orc_num_threads())


def set_threads(n: int) -> int:
    """OpenMP threads of later oracle calls; returns the previous count."""
    return int(load().orc_set_threads(int(n)))
