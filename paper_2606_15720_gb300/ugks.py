"""Python binding of the C ABI in include/ugks.h (argument marshalling only).

Every step of the UGKS path runs in the CUDA library libugks.so built by
``paper_2606_15720_gb300.build``; this module only converts numpy arrays and
dataclasses into the C structs and calls the entry points of the same names.
There is no fallback: if the library cannot be loaded, or a call fails, an
exception is raised.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

from . import build as _build
from .inputs import LIMITERS, MODELS, Gas, Mesh, VelocityGrid

STORAGE = {"f64": 0, "f32": 1, "f16": 2, "bf16": 3}
SWEEP = {"auto": 0, "tiled": 1, "blocked": 2, "blocked_fused": 3}
STATUS = {0: "UGKS_OK", 1: "UGKS_ERR_INVALID_ARGUMENT", 2: "UGKS_ERR_MESH", 3: "UGKS_ERR_VGRID",
          4: "UGKS_ERR_OUT_OF_MEMORY", 5: "UGKS_ERR_CUDA", 6: "UGKS_ERR_NONFINITE", 7: "UGKS_ERR_TIMEOUT",
          8: "UGKS_ERR_UNSUPPORTED"}

_lib = None


class UGKSError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class ugks_bc(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int32), ("rho", ctypes.c_double), ("u", ctypes.c_double * 3),
                ("T", ctypes.c_double)]


class ugks_mesh(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("n_cells", ctypes.c_int64), ("n_faces", ctypes.c_int64),
                ("cell_volume", ctypes.c_void_p), ("cell_centroid", ctypes.c_void_p),
                ("face_owner", ctypes.c_void_p), ("face_neighbor", ctypes.c_void_p),
                ("face_area", ctypes.c_void_p), ("face_normal", ctypes.c_void_p),
                ("face_centroid", ctypes.c_void_p), ("face_shift", ctypes.c_void_p),
                ("n_bc", ctypes.c_int32), ("bc", ctypes.c_void_p)]


class ugks_vgrid(ctypes.Structure):
    _fields_ = [("n_v", ctypes.c_int64), ("u", ctypes.c_void_p), ("weight", ctypes.c_void_p),
                ("tensor_n", ctypes.c_int32 * 3), ("axis", ctypes.c_void_p * 3)]


class ugks_params(ctypes.Structure):
    _fields_ = [("model", ctypes.c_int32), ("K", ctypes.c_int32), ("Pr", ctypes.c_double),
                ("omega", ctypes.c_double), ("mu_ref", ctypes.c_double), ("cfl", ctypes.c_double),
                ("dt_override", ctypes.c_double), ("limiter", ctypes.c_int32), ("venkat_K", ctypes.c_double),
                ("shock_tau_fix", ctypes.c_int32), ("storage", ctypes.c_int32), ("tile_cells", ctypes.c_int32),
                ("sweep", ctypes.c_int32), ("block_velocities", ctypes.c_int32)]


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Loads libugks.so (building it first if it is missing and nvcc exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.LIB) and build_if_missing:
        _build.build()
    lib = ctypes.CDLL(_build.LIB)
    P, I32, I64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    sig = {
        "ugks_create": [P, P, P, P, P, P],
        "ugks_step": [P, I32],
        "ugks_step_static_scratch": [P, I32],
        "ugks_moments": [P, P, P],
        "ugks_residual": [P, P],
        "ugks_dt": [P, P],
        "ugks_sizes": [P, P, P],
        "ugks_get_f": [P, P, I64, P],
        "ugks_get_state": [P, P, P, P],
        "ugks_set_state": [P, P, P, I64],
        "ugks_stats_enable": [P, I32],
        "ugks_stats": [P, I32, P, P, P, P],
        "ugks_solve": [P, P, P, P, I32, P, P],
        "ugks_surface": [P, P, I64, P, P, P, P],
        "ugks_moments13": [P, P],
        "ugks_init_moments13": [P, P],
        "ugks_batch_create": [I32, P, P, P, P, P, P],
        "ugks_batch_autotune": [P],
        "ugks_batch_step": [P, I32],
        "ugks_batch_context": [P, I32, P],
        "ugks_batch_tuning": [P, I32, P, P],
        "ugks_batch_shape": [P, I32, P, P, P, P, P],
        "ugks_batch_destroy": [P],
        "ugks_destroy": [P],
        "ugks_mesh_sizes": [P, P, P, P],
        "ugks_mlp_create": [I32, I32, I32, I32, ctypes.c_uint64, P, P],
        "ugks_mlp_set_scaling": [P, P, P, P, P],
        "ugks_mlp_get_scaling": [P, P, P, P, P],
        "ugks_mlp_fit_scaling": [P, P, P, I64],
        "ugks_mlp_param_count": [P, P],
        "ugks_mlp_get_params": [P, P],
        "ugks_mlp_set_params": [P, P],
        "ugks_mlp_gradients": [P, P, P, I64, P, P],
        "ugks_mlp_train": [P, P, P, I64, I32, I32, ctypes.c_float, ctypes.c_uint64, P],
        "ugks_mlp_predict": [P, P, I64, P],
        "ugks_mlp_features": [P, P, ctypes.c_double, ctypes.c_double, P],
        "ugks_mlp_warm_start": [P, P, P, ctypes.c_double, ctypes.c_double, P, P],
        "ugks_mlp_destroy": [P],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    lib.ugks_last_error.argtypes = [P]
    lib.ugks_last_error.restype = ctypes.c_char_p
    lib.ugks_mlp_last_error.argtypes = [P]
    lib.ugks_mlp_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data


class _MeshArgs:
    """Owns contiguous copies of the mesh / grid arrays while a call runs."""

    def __init__(self, mesh: Mesh, grid: VelocityGrid):
        f64 = lambda a: np.ascontiguousarray(a, dtype=np.float64)  # noqa: E731
        i64 = lambda a: np.ascontiguousarray(a, dtype=np.int64)  # noqa: E731
        self.arrays = [f64(mesh.cell_volume), f64(mesh.cell_centroid), i64(mesh.face_owner),
                       i64(mesh.face_neighbor), f64(mesh.face_area), f64(mesh.face_normal),
                       f64(mesh.face_centroid), f64(mesh.face_shift)]
        nbc = max(1, len(mesh.bc))
        self.bcs = (ugks_bc * nbc)()
        for i, b in enumerate(mesh.bc):
            self.bcs[i].type = int(b.type)
            self.bcs[i].rho = float(b.rho)
            for d in range(3):
                self.bcs[i].u[d] = float(b.u[d])
            self.bcs[i].T = float(b.T)
        a = self.arrays
        self.mesh = ugks_mesh(mesh.dim, mesh.n_cells, mesh.n_faces, *[_ptr(x) for x in a], len(mesh.bc),
                              ctypes.addressof(self.bcs))
        if grid is not None:
            self.u = f64(grid.u)
            self.w = f64(grid.weight)
            self.grid = ugks_vgrid(grid.n_v, _ptr(self.u), _ptr(self.w))
            if grid.axes is not None:   # declare the tensor product (checked by the library)
                self.axes = [f64(a) for a in grid.axes]
                for d, ax in enumerate(self.axes):
                    self.grid.tensor_n[d] = int(ax.size)
                    self.grid.axis[d] = _ptr(ax)


def make_params(gas: Gas, storage: str = "f32", tile_cells: int = 0, sweep: str = "auto",
                block_velocities: int = 0) -> ugks_params:
    return ugks_params(MODELS[gas.model], int(gas.K), float(gas.Pr), float(gas.omega), float(gas.mu_ref),
                       float(gas.cfl), float(gas.dt), LIMITERS[gas.limiter], float(gas.venkat_K),
                       int(bool(gas.shock_tau_fix)), STORAGE[storage], int(tile_cells), SWEEP[sweep],
                       int(block_velocities))


def _check(lib, status: int, ctx=None):
    if status != 0:
        msg = lib.ugks_last_error(ctx).decode(errors="replace")
        raise UGKSError(status, msg)


def current_stream_handle() -> Optional[int]:
    """cudaStream_t of torch's current stream (torch supplies streams), or None."""
    try:
        import torch
        if torch.cuda.is_available():
            return int(torch.cuda.current_stream().cuda_stream)
    except Exception:  # pragma: no cover - torch missing
        return None
    return None


class Solver:
    """One ugks_ctx: ugks_create / ugks_step / ugks_moments / ugks_residual."""

    def __init__(self, mesh: Mesh, grid: VelocityGrid, gas: Gas, W_init: Optional[np.ndarray] = None,
                 storage: str = "f32", tile_cells: int = 0, stream: Optional[int] = None, sweep: str = "auto",
                 block_velocities: int = 0):
        self._lib = load()
        self.mesh, self.grid, self.gas = mesh, grid, gas
        self.dim = mesh.dim
        args = _MeshArgs(mesh, grid)
        prm = make_params(gas, storage, tile_cells, sweep, block_velocities)
        W = None if W_init is None else np.ascontiguousarray(W_init, dtype=np.float64)
        if W is not None and W.shape != (mesh.n_cells, mesh.dim + 2):
            raise ValueError("W_init must be [n_cells, dim+2]")
        if stream is None:
            stream = current_stream_handle()
        ctx = ctypes.c_void_p()
        st = self._lib.ugks_create(ctypes.byref(args.mesh), ctypes.byref(args.grid), ctypes.byref(prm), _ptr(W),
                                   stream, ctypes.byref(ctx))
        _check(self._lib, st)
        self._ctx = ctx
        nr = ctypes.c_int32()
        nvp = ctypes.c_int64()
        self._lib.ugks_sizes(self._ctx, ctypes.byref(nr), ctypes.byref(nvp))
        self.n_reduced = nr.value
        self.n_v_padded = nvp.value

    @classmethod
    def _view(cls, lib, ctx, mesh: Mesh, grid: VelocityGrid, gas: Gas) -> "Solver":
        """A Solver over a context owned by someone else (a batch case)."""
        self = cls.__new__(cls)
        self._lib, self._ctx, self._owned = lib, ctx, False
        self.mesh, self.grid, self.gas, self.dim = mesh, grid, gas, mesh.dim
        nr, nvp = ctypes.c_int32(), ctypes.c_int64()
        lib.ugks_sizes(ctx, ctypes.byref(nr), ctypes.byref(nvp))
        self.n_reduced, self.n_v_padded = nr.value, nvp.value
        return self

    def _c(self, st):
        _check(self._lib, st, self._ctx)

    def step(self, n: int = 1) -> None:
        self._c(self._lib.ugks_step(self._ctx, int(n)))

    def step_static_scratch(self, n: int = 1) -> None:
        """ugks_step_static_scratch: the same step without any device allocation."""
        self._c(self._lib.ugks_step_static_scratch(self._ctx, int(n)))

    def moments(self, with_q: bool = False):
        W = np.zeros((self.mesh.n_cells, self.dim + 2))
        q = np.zeros((self.mesh.n_cells, self.dim)) if with_q else None
        self._c(self._lib.ugks_moments(self._ctx, _ptr(W), _ptr(q)))
        return (W, q) if with_q else W

    def residual(self) -> np.ndarray:
        r = np.zeros(self.dim + 2)
        self._c(self._lib.ugks_residual(self._ctx, _ptr(r)))
        return r

    @property
    def dt(self) -> float:
        v = ctypes.c_double()
        self._c(self._lib.ugks_dt(self._ctx, ctypes.byref(v)))
        return v.value

    def surface(self, freestream: Optional[Sequence[float]] = None):
        """ugks_surface: (faces, vals[:, p_w, tau_w[dim], q_w], coef[:, C_p, C_t, C_h] or None)
        of the diffuse-wall faces after the last step."""
        n = ctypes.c_int64()
        fs = None if freestream is None else np.ascontiguousarray(freestream, dtype=np.float64)
        cap = sum(1 for j in self.mesh.face_neighbor if j < 0 and self.mesh.bc[-j - 1].type == 1)
        faces = np.zeros(max(cap, 1), dtype=np.int64)
        vals = np.zeros((max(cap, 1), self.dim + 2))
        coef = np.zeros((max(cap, 1), 3))
        self._c(self._lib.ugks_surface(self._ctx, _ptr(fs), cap, ctypes.byref(n), _ptr(faces), _ptr(vals),
                                       _ptr(coef)))
        k = n.value
        return faces[:k], vals[:k], (coef[:k] if fs is not None else None)

    @property
    def n13(self) -> int:
        return 2 * self.dim + 2 + self.dim * (self.dim + 1) // 2

    def moments13(self) -> np.ndarray:
        """ugks_moments13: [n_cells, n13] = rho, U, T, sigma (xx, xy, (xz), yy, (yz), zz), q."""
        out = np.zeros((self.mesh.n_cells, self.n13))
        self._c(self._lib.ugks_moments13(self._ctx, _ptr(out)))
        return out

    def init_moments13(self, fields: np.ndarray) -> None:
        """ugks_init_moments13: Chapman-Enskog state of the given fields."""
        fields = np.ascontiguousarray(fields, dtype=np.float64)
        assert fields.shape == (self.mesh.n_cells, self.n13)
        self._c(self._lib.ugks_init_moments13(self._ctx, _ptr(fields)))

    def get_f(self, cells: Sequence[int]) -> np.ndarray:
        cells = np.ascontiguousarray(cells, dtype=np.int64)
        out = np.zeros((cells.size, self.n_reduced, self.grid.n_v))
        self._c(self._lib.ugks_get_f(self._ctx, _ptr(cells), cells.size, _ptr(out)))
        return out

    def get_state(self):
        W = np.zeros((self.mesh.n_cells, self.dim + 2))
        f = np.zeros((self.n_reduced, self.mesh.n_cells, self.grid.n_v))
        step = ctypes.c_int64()
        self._c(self._lib.ugks_get_state(self._ctx, _ptr(W), _ptr(f), ctypes.byref(step)))
        return W, f, step.value

    def set_state(self, W: np.ndarray, f: np.ndarray, step: int = 0) -> None:
        W = np.ascontiguousarray(W, dtype=np.float64)
        f = np.ascontiguousarray(f, dtype=np.float64)
        assert f.shape == (self.n_reduced, self.mesh.n_cells, self.grid.n_v)
        self._c(self._lib.ugks_set_state(self._ctx, _ptr(W), _ptr(f), int(step)))

    def stats_enable(self, on: bool = True) -> None:
        self._c(self._lib.ugks_stats_enable(self._ctx, int(bool(on))))

    def stats(self) -> dict:
        cap = 16
        names = (ctypes.c_char_p * cap)()
        ms = np.zeros(cap)
        cnt = np.zeros(cap, dtype=np.int64)
        n = ctypes.c_int32()
        self._c(self._lib.ugks_stats(self._ctx, cap, ctypes.addressof(names), _ptr(ms), _ptr(cnt), ctypes.byref(n)))
        return {names[i].decode(): (float(ms[i]), int(cnt[i])) for i in range(n.value)}

    def close(self) -> None:
        if getattr(self, "_ctx", None) and getattr(self, "_owned", True):
            self._lib.ugks_destroy(self._ctx)
        self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Batch:
    """ugks_batch_*: many cases stepped by one CUDA-graph launch per two steps."""

    def __init__(self, meshes, grids, gases, W_inits=None, storage: str = "f32", block_velocities: int = 0,
                 stream: Optional[int] = None):
        self._lib = load()
        n = len(meshes)
        self._args = [_MeshArgs(m, g) for m, g in zip(meshes, grids)]
        self.meshes, self.grids, self.gases = list(meshes), list(grids), list(gases)
        mptr = (ctypes.c_void_p * n)(*[ctypes.addressof(a.mesh) for a in self._args])
        gptr = (ctypes.c_void_p * n)(*[ctypes.addressof(a.grid) for a in self._args])
        prms = (ugks_params * n)(*[make_params(gs, storage, 0, "blocked", block_velocities) for gs in gases])
        self._W = None
        wptr = None
        if W_inits is not None:
            self._W = [np.ascontiguousarray(W, dtype=np.float64) for W in W_inits]
            wptr = (ctypes.c_void_p * n)(*[_ptr(W) for W in self._W])
        if stream is None:
            stream = current_stream_handle()
        b = ctypes.c_void_p()
        _check(self._lib, self._lib.ugks_batch_create(n, mptr, gptr, prms, wptr, stream, ctypes.byref(b)))
        self._b = b
        self.cases = []
        for i in range(n):
            c = ctypes.c_void_p()
            self._c(self._lib.ugks_batch_context(self._b, i, ctypes.byref(c)))
            self.cases.append(Solver._view(self._lib, c, meshes[i], grids[i], gases[i]))

    def _c(self, st):
        if st != 0:
            raise UGKSError(st, self._lib.ugks_last_error(None).decode(errors="replace"))

    def autotune(self) -> None:
        self._c(self._lib.ugks_batch_autotune(self._b))

    def step(self, n: int = 1) -> None:
        self._c(self._lib.ugks_batch_step(self._b, int(n)))

    def shape(self, i: int) -> dict:
        """ugks_batch_shape: the (tuned) shape of case i."""
        bv, fu, ch, tr = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        ms = ctypes.c_double()
        self._c(self._lib.ugks_batch_shape(self._b, int(i), ctypes.byref(bv), ctypes.byref(fu), ctypes.byref(ch),
                                           ctypes.byref(ms), ctypes.byref(tr)))
        return {"block_velocities": bv.value, "fused": bool(fu.value), "stage2_chunks": ch.value,
                "ms_per_step": ms.value, "trials": tr.value}

    def tuning(self, i: int):
        bv = ctypes.c_int32()
        ms = np.zeros(4)
        self._c(self._lib.ugks_batch_tuning(self._b, int(i), ctypes.byref(bv), _ptr(ms)))
        return bv.value, ms

    def close(self) -> None:
        if getattr(self, "_b", None):
            for c in self.cases:
                c._ctx = None
            self._lib.ugks_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class WarmStartNet:
    """ugks_mlp_*: the warm-start network (BF16 weights and activations, FP32
    accumulation, master weights and Adam state), trained and evaluated by the
    library's kernels.  Arrays are host numpy arrays (converted to FP32)."""

    N_FEATURES = 6

    def __init__(self, n_in: int, n_out: int, width: int = 256, hidden_layers: int = 6, seed: int = 0,
                 stream: Optional[int] = None):
        self._lib = load()
        self.n_in, self.n_out, self.width, self.hidden_layers = int(n_in), int(n_out), int(width), int(hidden_layers)
        self.sizes = [self.n_in] + [self.width] * self.hidden_layers + [self.n_out]
        net = ctypes.c_void_p()
        st = self._lib.ugks_mlp_create(self.n_in, self.n_out, self.width, self.hidden_layers,
                                       ctypes.c_uint64(int(seed)), stream, ctypes.byref(net))
        if st != 0:
            raise UGKSError(st, self._lib.ugks_mlp_last_error(None).decode(errors="replace"))
        self._net = net

    def _c(self, st):
        if st != 0:
            raise UGKSError(st, self._lib.ugks_mlp_last_error(self._net).decode(errors="replace"))

    @staticmethod
    def _f32(a, cols):
        a = np.ascontiguousarray(a, dtype=np.float32)
        if a.ndim != 2 or a.shape[1] != cols:
            raise ValueError(f"expected an array of shape (n, {cols}), got {a.shape}")
        return a

    def param_count(self) -> int:
        n = ctypes.c_int64()
        self._c(self._lib.ugks_mlp_param_count(self._net, ctypes.byref(n)))
        return n.value

    def get_params(self) -> np.ndarray:
        out = np.zeros(self.param_count(), dtype=np.float32)
        self._c(self._lib.ugks_mlp_get_params(self._net, _ptr(out)))
        return out

    def set_params(self, params: np.ndarray) -> None:
        p = np.ascontiguousarray(params, dtype=np.float32)
        if p.size != self.param_count():
            raise ValueError("wrong number of parameters")
        self._c(self._lib.ugks_mlp_set_params(self._net, _ptr(p)))

    def set_scaling(self, in_shift, in_scale, out_shift, out_scale) -> None:
        a = [np.ascontiguousarray(x, dtype=np.float32) for x in (in_shift, in_scale, out_shift, out_scale)]
        if a[0].size != self.n_in or a[1].size != self.n_in or a[2].size != self.n_out or a[3].size != self.n_out:
            raise ValueError("scaling arrays have the wrong sizes")
        self._c(self._lib.ugks_mlp_set_scaling(self._net, *[_ptr(x) for x in a]))

    def get_scaling(self):
        a = [np.zeros(k, dtype=np.float32) for k in (self.n_in, self.n_in, self.n_out, self.n_out)]
        self._c(self._lib.ugks_mlp_get_scaling(self._net, *[_ptr(x) for x in a]))
        return tuple(a)

    def fit_scaling(self, X, Y) -> None:
        X, Y = self._f32(X, self.n_in), self._f32(Y, self.n_out)
        self._c(self._lib.ugks_mlp_fit_scaling(self._net, _ptr(X), _ptr(Y), X.shape[0]))

    def gradients(self, X, Y):
        X, Y = self._f32(X, self.n_in), self._f32(Y, self.n_out)
        g = np.zeros(self.param_count(), dtype=np.float32)
        loss = ctypes.c_double()
        self._c(self._lib.ugks_mlp_gradients(self._net, _ptr(X), _ptr(Y), X.shape[0], _ptr(g), ctypes.byref(loss)))
        return g, loss.value

    def train(self, X, Y, epochs: int, batch: int = 1024, lr: float = 1e-3, seed: int = 0) -> float:
        X, Y = self._f32(X, self.n_in), self._f32(Y, self.n_out)
        loss = ctypes.c_double()
        self._c(self._lib.ugks_mlp_train(self._net, _ptr(X), _ptr(Y), X.shape[0], int(epochs), int(batch),
                                         ctypes.c_float(lr), ctypes.c_uint64(int(seed)), ctypes.byref(loss)))
        return loss.value

    def predict(self, X) -> np.ndarray:
        X = self._f32(X, self.n_in)
        Y = np.zeros((X.shape[0], self.n_out), dtype=np.float32)
        self._c(self._lib.ugks_mlp_predict(self._net, _ptr(X), X.shape[0], _ptr(Y)))
        return Y

    def features(self, mesh: Mesh, mach: float, kn: float) -> np.ndarray:
        args = _MeshArgs(mesh, None)
        out = np.zeros((mesh.n_cells, self.N_FEATURES), dtype=np.float32)
        self._c(self._lib.ugks_mlp_features(self._net, ctypes.byref(args.mesh), float(mach), float(kn), _ptr(out)))
        return out

    def warm_start(self, solver: "Solver", mesh: Mesh, mach: float, kn: float, freestream) -> int:
        """Resets the solver to the Chapman-Enskog start of the predicted
        fields; returns the number of cells that fell back to the freestream."""
        args = _MeshArgs(mesh, None)
        fs = np.ascontiguousarray(freestream, dtype=np.float64)
        if fs.size != mesh.dim + 2:
            raise ValueError("freestream = (rho, U[dim], T)")
        nf = ctypes.c_int64()
        self._c(self._lib.ugks_mlp_warm_start(self._net, solver._ctx, ctypes.byref(args.mesh), float(mach),
                                              float(kn), _ptr(fs), ctypes.byref(nf)))
        return nf.value

    def close(self) -> None:
        if getattr(self, "_net", None):
            self._lib.ugks_mlp_destroy(self._net)
            self._net = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve(mesh: Mesh, grid: VelocityGrid, gas: Gas, W_init: np.ndarray, n_steps: int, storage: str = "f32",
          tile_cells: int = 0, sweep: str = "auto", block_velocities: int = 0):
    """ugks_solve: one call with host buffers (create, n steps, W and residual, destroy)."""
    lib = load()
    args = _MeshArgs(mesh, grid)
    prm = make_params(gas, storage, tile_cells, sweep, block_velocities)
    W = np.ascontiguousarray(W_init, dtype=np.float64)
    Wout = np.zeros_like(W)
    res = np.zeros(mesh.dim + 2)
    st = lib.ugks_solve(ctypes.byref(args.mesh), ctypes.byref(args.grid), ctypes.byref(prm), _ptr(W), int(n_steps),
                        _ptr(Wout), _ptr(res))
    _check(lib, st)
    return Wout, res
