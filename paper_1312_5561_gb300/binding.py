"""Thin ctypes binding of the C ABI in include/fsi_solid.h.

Argument marshalling only: every step of the solid Newton step runs in the
CUDA kernels of libfsi_solid.so.  There is no CPU fallback; if the library
has not been built the import of this module raises.

Device arrays are torch CUDA tensors (FP64 [n_nodes, 4] states); the CUDA
stream passed to the library is torch's current stream.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os
from typing import Optional

import numpy as np

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "libfsi_solid.so")

FSI_OK = 0
STATUS = {0: "FSI_OK", -1: "FSI_ERR_ARG", -2: "FSI_ERR_CUDA", -3: "FSI_ERR_OOM", -4: "FSI_ERR_INVERTED",
          -5: "FSI_ERR_NOT_CONVERGED"}

# symbols declared in include/fsi_solid.h
EXPORTS = [
    "fsi_solid_default_opts", "fsi_solid_create", "fsi_solid_destroy", "fsi_solid_residual_tangent",
    "fsi_solid_get_bsr", "fsi_solid_spmv", "fsi_solid_linear_solve", "fsi_solid_newton_step",
    "fsi_solid_solve", "fsi_solid_get_colouring", "fsi_solid_get_levels", "fsi_solid_last_error",
    "fsi_solid_launch_count", "fsi_solid_kernel_timing", "fsi_dots_static",
    "fsi_mlp_create", "fsi_mlp_destroy", "fsi_mlp_num_params", "fsi_mlp_params", "fsi_mlp_forward",
    "fsi_mlp_train_step", "fsi_solid_newmark_advance", "fsi_dn_default_opts", "fsi_solid_dn_solve",
    "fsi_solid_get_tuning",
]

# kernel classes of fsi_solid_kernel_timing (FSI_KC_* in the header)
KERNEL_CLASSES = ["tangent", "residual", "jacobi0", "bsr0", "coarse_bsr", "transfer", "galerkin", "blockinv",
                  "coarse", "vector", "other", "level1_spmv"]


class MeshDesc(C.Structure):
    _fields_ = [("n_nodes", C.c_int32), ("n_elems", C.c_int32), ("X", C.c_void_p), ("tets", C.c_void_p),
                ("mat_id", C.c_void_p), ("fibre", C.c_void_p), ("dir_mask", C.c_void_p),
                ("n_faces", C.c_int32), ("neu_faces", C.c_void_p), ("n_segments", C.c_int32),
                ("seg_node", C.c_void_p)]


class MaterialDesc(C.Structure):
    _fields_ = [("model", C.c_int32), ("c10", C.c_double), ("c01", C.c_double), ("k1", C.c_double),
                ("k2", C.c_double), ("kappa", C.c_double), ("rho", C.c_double)]


class SolverOpts(C.Structure):
    _fields_ = [("precision", C.c_int32), ("krylov", C.c_int32), ("restart", C.c_int32),
                ("max_krylov", C.c_int32), ("max_newton", C.c_int32), ("smoother", C.c_int32),
                ("nu_pre", C.c_int32), ("nu_post", C.c_int32),
                ("coarse_max_nodes", C.c_int32), ("max_levels", C.c_int32), ("use_pspg", C.c_int32),
                ("adaptive_tol", C.c_int32), ("use_graphs", C.c_int32), ("nu_coarse", C.c_int32),
                ("omega", C.c_double), ("newton_rtol", C.c_double), ("krylov_rtol", C.c_double),
                ("fibre_factor", C.c_double), ("inertia_coef", C.c_double), ("amg_lag", C.c_int32),
                ("assembly", C.c_int32), ("precond", C.c_int32), ("schur_theta", C.c_double),
                ("vanka_omega", C.c_double), ("aggregation", C.c_int32), ("coarse_bf16", C.c_int32),
                ("coarse_smoother", C.c_int32), ("autotune", C.c_int32), ("segment_krylov", C.c_int32),
                ("exact_candidates", C.c_int32), ("power_steps", C.c_int32)]


class LoadDesc(C.Structure):
    _fields_ = [("dir_values", C.c_void_p), ("pressure", C.c_double), ("node_pressure", C.c_void_p),
                ("face_pressure", C.c_void_p), ("hist", C.c_void_p)]


class Info(C.Structure):
    _fields_ = [("newton_its", C.c_int32), ("krylov_its_total", C.c_int32), ("krylov_its_last", C.c_int32),
                ("status", C.c_int32), ("guess_accepted", C.c_int32), ("n_levels", C.c_int32),
                ("res0", C.c_double), ("res", C.c_double), ("inc_norm", C.c_double), ("lin_res", C.c_double),
                ("inc_mnorm", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class DnOpts(C.Structure):
    _fields_ = [("p0", C.c_double), ("added_mass", C.c_double), ("d_ref", C.c_void_p), ("omega0", C.c_double),
                ("tol", C.c_double), ("max_cycles", C.c_int32), ("aitken", C.c_int32)]


class DnInfo(C.Structure):
    _fields_ = [("cycles", C.c_int32), ("converged", C.c_int32), ("newton_its_total", C.c_int32),
                ("krylov_its_total", C.c_int32), ("n_interface", C.c_int32), ("res_first", C.c_double),
                ("res_last", C.c_double), ("omega_last", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def _load_library():
    if not os.path.exists(_LIB_PATH):
        raise ImportError(f"{_LIB_PATH} is missing: build it with `python -m paper_1312_5561_gb300.build` "
                          "(the solver has no CPU fallback)")
    lib = C.CDLL(_LIB_PATH)
    vp, i32 = C.c_void_p, C.c_int32
    lib.fsi_solid_default_opts.argtypes = [C.POINTER(SolverOpts)]
    lib.fsi_solid_default_opts.restype = None
    lib.fsi_solid_create.argtypes = [C.POINTER(MeshDesc), i32, C.POINTER(MaterialDesc), C.POINTER(SolverOpts),
                                     C.POINTER(vp)]
    lib.fsi_solid_create.restype = i32
    lib.fsi_solid_destroy.argtypes = [vp]
    lib.fsi_solid_destroy.restype = i32
    lib.fsi_solid_residual_tangent.argtypes = [vp, vp, C.POINTER(LoadDesc), vp, i32, vp]
    lib.fsi_solid_residual_tangent.restype = i32
    lib.fsi_solid_get_bsr.argtypes = [vp, C.POINTER(vp), C.POINTER(vp), C.POINTER(vp), C.POINTER(i32),
                                      C.POINTER(i32)]
    lib.fsi_solid_get_bsr.restype = i32
    lib.fsi_solid_spmv.argtypes = [vp, vp, vp, vp]
    lib.fsi_solid_spmv.restype = i32
    lib.fsi_solid_linear_solve.argtypes = [vp, vp, vp, C.POINTER(Info), vp]
    lib.fsi_solid_linear_solve.restype = i32
    lib.fsi_solid_newton_step.argtypes = [vp, vp, C.POINTER(LoadDesc), C.POINTER(Info), vp]
    lib.fsi_solid_newton_step.restype = i32
    lib.fsi_solid_solve.argtypes = [vp, vp, C.POINTER(LoadDesc), vp, C.POINTER(Info), vp]
    lib.fsi_solid_solve.restype = i32
    lib.fsi_solid_get_colouring.argtypes = [vp, vp, C.POINTER(i32)]
    lib.fsi_solid_get_colouring.restype = i32
    lib.fsi_solid_get_tuning.argtypes = [vp, vp, i32, C.POINTER(i32)]
    lib.fsi_solid_get_tuning.restype = i32
    lib.fsi_solid_get_levels.argtypes = [vp, vp, vp, i32, C.POINTER(i32)]
    lib.fsi_solid_get_levels.restype = i32
    lib.fsi_solid_last_error.argtypes = [vp]
    lib.fsi_solid_last_error.restype = C.c_char_p
    lib.fsi_solid_launch_count.argtypes = []
    lib.fsi_solid_launch_count.restype = C.c_int64
    lib.fsi_solid_kernel_timing.argtypes = [vp, i32, vp, vp]
    lib.fsi_solid_kernel_timing.restype = i32
    lib.fsi_dots_static.argtypes = [vp, C.c_int64, i32, vp, C.c_int64, vp, vp]
    lib.fsi_dots_static.restype = i32
    lib.fsi_mlp_create.argtypes = [i32, vp, C.c_uint64, C.POINTER(vp)]
    lib.fsi_mlp_create.restype = i32
    lib.fsi_mlp_destroy.argtypes = [vp]
    lib.fsi_mlp_destroy.restype = i32
    lib.fsi_mlp_num_params.argtypes = [vp]
    lib.fsi_mlp_num_params.restype = C.c_int64
    lib.fsi_mlp_params.argtypes = [vp, vp, i32]
    lib.fsi_mlp_params.restype = i32
    lib.fsi_mlp_forward.argtypes = [vp, vp, i32, vp, i32, vp]
    lib.fsi_mlp_forward.restype = i32
    lib.fsi_mlp_train_step.argtypes = [vp, vp, vp, i32, vp, C.c_float, i32, vp, vp, vp]
    lib.fsi_mlp_train_step.restype = i32
    lib.fsi_solid_newmark_advance.argtypes = [vp, vp, vp, vp, vp, vp, C.c_double, C.c_double, C.c_double, vp]
    lib.fsi_solid_newmark_advance.restype = i32
    lib.fsi_dn_default_opts.argtypes = [C.POINTER(DnOpts)]
    lib.fsi_dn_default_opts.restype = None
    lib.fsi_solid_dn_solve.argtypes = [vp, vp, C.POINTER(LoadDesc), C.POINTER(DnOpts), C.POINTER(DnInfo), vp]
    lib.fsi_solid_dn_solve.restype = i32
    return lib


lib = _load_library()


class FsiError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def default_opts(**kw) -> SolverOpts:
    o = SolverOpts()
    lib.fsi_solid_default_opts(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


@dataclasses.dataclass
class Load:
    """Load of one solve; tensors are CUDA FP64 (see fsi_load in the header)."""
    dir_values: Optional[object] = None
    pressure: float = 0.0
    node_pressure: Optional[object] = None
    face_pressure: Optional[object] = None
    hist: Optional[object] = None

    def desc(self) -> LoadDesc:
        def ptr(t):
            return None if t is None else _dev_ptr(t)
        return LoadDesc(ptr(self.dir_values), float(self.pressure), ptr(self.node_pressure),
                        ptr(self.face_pressure), ptr(self.hist))


def _dev_ptr(t):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError("expected a contiguous CUDA float64 tensor")
    return t.data_ptr()


def _stream():
    import torch
    return torch.cuda.current_stream().cuda_stream


class SolidSolver:
    """Owns one fsi_solid handle.  ``mesh`` needs the attributes X, tets,
    mat_id, fibre, dir_mask, neu_faces, materials (and optionally seg_node)."""

    def __init__(self, mesh, **opts):
        self.n_nodes = int(mesh.X.shape[0])
        self.n_elems = int(mesh.tets.shape[0])
        self._keep = []

        def arr(a, dt):
            a = np.ascontiguousarray(a, dtype=dt)
            self._keep.append(a)
            return a.ctypes.data

        d = MeshDesc()
        d.n_nodes = self.n_nodes
        d.n_elems = self.n_elems
        d.X = arr(mesh.X, np.float64)
        d.tets = arr(mesh.tets, np.int32)
        d.mat_id = arr(mesh.mat_id, np.int32)
        d.fibre = arr(mesh.fibre, np.float64) if getattr(mesh, "fibre", None) is not None else None
        d.dir_mask = arr(mesh.dir_mask, np.uint8)
        faces = np.asarray(mesh.neu_faces, dtype=np.int32).reshape(-1, 3)
        d.n_faces = int(faces.shape[0])
        d.neu_faces = arr(faces, np.int32) if len(faces) else None
        seg = getattr(mesh, "seg_node", None)
        d.n_segments = int(seg.max() + 1) if seg is not None else 1
        d.seg_node = arr(seg, np.int32) if seg is not None else None
        mats = (MaterialDesc * len(mesh.materials))()
        for i, m in enumerate(mesh.materials):
            mats[i] = MaterialDesc(int(m.model), m.c10, m.c01, m.k1, m.k2, m.kappa, m.rho)
        self.opts = default_opts(**opts)
        h = C.c_void_p()
        st = lib.fsi_solid_create(C.byref(d), len(mesh.materials), mats, C.byref(self.opts), C.byref(h))
        self._keep = []
        if st != FSI_OK:
            raise FsiError(st, lib.fsi_solid_last_error(None).decode())
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib.fsi_solid_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != FSI_OK:
            raise FsiError(st, lib.fsi_solid_last_error(self.h).decode())

    # ---------------------------------------------------------------- calls
    def residual_tangent(self, state, load: Optional[Load] = None, want_tangent=True, residual=None):
        import torch
        if residual is None:
            residual = torch.empty_like(state)
        ld = (load or Load()).desc()
        st = lib.fsi_solid_residual_tangent(self.h, _dev_ptr(state), C.byref(ld), _dev_ptr(residual),
                                            int(bool(want_tangent)), _stream())
        self._check(st)
        return residual

    def bsr(self):
        """Copies of the assembled matrix: (row_ptr, col_idx, vals [nb, 4, 4] float64)."""
        import torch
        rp, ci, vv = C.c_void_p(), C.c_void_p(), C.c_void_p()
        dt, nb = C.c_int32(), C.c_int32()
        self._check(lib.fsi_solid_get_bsr(self.h, C.byref(rp), C.byref(ci), C.byref(vv), C.byref(dt), C.byref(nb)))
        torch.cuda.synchronize()
        n = self.n_nodes
        row_ptr = np.empty(n + 1, np.int32)
        col_idx = np.empty(nb.value, np.int32)
        vals = np.empty((nb.value, 4, 4), np.float32 if dt.value == 1 else np.float64)
        cudart = _cudart()
        for host, dev in ((row_ptr, rp), (col_idx, ci), (vals, vv)):
            err = cudart.cudaMemcpy(host.ctypes.data, dev, host.nbytes, 2)   # 2: device to host
            if err != 0:
                raise FsiError(-2, f"cudaMemcpy of the assembled matrix failed with CUDA error {err}")
        return row_ptr, col_idx, vals

    def spmv(self, x, y=None):
        import torch
        y = torch.empty_like(x) if y is None else y
        self._check(lib.fsi_solid_spmv(self.h, _dev_ptr(x), _dev_ptr(y), _stream()))
        return y

    def linear_solve(self, b, x=None, check=True):
        import torch
        x = torch.zeros_like(b) if x is None else x
        info = Info()
        st = lib.fsi_solid_linear_solve(self.h, _dev_ptr(b), _dev_ptr(x), C.byref(info), _stream())
        if check:
            self._check(st)
        return x, info

    def newton_step(self, state, load: Optional[Load] = None, check=True):
        info = Info()
        ld = (load or Load()).desc()
        st = lib.fsi_solid_newton_step(self.h, _dev_ptr(state), C.byref(ld), C.byref(info), _stream())
        if check:
            self._check(st)
        return info

    def solve(self, state, load: Optional[Load] = None, guess=None, check=True):
        info = Info()
        ld = (load or Load()).desc()
        st = lib.fsi_solid_solve(self.h, _dev_ptr(state), C.byref(ld), None if guess is None else _dev_ptr(guess),
                                 C.byref(info), _stream())
        if check:
            self._check(st)
        return info

    def tuning(self):
        """Launch shapes chosen by the autotuner: [element CTA size, level-0 CTA
        size, shape of level 1, ...] (see fsi_solid_get_tuning)."""
        out = np.zeros(64, np.int32)
        n = C.c_int32()
        self._check(lib.fsi_solid_get_tuning(self.h, out.ctypes.data, 64, C.byref(n)))
        return out[:n.value].tolist()

    def colouring(self):
        out = np.empty(self.n_elems, np.int32)
        nc = C.c_int32()
        self._check(lib.fsi_solid_get_colouring(self.h, out.ctypes.data, C.byref(nc)))
        return out, nc.value

    def newmark_advance(self, state, disp, vel, acc, hist, beta, gamma, dt):
        """Newmark-beta update after a converged step (see the header)."""
        self._check(lib.fsi_solid_newmark_advance(self.h, _dev_ptr(state), _dev_ptr(disp), _dev_ptr(vel),
                                                  _dev_ptr(acc), _dev_ptr(hist), float(beta), float(gamma),
                                                  float(dt), _stream()))

    def dn_solve(self, state, p0, added_mass, d_ref=None, load: Optional[Load] = None, check=True, **kw):
        """Dirichlet-Neumann coupling loop with Aitken relaxation around the solid
        solve, with the surrogate added-mass fluid map (see the header).  kw:
        omega0, tol, max_cycles, aitken."""
        o = DnOpts()
        lib.fsi_dn_default_opts(C.byref(o))
        o.p0, o.added_mass = float(p0), float(added_mass)
        o.d_ref = None if d_ref is None else _dev_ptr(d_ref)
        for k, v in kw.items():
            if not hasattr(o, k):
                raise TypeError(f"unknown DN option {k}")
            setattr(o, k, v)
        info = DnInfo()
        ld = (load or Load()).desc()
        st = lib.fsi_solid_dn_solve(self.h, _dev_ptr(state), C.byref(ld), C.byref(o), C.byref(info), _stream())
        if check:
            self._check(st)
        return info

    def kernel_timing(self, enable: bool):
        """Per-class device time (ms) and launch counts since the last call;
        ``enable`` switches event recording on or off for later calls."""
        ms = np.zeros(len(KERNEL_CLASSES), np.float64)
        cnt = np.zeros(len(KERNEL_CLASSES), np.int64)
        self._check(lib.fsi_solid_kernel_timing(self.h, int(bool(enable)), ms.ctypes.data, cnt.ctypes.data))
        return {k: (float(ms[i]), int(cnt[i])) for i, k in enumerate(KERNEL_CLASSES)}

    def levels(self):
        cap = 32
        nodes = np.zeros(cap, np.int32)
        blocks = np.zeros(cap, np.int32)
        nl = C.c_int32()
        self._check(lib.fsi_solid_get_levels(self.h, nodes.ctypes.data, blocks.ctypes.data, cap, C.byref(nl)))
        return list(zip(nodes[:nl.value].tolist(), blocks[:nl.value].tolist()))


def _f32_ptr(t):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
        raise TypeError("expected a contiguous CUDA float32 tensor")
    return t.data_ptr()


class Mlp:
    """Per-node MLP of the learned initial guess (fsi_mlp_* in the header)."""

    def __init__(self, sizes, seed=0):
        self.sizes = [int(s) for s in sizes]
        arr = np.asarray(self.sizes, dtype=np.int32)
        h = C.c_void_p()
        st = lib.fsi_mlp_create(len(self.sizes) - 1, arr.ctypes.data, int(seed), C.byref(h))
        if st != FSI_OK:
            raise FsiError(st, "fsi_mlp_create failed")
        self.h = h
        self.n_params = int(lib.fsi_mlp_num_params(h))

    def close(self):
        if getattr(self, "h", None):
            lib.fsi_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_params(self):
        out = np.empty(self.n_params, np.float32)
        st = lib.fsi_mlp_params(self.h, out.ctypes.data, 0)
        if st != FSI_OK:
            raise FsiError(st, "fsi_mlp_params")
        return out

    def set_params(self, flat):
        arr = np.ascontiguousarray(flat, dtype=np.float32)
        st = lib.fsi_mlp_params(self.h, arr.ctypes.data, 1)
        if st != FSI_OK:
            raise FsiError(st, "fsi_mlp_params")

    def forward(self, X, bf16=False):
        import torch
        Y = torch.empty((X.shape[0], self.sizes[-1]), device=X.device, dtype=torch.float32)
        st = lib.fsi_mlp_forward(self.h, _f32_ptr(X), int(X.shape[0]), _f32_ptr(Y), int(bool(bf16)), _stream())
        if st != FSI_OK:
            raise FsiError(st, "fsi_mlp_forward")
        return Y

    def train_step(self, X, T, lr=1e-3, w_out=None, apply=True, want_grad=False):
        loss = C.c_float()
        grad = np.empty(self.n_params, np.float32) if want_grad else None
        st = lib.fsi_mlp_train_step(self.h, _f32_ptr(X), _f32_ptr(T), int(X.shape[0]),
                                    None if w_out is None else _f32_ptr(w_out), float(lr), int(bool(apply)),
                                    C.byref(loss), None if grad is None else grad.ctypes.data, _stream())
        if st != FSI_OK:
            raise FsiError(st, "fsi_mlp_train_step")
        return (loss.value, grad) if want_grad else loss.value


def launch_count() -> int:
    return int(lib.fsi_solid_launch_count())


_CUDART = None


def _cudart():
    global _CUDART
    if _CUDART is None:
        for name in ("libcudart.so.13", "libcudart.so", "/usr/local/cuda/lib64/libcudart.so.13"):
            try:
                _CUDART = C.CDLL(name)
                break
            except OSError:
                continue
        if _CUDART is None:
            raise ImportError("libcudart not found")
        _CUDART.cudaMemcpy.argtypes = [C.c_void_p, C.c_void_p, C.c_size_t, C.c_int]
        _CUDART.cudaMemcpy.restype = C.c_int
    return _CUDART
