"""Thin ctypes binding over libsylv.so (include/sylv.h).

Argument marshalling only: every step of the solve runs in the library's
sm_103a kernels.  PyTorch provides device memory and streams.  Tensors are
flat contiguous buffers whose element order is column-major
(n_1 x ... x n_N x nrhs, i_1 fastest); use `to_device` / `from_device` to move
numpy arrays in Fortran order.  If the shared library is missing, every call
raises: there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
from typing import List, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsylv.so")

SYLV_FP64 = 0
SYLV_MIXED_FP32 = 1
SYLV_MIXED_FP32_EMU = 2
PRECISIONS = {"fp64": SYLV_FP64, "mixed": SYLV_MIXED_FP32, "mixed_fp32": SYLV_MIXED_FP32,
              "mixed_emu": SYLV_MIXED_FP32_EMU}

PHASES = ("forward", "sweep", "back", "residual", "update", "total", "evolve")

STATUS = {0: "SYLV_OK", 1: "SYLV_ERR_INVALID_ARG", 2: "SYLV_ERR_SHAPE", 3: "SYLV_ERR_SINGULAR",
          4: "SYLV_ERR_NOT_CONVERGED", 5: "SYLV_ERR_TIMEOUT", 6: "SYLV_ERR_OOM",
          7: "SYLV_ERR_CUDA", 8: "SYLV_ERR_SCHUR", 9: "SYLV_ERR_WORKSPACE"}

EXPORTED = ("sylv_plan_create", "sylv_plan_destroy", "sylv_workspace_size", "sylv_solve",
            "sylv_workspace_size_batched", "sylv_solve_batched", "sylv_forward", "sylv_sweep",
            "sylv_back", "sylv_residual", "sylv_plan_factors", "sylv_plan_set_timing",
            "sylv_plan_timing", "sylv_schur", "sylv_status_string", "sylv_version",
            "sylv_sweep_static", "sylv_plan_autotune", "sylv_evolve_workspace_size",
            "sylv_evolve", "sylv_expm", "sylv_schur_real", "sylv_plan_create_real",
            "sylv_plan_describe")


class SylvError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = _lib().sylv_status_string(status).decode() if _LIB is not None else ""
        super().__init__(f"{where}: {STATUS.get(status, status)} ({msg})")


class Info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("refine_iters", ctypes.c_int32),
                ("launches", ctypes.c_int32), ("path", ctypes.c_int32),
                ("last_corr_rel", ctypes.c_double), ("est_rel_err", ctypes.c_double),
                ("min_abs_den", ctypes.c_double), ("max_abs_den", ctypes.c_double)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["diagonal_sweep"] = bool(self.path & 1)
        d["tensor_core_residual"] = bool(self.path & 2)
        d["real"] = bool(self.path & 4)
        return d


class Timing(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * 8), ("launches", ctypes.c_int64 * 8),
                ("solves", ctypes.c_int64)]


class Desc(ctypes.Structure):
    _fields_ = [("transform_passes", ctypes.c_int32), ("transform_tc_passes", ctypes.c_int32),
                ("residual_passes", ctypes.c_int32), ("residual_tc", ctypes.c_int32),
                ("diag_sweep", ctypes.c_int32), ("sweep_threads", ctypes.c_int32),
                ("sweep_ctas_per_sm", ctypes.c_int32), ("sweep_grid", ctypes.c_int32),
                ("sweep_tiles", ctypes.c_int64), ("sweep_tile_entries", ctypes.c_int32),
                ("sweep_tile_levels", ctypes.c_int32), ("sweep_inv_table", ctypes.c_int32),
                ("sweep_far_split", ctypes.c_int32), ("sweep_block", ctypes.c_int32 * 64),
                ("sweep_lanes", ctypes.c_int32), ("transform_tma", ctypes.c_int32),
                ("transform_group_max", ctypes.c_int32), ("sweep_3m", ctypes.c_int32),
                ("transform_fib_passes", ctypes.c_int32)]


class Tuning(ctypes.Structure):
    _fields_ = [("block", ctypes.c_int32 * 64), ("group_max", ctypes.c_int32),
                ("sweep_threads", ctypes.c_int32), ("no_tensor_cores", ctypes.c_int32),
                ("timeout_ms", ctypes.c_int32), ("fault_tile", ctypes.c_int32),
                ("general_sweep", ctypes.c_int32), ("sweep_ctas_per_sm", ctypes.c_int32),
                ("tc_plain", ctypes.c_int32)]


_LIB = None
vp = ctypes.c_void_p


def _lib():
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libsylv.so not built ({LIB_PATH}); run "
                               "`python -m paper_2412_15840_gb300.build` first")
        L = ctypes.CDLL(LIB_PATH)
        st = ctypes.c_int
        L.sylv_plan_create.restype = st
        L.sylv_plan_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int,
                                       ctypes.POINTER(ctypes.c_int64), ctypes.c_int64,
                                       ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp),
                                       ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                       ctypes.POINTER(Tuning)]
        L.sylv_plan_create_real.restype = st
        L.sylv_plan_create_real.argtypes = [ctypes.POINTER(vp), ctypes.c_int,
                                            ctypes.POINTER(ctypes.c_int64), ctypes.c_int64,
                                            ctypes.POINTER(vp), ctypes.c_int, ctypes.c_double,
                                            ctypes.c_int, ctypes.c_int, ctypes.POINTER(Tuning)]
        L.sylv_plan_destroy.restype = st
        L.sylv_plan_destroy.argtypes = [vp]
        L.sylv_workspace_size.restype = st
        L.sylv_workspace_size.argtypes = [vp, ctypes.POINTER(ctypes.c_size_t)]
        L.sylv_solve.restype = st
        L.sylv_solve.argtypes = [vp, vp, vp, vp, ctypes.c_size_t, vp, ctypes.POINTER(Info)]
        L.sylv_workspace_size_batched.restype = st
        L.sylv_workspace_size_batched.argtypes = [ctypes.c_int, ctypes.POINTER(vp),
                                                  ctypes.POINTER(ctypes.c_size_t)]
        L.sylv_solve_batched.restype = st
        L.sylv_solve_batched.argtypes = [ctypes.c_int, ctypes.POINTER(vp), ctypes.POINTER(vp),
                                         ctypes.POINTER(vp), vp, ctypes.c_size_t, vp,
                                         ctypes.POINTER(Info)]
        for f in ("sylv_forward", "sylv_sweep", "sylv_back"):
            getattr(L, f).restype = st
            getattr(L, f).argtypes = [vp, vp, vp, ctypes.c_size_t, vp]
        L.sylv_plan_autotune.restype = st
        L.sylv_plan_autotune.argtypes = [vp, vp, vp, ctypes.c_size_t, vp,
                                         ctypes.POINTER(ctypes.c_int32),
                                         ctypes.POINTER(ctypes.c_float)]
        L.sylv_sweep_static.restype = st
        L.sylv_sweep_static.argtypes = [vp, vp, vp]
        L.sylv_residual.restype = st
        L.sylv_residual.argtypes = [vp, vp, vp, vp, vp]
        L.sylv_plan_factors.restype = st
        L.sylv_plan_factors.argtypes = [vp, ctypes.c_int, vp, vp]
        L.sylv_plan_describe.restype = st
        L.sylv_plan_describe.argtypes = [vp, ctypes.POINTER(Desc)]
        L.sylv_plan_set_timing.restype = st
        L.sylv_plan_set_timing.argtypes = [vp, ctypes.c_int]
        L.sylv_plan_timing.restype = st
        L.sylv_plan_timing.argtypes = [vp, ctypes.POINTER(Timing), ctypes.c_int]
        L.sylv_schur.restype = st
        L.sylv_schur.argtypes = [ctypes.c_int64, vp, vp, vp]
        L.sylv_schur_real.restype = st
        L.sylv_schur_real.argtypes = [ctypes.c_int64, vp, vp, vp]
        L.sylv_expm.restype = st
        L.sylv_expm.argtypes = [ctypes.c_int64, vp, vp]
        L.sylv_evolve_workspace_size.restype = st
        L.sylv_evolve_workspace_size.argtypes = [vp, ctypes.POINTER(ctypes.c_size_t)]
        L.sylv_evolve.restype = st
        L.sylv_evolve.argtypes = [vp, ctypes.c_double, vp, vp, vp, vp, ctypes.c_size_t, vp,
                                  ctypes.POINTER(Info)]
        L.sylv_status_string.restype = ctypes.c_char_p
        L.sylv_status_string.argtypes = [ctypes.c_int]
        L.sylv_version.restype = ctypes.c_int
        L.sylv_version.argtypes = []
        _LIB = L
    return _LIB


def lib():
    return _lib()


def _check(status: int, where: str):
    if status != 0:
        raise SylvError(status, where)


def _cmat(M) -> np.ndarray:
    """complex matrix -> column-major interleaved complex128 host buffer."""
    a = np.asarray(M, dtype=np.complex128)
    if a.ndim == 0:
        a = a.reshape(1, 1)
    return np.asfortranarray(a)


def schur(A) -> tuple:
    """Host complex Schur A = Q T Q^* computed by the library (no GPU needed)."""
    a = _cmat(A)
    n = a.shape[0]
    Q = np.zeros((n, n), dtype=np.complex128, order="F")
    T = np.zeros((n, n), dtype=np.complex128, order="F")
    _check(_lib().sylv_schur(n, a.ctypes.data, Q.ctypes.data, T.ctypes.data), "sylv_schur")
    return Q, T


def schur_real(A) -> tuple:
    """Host real Schur A = Q T Q^T computed by the library (no GPU needed): T
    quasi-upper-triangular, its 2 x 2 blocks at even offsets."""
    a = np.asfortranarray(np.asarray(A, dtype=np.float64).reshape(np.shape(A) or (1, 1)))
    n = a.shape[0]
    Q = np.zeros((n, n), dtype=np.float64, order="F")
    T = np.zeros((n, n), dtype=np.float64, order="F")
    _check(_lib().sylv_schur_real(n, a.ctypes.data, Q.ctypes.data, T.ctypes.data),
           "sylv_schur_real")
    return Q, T


def expm(M) -> np.ndarray:
    """Host matrix exponential computed by the library (no GPU needed)."""
    m = _cmat(M)
    n = m.shape[0]
    E = np.zeros((n, n), dtype=np.complex128, order="F")
    _check(_lib().sylv_expm(n, m.ctypes.data, E.ctypes.data), "sylv_expm")
    return E


def _stream_handle(stream) -> Optional[int]:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _ptr(t) -> int:
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return t.data_ptr()


def check_tensor(t, dtype, numel: int, device: int, what: str):
    """Refuse a tensor the library would misuse: it reads and writes `numel`
    elements of `dtype` on the plan's device, so a tensor of another type or
    size would be overrun, and one on another GPU would be dereferenced from
    the plan's device (an illegal address without peer access)."""
    if t.dtype != dtype or t.numel() != numel or not t.is_cuda:
        raise ValueError(f"{what} must be a CUDA {dtype} tensor with prod(shape)*nrhs "
                         f"= {numel} elements")
    if t.device.index is not None and t.device.index != device:
        raise ValueError(f"{what} is on cuda:{t.device.index}, the plan on cuda:{device}")


def check_workspace(ws, device: int, what: str = "workspace"):
    """A workspace is device memory of the plan's GPU (any dtype, contiguous)."""
    if not ws.is_cuda:
        raise ValueError(f"{what} must be a CUDA tensor on cuda:{device}")
    if ws.device.index is not None and ws.device.index != device:
        raise ValueError(f"{what} is on cuda:{ws.device.index}, the plan on cuda:{device}")
    if not ws.is_contiguous():
        raise ValueError(f"{what} must be contiguous")


def to_device(x: np.ndarray, device="cuda", dtype=None):
    """numpy array (logical shape, any order) -> flat device tensor in column-major order."""
    import torch
    flat = np.asarray(x).reshape(-1, order="F")
    t = torch.from_numpy(np.ascontiguousarray(flat))
    if dtype is not None:
        t = t.to(dtype)
    return t.to(device)


def from_device(t, shape) -> np.ndarray:
    """flat device tensor in column-major order -> numpy array of logical `shape`."""
    return t.detach().cpu().numpy().reshape(tuple(shape), order="F")


class Plan:
    """One equation shape, its Schur factors and launch tables (sylv_plan_create).

    real=True: the real-arithmetic variant (sylv_plan_create_real) for real A
    (float64 matrices); B and X are then float64 device tensors."""

    def __init__(self, A: Optional[Sequence] = None, Q: Optional[Sequence] = None,
                 T: Optional[Sequence] = None, nrhs: int = 1, prec: str = "fp64",
                 rtol: float = 1e-10, max_refine: int = 5, device: int = 0,
                 block: Optional[Sequence[int]] = None, group_max: int = 0,
                 sweep_threads: int = 0, tensor_cores: bool = True, timeout_ms: int = 0,
                 fault_tile: int = 0, general_sweep: bool = False, sweep_ctas_per_sm: int = 0,
                 real: bool = False, tc_pipeline: bool = True):
        L = _lib()
        self.real = bool(real)
        if self.real and (A is None or Q is not None or T is not None):
            raise ValueError("a real plan takes A only")
        if (A is None) == (Q is None or T is None) and not self.real:
            raise ValueError("give A, or both Q and T")
        if self.real and any(np.iscomplexobj(a) and np.any(np.imag(a) != 0) for a in A):
            raise ValueError("a real plan takes real A_j (an operator has imaginary parts)")
        mats = [np.atleast_2d(np.asarray(np.real(a), dtype=np.float64)) if self.real else _cmat(a)
                for a in (A if A is not None else T)]
        self.shape = tuple(int(m.shape[0]) for m in mats)
        self.N = len(self.shape)
        self.nrhs = int(nrhs)
        self.prec = PRECISIONS[prec] if isinstance(prec, str) else int(prec)
        self.device = device
        n = (ctypes.c_int64 * self.N)(*self.shape)
        keep = []

        def ptrs(seq):
            arr = [np.asfortranarray(m) for m in mats] if self.real else [_cmat(m) for m in seq]
            keep.extend(arr)
            return (vp * self.N)(*[a.ctypes.data for a in arr])

        pA = ptrs(A) if A is not None else None
        pQ = ptrs(Q) if Q is not None else None
        pT = ptrs(T) if T is not None else None
        tun = None
        if block is not None or group_max or sweep_threads or not tensor_cores or timeout_ms \
                or fault_tile or general_sweep or sweep_ctas_per_sm or not tc_pipeline:
            tun = Tuning()
            if block is not None:
                for j, b in enumerate(block):
                    tun.block[j] = int(b)
            tun.group_max = int(group_max)
            tun.sweep_threads = int(sweep_threads)
            tun.no_tensor_cores = 0 if tensor_cores else 1
            tun.timeout_ms = int(timeout_ms)
            tun.fault_tile = int(fault_tile)
            tun.general_sweep = int(bool(general_sweep))
            tun.sweep_ctas_per_sm = int(sweep_ctas_per_sm)
            tun.tc_plain = 0 if tc_pipeline else 1
        h = vp()
        tp = ctypes.byref(tun) if tun is not None else None
        if self.real:
            s = L.sylv_plan_create_real(ctypes.byref(h), self.N, n, self.nrhs, pA, self.prec,
                                        float(rtol), int(max_refine), int(device), tp)
            _check(s, "sylv_plan_create_real")
        else:
            s = L.sylv_plan_create(ctypes.byref(h), self.N, n, self.nrhs, pA, pQ, pT, self.prec,
                                   float(rtol), int(max_refine), int(device), tp)
            _check(s, "sylv_plan_create")
        self._h = h
        sz = ctypes.c_size_t()
        _check(L.sylv_workspace_size(h, ctypes.byref(sz)), "sylv_workspace_size")
        self.workspace_bytes = int(sz.value)
        self._ws = None

    # ------------------------------------------------------------------
    @property
    def handle(self):
        return self._h

    @property
    def numel(self) -> int:
        return int(np.prod(self.shape, dtype=np.int64)) * self.nrhs

    def workspace(self):
        import torch
        if self._ws is None:
            self._ws = torch.empty(max(self.workspace_bytes, 256), dtype=torch.uint8,
                                   device=f"cuda:{self.device}")
        return self._ws

    def _wsargs(self, workspace):
        ws = self.workspace() if workspace is None else workspace
        check_workspace(ws, self.device, "workspace")
        return ws.data_ptr(), ws.numel() * ws.element_size()

    @property
    def dtype(self):
        """dtype of B and X: complex128, or float64 for a real plan."""
        import torch
        return torch.float64 if self.real else torch.complex128

    @property
    def work_dtype(self):
        """dtype of the working-precision tensors of sylv_forward / sweep / back."""
        import torch
        if self.prec == SYLV_FP64:
            return torch.float64 if self.real else torch.complex128
        return torch.float32 if self.real else torch.complex64

    def solve(self, B, X=None, workspace=None, stream=None, info: bool = False):
        """X with sum_j A_j (x)_j X = B; B, X flat complex128 (float64 for a real
        plan) device tensors."""
        import torch
        self._check_tensor(B, self.dtype, "B")
        if X is None:
            X = torch.empty_like(B)
        self._check_tensor(X, self.dtype, "X")
        wp, wb = self._wsargs(workspace)
        inf = Info() if info else None
        s = _lib().sylv_solve(self._h, _ptr(B), _ptr(X), wp, wb, _stream_handle(stream),
                              ctypes.byref(inf) if inf is not None else None)
        if info:
            if s not in (0, 4):
                _check(s, "sylv_solve")
            return X, inf.as_dict()
        _check(s, "sylv_solve")
        return X

    def evolve_workspace_bytes(self) -> int:
        sz = ctypes.c_size_t()
        _check(_lib().sylv_evolve_workspace_size(self._h, ctypes.byref(sz)),
               "sylv_evolve_workspace_size")
        return int(sz.value)

    def evolve(self, t: float, B, X0, X=None, workspace=None, stream=None, info: bool = False):
        """X(t) of X_t = sum_j A_j (x)_j X + B, X(0) = X0 (Theorem 1); flat complex128
        device tensors.  `workspace` holds at least evolve_workspace_bytes()."""
        import torch
        for v, what in ((B, "B"), (X0, "X0")):
            self._check_tensor(v, torch.complex128, what)
        if X is None:
            X = torch.empty_like(B)
        self._check_tensor(X, torch.complex128, "X")
        if workspace is None:
            workspace = torch.empty(self.evolve_workspace_bytes(), dtype=torch.uint8,
                                    device=f"cuda:{self.device}")
        check_workspace(workspace, self.device, "workspace")
        inf = Info() if info else None
        s = _lib().sylv_evolve(self._h, float(t), _ptr(B), _ptr(X0), _ptr(X),
                               workspace.data_ptr(), workspace.numel(), _stream_handle(stream),
                               ctypes.byref(inf) if inf is not None else None)
        if info:
            if s not in (0, 4):
                _check(s, "sylv_evolve")
            return X, inf.as_dict()
        _check(s, "sylv_evolve")
        return X

    def _check_tensor(self, t, dtype, what):
        check_tensor(t, dtype, self.numel, self.device, what)

    def forward(self, Tns, workspace=None, stream=None):
        self._check_tensor(Tns, self.work_dtype, "the tensor")
        wp, wb = self._wsargs(workspace)
        _check(_lib().sylv_forward(self._h, _ptr(Tns), wp, wb, _stream_handle(stream)),
               "sylv_forward")
        return Tns

    def sweep(self, Tns, workspace=None, stream=None):
        self._check_tensor(Tns, self.work_dtype, "the tensor")
        wp, wb = self._wsargs(workspace)
        _check(_lib().sylv_sweep(self._h, _ptr(Tns), wp, wb, _stream_handle(stream)),
               "sylv_sweep")
        return Tns

    def sweep_static(self, Tns, stream=None):
        """sylv_sweep_static: the sweep with the library's fixed scratch array
        (no workspace, no allocation); see include/sylv.h for its limits."""
        self._check_tensor(Tns, self.work_dtype, "the tensor")
        _check(_lib().sylv_sweep_static(self._h, _ptr(Tns), _stream_handle(stream)),
               "sylv_sweep_static")
        return Tns

    def back(self, Tns, workspace=None, stream=None):
        self._check_tensor(Tns, self.work_dtype, "the tensor")
        wp, wb = self._wsargs(workspace)
        _check(_lib().sylv_back(self._h, _ptr(Tns), wp, wb, _stream_handle(stream)),
               "sylv_back")
        return Tns

    def residual(self, B, X, R=None, stream=None):
        import torch
        if R is None:
            R = torch.empty_like(B)
        for t, what in ((B, "B"), (X, "X"), (R, "R")):
            self._check_tensor(t, self.dtype, what)
        _check(_lib().sylv_residual(self._h, _ptr(B), _ptr(X), _ptr(R), _stream_handle(stream)),
               "sylv_residual")
        return R

    def autotune(self, scratch=None, workspace=None, stream=None):
        """sylv_plan_autotune: time candidate sweep tilings, keep the fastest.
        Returns (block extents per input mode, best sweep time in ms)."""
        import torch
        if scratch is None:
            scratch = torch.empty(self.numel, dtype=self.work_dtype,
                                  device=f"cuda:{self.device}")
        self._check_tensor(scratch, self.work_dtype, "the scratch tensor")
        wp, wb = self._wsargs(workspace)
        blk = (ctypes.c_int32 * self.N)()
        ms = ctypes.c_float()
        _check(_lib().sylv_plan_autotune(self._h, _ptr(scratch), wp, wb, _stream_handle(stream),
                                         blk, ctypes.byref(ms)), "sylv_plan_autotune")
        return tuple(int(b) for b in blk), float(ms.value)

    def factors(self, j: int):
        n = self.shape[j]
        Q = np.zeros((n, n), dtype=np.complex128, order="F")
        T = np.zeros((n, n), dtype=np.complex128, order="F")
        _check(_lib().sylv_plan_factors(self._h, j, Q.ctypes.data, T.ctypes.data),
               "sylv_plan_factors")
        return Q, T

    def describe(self) -> dict:
        """sylv_plan_describe: passes, tiles and launch shapes the plan chose."""
        d = Desc()
        _check(_lib().sylv_plan_describe(self._h, ctypes.byref(d)), "sylv_plan_describe")
        out = {k: getattr(d, k) for k, _ in Desc._fields_ if k != "sweep_block"}
        out["sweep_block"] = tuple(int(d.sweep_block[j]) for j in range(self.N))
        return out

    def set_timing(self, enable: bool = True):
        _check(_lib().sylv_plan_set_timing(self._h, int(bool(enable))), "sylv_plan_set_timing")

    def timing(self, reset: bool = True) -> dict:
        t = Timing()
        _check(_lib().sylv_plan_timing(self._h, ctypes.byref(t), int(reset)), "sylv_plan_timing")
        return {"ms": {PHASES[i]: t.ms[i] for i in range(len(PHASES))},
                "launches": {PHASES[i]: int(t.launches[i]) for i in range(len(PHASES))},
                "solves": int(t.solves)}

    def close(self):
        if getattr(self, "_h", None):
            _lib().sylv_plan_destroy(self._h)
            self._h = None
            self._ws = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def workspace_size_batched(plans: Sequence[Plan]) -> int:
    hs = (vp * len(plans))(*[p.handle for p in plans])
    sz = ctypes.c_size_t()
    _check(_lib().sylv_workspace_size_batched(len(plans), hs, ctypes.byref(sz)),
           "sylv_workspace_size_batched")
    return int(sz.value)


def solve_batched(plans: Sequence[Plan], Bs: Sequence, Xs: Sequence, workspace, stream=None,
                  info: bool = False):
    """sylv_solve_batched over independent equations (any shapes)."""
    m = len(plans)
    if len(Bs) != m or len(Xs) != m:
        raise ValueError("plans, Bs and Xs must have the same length")
    for p, b, x in zip(plans, Bs, Xs):
        p._check_tensor(b, p.dtype, "B")
        p._check_tensor(x, p.dtype, "X")
    if m:
        check_workspace(workspace, plans[0].device, "workspace")
    hs = (vp * m)(*[p.handle for p in plans])
    pb = (vp * m)(*[_ptr(b) for b in Bs])
    px = (vp * m)(*[_ptr(x) for x in Xs])
    infos = (Info * m)() if info else None
    s = _lib().sylv_solve_batched(m, hs, pb, px, workspace.data_ptr(),
                                  workspace.numel() * workspace.element_size(),
                                  _stream_handle(stream), infos)
    if info:
        if s not in (0, 4):
            _check(s, "sylv_solve_batched")
        return [i.as_dict() for i in infos]
    _check(s, "sylv_solve_batched")
    return None
