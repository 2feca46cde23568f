"""GB300 (sm_103a) two-site DMRG effective-Hamiltonian library: Python binding.

This module only marshals arguments to the C ABI of libdmrg_gb300.so (declared
in include/dmrg_heff.h); every step of H_eff*psi and of the Davidson solver runs
in the library's CUDA kernels.  Importing it fails if the library has not been
built (``python paper_2407_07411_gb300/build.py``): there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdmrg_gb300.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with `python paper_2407_07411_gb300/build.py`")

_lib = ctypes.CDLL(LIB_PATH)

PREC_FP64 = 0
PREC_SPLIT_BF16 = 1
FLAG_PLAN_ONLY = 1
FLAG_NO_GRAPH = 2
_PREC = {"fp64": PREC_FP64, "split_bf16": PREC_SPLIT_BF16, "split": PREC_SPLIT_BF16}

#: Every symbol the C ABI exports (include/dmrg_heff.h).
SYMBOLS = ("dmrg_heff_create", "dmrg_heff_dim", "dmrg_heff_flops", "dmrg_heff_plan_dump",
           "dmrg_heff_apply", "dmrg_heff_apply_host", "dmrg_heff_diagonal", "dmrg_davidson",
           "dmrg_heff_destroy", "dmrg_strerror", "dmrg_last_error", "dmrg_heff_profile",
           "dmrg_heff_profile_read", "dmrg_probe_fp64_peak", "dmrg_heff_apply_noalloc",
           "dmrg_selftest_wait_timeout", "dmrg_heff_schedule_get", "dmrg_heff_schedule_set",
           "dmrg_heff_autotune", "dmrg_heff_gemm_count", "dmrg_lanczos", "dmrg_renormalise",
           "dmrg_heff_psi_blocks", "dmrg_svd_truncate", "dmrg_heff_create_su2", "dmrg_su2_recoupling",
           "dmrg_heff_memory", "dmrg_renorm_create", "dmrg_renorm_run", "dmrg_renorm_destroy")


class Opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("n_slices", ctypes.c_int32),
                ("max_nvec", ctypes.c_int32), ("flags", ctypes.c_int32), ("split_mid_bytes", ctypes.c_int64)]


class Memory(ctypes.Structure):
    _fields_ = [("operators", ctypes.c_int64), ("operator_slices", ctypes.c_int64),
                ("apply_buffers", ctypes.c_int64), ("setup_peak", ctypes.c_int64), ("total", ctypes.c_int64)]


class DavidsonInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("matvecs", ctypes.c_int32),
                ("converged", ctypes.c_int32), ("restarts", ctypes.c_int32),
                ("resid_max", ctypes.c_double), ("seconds", ctypes.c_double),
                ("hist_theta", ctypes.c_void_p), ("hist_time", ctypes.c_void_p),
                ("hist_cap", ctypes.c_int32), ("pad", ctypes.c_int32)]


class KernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 48), ("launches", ctypes.c_int64), ("ms_total", ctypes.c_double),
                ("flops_total", ctypes.c_double), ("bytes_total", ctypes.c_double)]


class Schedule(ctypes.Structure):
    _fields_ = [("fp64_kchunk", ctypes.c_int32 * 3), ("fp64_ctas_per_sm", ctypes.c_int32),
                ("split_kchunk", ctypes.c_int32 * 3), ("per_gemm", ctypes.c_int32), ("fp64_tile", ctypes.c_int32)]

    def to_dict(self) -> dict:
        return dict(fp64_kchunk=list(self.fp64_kchunk), fp64_ctas_per_sm=self.fp64_ctas_per_sm,
                    split_kchunk=list(self.split_kchunk), per_gemm=self.per_gemm, fp64_tile=self.fp64_tile)

    @classmethod
    def from_dict(cls, d: dict) -> "Schedule":
        s = cls()
        for i, v in enumerate(d["fp64_kchunk"]):
            s.fp64_kchunk[i] = int(v)
        for i, v in enumerate(d["split_kchunk"]):
            s.split_kchunk[i] = int(v)
        s.fp64_ctas_per_sm = int(d["fp64_ctas_per_sm"])
        s.per_gemm = int(d["per_gemm"])
        s.fp64_tile = int(d.get("fp64_tile", 0))
        return s


class TuneReport(ctypes.Structure):
    _fields_ = [("trials", ctypes.c_int32), ("nvec", ctypes.c_int32), ("default_ms", ctypes.c_double),
                ("best_ms", ctypes.c_double), ("best", Schedule), ("tile_m", ctypes.c_int32),
                ("tile_n", ctypes.c_int32)]


_P = ctypes.c_void_p
_i32, _i64, _f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
_lib.dmrg_heff_create.argtypes = [_P, _i32, _P, _i32, _i32, _i32, _P, _P, _P, _P, _P, _i64, _P, _i64,
                                  ctypes.POINTER(Opts), ctypes.POINTER(_P)]
_lib.dmrg_heff_create.restype = ctypes.c_int
_lib.dmrg_heff_create_su2.argtypes = [_P, _i32, _P, _i32, _i32, _i32, _P, _P, _P, _P, _i64, _P, _i64, _P, _i64,
                                      _P, _i64, ctypes.POINTER(Opts), ctypes.POINTER(ctypes.c_void_p)]
_lib.dmrg_heff_create_su2.restype = ctypes.c_int
_lib.dmrg_su2_recoupling.argtypes = [_i32, _i32, _i32, _i32, _i32, _i32, ctypes.POINTER(_f64)]
_lib.dmrg_heff_dim.argtypes = [_P]
_lib.dmrg_heff_dim.restype = _i64
_lib.dmrg_heff_flops.argtypes = [_P, ctypes.POINTER(_i64)]
_lib.dmrg_heff_memory.argtypes = [_P, ctypes.POINTER(Memory)]
_lib.dmrg_heff_plan_dump.argtypes = [_P, _P, ctypes.POINTER(_i64)]
_lib.dmrg_heff_apply.argtypes = [_P, _P, _P, _i32, _P]
_lib.dmrg_heff_apply_host.argtypes = [_P, _P, _P, _i32]
_lib.dmrg_heff_diagonal.argtypes = [_P, _P, _P]
_lib.dmrg_davidson.argtypes = [_P, _i32, _f64, _i32, _i32, _i32, _P, _P, ctypes.POINTER(DavidsonInfo)]
_lib.dmrg_heff_schedule_get.argtypes = [_P, ctypes.POINTER(Schedule)]
_lib.dmrg_heff_schedule_set.argtypes = [_P, ctypes.POINTER(Schedule)]
_lib.dmrg_heff_autotune.argtypes = [_P, _i32, _i32, ctypes.POINTER(TuneReport)]
_lib.dmrg_heff_gemm_count.argtypes = [_P, _i32, _P]
_lib.dmrg_lanczos.argtypes = [_P, _f64, _i32, _i32, _P, _P, ctypes.POINTER(DavidsonInfo)]
_lib.dmrg_renormalise.argtypes = [_i32, _P, _P, _P, _P, _i64, _P, _i64, _P, _i64, _P, _P]
_lib.dmrg_renorm_create.argtypes = [_i32, _P, _P, _P, _i64, _i64, _i64, _P, ctypes.POINTER(_P)]
_lib.dmrg_renorm_run.argtypes = [_P, _P, _P, _P, _P]
_lib.dmrg_renorm_destroy.argtypes = [_P]
_lib.dmrg_heff_psi_blocks.argtypes = [_P, _P, ctypes.POINTER(_i64)]
_lib.dmrg_svd_truncate.argtypes = [_P, _P, _i32, _P, _P, _P, _i64, _P, ctypes.POINTER(_f64)]
_lib.dmrg_heff_destroy.argtypes = [_P]
_lib.dmrg_heff_destroy.restype = None
_lib.dmrg_strerror.argtypes = [ctypes.c_int]
_lib.dmrg_strerror.restype = ctypes.c_char_p
_lib.dmrg_last_error.argtypes = []
_lib.dmrg_last_error.restype = ctypes.c_char_p

_lib.dmrg_heff_profile.argtypes = [_P, _i32]
_lib.dmrg_heff_profile_read.argtypes = [_P, ctypes.POINTER(KernelStat), ctypes.POINTER(_i32)]
_lib.dmrg_probe_fp64_peak.argtypes = [ctypes.POINTER(_f64)]
_lib.dmrg_selftest_wait_timeout.argtypes = [_i64]
_lib.dmrg_heff_apply_noalloc.argtypes = [_P, _i32, _P, _i32, _i32, _i32, _P, _P, _P, _P, _P, _i64, _P, _i64,
                                         _P, _P, _P]
_lib.dmrg_heff_apply_noalloc.restype = ctypes.c_int

ERR_INVALID_ARG, ERR_NOT_CONVERGED = -1, -6


class DmrgError(RuntimeError):
    def __init__(self, code: int):
        self.code = code
        msg = _lib.dmrg_strerror(code).decode()
        detail = _lib.dmrg_last_error().decode()
        super().__init__(f"{msg} ({code}): {detail}")


def _check(rc: int) -> int:
    if rc != 0:
        raise DmrgError(rc)
    return rc


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p) if a.size else None


def _dev_ptr(t, n: int, what: str):
    """Device pointer of a contiguous CUDA float64 tensor with >= n elements."""
    if isinstance(t, int):
        return ctypes.c_void_p(t)
    if not (t.is_cuda and t.dtype.is_floating_point and t.element_size() == 8 and t.is_contiguous()):
        raise ValueError(f"{what} must be a contiguous CUDA float64 tensor")
    if t.numel() < n:
        raise ValueError(f"{what} holds {t.numel()} values, {n} needed")
    return ctypes.c_void_p(t.data_ptr())


def _stream_ptr(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


class HEff:
    """Handle of one effective Hamiltonian on the current CUDA device."""

    def __init__(self, left, right, target, coef, delta, parity, a_off, b_off, op_data,
                 precision: str = "fp64", max_nvec: int = 1, n_slices: int = 0, plan_only: bool = False,
                 graphs: bool = True, split_mid_bytes: int = 0):
        self._h = None
        arr = lambda a, dt: np.ascontiguousarray(np.asarray(a, dtype=dt))
        self._left = arr(left, np.int32).reshape(-1, 3)
        self._right = arr(right, np.int32).reshape(-1, 3)
        coef, delta = arr(coef, np.float64), arr(delta, np.int32).reshape(-1, 2)
        parity = arr(parity, np.int32)
        T = coef.shape[0]
        a_off = arr(a_off, np.int64).reshape(T, len(self._left))
        b_off = arr(b_off, np.int64).reshape(T, len(self._right))
        op_data = arr(op_data, np.float64)
        opts = Opts(_PREC[precision] if isinstance(precision, str) else int(precision), n_slices, max_nvec,
                    (FLAG_PLAN_ONLY if plan_only else 0) | (0 if graphs else FLAG_NO_GRAPH), int(split_mid_bytes))
        h = ctypes.c_void_p()
        _check(_lib.dmrg_heff_create(_ptr(self._left), len(self._left), _ptr(self._right), len(self._right),
                                     int(target[0]), int(target[1]), _ptr(coef), _ptr(delta), _ptr(parity),
                                     _ptr(a_off), _ptr(b_off), T, _ptr(op_data), op_data.size,
                                     ctypes.byref(opts), ctypes.byref(h)))
        self._h = h
        self.max_nvec = max_nvec
        self.precision = precision

    @classmethod
    def from_problem(cls, p, **kw) -> "HEff":
        """Build from any object with the fields of a two-site problem
        (left, right, target, coef, delta, parity, a_off, b_off, op_data), or of a
        spin-adapted one (see from_su2)."""
        if hasattr(p, "rank2"):
            return cls.from_su2(p, **kw)
        return cls(p.left, p.right, p.target, p.coef, p.delta, p.parity, p.a_off, p.b_off, p.op_data, **kw)

    @classmethod
    def from_su2(cls, p, precision: str = "fp64", max_nvec: int = 1, n_slices: int = 0, plan_only: bool = False,
                 graphs: bool = True, split_mid_bytes: int = 0) -> "HEff":
        """Spin-adapted handle (dmrg_heff_create_su2) from an object with the fields
        left, right, target, coef, rank2, dn, parity, a_blocks, b_blocks, op_data."""
        self = cls.__new__(cls)
        self._h = None
        arr = lambda a, dt: np.ascontiguousarray(np.asarray(a, dtype=dt))  # noqa: E731
        self._left = arr(p.left, np.int32).reshape(-1, 3)
        self._right = arr(p.right, np.int32).reshape(-1, 3)
        coef = arr(p.coef, np.float64)
        rank2, dn, parity = arr(p.rank2, np.int32), arr(p.dn, np.int32), arr(p.parity, np.int32)
        ab = arr(p.a_blocks, np.int64).reshape(-1, 4)
        bb = arr(p.b_blocks, np.int64).reshape(-1, 4)
        op_data = arr(p.op_data, np.float64)
        opts = Opts(_PREC[precision] if isinstance(precision, str) else int(precision), n_slices, max_nvec,
                    (FLAG_PLAN_ONLY if plan_only else 0) | (0 if graphs else FLAG_NO_GRAPH), int(split_mid_bytes))
        h = ctypes.c_void_p()
        _check(_lib.dmrg_heff_create_su2(_ptr(self._left), len(self._left), _ptr(self._right), len(self._right),
                                         int(p.target[0]), int(p.target[1]), _ptr(coef), _ptr(rank2), _ptr(dn),
                                         _ptr(parity), coef.shape[0], _ptr(ab), ab.shape[0], _ptr(bb), bb.shape[0],
                                         _ptr(op_data), op_data.size, ctypes.byref(opts), ctypes.byref(h)))
        self._h = h
        self.max_nvec = max_nvec
        self.precision = precision
        return self

    def close(self):
        if self._h:
            _lib.dmrg_heff_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def dim(self) -> int:
        return int(_lib.dmrg_heff_dim(self._h))

    @property
    def flops(self) -> int:
        f = _i64()
        _check(_lib.dmrg_heff_flops(self._h, ctypes.byref(f)))
        return int(f.value)

    def memory(self) -> dict:
        """Device bytes of the handle (dmrg_heff_memory): operators, operator_slices,
        apply_buffers, setup_peak, total."""
        m = Memory()
        _check(_lib.dmrg_heff_memory(self._h, ctypes.byref(m)))
        return {k: int(getattr(m, k)) for k, _ in Memory._fields_}

    def plan_dump(self) -> np.ndarray:
        n = _i64(0)
        _check(_lib.dmrg_heff_plan_dump(self._h, None, ctypes.byref(n)))
        buf = np.zeros((n.value, 5), np.int64)
        _check(_lib.dmrg_heff_plan_dump(self._h, _ptr(buf), ctypes.byref(n)))
        return buf

    def apply(self, x, y, nvec: int = 1, stream=None):
        """y = H_eff x for nvec vectors; x, y CUDA float64 tensors (or raw device
        pointers), asynchronous on `stream` (default: torch's current stream)."""
        n = nvec * self.dim
        _check(_lib.dmrg_heff_apply(self._h, _dev_ptr(x, n, "x"), _dev_ptr(y, n, "y"), nvec,
                                    _stream_ptr(stream)))
        return y

    def apply_host(self, x: np.ndarray) -> np.ndarray:
        """y = H_eff x with host arrays (nvec, dim) or (dim,), synchronous."""
        x = np.ascontiguousarray(x, np.float64)
        nvec = 1 if x.ndim == 1 else x.shape[0]
        if x.size != nvec * self.dim:
            raise ValueError("x has the wrong size")
        y = np.empty_like(x)
        _check(_lib.dmrg_heff_apply_host(self._h, _ptr(x), _ptr(y), nvec))
        return y

    def apply_host_ptr(self, x_ptr: int, y_ptr: int, nvec: int):
        """apply_host on raw host pointers (for pinned buffers)."""
        _check(_lib.dmrg_heff_apply_host(self._h, ctypes.c_void_p(x_ptr), ctypes.c_void_p(y_ptr), nvec))

    @property
    def schedule(self) -> dict:
        """Current work-list schedule (see dmrg_schedule in the C header)."""
        s = Schedule()
        _check(_lib.dmrg_heff_schedule_get(self._h, ctypes.byref(s)))
        return s.to_dict()

    @schedule.setter
    def schedule(self, d: dict):
        s = Schedule.from_dict(d)
        _check(_lib.dmrg_heff_schedule_set(self._h, ctypes.byref(s)))

    def autotune(self, nvec: int = 1, reps: int = 3) -> dict:
        """Time candidate schedules on this handle and keep the fastest; returns the
        report (trials, nvec, default_ms, best_ms, best)."""
        r = TuneReport()
        _check(_lib.dmrg_heff_autotune(self._h, nvec, reps, ctypes.byref(r)))
        return dict(trials=r.trials, nvec=r.nvec, default_ms=r.default_ms, best_ms=r.best_ms,
                    best=r.best.to_dict(), tile=[r.tile_m, r.tile_n])

    def psi_blocks(self) -> np.ndarray:
        """Wave-function layout: rows (left sector, right sector, rows, cols, offset)."""
        n = _i64(0)
        _check(_lib.dmrg_heff_psi_blocks(self._h, None, ctypes.byref(n)))
        buf = np.zeros((max(n.value, 1), 5), np.int64)
        _check(_lib.dmrg_heff_psi_blocks(self._h, _ptr(buf), ctypes.byref(n)))
        return buf[:n.value]

    def svd_matrices(self) -> np.ndarray:
        """Matrices of the two-site decomposition: rows (left sector, rows, cols, offset of
        its first block) -- per left sector its wave-function blocks side by side."""
        out = []
        for iL, _, rows, cols, off in self.psi_blocks():
            if out and out[-1][0] == iL:
                out[-1][2] += int(cols)
            else:
                out.append([int(iL), int(rows), int(cols), int(off)])
        return np.array(out, np.int64).reshape(-1, 4)

    def svd_truncate(self, psi, D: int) -> dict:
        """SVD per left sector of the device wave function psi (its blocks side by side,
        see svd_matrices) and truncation to the D largest singular values; returns
        dict(sectors, sv=[per matrix], kept, U=device tensor of the kept left vectors,
        u_off, discarded)."""
        import torch
        mats = self.svd_matrices()
        rows, cols = mats[:, 1], mats[:, 2]
        nsv = int(np.minimum(rows, cols).sum())
        sv = np.zeros(max(nsv, 1), np.float64)
        kept = np.zeros(max(len(mats), 1), np.int32)
        u_off = np.zeros(max(len(mats), 1), np.int64)
        disc = _f64(0.0)
        cap = int((rows * np.minimum(np.minimum(rows, cols), D)).sum())
        U = torch.empty(max(cap, 1), dtype=torch.float64, device="cuda")
        _check(_lib.dmrg_svd_truncate(self._h, _dev_ptr(psi, self.dim, "psi"), D, _ptr(sv), _ptr(kept),
                                      ctypes.c_void_p(U.data_ptr()), int(U.numel()), _ptr(u_off), ctypes.byref(disc)))
        k = np.minimum(rows, cols)
        parts = np.split(sv[:nsv], np.cumsum(k)[:-1]) if len(mats) else []
        return dict(sectors=mats[:, 0].copy(), sv=parts, kept=kept[:len(mats)], U=U, u_off=u_off[:len(mats)],
                    discarded=disc.value)

    def gemm_count(self, nvec: int = 1) -> tuple:
        """(stage-1, stage-2) grouped GEMMs of the plan for nvec vectors."""
        c = (_i64 * 2)()
        _check(_lib.dmrg_heff_gemm_count(self._h, nvec, c))
        return int(c[0]), int(c[1])

    def profile(self, enable: bool = True):
        """Start (reset) or stop per-kernel CUDA-event timing of this handle."""
        _check(_lib.dmrg_heff_profile(self._h, 1 if enable else 0))

    def profile_read(self) -> list:
        """Per-kernel dicts: name, launches, ms_total, flops_total, bytes_total."""
        n = _i32(0)
        _check(_lib.dmrg_heff_profile_read(self._h, None, ctypes.byref(n)))
        buf = (KernelStat * max(n.value, 1))()
        _check(_lib.dmrg_heff_profile_read(self._h, buf, ctypes.byref(n)))
        return [dict(name=s.name.decode(), launches=s.launches, ms_total=s.ms_total,
                     flops_total=s.flops_total, bytes_total=s.bytes_total) for s in buf[:n.value]]

    def diagonal(self, out, stream=None):
        _check(_lib.dmrg_heff_diagonal(self._h, _dev_ptr(out, self.dim, "diag"), _stream_ptr(stream)))
        return out

    def davidson(self, x0, k_eig: int = 1, tol: float = 1e-8, max_iter: int = 300, block: int | None = None,
                 n_iter: int = 0):
        """Lowest k_eig eigenpairs.  x0: CUDA float64 tensor with max(block, k_eig)
        rows of length dim; its first `block` rows are the start block, and its
        first k_eig rows are overwritten with the Ritz vectors.
        Returns (evals ndarray, info dict); info['converged'] is False when tol
        was not met within max_iter."""
        block = block or (x0.shape[0] if x0.dim() == 2 else 1)
        ev = np.zeros(max(k_eig, 1), np.float64)
        cap = max(max_iter, n_iter, 1)
        th = np.full(cap, np.nan)
        tm = np.full(cap, np.nan)
        info = DavidsonInfo()
        info.hist_theta, info.hist_time, info.hist_cap = th.ctypes.data, tm.ctypes.data, cap
        rc = _lib.dmrg_davidson(self._h, k_eig, tol, max_iter, block, n_iter,
                                _dev_ptr(x0, max(block, k_eig) * self.dim, "x0"), _ptr(ev), ctypes.byref(info))
        if rc not in (0, ERR_NOT_CONVERGED):
            raise DmrgError(rc)
        n = info.iters
        return ev[:k_eig], dict(iters=n, matvecs=info.matvecs, converged=bool(info.converged),
                                restarts=info.restarts, resid_max=info.resid_max, seconds=info.seconds,
                                theta=th[:n].copy(), time=tm[:n].copy())

    def lanczos(self, x0, tol: float = 1e-8, max_iter: int = 300, m_max: int = 63):
        """Lowest eigenpair by restarted Lanczos.  x0: CUDA float64 tensor of dim values
        (the start vector), overwritten with the unit Ritz vector.
        Returns (eval, info dict) as davidson does; info['resid_max'] is the explicit
        residual of the returned vector."""
        ev = np.zeros(1, np.float64)
        cap = max(max_iter, 1)
        th = np.full(cap, np.nan)
        tm = np.full(cap, np.nan)
        info = DavidsonInfo()
        info.hist_theta, info.hist_time, info.hist_cap = th.ctypes.data, tm.ctypes.data, cap
        rc = _lib.dmrg_lanczos(self._h, tol, max_iter, m_max, _dev_ptr(x0, self.dim, "x0"), _ptr(ev),
                               ctypes.byref(info))
        if rc not in (0, ERR_NOT_CONVERGED):
            raise DmrgError(rc)
        n = info.iters
        return float(ev[0]), dict(iters=n, matvecs=info.matvecs, converged=bool(info.converged),
                                  restarts=info.restarts, resid_max=info.resid_max, seconds=info.seconds,
                                  theta=th[:n].copy(), time=tm[:n].copy())


def renormalise(dims, dims_new, U, blocks, op, out, stream=None) -> np.ndarray:
    """O'[p<-q] = U_p^T O[p<-q] U_q for each row (q, p, offset) of blocks.  dims and
    dims_new: per-sector old and new dims; U, op, out: contiguous CUDA float64 tensors;
    returns the offsets of the results in out."""
    dims = np.ascontiguousarray(dims, np.int32)
    dims_new = np.ascontiguousarray(dims_new, np.int32)
    blocks = np.ascontiguousarray(np.asarray(blocks, np.int64).reshape(-1, 3))
    out_off = np.zeros(max(len(blocks), 1), np.int64)
    nu = int((dims.astype(np.int64) * dims_new).sum())
    _check(_lib.dmrg_renormalise(len(dims), _ptr(dims), _ptr(dims_new), _dev_ptr(U, nu, "U"), _ptr(blocks),
                                 len(blocks), _dev_ptr(op, 0, "op"), int(op.numel()), _dev_ptr(out, 0, "out"),
                                 int(out.numel()), _ptr(out_off), _stream_ptr(stream)))
    return out_off[:len(blocks)]


class Renorm:
    """A renormalisation plan (dmrg_renorm_create): the block list's GEMM lists and device
    buffers, built once; run() launches on a stream without allocating or synchronising."""

    def __init__(self, dims, dims_new, blocks, op_len: int, out_len: int):
        self._p = None
        self.dims = np.ascontiguousarray(dims, np.int32)
        self.dims_new = np.ascontiguousarray(dims_new, np.int32)
        b = np.ascontiguousarray(np.asarray(blocks, np.int64).reshape(-1, 3))
        out_off = np.zeros(max(len(b), 1), np.int64)
        p = ctypes.c_void_p()
        _check(_lib.dmrg_renorm_create(len(self.dims), _ptr(self.dims), _ptr(self.dims_new), _ptr(b), len(b),
                                       int(op_len), int(out_len), _ptr(out_off), ctypes.byref(p)))
        self._p = p
        self.out_off = out_off[:len(b)]
        self.nu = int((self.dims.astype(np.int64) * self.dims_new).sum())

    def run(self, U, op, out, stream=None):
        _check(_lib.dmrg_renorm_run(self._p, _dev_ptr(U, self.nu, "U"), _dev_ptr(op, 0, "op"),
                                    _dev_ptr(out, 0, "out"), _stream_ptr(stream)))
        return out

    def close(self):
        if self._p:
            _lib.dmrg_renorm_destroy(self._p)
            self._p = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def su2_recoupling(two_sl_out: int, two_sr_out: int, two_sl_in: int, two_sr_in: int, two_k: int,
                   two_s: int) -> float:
    """Recoupling coefficient the spin-adapted planner applies (dmrg_su2_recoupling);
    host only, arguments twice the spins."""
    w = _f64()
    _check(_lib.dmrg_su2_recoupling(two_sl_out, two_sr_out, two_sl_in, two_sr_in, two_k, two_s, ctypes.byref(w)))
    return float(w.value)


def probe_fp64_peak() -> float:
    """FP64 tensor-core (DMMA m16n8k16) throughput of the current GPU, TFLOP/s."""
    v = _f64()
    _check(_lib.dmrg_probe_fp64_peak(ctypes.byref(v)))
    return float(v.value)
