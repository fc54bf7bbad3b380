"""ctypes binding of libseqaccel: structs mirroring include/seqaccel.h and thin
wrappers with the same names.  Argument marshalling only."""
from __future__ import annotations

import ctypes
import dataclasses
import os
from typing import Optional

import torch

from . import build as _build

STATUS = {0: "SEQ_OK", 1: "SEQ_NOT_CONVERGED", 2: "SEQ_FALLBACK_USED", -1: "SEQ_EINVAL",
          -2: "SEQ_ENOMEM", -3: "SEQ_ECUDA", -4: "SEQ_EBREAKDOWN", -5: "SEQ_ENONFINITE",
          -6: "SEQ_ETIMEOUT"}
PRECISION = {"f64": 0, "mixed": 1, "mixed_krylov": 2}
GUESS = {"zero": 0, "prev": 1, "sketch": 2, "learned": 3, "pod": 4, "rand": 5}
KRYLOV = {"cg": 0, "gmres": 1}


class SeqError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class _Csr(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("nnz", ctypes.c_int32),
                ("rowptr", ctypes.c_void_p), ("colind", ctypes.c_void_p),
                ("values", ctypes.c_void_p), ("values_f32", ctypes.c_void_p)]


class _Config(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("M", ctypes.c_int32), ("s", ctypes.c_int32),
                ("zeta", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("precision", ctypes.c_int32), ("guess", ctypes.c_int32),
                ("krylov", ctypes.c_int32), ("restart", ctypes.c_int32),
                ("max_iters", ctypes.c_int32), ("inner_tol", ctypes.c_double),
                ("rank_tol", ctypes.c_double), ("basis_m", ctypes.c_int32),
                ("refresh", ctypes.c_int32), ("precond_sweeps", ctypes.c_int32),
                ("precond_omega", ctypes.c_double), ("precond_kind", ctypes.c_int32),
                ("precond_ratio", ctypes.c_double), ("precond_lmax", ctypes.c_double)]

PRECOND = {"jacobi": 0, "chebyshev": 1}


class SeqInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("refinements", ctypes.c_int32),
                ("history_cols", ctypes.c_int32), ("rank", ctypes.c_int32),
                ("guess_relres", ctypes.c_double), ("sketch_resid", ctypes.c_double),
                ("final_relres", ctypes.c_double), ("status", ctypes.c_int32),
                ("launches", ctypes.c_int32), ("net_resid", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class KernelStat(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64), ("ms", ctypes.c_double),
                ("bytes", ctypes.c_double), ("flops", ctypes.c_double)]


KERNEL_KINDS = ["spmv", "cgs_dot", "cgs_pass2", "cgs_pass3", "update", "restart", "precond"]

_LIB = None

_SIGS = {
    "seq_create": (ctypes.c_int, [ctypes.POINTER(_Config), ctypes.c_void_p,
                                  ctypes.POINTER(ctypes.c_void_p)]),
    "seq_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "seq_push_solution": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "seq_history_size": (ctypes.c_int, [ctypes.c_void_p]),
    "seq_guess": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(_Csr), ctypes.c_void_p,
                                 ctypes.c_void_p, ctypes.POINTER(SeqInfo)]),
    "seq_solve": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(_Csr), ctypes.c_void_p,
                                 ctypes.c_double, ctypes.c_void_p, ctypes.POINTER(SeqInfo)]),
    "seq_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "seq_last_sketch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "seq_sketch_columns": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                          ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_void_p]),
    "seq_probe_fp64_peak": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]),
    "seq_sketch_block_noalloc": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                                ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                                ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                                ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64,
                                                ctypes.c_void_p, ctypes.c_void_p]),
    "seq_batch_create": (ctypes.c_int, [ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32,
                                        ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64,
                                        ctypes.c_int32, ctypes.c_double, ctypes.c_void_p,
                                        ctypes.POINTER(ctypes.c_void_p)]),
    "seq_batch_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "seq_batch_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p]),
    "seq_batch_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p]),
    "seq_batch_push": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p]),
    "seq_batch_set_autopush": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "seq_batch_set_schedule": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                              ctypes.c_int32]),
    "seq_batch_set_cluster": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                             ctypes.c_int32]),
    "seq_batch_get_schedule": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "seq_mlp_create": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                      ctypes.c_uint64, ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    "seq_mlp_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "seq_mlp_param_count": (ctypes.c_int, [ctypes.c_void_p]),
    "seq_mlp_get_params": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "seq_mlp_set_params": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "seq_mlp_fit_normalization": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32]),
    "seq_mlp_loss_grad": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                         ctypes.c_void_p, ctypes.c_void_p]),
    "seq_mlp_train": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                     ctypes.c_int32, ctypes.c_float, ctypes.c_uint64, ctypes.c_void_p]),
    "seq_mlp_predict": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p]),
    "seq_set_learned": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "seq_last_sample": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "seq_learned_train": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                         ctypes.c_int32, ctypes.c_uint64]),
    "seq_learned_save": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                        ctypes.POINTER(ctypes.c_size_t)]),
    "seq_learned_load": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t]),
    "seq_rand_state": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_void_p, ctypes.c_void_p]),
    "seq_pod_state": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_void_p]),
    "seq_set_profiling": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "seq_kernel_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
}


def lib_path() -> str:
    return _build.LIB


def load(build_if_needed: bool = True) -> ctypes.CDLL:
    """Load libseqaccel.so (building it first when sources are newer)."""
    global _LIB
    if _LIB is None:
        path = _build.build() if build_if_needed else _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"libseqaccel.so is not built ({path}); run __graft_entry__.build()")
        lib = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = lib
    return _LIB


def _stream() -> int:
    return torch.cuda.current_stream().cuda_stream


def _ptr(t: Optional[torch.Tensor], dtype: torch.dtype, n: Optional[int] = None) -> int:
    if t is None:
        return 0
    if not t.is_cuda or t.dtype != dtype or not t.is_contiguous():
        raise ValueError(f"expected a contiguous CUDA tensor of {dtype}, got {t.dtype} on {t.device}")
    if n is not None and t.numel() < n:
        raise ValueError(f"tensor has {t.numel()} elements, need {n}")
    return t.data_ptr()


@dataclasses.dataclass
class CSR:
    """A device CSR matrix: int32 rowptr (n+1), int32 colind (nnz), float64 values
    and an optional float32 copy for mixed precision."""
    rowptr: torch.Tensor
    colind: torch.Tensor
    values: torch.Tensor
    values_f32: Optional[torch.Tensor] = None

    @property
    def n(self) -> int:
        return self.rowptr.numel() - 1

    @property
    def nnz(self) -> int:
        return self.colind.numel()

    def _c(self) -> _Csr:
        return _Csr(self.n, self.nnz, _ptr(self.rowptr, torch.int32, self.n + 1),
                    _ptr(self.colind, torch.int32, self.nnz),
                    _ptr(self.values, torch.float64, self.nnz),
                    _ptr(self.values_f32, torch.float32, self.nnz))


class Sequence:
    """One sequence of systems A(t_i) x = b(t_i) sharing a history of M solutions
    (seq_create / seq_push_solution / seq_guess / seq_solve)."""

    def __init__(self, n: int, M: int, s: int, zeta: int = 8, seed: int = 0x5EEDBA5E,
                 precision: str = "f64", guess: str = "sketch", krylov: str = "gmres",
                 restart: int = 30, max_iters: int = 30000, inner_tol: float = 0.0,
                 rank_tol: float = 0.0, basis_m: int = 0, refresh: int = 0,
                 precond_sweeps: int = 0, precond_omega: float = 0.0,
                 precond_kind: str = "jacobi", precond_ratio: float = 0.0,
                 precond_lmax: float = 0.0):
        self._lib = load()
        cfg = _Config(n, M, s, zeta, seed, PRECISION[precision], GUESS[guess], KRYLOV[krylov],
                      restart, max_iters, inner_tol, rank_tol, basis_m, refresh,
                      precond_sweeps, precond_omega, PRECOND[precond_kind], precond_ratio,
                      precond_lmax)
        h = ctypes.c_void_p()
        rc = self._lib.seq_create(ctypes.byref(cfg), ctypes.c_void_p(_stream()), ctypes.byref(h))
        if rc != 0:
            raise SeqError(rc, "seq_create failed")
        self._h = h
        self.n, self.M, self.s, self.basis_m = n, M, s, basis_m

    def close(self) -> None:
        if getattr(self, "_h", None):
            self._lib.seq_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc: int, info: Optional[SeqInfo] = None, allow=(0, 1)) -> None:
        if rc not in allow:
            msg = self._lib.seq_last_error(self._h)
            raise SeqError(rc, msg.decode() if msg else "")

    def history_size(self) -> int:
        return self._lib.seq_history_size(self._h)

    def push(self, x: torch.Tensor) -> None:
        self._check(self._lib.seq_push_solution(self._h, _ptr(x, torch.float64, self.n)))

    def guess(self, A: CSR, b: torch.Tensor, x0: torch.Tensor) -> dict:
        info = SeqInfo()
        rc = self._lib.seq_guess(self._h, ctypes.byref(A._c()), _ptr(b, torch.float64, self.n),
                                 _ptr(x0, torch.float64, self.n), ctypes.byref(info))
        self._check(rc, info, allow=(0, 2))
        d = info.as_dict()
        d["fallback"] = rc == 2
        return d

    def solve(self, A: CSR, b: torch.Tensor, tol: float, x: torch.Tensor,
              allow=(0, 1)) -> dict:
        info = SeqInfo()
        rc = self._lib.seq_solve(self._h, ctypes.byref(A._c()), _ptr(b, torch.float64, self.n),
                                 ctypes.c_double(tol), _ptr(x, torch.float64, self.n),
                                 ctypes.byref(info))
        self._check(rc, info, allow)
        d = info.as_dict()
        d["rc"] = rc
        return d

    def set_profiling(self, on: bool) -> None:
        self._check(self._lib.seq_set_profiling(self._h, int(bool(on))))

    def kernel_stats(self, reset: bool = False) -> dict:
        """Per kernel kind: launches, device ms, algorithmic bytes and flops."""
        arr = (KernelStat * len(KERNEL_KINDS))()
        self._check(self._lib.seq_kernel_stats(self._h, ctypes.byref(arr), int(reset)))
        return {k: {"launches": arr[i].launches, "ms": arr[i].ms, "bytes": arr[i].bytes,
                    "flops": arr[i].flops} for i, k in enumerate(KERNEL_KINDS)}

    def set_learned(self, mlp) -> None:
        self._check(self._lib.seq_set_learned(self._h, mlp._h if mlp is not None else None))
        self._mlp = mlp

    def learned_train(self, samples: torch.Tensor, epochs: int, seed: int) -> None:
        """seq_learned_train on (count, stride) CUDA float32 samples."""
        self._check(self._lib.seq_learned_train(self._h, _ptr(samples, torch.float32),
                                                samples.shape[0], epochs, seed), allow=(0,))
        self._mlp = None

    def learned_save(self) -> bytes:
        """seq_learned_save: the attached predictor serialised (host bytes)."""
        need = ctypes.c_size_t()
        self._check(self._lib.seq_learned_save(self._h, None, 0, ctypes.byref(need)), allow=(0,))
        buf = ctypes.create_string_buffer(need.value)
        self._check(self._lib.seq_learned_save(self._h, buf, need.value, ctypes.byref(need)),
                    allow=(0,))
        return buf.raw

    def learned_load(self, blob: bytes) -> None:
        """seq_learned_load from host bytes."""
        self._check(self._lib.seq_learned_load(self._h, blob, len(blob)), allow=(0,))
        self._mlp = None

    def last_sample(self, out: torch.Tensor) -> None:
        """Write the training sample of the last guess into out (CUDA float32)."""
        self._check(self._lib.seq_last_sample(self._h, _ptr(out, torch.float32)), allow=(0,))

    def rand_state(self):
        """(Omega n x m, Z history_size x m, draws, updates) of Algorithm 4 (host arrays)."""
        import numpy as np
        om = np.zeros((self.n, self.basis_m))
        Z = np.zeros((self.history_size(), self.basis_m))
        draws = ctypes.c_uint64()
        upd = ctypes.c_int32()
        self._check(self._lib.seq_rand_state(self._h, om.ctypes.data, Z.ctypes.data,
                                             ctypes.byref(draws), ctypes.byref(upd)), allow=(0,))
        return om, Z, draws.value, upd.value

    def pod_state(self):
        """(V_k m_i x k, eigenvalues m_i, sweeps) of the last POD guess."""
        import numpy as np
        dims = (ctypes.c_int32 * 3)()
        self._check(self._lib.seq_pod_state(self._h, None, None, dims), allow=(0,))
        mi, kk = dims[0], dims[1]
        V = np.zeros(max(mi * kk, 1))
        lam = np.zeros(max(mi, 1))
        self._check(self._lib.seq_pod_state(self._h, V.ctypes.data, lam.ctypes.data, dims), allow=(0,))
        return V[:mi * kk].reshape(kk, mi).T.copy(), lam[:mi].copy(), dims[2]

    def last_sketch(self):
        """(W, y) of the last guess as float64 host arrays, oldest history column first."""
        import numpy as np
        W = np.zeros(self.s * (self.M + 1))
        y = np.zeros(self.M)
        rc = self._lib.seq_last_sketch(self._h, W.ctypes.data, y.ctypes.data)
        self._check(rc)
        return W, y


def sketch_columns(n: int, s: int, zeta: int, seed: int):
    """(rows int32 [n, zeta], signs int8 [n, zeta]) of the sparse-sign sketch, on the device."""
    lib = load()
    rows = torch.empty((n, zeta), dtype=torch.int32, device="cuda")
    signs = torch.empty((n, zeta), dtype=torch.int8, device="cuda")
    rc = lib.seq_sketch_columns(n, s, zeta, seed, rows.data_ptr(), signs.data_ptr(),
                                ctypes.c_void_p(_stream()))
    if rc != 0:
        raise SeqError(rc, "seq_sketch_columns failed")
    return rows, signs


def probe_fp64_peak() -> float:
    """Measured FP64 FMA throughput of the current device in TFLOP/s."""
    lib = load()
    out = ctypes.c_double()
    rc = lib.seq_probe_fp64_peak(ctypes.c_void_p(_stream()), ctypes.byref(out))
    if rc != 0:
        raise SeqError(rc, "seq_probe_fp64_peak failed")
    return out.value


def sketch_block_noalloc(A: CSR, X: torch.Tensor, b: torch.Tensor, s: int, zeta: int, seed: int,
                         W: torch.Tensor) -> None:
    """W <- S [A X | b] into the caller's (s, M+1) float64 tensor, without any
    allocation inside the library (seq_sketch_block_noalloc).  X is (n, M)
    float64, row-major, each column one history vector."""
    lib = load()
    n, M = X.shape
    if W.shape != (s, M + 1):
        raise ValueError(f"W must have shape ({s}, {M + 1})")
    rc = lib.seq_sketch_block_noalloc(n, A.nnz, _ptr(A.rowptr, torch.int32, n + 1),
                                      _ptr(A.colind, torch.int32, A.nnz),
                                      _ptr(A.values, torch.float64, A.nnz),
                                      _ptr(X, torch.float64, n * M), X.stride(0), M,
                                      _ptr(b, torch.float64, n), s, zeta, seed,
                                      _ptr(W, torch.float64, s * (M + 1)),
                                      ctypes.c_void_p(_stream()))
    if rc != 0:
        raise SeqError(rc, "seq_sketch_block_noalloc failed")


class Batch:
    """Many independent SPD sequences advanced one time step per call
    (seq_batch_create / seq_batch_step / seq_batch_autotune)."""

    def __init__(self, patterns, M: int, s: int, zeta: int = 8, seed: int = 0x5EEDBA5E,
                 max_iters: int = 100000, inner_tol: float = 0.0):
        """patterns: list of (rowptr, colind) int32 CUDA tensors (kept alive here)."""
        self._lib = load()
        self._patterns = [(rp, ci) for rp, ci in patterns]
        arr = (_Csr * len(patterns))()
        for k, (rp, ci) in enumerate(self._patterns):
            n = rp.numel() - 1
            arr[k] = _Csr(n, ci.numel(), _ptr(rp, torch.int32, n + 1), _ptr(ci, torch.int32), 0, 0)
        h = ctypes.c_void_p()
        rc = self._lib.seq_batch_create(len(patterns), ctypes.byref(arr), M, s, zeta, seed,
                                        max_iters, inner_tol, ctypes.c_void_p(_stream()),
                                        ctypes.byref(h))
        if rc != 0:
            raise SeqError(rc, "seq_batch_create failed")
        self._h = h
        self.count = len(patterns)
        self.sizes = [rp.numel() - 1 for rp, _ in self._patterns]

    def close(self) -> None:
        if getattr(self, "_h", None):
            self._lib.seq_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _arrays(self, values, b, x):
        P = ctypes.c_void_p * self.count
        va = P(*[_ptr(v, torch.float64) for v in values])
        ba = P(*[_ptr(t, torch.float64, nn) for t, nn in zip(b, self.sizes)])
        xa = P(*[_ptr(t, torch.float64, nn) for t, nn in zip(x, self.sizes)])
        return va, ba, xa

    def step(self, values, b, x, tol: float, allow=(0, 1)):
        """values, b, x: lists of CUDA float64 tensors (one per sequence).
        Returns the list of per-sequence info dicts."""
        va, ba, xa = self._arrays(values, b, x)
        infos = (SeqInfo * self.count)()
        rc = self._lib.seq_batch_step(self._h, va, ba, xa, ctypes.c_double(tol), infos)
        if rc not in allow:
            raise SeqError(rc, "seq_batch_step failed")
        return [infos[k].as_dict() for k in range(self.count)]

    def autotune(self, values, b, x, tol: float):
        va, ba, xa = self._arrays(values, b, x)
        chosen = (ctypes.c_int32 * 3)()
        rc = self._lib.seq_batch_autotune(self._h, va, ba, xa, ctypes.c_double(tol), chosen)
        if rc != 0:
            raise SeqError(rc, "seq_batch_autotune failed")
        return self.schedule()

    def schedule(self) -> dict:
        """The schedule in use (seq_batch_get_schedule)."""
        out = (ctypes.c_int32 * 4)()
        rc = self._lib.seq_batch_get_schedule(self._h, out)
        if rc != 0:
            raise SeqError(rc, "seq_batch_get_schedule failed")
        return {"threads": out[0], "blocks_per_sm": out[1],
                "order": "largest first" if out[2] == 0 else "given", "ctas_per_sequence": out[3]}

    def set_autopush(self, on: bool) -> None:
        rc = self._lib.seq_batch_set_autopush(self._h, int(bool(on)))
        if rc != 0:
            raise SeqError(rc, "seq_batch_set_autopush failed")

    def push(self, k: int, x: torch.Tensor) -> None:
        rc = self._lib.seq_batch_push(self._h, k, _ptr(x, torch.float64, self.sizes[k]))
        if rc != 0:
            raise SeqError(rc, "seq_batch_push failed")

    def set_schedule(self, threads: int, blocks_per_sm: int, order: int) -> None:
        rc = self._lib.seq_batch_set_schedule(self._h, threads, blocks_per_sm, order)
        if rc != 0:
            raise SeqError(rc, "seq_batch_set_schedule failed")

    def set_cluster(self, ctas: int, threads: int = 1024, order: int = 0) -> None:
        """One thread-block cluster of `ctas` CTAs per sequence (seq_batch_set_cluster)."""
        rc = self._lib.seq_batch_set_cluster(self._h, ctas, threads, order)
        if rc != 0:
            raise SeqError(rc, "seq_batch_set_cluster failed")


class MLP:
    """The learned coefficient predictor (seq_mlp_*)."""

    def __init__(self, M: int, s: int, hidden: int = 256, max_batch: int = 256, seed: int = 1):
        self._lib = load()
        h = ctypes.c_void_p()
        rc = self._lib.seq_mlp_create(M, s, hidden, max_batch, seed, ctypes.c_void_p(_stream()),
                                      ctypes.byref(h))
        if rc != 0:
            raise SeqError(rc, "seq_mlp_create failed")
        self._h = h
        self.M, self.s, self.hidden = M, s, hidden
        self.inp = 4 * M + s
        self.stride = self.inp + M + M * M + 1
        self.nparams = self._lib.seq_mlp_param_count(h)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.seq_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _rc(self, rc, what):
        if rc != 0:
            raise SeqError(rc, what)

    def get_params(self):
        import numpy as np
        p = np.zeros(self.nparams, np.float32)
        nrm = np.zeros(2 * self.inp + self.M, np.float32)
        self._rc(self._lib.seq_mlp_get_params(self._h, p.ctypes.data, nrm.ctypes.data), "get_params")
        return p, nrm

    def set_params(self, params, norm=None):
        import numpy as np
        p = np.ascontiguousarray(params, np.float32)
        nrm = None if norm is None else np.ascontiguousarray(norm, np.float32)
        self._rc(self._lib.seq_mlp_set_params(self._h, p.ctypes.data,
                                              None if nrm is None else nrm.ctypes.data), "set_params")

    def fit_normalization(self, samples: torch.Tensor) -> None:
        self._rc(self._lib.seq_mlp_fit_normalization(self._h, _ptr(samples, torch.float32),
                                                     samples.shape[0]), "fit_normalization")

    def loss_grad(self, samples: torch.Tensor):
        import numpy as np
        g = np.zeros(self.nparams, np.float32)
        loss = ctypes.c_float()
        self._rc(self._lib.seq_mlp_loss_grad(self._h, _ptr(samples, torch.float32), samples.shape[0],
                                             ctypes.byref(loss), g.ctypes.data), "loss_grad")
        return loss.value, g

    def train(self, samples: torch.Tensor, epochs: int, batch: int, lr: float = 1e-3, seed: int = 7):
        import numpy as np
        losses = np.zeros(max(epochs, 1), np.float32)
        self._rc(self._lib.seq_mlp_train(self._h, _ptr(samples, torch.float32), samples.shape[0],
                                         epochs, batch, ctypes.c_float(lr), seed, losses.ctypes.data),
                 "train")
        return losses[:epochs]

    def predict(self, samples: torch.Tensor) -> torch.Tensor:
        y = torch.empty((samples.shape[0], self.M), dtype=torch.float32, device=samples.device)
        self._rc(self._lib.seq_mlp_predict(self._h, _ptr(samples, torch.float32), samples.shape[0],
                                           _ptr(y, torch.float32)), "predict")
        return y
