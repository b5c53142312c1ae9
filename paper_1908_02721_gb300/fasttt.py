"""Thin ctypes binding of libfasttt.so (argument marshalling only).

The names match the C ABI in include/fasttt.h: ``fasttt_decompose``,
``tt_eval_at`` and ``tt_eval_backward``; every step of the computation runs in
the library's CUDA kernels.  PyTorch only provides device memory and the CUDA
stream.  Importing this module raises ImportError when the library has not been
built (``python -m paper_1908_02721_gb300.build``); there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfasttt.so")
if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_1908_02721_gb300.build`")
_lib = ctypes.CDLL(LIB_PATH)

MAX_D = 64
OK, EINVAL, EDUP, ENOMEM, ETIMEOUT, ENUMERIC, ERANK, ECUDA = 0, -1, -2, -3, -4, -5, -6, -7
F64, F32 = 0, 1
PREC_FP64, PREC_MIXED = 0, 1
STATIC, DYNAMIC = 0, 1
STAGE_FULL, STAGE_EXACT, STAGE_DEPAR = 0, 1, 2
STAGES = {"full": STAGE_FULL, "exact": STAGE_EXACT, "depar": STAGE_DEPAR}
SWEEP_MODES = {"auto": 0, "sparse": 1, "dense": 2}
GEMM_ENGINES = {"tensor": 0, "dfma": 1}
ARR = {name: i for i, name in enumerate([
    "core", "left_parent", "left_index", "right_index", "right_child", "mid_row", "mid_col", "mid_val",
    "row_id", "row_class", "row_pref", "col_id", "col_class", "col_pref", "dp_row", "dp_col", "dp_val",
    "lam_s", "lam_t", "sigma"])}
_ARR_DTYPE = {"core": torch.float64, "left_parent": torch.int32, "left_index": torch.int32,
              "right_index": torch.int32, "right_child": torch.int32, "mid_row": torch.int64,
              "mid_col": torch.int64, "mid_val": torch.float64, "row_id": torch.int64,
              "row_class": torch.int32, "row_pref": torch.float64, "col_id": torch.int64,
              "col_class": torch.int32, "col_pref": torch.float64, "dp_row": torch.int32,
              "dp_col": torch.int32, "dp_val": torch.float64, "lam_s": torch.float64,
              "lam_t": torch.float64, "sigma": torch.float64}


class Opts(ctypes.Structure):
    _fields_ = [("p", ctypes.c_int), ("precision", ctypes.c_int), ("rounding", ctypes.c_int),
                ("depar_values", ctypes.c_int), ("stage", ctypes.c_int), ("keep_intermediates", ctypes.c_int),
                ("max_rank", ctypes.c_int64), ("max_sweeps", ctypes.c_int64), ("sparse_sweep", ctypes.c_int),
                ("gemm_engine", ctypes.c_int), ("max_spin", ctypes.c_int64)]


class Stats(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int), ("p", ctypes.c_int), ("nnz_in", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("dropped", ctypes.c_int64), ("R", ctypes.c_int64), ("Rs", ctypes.c_int64 * MAX_D),
                ("rt", ctypes.c_int64 * (MAX_D + 1)), ("ranks", ctypes.c_int64 * (MAX_D + 1)),
                ("beta_r", ctypes.c_int64), ("beta_c", ctypes.c_int64), ("jacobi_sweeps", ctypes.c_int64),
                ("launches", ctypes.c_int64), ("jacobi_block_sweeps", ctypes.c_int64),
                ("coop_launch_error", ctypes.c_int64),
                ("norm2", ctypes.c_double), ("err2", ctypes.c_double),
                ("deltas", ctypes.c_double * (MAX_D + 1)), ("ms_ingest", ctypes.c_double),
                ("ms_group", ctypes.c_double), ("ms_depar", ctypes.c_double), ("ms_round", ctypes.c_double),
                ("ms_total", ctypes.c_double), ("ms_gemm", ctypes.c_double), ("flop_gemm", ctypes.c_double),
                ("ms_jacobi", ctypes.c_double), ("flop_jacobi", ctypes.c_double), ("ms_sort", ctypes.c_double),
                ("bytes_sort", ctypes.c_double), ("ms_jacobi32", ctypes.c_double),
                ("flop_jacobi32", ctypes.c_double), ("ms_gemm_tc", ctypes.c_double),
                ("flop_gemm_tc", ctypes.c_double), ("sparse_bonds", ctypes.c_int64),
                ("ms_tridiag", ctypes.c_double), ("flop_tridiag", ctypes.c_double), ("ms_tdeig", ctypes.c_double),
                ("eig_tridiag", ctypes.c_int64), ("eig_fallbacks", ctypes.c_int64),
                ("ms_gemm_oz", ctypes.c_double), ("flop_gemm_oz", ctypes.c_double),
                ("ms_tridiag32", ctypes.c_double), ("flop_tridiag32", ctypes.c_double),
                ("ms_tsqr", ctypes.c_double), ("flop_tsqr", ctypes.c_double), ("eig_fast", ctypes.c_int64),
                ("qr_cholqr2", ctypes.c_int64), ("qr_svd", ctypes.c_int64), ("mixed_fp32_bonds", ctypes.c_int64),
                ("mixed_fp64_bonds", ctypes.c_int64), ("wait_timeouts", ctypes.c_int64)]

    def to_dict(self):
        d = self.d
        return {"d": d, "p": self.p, "nnz_in": self.nnz_in, "nnz": self.nnz, "dropped": self.dropped,
                "R": self.R, "Rs": list(self.Rs[:d]), "rt": list(self.rt[:d + 1]),
                "ranks": list(self.ranks[:d + 1]), "beta_r": self.beta_r, "beta_c": self.beta_c,
                "jacobi_sweeps": self.jacobi_sweeps, "launches": self.launches,
                "jacobi_block_sweeps": self.jacobi_block_sweeps, "coop_launch_error": self.coop_launch_error,
                "norm2": self.norm2,
                "err2": self.err2,
                "deltas": list(self.deltas[:d + 1]), "ms_ingest": self.ms_ingest, "ms_group": self.ms_group,
                "ms_depar": self.ms_depar, "ms_round": self.ms_round, "ms_total": self.ms_total,
                "ms_gemm": self.ms_gemm, "flop_gemm": self.flop_gemm, "ms_jacobi": self.ms_jacobi,
                "flop_jacobi": self.flop_jacobi, "ms_sort": self.ms_sort, "bytes_sort": self.bytes_sort,
                "ms_jacobi32": self.ms_jacobi32, "flop_jacobi32": self.flop_jacobi32,
                "ms_gemm_tc": self.ms_gemm_tc, "flop_gemm_tc": self.flop_gemm_tc,
                "sparse_bonds": self.sparse_bonds, "ms_tridiag": self.ms_tridiag,
                "flop_tridiag": self.flop_tridiag, "ms_tdeig": self.ms_tdeig, "eig_tridiag": self.eig_tridiag,
                "eig_fallbacks": self.eig_fallbacks, "ms_gemm_oz": self.ms_gemm_oz,
                "flop_gemm_oz": self.flop_gemm_oz, "ms_tridiag32": self.ms_tridiag32,
                "flop_tridiag32": self.flop_tridiag32, "ms_tsqr": self.ms_tsqr, "flop_tsqr": self.flop_tsqr,
                "eig_fast": self.eig_fast, "qr_cholqr2": self.qr_cholqr2, "qr_svd": self.qr_svd,
                "mixed_fp32_bonds": self.mixed_fp32_bonds, "mixed_fp64_bonds": self.mixed_fp64_bonds,
                "wait_timeouts": self.wait_timeouts}


_P = ctypes.c_void_p
_I64P = ctypes.POINTER(ctypes.c_int64)
_lib.fasttt_default_opts.argtypes = [ctypes.POINTER(Opts)]
_lib.fasttt_decompose.argtypes = [ctypes.c_int, _I64P, ctypes.c_int64, _P, _P, ctypes.c_int, ctypes.c_double,
                                  ctypes.POINTER(Opts), _P, ctypes.POINTER(_P), ctypes.POINTER(Stats)]
_lib.fasttt_decompose.restype = ctypes.c_int
_lib.fasttt_tt_free.argtypes = [_P]
_lib.fasttt_tt_stats.argtypes = [_P, ctypes.POINTER(Stats)]
_lib.fasttt_tt_ranks.argtypes = [_P, _I64P]
_lib.fasttt_tt_core.argtypes = [_P, ctypes.c_int, ctypes.POINTER(_P)]
_lib.fasttt_tt_count.argtypes = [_P, ctypes.c_int, ctypes.c_int]
_lib.fasttt_tt_count.restype = ctypes.c_int64
_lib.fasttt_tt_copy.argtypes = [_P, ctypes.c_int, ctypes.c_int, _P, ctypes.c_int64]
_lib.tt_eval_at.argtypes = [ctypes.c_int, _I64P, _I64P, ctypes.POINTER(_P), ctypes.c_int, ctypes.c_int64, _P, _P, _P]
_lib.tt_eval_backward.argtypes = [ctypes.c_int, _I64P, _I64P, ctypes.POINTER(_P), ctypes.c_int, ctypes.c_int64,
                                  _P, _P, ctypes.POINTER(_P), ctypes.c_int, _P]
_lib.tt_eval_backward_noalloc.argtypes = [ctypes.c_int, _I64P, _I64P, ctypes.POINTER(_P), ctypes.c_int,
                                          ctypes.c_int64, _P, _P, ctypes.POINTER(_P), _P]
_lib.fasttt_tt_round.argtypes = [ctypes.c_int, _I64P, _I64P, ctypes.POINTER(_P), ctypes.c_double,
                                 ctypes.POINTER(Opts), _P, ctypes.POINTER(_P), ctypes.POINTER(Stats)]
_lib.fasttt_tt_round.restype = ctypes.c_int
_lib.fasttt_tt_add.argtypes = [ctypes.c_int, _I64P, _I64P, ctypes.POINTER(_P), _I64P, ctypes.POINTER(_P),
                               ctypes.c_double, _P, ctypes.POINTER(_P)]
_lib.fasttt_tt_add.restype = ctypes.c_int
_lib.tt_fit_gd.argtypes = [ctypes.c_int, _I64P, _I64P, ctypes.POINTER(_P), ctypes.c_int, ctypes.c_int64, _P, _P,
                           ctypes.c_int64, ctypes.c_double, ctypes.POINTER(ctypes.c_double), _P]
_lib.tt_fit_gd.restype = ctypes.c_int
_lib.fasttt_debug_select_p.argtypes = [ctypes.c_int, _I64P, _I64P, ctypes.c_int64]
_lib.fasttt_debug_select_p.restype = ctypes.c_int
_lib.fasttt_debug_rank_rule.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.c_int64, ctypes.c_double, ctypes.c_int,
                                        ctypes.c_int, _I64P, ctypes.c_int, ctypes.c_int64]
_lib.fasttt_debug_rank_rule.restype = ctypes.c_int64
_lib.fasttt_last_error.restype = ctypes.c_char_p
_lib.fasttt_version.restype = ctypes.c_char_p
_lib.fasttt_debug_fail_alloc_after.argtypes = [ctypes.c_int64]
_lib.fasttt_debug_sym_eig.argtypes = [_P, ctypes.c_int64, _P, ctypes.POINTER(ctypes.c_double), ctypes.c_int, _P]
_lib.fasttt_debug_gemm.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, _P, _P, _P, ctypes.c_int, _P]
_lib.fasttt_debug_cholqr.argtypes = [ctypes.c_int64, ctypes.c_int64, _P, _P, ctypes.c_int, _P]
_lib.fasttt_debug_gram.argtypes = [ctypes.c_int64, ctypes.c_int64, _P, _P, ctypes.c_int, _P]
_lib.fasttt_debug_svd.argtypes = [ctypes.c_int64, ctypes.c_int64, _P, ctypes.POINTER(ctypes.c_double), _P, _P,
                                  ctypes.c_int, _P]

EXPORTS = ["fasttt_default_opts", "fasttt_decompose", "fasttt_tt_free", "fasttt_tt_stats", "fasttt_tt_ranks",
           "fasttt_tt_core", "fasttt_tt_count", "fasttt_tt_copy", "tt_eval_at", "tt_eval_backward",
           "tt_eval_backward_noalloc",
           "fasttt_last_error", "fasttt_version", "fasttt_debug_fail_alloc_after", "fasttt_debug_sym_eig",
           "fasttt_debug_gemm", "fasttt_debug_gram", "fasttt_debug_cholqr", "fasttt_debug_svd", "fasttt_tt_round", "fasttt_tt_add", "tt_fit_gd",
           "fasttt_debug_select_p", "fasttt_debug_rank_rule"]


class FastTTError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"[{code}] {msg}")
        self.code = code
        self.stats = None


def _check(rc, stats=None):
    if rc != OK:
        err = FastTTError(rc, _lib.fasttt_last_error().decode())
        err.stats = stats.to_dict() if stats is not None else None
        raise err


def version() -> str:
    return _lib.fasttt_version().decode()


def debug_fail_alloc_after(n: int) -> None:
    _lib.fasttt_debug_fail_alloc_after(int(n))


def debug_select_p(dims, Rs, max_rank=0) -> int:
    """Alg. 9's split index as the library's host code computes it (no device work)."""
    p = _lib.fasttt_debug_select_p(len(dims), _i64arr(dims), _i64arr(Rs), int(max_rank))
    if p < 0:
        raise FastTTError(p, _lib.fasttt_last_error().decode())
    return int(p)


def debug_rank_rule(sigma, delta, eps_zero, dims, bond, max_rank=0) -> int:
    """The rounding's rank decision at `bond` as the library's host code takes it (no device work)."""
    s = np.ascontiguousarray(np.asarray(sigma, dtype=np.float64))
    r = _lib.fasttt_debug_rank_rule(s.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), s.size, float(delta),
                                    1 if eps_zero else 0, len(dims), _i64arr(dims), int(bond), int(max_rank))
    if r < 0:
        raise FastTTError(int(r), _lib.fasttt_last_error().decode())
    return int(r)


EIG_METHODS = {"tridiagonal": 0, "iterative": 1, "auto": 2, "fast": 3}


def debug_sym_eig(G, method="auto", stream=None):
    """Eigendecomposition of the symmetric FP64 CUDA matrix G through the library's
    Gram eigensolver (a test hook).  Returns (lam (n,) numpy, V (n, n) torch) with
    V[j] the eigenvector of lam[j]."""
    _require_cuda()
    G = _dev(G, torch.float64)
    n = int(G.shape[0])
    if G.dim() != 2 or G.shape[1] != n:
        raise FastTTError(EINVAL, "G must be square")
    V = torch.empty((n, n), dtype=torch.float64, device=G.device)
    lam = np.zeros(n, dtype=np.float64)
    rc = _lib.fasttt_debug_sym_eig(ctypes.c_void_p(G.data_ptr()), n, ctypes.c_void_p(V.data_ptr()),
                                   lam.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), EIG_METHODS[method],
                                   _stream(stream))
    _check(rc)
    return lam, V


GEMM_TEST_ENGINES = {"dfma": 0, "tensor_f64": 1, "tensor_f32": 2, "tf32x3": 3}


def debug_gemm(A, B, engine, stream=None):
    """C = A @ B for FP64 CUDA matrices through one of the library's GEMM kernels (a test hook)."""
    _require_cuda()
    A = _dev(A, torch.float64)
    B = _dev(B, torch.float64)
    M, K = A.shape
    K2, N = B.shape
    if K2 != K:
        raise FastTTError(EINVAL, "inner dimensions differ")
    C = torch.empty((M, N), dtype=torch.float64, device=A.device)
    rc = _lib.fasttt_debug_gemm(M, N, K, ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(B.data_ptr()),
                                ctypes.c_void_p(C.data_ptr()), GEMM_TEST_ENGINES[engine], _stream(stream))
    _check(rc)
    return C


def debug_svd(Z, precision="fp64", stream=None):
    """Full SVD Z = U diag(sigma) Vt of an FP64 CUDA matrix through the library's rounding SVD
    (a test hook).  Returns (sigma (r,) numpy descending, U (M, r) torch, Vt (r, N) torch)."""
    _require_cuda()
    Z = _dev(Z, torch.float64)
    M, N = Z.shape
    r = min(M, N)
    U = torch.empty((M, r), dtype=torch.float64, device=Z.device)
    Vt = torch.empty((r, N), dtype=torch.float64, device=Z.device)
    sigma = np.zeros(r, dtype=np.float64)
    if precision not in ("fp64", "mixed"):
        raise FastTTError(EINVAL, "precision must be 'fp64' or 'mixed'")
    prec = PREC_FP64 if precision == "fp64" else PREC_MIXED
    rc = _lib.fasttt_debug_svd(M, N, ctypes.c_void_p(Z.data_ptr()), sigma.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                               ctypes.c_void_p(U.data_ptr()), ctypes.c_void_p(Vt.data_ptr()), prec, _stream(stream))
    _check(rc)
    return sigma, U, Vt


def debug_cholqr(Z, precision="fp64", stream=None):
    """CholeskyQR2 of the rows of an FP64 CUDA matrix Z (M x N, M <= N) through the library
    (a test hook).  Returns (Q (M, N) torch with orthonormal rows, R (M, M) torch upper) with Z = R^T Q."""
    _require_cuda()
    Q = _dev(Z, torch.float64).clone()
    M, N = Q.shape
    if precision not in ("fp64", "mixed"):
        raise FastTTError(EINVAL, "precision must be 'fp64' or 'mixed'")
    R = torch.empty((M, M), dtype=torch.float64, device=Q.device)
    rc = _lib.fasttt_debug_cholqr(M, N, ctypes.c_void_p(Q.data_ptr()), ctypes.c_void_p(R.data_ptr()),
                                  PREC_FP64 if precision == "fp64" else PREC_MIXED, _stream(stream))
    _check(rc)
    return Q, R


def debug_gram(A, engine, stream=None):
    """C = A @ A.T for an FP64 CUDA matrix through the symmetric path of one GEMM kernel (a test hook)."""
    _require_cuda()
    A = _dev(A, torch.float64)
    M, K = A.shape
    C = torch.empty((M, M), dtype=torch.float64, device=A.device)
    rc = _lib.fasttt_debug_gram(M, K, ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(C.data_ptr()),
                                GEMM_TEST_ENGINES[engine], _stream(stream))
    _check(rc)
    return C


def _require_cuda():
    if not torch.cuda.is_available():
        raise FastTTError(ECUDA, "no CUDA device: libfasttt has no CPU path")


def _stream(stream):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _dev(x, dtype):
    if isinstance(x, np.ndarray):
        x = torch.from_numpy(np.ascontiguousarray(x))
    if x.device.type != "cuda" or x.dtype != dtype or not x.is_contiguous():
        x = x.to(device="cuda", dtype=dtype).contiguous()
    return x


def _i64arr(vals):
    return (ctypes.c_int64 * len(vals))(*[int(v) for v in vals])


class TT:
    """Result handle of fasttt_decompose; owns the library's device memory."""

    def __init__(self, handle, dims):
        self._h = ctypes.c_void_p(handle)
        self.dims = [int(n) for n in dims]
        self.d = len(self.dims)
        r = (ctypes.c_int64 * (self.d + 1))()
        _check(_lib.fasttt_tt_ranks(self._h, r))
        self.ranks = list(r)
        st = Stats()
        _check(_lib.fasttt_tt_stats(self._h, ctypes.byref(st)))
        self.stats = st.to_dict()

    def count(self, what, k=0) -> int:
        n = _lib.fasttt_tt_count(self._h, ARR[what], int(k))
        if n < 0:
            raise FastTTError(int(n), _lib.fasttt_last_error().decode())
        return int(n)

    def array(self, what, k=0, device="cuda") -> torch.Tensor:
        n = self.count(what, k)
        out = torch.empty(n, dtype=_ARR_DTYPE[what], device=device)
        if n:
            _check(_lib.fasttt_tt_copy(self._h, ARR[what], int(k), ctypes.c_void_p(out.data_ptr()), n))
        return out

    def core(self, k, device="cuda") -> torch.Tensor:
        """Copy of core k (1-based), shape (r_{k-1}, n_k, r_k)."""
        return self.array("core", k, device).view(self.ranks[k - 1], self.dims[k - 1], self.ranks[k])

    def cores(self, device="cuda"):
        return [self.core(k, device) for k in range(1, self.d + 1)]

    def free(self):
        if self._h:
            _lib.fasttt_tt_free(self._h)
            self._h = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def fasttt_decompose(idx, vals, dims, eps, *, p=0, max_rank=0, depar_values=True, rounding="static",
                     stage="full", keep_intermediates=False, max_sweeps=0, precision="fp64", sparse_sweep="auto",
                     gemm_engine="tensor", max_spin=0, stream=None) -> TT:
    """FastTT (Alg. 7) of the COO tensor (idx (d, nnz) int32, vals float64/float32).

    sparse_sweep: "auto", "sparse" or "dense", how the first SVD sweep holds its cores.
    gemm_engine: "tensor" (large FP64 products on the tensor cores from exact bf16 slices)
    or "dfma" (FP64 DFMA only).  max_spin > 0 bounds every device spin-wait at that many
    polls; a wait that gives up fails the call with ETIMEOUT.  On failure the raised
    FastTTError carries the call's statistics in .stats."""
    _require_cuda()
    idx = _dev(idx, torch.int32)
    if isinstance(vals, np.ndarray):
        vals = torch.from_numpy(np.ascontiguousarray(vals))
    vdtype = F32 if vals.dtype == torch.float32 else F64
    vals = _dev(vals, torch.float32 if vdtype == F32 else torch.float64)
    d = len(dims)
    if idx.dim() != 2 or idx.shape[0] != d or vals.shape != (idx.shape[1],):
        raise FastTTError(EINVAL, "idx must be (d, nnz) and vals (nnz,)")
    o = Opts()
    _lib.fasttt_default_opts(ctypes.byref(o))
    o.p = int(p)
    o.max_rank = int(max_rank)
    o.depar_values = 1 if depar_values else 0
    o.rounding = DYNAMIC if rounding == "dynamic" else STATIC
    if stage not in STAGES:
        raise FastTTError(EINVAL, "stage must be 'full', 'exact' or 'depar'")
    o.stage = STAGES[stage]
    o.keep_intermediates = 1 if keep_intermediates else 0
    o.max_sweeps = int(max_sweeps)
    o.precision = PREC_MIXED if precision == "mixed" else PREC_FP64
    if sparse_sweep not in SWEEP_MODES:
        raise FastTTError(EINVAL, "sparse_sweep must be 'auto', 'sparse' or 'dense'")
    o.sparse_sweep = SWEEP_MODES[sparse_sweep]
    if gemm_engine not in GEMM_ENGINES:
        raise FastTTError(EINVAL, "gemm_engine must be 'tensor' or 'dfma'")
    o.gemm_engine = GEMM_ENGINES[gemm_engine]
    o.max_spin = int(max_spin)
    out = ctypes.c_void_p(0)
    st = Stats()
    rc = _lib.fasttt_decompose(d, _i64arr(dims), int(idx.shape[1]), ctypes.c_void_p(idx.data_ptr()),
                               ctypes.c_void_p(vals.data_ptr()), vdtype, float(eps), ctypes.byref(o),
                               _stream(stream), ctypes.byref(out), ctypes.byref(st))
    _check(rc, st)
    return TT(out.value, dims)


def _fp64_tt(x):
    """(d, dims, ranks, core pointer array, keep-alive) of a TT handle (borrowed cores)
    or of a list of FP64 CUDA cores (r_{k-1}, n_k, r_k)."""
    if isinstance(x, TT):
        ptrs = (ctypes.c_void_p * x.d)()
        for k in range(1, x.d + 1):
            p = ctypes.c_void_p(0)
            _check(_lib.fasttt_tt_core(x._h, k, ctypes.byref(p)))
            ptrs[k - 1] = p.value
        return x.d, list(x.dims), list(x.ranks), ptrs, x
    cores = [_dev(G, torch.float64) for G in x]
    if not cores or any(G.dim() != 3 for G in cores):
        raise FastTTError(EINVAL, "cores must be a non-empty list of (r0, n, r1) tensors")
    d = len(cores)
    dims = [int(G.shape[1]) for G in cores]
    ranks = [int(cores[0].shape[0])] + [int(G.shape[2]) for G in cores]
    if any(int(cores[k].shape[0]) != ranks[k] for k in range(d)):
        raise FastTTError(EINVAL, "core ranks do not chain")
    ptrs = (ctypes.c_void_p * d)(*[G.data_ptr() for G in cores])
    return d, dims, ranks, ptrs, cores


def tt_round(tt, eps, *, max_rank=0, precision="fp64", max_sweeps=0, gemm_engine="tensor",
             keep_intermediates=False, max_spin=0, stream=None) -> TT:
    """TT-rounding (Alg. 2) of a TT given as a handle or as FP64 CUDA cores, to relative
    accuracy eps (eps = 0: numerical ranks); max_rank caps every rank.  Returns a new handle."""
    _require_cuda()
    d, dims, ranks, ptrs, keep = _fp64_tt(tt)
    o = Opts()
    _lib.fasttt_default_opts(ctypes.byref(o))
    o.max_rank = int(max_rank)
    o.max_sweeps = int(max_sweeps)
    o.keep_intermediates = 1 if keep_intermediates else 0
    if precision not in ("fp64", "mixed"):
        raise FastTTError(EINVAL, "precision must be 'fp64' or 'mixed'")
    o.precision = PREC_MIXED if precision == "mixed" else PREC_FP64
    if gemm_engine not in GEMM_ENGINES:
        raise FastTTError(EINVAL, "gemm_engine must be 'tensor' or 'dfma'")
    o.gemm_engine = GEMM_ENGINES[gemm_engine]
    o.max_spin = int(max_spin)
    out = ctypes.c_void_p(0)
    st = Stats()
    rc = _lib.fasttt_tt_round(d, _i64arr(dims), _i64arr(ranks), ptrs, float(eps), ctypes.byref(o), _stream(stream),
                              ctypes.byref(out), ctypes.byref(st))
    del keep
    _check(rc)
    return TT(out.value, dims)


def tt_add(a, b, beta=1.0, stream=None) -> TT:
    """Cores of A + beta B (Lemma 2) for TTs given as handles or FP64 CUDA cores."""
    _require_cuda()
    d, dims, ra, pa, keep_a = _fp64_tt(a)
    db, dims_b, rb, pb, keep_b = _fp64_tt(b)
    if db != d or dims_b != dims:
        raise FastTTError(EINVAL, "tt_add: the TTs have different mode sizes")
    out = ctypes.c_void_p(0)
    rc = _lib.fasttt_tt_add(d, _i64arr(dims), _i64arr(ra), pa, _i64arr(rb), pb, float(beta), _stream(stream),
                            ctypes.byref(out))
    del keep_a, keep_b
    _check(rc)
    return TT(out.value, dims)


def _check_cores(cores):
    """Shapes and dtypes of a TT's cores, before any device is needed: d >= 1 contiguous
    (r_{k-1}, n_k, r_k) tensors of one dtype (float64 or float32), r_0 = r_d = 1 and
    adjacent ranks equal.  Returns d."""
    if not isinstance(cores, (list, tuple)) or len(cores) < 1 or len(cores) > MAX_D:
        raise FastTTError(EINVAL, "cores must be a list of 1..64 tensors")
    dtype = getattr(cores[0], "dtype", None)
    if dtype not in (torch.float64, torch.float32):
        raise FastTTError(EINVAL, "cores must be float64 or float32")
    for G in cores:
        if not isinstance(G, torch.Tensor) or G.dtype != dtype or G.dim() != 3 or not G.is_contiguous():
            raise FastTTError(EINVAL, "cores must be contiguous tensors (r0, n, r1) of one dtype")
    if cores[0].shape[0] != 1 or cores[-1].shape[2] != 1:
        raise FastTTError(EINVAL, "r_0 and r_d must be 1")
    for a, b in zip(cores[:-1], cores[1:]):
        if a.shape[2] != b.shape[0]:
            raise FastTTError(EINVAL, "adjacent cores disagree on their rank")
    return len(cores)


def _check_entries(d, idx, grad_out=None):
    """idx (d, m) and, for the adjoint, grad_out (m,), before any device is needed."""
    shape = tuple(getattr(idx, "shape", np.shape(idx)))
    if len(shape) != 2 or shape[0] != d:
        raise FastTTError(EINVAL, "idx must have shape (d, m)")
    if grad_out is not None:
        gshape = tuple(getattr(grad_out, "shape", np.shape(grad_out)))
        if gshape != (shape[1],):
            raise FastTTError(EINVAL, "grad_out must have shape (m,)")
    return shape[1]


def _check_grad_cores(cores, grad_cores):
    """Caller-provided gradient cores: one per core, each of its core's shape, dtype and
    device, contiguous (the kernels add into them at the core's layout)."""
    if not isinstance(grad_cores, (list, tuple)) or len(grad_cores) != len(cores):
        raise FastTTError(EINVAL, "grad_cores must hold one tensor per core")
    for g, G in zip(grad_cores, cores):
        if (not isinstance(g, torch.Tensor) or g.shape != G.shape or g.dtype != G.dtype or g.device != G.device
                or not g.is_contiguous()):
            raise FastTTError(EINVAL, "every gradient core must be a contiguous tensor of its core's shape, dtype "
                                      "and device")


def _core_args(cores):
    _check_cores(cores)
    d = len(cores)
    dtype = cores[0].dtype
    for G in cores:
        if G.device.type != "cuda":
            raise FastTTError(EINVAL, "cores must be CUDA tensors")
    dims = [int(G.shape[1]) for G in cores]
    ranks = [int(cores[0].shape[0])] + [int(G.shape[2]) for G in cores]
    ptrs = (ctypes.c_void_p * d)(*[G.data_ptr() for G in cores])
    return d, dims, ranks, ptrs, (F64 if dtype == torch.float64 else F32), dtype


def tt_fit_gd(cores, idx, vals, steps, lr, stream=None):
    """Fixed-rank fitting of the TT to the entries (idx (d, m) int32, vals (m,) in the
    cores' dtype) by gradient descent with the adjoint; the cores (contiguous CUDA
    tensors) are updated in place.  Returns the steps + 1 losses 1/2 sum (a - v)^2."""
    _require_cuda()
    d, dims, ranks, ptrs, code, dtype = _core_args(cores)
    idx = _dev(idx, torch.int32)
    vals = _dev(vals, dtype)
    if idx.dim() != 2 or idx.shape[0] != d or vals.shape != (idx.shape[1],):
        raise FastTTError(EINVAL, "idx must be (d, m) and vals (m,)")
    losses = np.zeros(int(steps) + 1, dtype=np.float64)
    rc = _lib.tt_fit_gd(d, _i64arr(dims), _i64arr(ranks), ptrs, code, int(idx.shape[1]),
                        ctypes.c_void_p(idx.data_ptr()), ctypes.c_void_p(vals.data_ptr()), int(steps), float(lr),
                        losses.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), _stream(stream))
    _check(rc)
    return losses


def tt_eval_at(cores, idx, stream=None) -> torch.Tensor:
    """a(i^e) = G_1[i_1] ... G_d[i_d] for every column of idx (d, m)."""
    _check_entries(_check_cores(cores), idx)
    _require_cuda()
    d, dims, ranks, ptrs, code, dtype = _core_args(cores)
    idx = _dev(idx, torch.int32)
    m = int(idx.shape[1])
    out = torch.empty(m, dtype=dtype, device="cuda")
    _check(_lib.tt_eval_at(d, _i64arr(dims), _i64arr(ranks), ptrs, code, m, ctypes.c_void_p(idx.data_ptr()),
                           ctypes.c_void_p(out.data_ptr()), _stream(stream)))
    return out


def tt_eval_backward(cores, idx, grad_out, grad_cores=None, recompute=False, stream=None):
    """Adds dL/dG_k for L = sum_e grad_out[e] a(i^e) into grad_cores (zeros if None); returns them."""
    _check_entries(_check_cores(cores), idx, grad_out)
    if grad_cores is not None:
        _check_grad_cores(cores, grad_cores)
    _require_cuda()
    d, dims, ranks, ptrs, code, dtype = _core_args(cores)
    idx = _dev(idx, torch.int32)
    grad_out = _dev(grad_out, dtype)
    if grad_cores is None:
        grad_cores = [torch.zeros_like(G) for G in cores]
    gptrs = (ctypes.c_void_p * d)(*[g.data_ptr() for g in grad_cores])
    _check(_lib.tt_eval_backward(d, _i64arr(dims), _i64arr(ranks), ptrs, code, int(idx.shape[1]),
                                 ctypes.c_void_p(idx.data_ptr()), ctypes.c_void_p(grad_out.data_ptr()), gptrs,
                                 1 if recompute else 0, _stream(stream)))
    return grad_cores


def tt_eval_backward_noalloc(cores, idx, grad_out, grad_cores, stream=None):
    """tt_eval_backward for callers that cannot allocate device memory (a framework
    that owns all device memory through its own pool, a runtime with a fixed memory
    budget): the library works in its fixed, process-lifetime scratch array instead.
    The caller provides every input and the (pre-allocated) gradient cores, which
    receive the gradient ADDED to their contents.  Every argument is checked here
    before the call, since the kernels read and add at the shapes given.  Calls
    sharing the scratch must not overlap on the GPU."""
    _check_entries(_check_cores(cores), idx, grad_out)
    _check_grad_cores(cores, grad_cores)
    _require_cuda()
    d, dims, ranks, ptrs, code, dtype = _core_args(cores)
    if idx.device.type != "cuda" or idx.dtype != torch.int32 or not idx.is_contiguous():
        raise FastTTError(EINVAL, "idx must be a contiguous int32 CUDA tensor")
    if grad_out.device.type != "cuda" or grad_out.dtype != dtype or not grad_out.is_contiguous():
        raise FastTTError(EINVAL, "grad_out must be a contiguous CUDA tensor of the cores' dtype")
    gptrs = (ctypes.c_void_p * d)(*[g.data_ptr() for g in grad_cores])
    _check(_lib.tt_eval_backward_noalloc(d, _i64arr(dims), _i64arr(ranks), ptrs, code, int(idx.shape[1]),
                                         ctypes.c_void_p(idx.data_ptr()), ctypes.c_void_p(grad_out.data_ptr()),
                                         gptrs, _stream(stream)))
    return grad_cores


class TTEval(torch.autograd.Function):
    """Differentiable entry evaluation: forward = tt_eval_at, backward = tt_eval_backward."""

    @staticmethod
    def forward(ctx, idx, recompute, *cores):
        cores = [G.contiguous() for G in cores]
        ctx.save_for_backward(idx, *cores)
        ctx.recompute = bool(recompute)
        return tt_eval_at(cores, idx)

    @staticmethod
    def backward(ctx, grad_out):
        idx, *cores = ctx.saved_tensors
        grads = tt_eval_backward(cores, idx, grad_out.contiguous(), recompute=ctx.recompute)
        return (None, None, *grads)


def tt_eval(cores, idx, recompute=False):
    return TTEval.apply(idx, recompute, *cores)
