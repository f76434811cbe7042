"""Thin Python binding of libaccord (include/accord.h).

Argument marshalling only: tensors supply device pointers and the stream,
every step of the computation runs in the library's CUDA kernels.  There is
no CPU fallback; calls fail loudly if the library is missing or the device is
not a GB300 (sm_103).
"""

from __future__ import annotations

import ctypes
import dataclasses
import os

import numpy as np
import torch

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "lib", "libaccord.so")

OK, NOT_CONVERGED = 0, 1
EINVAL, EDOMAIN, ENONFINITE, EBACKTRACK, ENOMEM, ECUDA, EUNSUPPORTED = -1, -2, -3, -4, -5, -6, -7
FP64, MIXED_BF16X3, MIXED_TF32X3 = 0, 1, 2
PRECISIONS = {"fp64": FP64, "mixed": MIXED_BF16X3, "bf16x3": MIXED_BF16X3, "tf32x3": MIXED_TF32X3}
TRACE_FIELDS = 8
TRACE_COLUMNS = ("f", "kkt", "tau", "ntrials", "nnz", "delta", "g", "reserved")


class AccordOpts(ctypes.Structure):
    _fields_ = [
        ("precision", ctypes.c_int32), ("tau_warm", ctypes.c_int32), ("max_iter", ctypes.c_int32),
        ("max_backtracks", ctypes.c_int32), ("penalize_diag", ctypes.c_int32),
        ("init_from_omega", ctypes.c_int32), ("lipschitz_max_iter", ctypes.c_int32), ("profile", ctypes.c_int32),
        ("sparse_update", ctypes.c_int32), ("autotune", ctypes.c_int32),
        ("tau0", ctypes.c_double), ("beta", ctypes.c_double), ("kkt_tol", ctypes.c_double),
        ("lipschitz", ctypes.c_double), ("lipschitz_tol", ctypes.c_double), ("epbic_gamma", ctypes.c_double),
        ("stream", ctypes.c_void_p),
        ("trace", ctypes.POINTER(ctypes.c_double)), ("trace_cap", ctypes.c_int64),
        ("y_refresh", ctypes.c_int32), ("reserved1", ctypes.c_int32), ("coarse_kkt", ctypes.c_double),
    ]


class AccordStats(ctypes.Structure):
    _fields_ = [
        ("iters", ctypes.c_int32), ("trials", ctypes.c_int32), ("status", ctypes.c_int32),
        ("y_refreshes", ctypes.c_int32), ("f", ctypes.c_double), ("g", ctypes.c_double), ("kkt", ctypes.c_double),
        ("tau_last", ctypes.c_double), ("L", ctypes.c_double), ("nnz_offdiag", ctypes.c_int64),
        ("t_setup_ms", ctypes.c_double), ("t_solve_ms", ctypes.c_double), ("n_prox_gemm", ctypes.c_int32),
        ("n_y_gemm", ctypes.c_int32), ("t_prox_gemm_ms", ctypes.c_double), ("t_y_gemm_ms", ctypes.c_double),
        ("n_launches", ctypes.c_int64), ("logdet_d", ctypes.c_double), ("epbic", ctypes.c_double),
        ("tile_group_m", ctypes.c_int32), ("tile_pairs", ctypes.c_int32), ("delta_entries", ctypes.c_int64),
        ("y_drift", ctypes.c_double), ("t_graph_idle_ms", ctypes.c_double),
        ("coarse_prox", ctypes.c_int32), ("reserved2", ctypes.c_int32),
    ]


class AccordPathEntry(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int32), ("iters", ctypes.c_int32), ("trials", ctypes.c_int32),
        ("y_refreshes", ctypes.c_int32), ("lambda_", ctypes.c_double), ("f", ctypes.c_double),
        ("g", ctypes.c_double), ("kkt", ctypes.c_double), ("logdet_d", ctypes.c_double),
        ("epbic", ctypes.c_double), ("tau_last", ctypes.c_double), ("nnz_offdiag", ctypes.c_int64),
        ("y_drift", ctypes.c_double),
    ]


EXPORTS = ("accord_default_opts", "accord_workspace_bytes", "accord_fit", "accord_fit_f64", "accord_refit", "accord_loss",
           "accord_grad", "accord_status_string", "accord_device_check", "accord_last_error",
           "accord_loss_f64_noalloc", "accord_path", "accord_path_workspace_bytes", "accord_grad_x",
           "accord_dloss_dloglam", "accord_postprocess", "accord_to_csr", "accord_test_wait_limit", "accord_test_refresh",
           "accord_fit_rows", "accord_fit_rows_workspace_bytes")

# exchange(sums, nsums, maxes, nmaxes, ctx) of accord_fit_rows
EXCHANGE_FN = ctypes.CFUNCTYPE(ctypes.c_int32, ctypes.POINTER(ctypes.c_double), ctypes.c_int32,
                               ctypes.POINTER(ctypes.c_double), ctypes.c_int32, ctypes.c_void_p)

_lib = None


def load_library(path: str | None = None) -> ctypes.CDLL:
    """Load libaccord.so (built by paper_2412_11554_gb300.build) and declare
    every exported signature."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    path = path or _LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"libaccord.so not found at {path}: run paper_2412_11554_gb300.build.build() first")
    lib = ctypes.CDLL(path)
    P, i64, dbl, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_int
    opts_p, stats_p = ctypes.POINTER(AccordOpts), ctypes.POINTER(AccordStats)
    lib.accord_default_opts.argtypes = [opts_p]
    lib.accord_default_opts.restype = None
    lib.accord_workspace_bytes.argtypes = [i64, i64, opts_p]
    lib.accord_workspace_bytes.restype = ctypes.c_size_t
    lib.accord_fit.argtypes = [P, i64, i64, dbl, opts_p, P, P, ctypes.c_size_t, stats_p]
    lib.accord_fit.restype = i32
    lib.accord_fit_f64.argtypes = [P, i64, i64, dbl, opts_p, P, P, ctypes.c_size_t, stats_p]
    lib.accord_fit_f64.restype = i32
    lib.accord_refit.argtypes = [P, i64, i64, dbl, dbl, P, opts_p, P, P, ctypes.c_size_t, stats_p]
    lib.accord_refit.restype = i32
    lib.accord_loss.argtypes = [P, i64, i64, P, dbl, opts_p, ctypes.POINTER(dbl), ctypes.POINTER(dbl)]
    lib.accord_loss.restype = i32
    lib.accord_grad.argtypes = [P, i64, i64, P, i32, opts_p, P]
    lib.accord_grad.restype = i32
    lib.accord_status_string.argtypes = [i32]
    lib.accord_status_string.restype = ctypes.c_char_p
    lib.accord_device_check.argtypes = []
    lib.accord_device_check.restype = i32
    lib.accord_last_error.argtypes = []
    lib.accord_last_error.restype = ctypes.c_char_p
    lib.accord_loss_f64_noalloc.argtypes = [P, i64, i64, P, dbl, i32, P, P]
    lib.accord_test_wait_limit.restype = i32
    lib.accord_test_wait_limit.argtypes = [i64, i32]
    lib.accord_test_refresh.restype = i32
    lib.accord_test_refresh.argtypes = [i32, i32]
    lib.accord_fit_rows.argtypes = [P, i64, i64, i64, i64, dbl, opts_p, EXCHANGE_FN, P, P, P, ctypes.c_size_t, stats_p]
    lib.accord_fit_rows.restype = i32
    lib.accord_fit_rows_workspace_bytes.argtypes = [i64, i64, i64, opts_p]
    lib.accord_fit_rows_workspace_bytes.restype = ctypes.c_size_t
    lib.accord_loss_f64_noalloc.restype = i32
    lib.accord_path.argtypes = [P, i64, i64, P, P, i64, P, i64, opts_p, ctypes.POINTER(AccordPathEntry), P, P, P, P,
                                ctypes.c_size_t, stats_p]
    lib.accord_path.restype = i32
    lib.accord_path_workspace_bytes.argtypes = [i64, i64, P, P, i64, i64, opts_p]
    lib.accord_path_workspace_bytes.restype = ctypes.c_size_t
    lib.accord_postprocess.argtypes = [i64, P, opts_p, P, P]
    lib.accord_postprocess.restype = i32
    lib.accord_to_csr.argtypes = [i64, P, opts_p, P, P, P, i64, ctypes.POINTER(i64)]
    lib.accord_to_csr.restype = i32
    lib.accord_grad_x.argtypes = [P, i64, i64, P, opts_p, P]
    lib.accord_grad_x.restype = i32
    lib.accord_dloss_dloglam.argtypes = [P, i64, P, i64, i64, P, dbl, opts_p, ctypes.POINTER(dbl),
                                         ctypes.POINTER(dbl), P]
    lib.accord_dloss_dloglam.restype = i32
    if path == _LIB_PATH:
        _lib = lib
    return lib


class AccordError(RuntimeError):
    def __init__(self, status: int, where: str):
        lib = load_library()
        msg = lib.accord_status_string(status).decode()
        detail = lib.accord_last_error().decode()
        super().__init__(f"{where}: status {status} ({msg})" + (f" [{detail}]" if detail else ""))
        self.status = status


@dataclasses.dataclass
class FitStats:
    iters: int
    trials: int
    status: int
    f: float
    g: float
    kkt: float
    tau_last: float
    L: float
    nnz_offdiag: int
    t_setup_ms: float
    t_solve_ms: float
    n_prox_gemm: int = 0
    n_y_gemm: int = 0
    t_prox_gemm_ms: float = 0.0
    t_y_gemm_ms: float = 0.0
    n_launches: int = 0
    logdet_d: float = 0.0
    epbic: float = 0.0
    trace: np.ndarray | None = None
    tile_group_m: int = 0
    tile_pairs: int = 0
    delta_entries: int = 0
    y_refreshes: int = 0
    y_drift: float = 0.0
    t_graph_idle_ms: float = 0.0
    coarse_prox: int = 0


def _stream_handle(stream) -> int | None:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream) or None


def accord_default_opts(**kw) -> AccordOpts:
    """AccordOpts with the library defaults, overridden by keyword fields
    (precision may be given as 'fp64' / 'mixed')."""
    o = AccordOpts()
    load_library().accord_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        if k == "precision" and isinstance(v, str):
            v = PRECISIONS[v]
        if isinstance(v, bool):
            v = int(v)
        setattr(o, k, v)
    return o


def accord_workspace_bytes(n: int, p: int, **kw) -> int:
    return int(load_library().accord_workspace_bytes(n, p, ctypes.byref(accord_default_opts(**kw))))


def _check_tensor(t, name: str, dtype, shape=None, ndim: int | None = None) -> None:
    """Raise ValueError unless t is a contiguous tensor of the given dtype (one
    dtype or a tuple) and shape, on the current CUDA device.  The library reads
    raw device pointers with the element type and extents it is told, so a
    host tensor, a narrower dtype or a smaller shape must never reach it.
    dtype and shape are checked first, so they are reported for host tensors too."""
    if not isinstance(t, torch.Tensor):
        raise ValueError(f"{name} must be a torch.Tensor")
    dts = dtype if isinstance(dtype, tuple) else (dtype,)
    if t.dtype not in dts:
        raise ValueError(f"{name} must be {' or '.join(str(d) for d in dts)}, got {t.dtype}")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    if ndim is not None and t.dim() != ndim:
        raise ValueError(f"{name} must be {ndim}-D, got {t.dim()}-D")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.device.index != torch.cuda.current_device():
        raise ValueError(f"{name} is on {t.device}, not the current device cuda:{torch.cuda.current_device()}")


def _check_x(X: torch.Tensor, dtype=torch.float32, name: str = "X") -> None:
    _check_tensor(X, name, dtype, ndim=2)


def _omega_dtype(prec: int) -> torch.dtype:
    """Element type of Omega (and of every p x p output) in a precision mode."""
    return torch.float64 if prec == FP64 else torch.float32


def _check_workspace(workspace: torch.Tensor | None) -> tuple[int | None, int]:
    if workspace is None:
        return None, 0
    if not isinstance(workspace, torch.Tensor):
        raise ValueError("workspace must be a torch.Tensor")
    _check_tensor(workspace, "workspace", workspace.dtype)
    return workspace.data_ptr(), workspace.numel() * workspace.element_size()


def _precision_of(precision: str | None, Omega: torch.Tensor) -> int:
    """The named mode, else the one Omega's dtype implies (float64: FP64,
    otherwise BF16x3); a named mode must then match Omega's dtype."""
    if precision:
        return PRECISIONS[precision]
    return FP64 if isinstance(Omega, torch.Tensor) and Omega.dtype == torch.float64 else MIXED_BF16X3


def _check_square(Omega: torch.Tensor) -> int:
    """p of a square float32 / float64 Omega on the current CUDA device."""
    if not isinstance(Omega, torch.Tensor) or Omega.dim() != 2:
        raise ValueError("Omega must be a 2-D torch.Tensor")
    p = Omega.shape[0]
    _check_tensor(Omega, "Omega", (torch.float32, torch.float64), (p, p))
    return p


def accord_refit(X: torch.Tensor, lam: float, phi: float, Omega_hat: torch.Tensor, **kw) -> tuple[torch.Tensor, FitStats]:
    """Bias-corrected refit of Eq. 3.8 on the support of Omega_hat (same
    keyword arguments as accord_fit)."""
    return accord_fit(X, lam, _refit=(float(phi), Omega_hat), **kw)


def accord_fit(X: torch.Tensor, lam: float, *, precision: str = "mixed", Omega: torch.Tensor | None = None,
               init_from_omega: bool = False, workspace: torch.Tensor | None = None, trace: bool = False,
               stream=None, check: bool = True, _refit=None, **opts) -> tuple[torch.Tensor, FitStats]:
    """Fit Omega-hat (Eq. 3.2) with ACCORD-FBS.  X: CUDA float32 (or float64
    with precision='fp64'), n x p.  Remaining keyword arguments set
    accord_opts fields (tau0, beta, tau_warm, max_iter, max_backtracks,
    kkt_tol, penalize_diag, lipschitz, lipschitz_max_iter, lipschitz_tol, profile)."""
    lib = load_library()
    prec = PRECISIONS[precision]
    x64 = X.dtype == torch.float64
    _check_x(X, torch.float64 if x64 else torch.float32)
    if x64 and prec != FP64:
        raise ValueError("float64 X requires precision='fp64'")
    n, p = X.shape
    odt = _omega_dtype(prec)
    ws_ptr, ws_bytes = _check_workspace(workspace)
    if _refit is not None:
        if x64:
            raise ValueError("refit needs float32 X")
        _check_tensor(_refit[1], "Omega_hat", odt, (p, p))
    if Omega is None:
        if init_from_omega:
            raise ValueError("init_from_omega needs Omega")
        Omega = torch.empty((p, p), dtype=odt, device=X.device)
    else:
        _check_tensor(Omega, "Omega", odt, (p, p))
    o = accord_default_opts(precision=prec, init_from_omega=int(init_from_omega), **opts)
    o.stream = _stream_handle(stream)
    tr = None
    if trace:
        tr = np.full((o.max_iter + 2, TRACE_FIELDS), np.nan)
        o.trace = tr.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        o.trace_cap = tr.shape[0]
    st = AccordStats()
    if _refit is not None:
        phi, Oh = _refit
        status = lib.accord_refit(X.data_ptr(), n, p, float(lam), phi, Oh.data_ptr(), ctypes.byref(o),
                                  Omega.data_ptr(), ws_ptr, ws_bytes, ctypes.byref(st))
    else:
        fn = lib.accord_fit_f64 if x64 else lib.accord_fit
        status = fn(X.data_ptr(), n, p, float(lam), ctypes.byref(o), Omega.data_ptr(), ws_ptr, ws_bytes,
                    ctypes.byref(st))
    stats = FitStats(st.iters, st.trials, st.status, st.f, st.g, st.kkt, st.tau_last, st.L, st.nnz_offdiag,
                     st.t_setup_ms, st.t_solve_ms, st.n_prox_gemm, st.n_y_gemm, st.t_prox_gemm_ms,
                     st.t_y_gemm_ms, st.n_launches, st.logdet_d, st.epbic, None,
                     delta_entries=st.delta_entries, y_refreshes=st.y_refreshes, y_drift=st.y_drift,
                     coarse_prox=st.coarse_prox)
    if tr is not None:
        stats.trace = tr[: st.iters + 1].copy()
    if check and status < 0:
        raise AccordError(status, "accord_fit")
    return Omega, stats


def accord_fit_rows(X: torch.Tensor, lam: float, row0: int, rows: int, exchange, *, precision: str = "mixed",
                    Omega: torch.Tensor | None = None, init_from_omega: bool = False,
                    workspace: torch.Tensor | None = None, trace: bool = False, stream=None, check: bool = True,
                    **opts) -> tuple[torch.Tensor, FitStats]:
    """Fit rows row0 .. row0 + rows - 1 of Omega-hat as one block of a fit
    split by rows (include/accord.h, accord_fit_rows).  exchange(sums, maxes)
    receives this block's 9 sums and 1 maximum as float64 numpy arrays and
    must overwrite them, in place, with the sums and maxima over all blocks;
    it is called once before the first trial and once per trial, the same
    number of times in every block.  Returns the block's rows (rows x p) and
    the stats of the whole fit."""
    lib = load_library()
    prec = PRECISIONS[precision]
    _check_x(X, torch.float32)
    n, p = X.shape
    odt = _omega_dtype(prec)
    ws_ptr, ws_bytes = _check_workspace(workspace)
    if Omega is None:
        if init_from_omega:
            raise ValueError("init_from_omega needs Omega")
        Omega = torch.empty((int(rows), p), dtype=odt, device=X.device)
    else:
        _check_tensor(Omega, "Omega", odt, (int(rows), p))
    o = accord_default_opts(precision=prec, init_from_omega=int(init_from_omega), **opts)
    o.stream = _stream_handle(stream)
    tr = None
    if trace:
        tr = np.full((o.max_iter + 2, TRACE_FIELDS), np.nan)
        o.trace = tr.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        o.trace_cap = tr.shape[0]
    failure = []

    def _cb(sums_p, nsums, maxes_p, nmaxes, _ctx):
        try:
            sums = np.ctypeslib.as_array(sums_p, shape=(nsums,))
            maxes = np.ctypeslib.as_array(maxes_p, shape=(nmaxes,))
            exchange(sums, maxes)
            return 0
        except Exception as e:  # no Python exception may cross the C boundary
            failure.append(e)
            return 1

    cb = EXCHANGE_FN(_cb)
    st = AccordStats()
    status = lib.accord_fit_rows(X.data_ptr(), n, p, int(row0), int(rows), float(lam), ctypes.byref(o), cb, None,
                                 Omega.data_ptr(), ws_ptr, ws_bytes, ctypes.byref(st))
    stats = FitStats(st.iters, st.trials, st.status, st.f, st.g, st.kkt, st.tau_last, st.L, st.nnz_offdiag,
                     st.t_setup_ms, st.t_solve_ms, st.n_prox_gemm, st.n_y_gemm, st.t_prox_gemm_ms,
                     st.t_y_gemm_ms, st.n_launches, st.logdet_d, st.epbic, None,
                     delta_entries=st.delta_entries, y_refreshes=st.y_refreshes, y_drift=st.y_drift,
                     coarse_prox=st.coarse_prox)
    if tr is not None:
        stats.trace = tr[: st.iters + 1].copy()
    if failure:
        raise failure[0]
    if check and status < 0:
        raise AccordError(status, "accord_fit_rows")
    return Omega, stats


def accord_fit_rows_workspace_bytes(n: int, p: int, rows: int, **kw) -> int:
    return int(load_library().accord_fit_rows_workspace_bytes(n, p, rows, ctypes.byref(accord_default_opts(**kw))))


def dist_exchange(group=None):
    """An exchange for accord_fit_rows between the ranks of a torch.distributed
    process group whose backend takes host tensors (gloo), one row block per
    rank.  Each call all-gathers every rank's 9 sums and 1 maximum; every rank
    then adds the sums in rank order and takes the maxima, so all ranks hold
    the same bits and take the same accept / stop decisions.  A collective
    that fails (a rank that left, the group's timeout) raises here, and
    accord_fit_rows then ends the fit and re-raises it."""
    import torch.distributed as dist
    world = dist.get_world_size(group)

    def exchange(sums: np.ndarray, maxes: np.ndarray) -> None:
        mine = torch.from_numpy(np.concatenate([sums, maxes]))
        parts = [torch.empty_like(mine) for _ in range(world)]
        dist.all_gather(parts, mine, group=group)
        allv = torch.stack(parts).numpy()
        ns = sums.shape[0]
        tot = allv[0, :ns].copy()
        for r in range(1, world):
            tot += allv[r, :ns]
        sums[:] = tot
        maxes[:] = allv[:, ns:].max(axis=0)

    return exchange


def accord_loss(X: torch.Tensor, Omega: torch.Tensor, lam: float, *, precision: str | None = None,
                penalize_diag: bool = True, stream=None) -> tuple[float, float]:
    """(f, g) of Eq. 3.2 / Eq. 3.4 at Omega; precision follows Omega's dtype."""
    lib = load_library()
    _check_x(X)
    n, p = X.shape
    prec = _precision_of(precision, Omega)
    _check_tensor(Omega, "Omega", _omega_dtype(prec), (p, p))
    o = accord_default_opts(precision=prec, penalize_diag=int(penalize_diag))
    o.stream = _stream_handle(stream)
    f, g = ctypes.c_double(), ctypes.c_double()
    status = lib.accord_loss(X.data_ptr(), n, p, Omega.data_ptr(), float(lam), ctypes.byref(o), ctypes.byref(f),
                             ctypes.byref(g))
    if status != OK:
        raise AccordError(status, "accord_loss")
    return f.value, g.value


def accord_grad(X: torch.Tensor, Omega: torch.Tensor, smooth: bool = False, *, precision: str | None = None,
                out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Omega S (smooth=False) or -Omega_D^-1 + Omega S (smooth=True)."""
    lib = load_library()
    _check_x(X)
    n, p = X.shape
    prec = _precision_of(precision, Omega)
    _check_tensor(Omega, "Omega", _omega_dtype(prec), (p, p))
    if out is None:
        out = torch.empty_like(Omega)
    else:
        _check_tensor(out, "out", Omega.dtype, (p, p))
        if out.data_ptr() == Omega.data_ptr():
            raise ValueError("out must not alias Omega")
    o = accord_default_opts(precision=prec)
    o.stream = _stream_handle(stream)
    status = lib.accord_grad(X.data_ptr(), n, p, Omega.data_ptr(), int(bool(smooth)), ctypes.byref(o),
                             out.data_ptr())
    if status != OK:
        raise AccordError(status, "accord_grad")
    return out


def accord_loss_f64_noalloc(X: torch.Tensor, Omega: torch.Tensor, lam: float, fg_out: torch.Tensor, *,
                            penalize_diag: bool = True, stream=None) -> None:
    """(f, g) of Eq. 3.2 / Eq. 3.4 into the device tensor fg_out (2 doubles)
    without any device allocation by the library (its scratch is a static
    device array; see include/accord.h).  X and Omega are CUDA float64."""
    lib = load_library()
    _check_x(X, torch.float64)
    n, p = X.shape
    _check_tensor(Omega, "Omega", torch.float64, (p, p))
    _check_tensor(fg_out, "fg_out", torch.float64)
    if fg_out.numel() < 2:
        raise ValueError("fg_out must hold at least 2 elements")
    status = lib.accord_loss_f64_noalloc(X.data_ptr(), n, p, Omega.data_ptr(), float(lam), int(bool(penalize_diag)),
                                         _stream_handle(stream), fg_out.data_ptr())
    if status != OK:
        raise AccordError(status, "accord_loss_f64_noalloc")


def accord_postprocess(Omega: torch.Tensor, *, theta: bool = True, rho: bool = True, stream=None):
    """(Theta-hat = Omega_D Omega, partial correlations) of an estimate (Sec 3.1);
    either may be skipped (None).  Precision follows Omega's dtype."""
    lib = load_library()
    p = _check_square(Omega)
    prec = FP64 if Omega.dtype == torch.float64 else MIXED_BF16X3
    o = accord_default_opts(precision=prec)
    o.stream = _stream_handle(stream)
    T = torch.empty_like(Omega) if theta else None
    Rh = torch.empty_like(Omega) if rho else None
    status = lib.accord_postprocess(p, Omega.data_ptr(), ctypes.byref(o), T.data_ptr() if T is not None else None,
                                    Rh.data_ptr() if Rh is not None else None)
    if status != OK:
        raise AccordError(status, "accord_postprocess")
    return T, Rh


def accord_to_csr(Omega: torch.Tensor, *, nnz_hint: int | None = None, stream=None):
    """(row_ptr int64 [p + 1], col_idx int32 [nnz], vals [nnz]) CUDA tensors of
    the nonzero entries of Omega, row by row in column order.  nnz_hint sizes
    the first attempt (e.g. FitStats.nnz_offdiag + p); a short buffer costs one
    more call.  The element type follows Omega's dtype."""
    lib = load_library()
    p = _check_square(Omega)
    prec = FP64 if Omega.dtype == torch.float64 else MIXED_BF16X3
    o = accord_default_opts(precision=prec)
    o.stream = _stream_handle(stream)
    row_ptr = torch.empty(p + 1, dtype=torch.int64, device=Omega.device)
    cap = int(nnz_hint) if nnz_hint is not None else p
    nnz = ctypes.c_int64()
    for _ in range(2):
        cols = torch.empty(max(cap, 1), dtype=torch.int32, device=Omega.device)
        vals = torch.empty(max(cap, 1), dtype=Omega.dtype, device=Omega.device)
        status = lib.accord_to_csr(p, Omega.data_ptr(), ctypes.byref(o), row_ptr.data_ptr(), cols.data_ptr(),
                                   vals.data_ptr(), cap, ctypes.byref(nnz))
        if status == ENOMEM and nnz.value > cap:
            cap = nnz.value
            continue
        break
    if status != OK:
        raise AccordError(status, "accord_to_csr")
    k = nnz.value
    return row_ptr, cols[:k], vals[:k]


def accord_grad_x(X: torch.Tensor, Omega: torch.Tensor, *, precision: str | None = None,
                  out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """dL/dX = (1/n) X Omega^T Omega of the smooth loss (n x p); precision
    defaults to Omega's dtype (float64: FP64 mode, float32: BF16x3)."""
    lib = load_library()
    _check_x(X)
    n, p = X.shape
    prec = _precision_of(precision, Omega)
    _check_tensor(Omega, "Omega", _omega_dtype(prec), (p, p))
    if out is None:
        out = torch.empty((n, p), dtype=Omega.dtype, device=X.device)
    else:
        _check_tensor(out, "out", Omega.dtype, (n, p))
    o = accord_default_opts(precision=prec)
    o.stream = _stream_handle(stream)
    status = lib.accord_grad_x(X.data_ptr(), n, p, Omega.data_ptr(), ctypes.byref(o), out.data_ptr())
    if status != OK:
        raise AccordError(status, "accord_grad_x")
    return out


def accord_dloss_dloglam(X_train: torch.Tensor, X_val: torch.Tensor, Omega_hat: torch.Tensor, lam: float, *,
                         penalize_diag: bool = True, want_domega: bool = False, precision: str | None = None,
                         stream=None):
    """(d L_val / d log lambda, L_val, dOmega-hat / d log lambda or None) by
    implicit differentiation on the active set of Omega_hat (a converged
    estimate for X_train at lam); precision defaults to Omega_hat's dtype
    (float64: FP64 mode, float32: BF16x3)."""
    lib = load_library()
    _check_x(X_train, name="X_train")
    _check_x(X_val, name="X_val")
    n, p = X_train.shape
    if X_val.shape[1] != p:
        raise ValueError("X_train and X_val need the same number of columns")
    prec = _precision_of(precision, Omega_hat)
    _check_tensor(Omega_hat, "Omega_hat", _omega_dtype(prec), (p, p))
    o = accord_default_opts(precision=prec, penalize_diag=int(penalize_diag))
    o.stream = _stream_handle(stream)
    d, lv = ctypes.c_double(), ctypes.c_double()
    dO = torch.empty((p, p), dtype=Omega_hat.dtype, device=X_train.device) if want_domega else None
    status = lib.accord_dloss_dloglam(X_train.data_ptr(), n, X_val.data_ptr(), X_val.shape[0], p,
                                      Omega_hat.data_ptr(), float(lam), ctypes.byref(o), ctypes.byref(d),
                                      ctypes.byref(lv), dO.data_ptr() if dO is not None else None)
    if status != OK:
        raise AccordError(status, "accord_dloss_dloglam")
    return d.value, lv.value, dO


@dataclasses.dataclass
class PathResult:
    """accord_path output.  Arrays are (n_lambda, n_sub): entry [k, s] is the
    estimate of subsample s at lambdas[k]."""
    status: int
    lambdas: np.ndarray
    entry_status: np.ndarray
    iters: np.ndarray
    trials: np.ndarray
    f: np.ndarray
    g: np.ndarray
    kkt: np.ndarray
    logdet_d: np.ndarray
    epbic: np.ndarray
    tau_last: np.ndarray
    nnz_offdiag: np.ndarray
    best_index: np.ndarray                   # (n_sub,) index k of the smallest epBIC, -1 if none
    omega_best: torch.Tensor | None          # (n_sub, p, p) estimates at best_index
    support: torch.Tensor | None             # (n_lambda, n_sub, p, ceil(p/32)) int32 bit words
    stats: FitStats
    y_refreshes: np.ndarray | None = None    # mixed modes: refreshes of Y per (penalty, subsample)
    y_drift: np.ndarray | None = None        # ... and the largest relative drift of Y they found


def _subsample_arrays(subsamples) -> tuple[np.ndarray, np.ndarray]:
    idx = [np.ascontiguousarray(np.asarray(s, dtype=np.int32).ravel()) for s in subsamples]
    rows = np.ascontiguousarray(np.concatenate(idx) if idx else np.zeros(0, np.int32))
    offs = np.ascontiguousarray(np.concatenate([[0], np.cumsum([len(s) for s in idx])]).astype(np.int64))
    return rows, offs


def accord_path_workspace_bytes(n: int, p: int, subsamples, n_lambda: int, **kw) -> int:
    rows, offs = _subsample_arrays(subsamples)
    o = accord_default_opts(**kw)
    return int(load_library().accord_path_workspace_bytes(n, p, rows.ctypes.data, offs.ctypes.data, len(offs) - 1,
                                                          n_lambda, ctypes.byref(o)))


def accord_path(X: torch.Tensor, subsamples, lambdas, *, precision: str = "mixed", support: bool = False,
                omega_best: bool = True, workspace: torch.Tensor | None = None, stream=None, check: bool = True,
                **opts) -> PathResult:
    """Lambda path over subsamples (Sec 3.4): X is the CUDA float32 n x p data
    set, subsamples a list of row-index arrays (repeats allowed), lambdas the
    penalties in solve order.  Remaining keyword arguments set accord_opts
    fields (kkt_tol, max_iter, epbic_gamma, ...)."""
    lib = load_library()
    _check_x(X, torch.float32)
    n, p = X.shape
    ws_ptr, ws_bytes = _check_workspace(workspace)
    rows, offs = _subsample_arrays(subsamples)
    lam = np.ascontiguousarray(np.asarray(lambdas, dtype=np.float64).ravel())
    ns, nl = len(offs) - 1, len(lam)
    prec = PRECISIONS[precision]
    odt = torch.float64 if prec == FP64 else torch.float32
    o = accord_default_opts(precision=prec, **opts)
    o.stream = _stream_handle(stream)
    ent = (AccordPathEntry * max(nl * ns, 1))()
    sup = None
    if support:
        sup = torch.zeros((nl, ns, p, (p + 31) // 32), dtype=torch.int32, device=X.device)
    best = torch.zeros((ns, p, p), dtype=odt, device=X.device) if omega_best else None
    bidx = np.full(max(ns, 1), -1, dtype=np.int32)
    st = AccordStats()
    status = lib.accord_path(X.data_ptr(), n, p, rows.ctypes.data, offs.ctypes.data, ns, lam.ctypes.data, nl,
                             ctypes.byref(o), ent, sup.data_ptr() if sup is not None else None,
                             best.data_ptr() if best is not None else None, bidx.ctypes.data, ws_ptr, ws_bytes,
                             ctypes.byref(st))
    if check and status < 0:
        raise AccordError(status, "accord_path")

    def col(name, dt):
        return np.array([getattr(ent[i], name) for i in range(nl * ns)], dtype=dt).reshape(nl, ns)

    stats = FitStats(st.iters, st.trials, st.status, st.f, st.g, st.kkt, st.tau_last, st.L, st.nnz_offdiag,
                     st.t_setup_ms, st.t_solve_ms, st.n_prox_gemm, st.n_y_gemm, st.t_prox_gemm_ms, st.t_y_gemm_ms,
                     st.n_launches, st.logdet_d, st.epbic, None, st.tile_group_m, st.tile_pairs,
                     y_refreshes=st.y_refreshes, y_drift=st.y_drift, t_graph_idle_ms=st.t_graph_idle_ms,
                     coarse_prox=st.coarse_prox)
    return PathResult(status, col("lambda_", np.float64), col("status", np.int32), col("iters", np.int32),
                      col("trials", np.int32), col("f", np.float64), col("g", np.float64), col("kkt", np.float64),
                      col("logdet_d", np.float64), col("epbic", np.float64), col("tau_last", np.float64),
                      col("nnz_offdiag", np.int64), bidx[:ns].copy(), best, sup, stats,
                      col("y_refreshes", np.int32), col("y_drift", np.float64))


def accord_status_string(status: int) -> str:
    return load_library().accord_status_string(status).decode()


def accord_device_check() -> int:
    return int(load_library().accord_device_check())


def accord_last_error() -> str:
    return load_library().accord_last_error().decode()


def accord_test_wait_limit(wait_limit_ns: int, withhold_next_prox: bool = False) -> int:
    """Testing hook of the bounded device waits (see include/accord.h)."""
    return int(load_library().accord_test_wait_limit(int(wait_limit_ns), int(bool(withhold_next_prox))))


def accord_test_refresh(list_cap: int = 0, form: int = 0) -> int:
    """Testing hook of the refresh of Y (see include/accord.h): the walk's
    list capacity (0: full) and the form (0: by nonzero count, 1: walk,
    2: blocked)."""
    return int(load_library().accord_test_refresh(int(list_cap), int(form)))
