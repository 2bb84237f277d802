"""Python binding of the C ABI in include/lse.h (ctypes; argument marshalling only).

Every function named ``lse_*`` here calls the C function of the same name in
``_build/liblse.so``; all computation happens in the CUDA kernels behind it.
There is no CPU fallback: if the library is missing or fails to load, the
first call raises ``RuntimeError``.

Host-array functions take and return numpy arrays.  The ``*_d`` functions
take torch CUDA tensors (device memory) and a torch stream, so callers can
keep inputs resident on the device.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "liblse.so")

LSE_OK, LSE_EINVAL, LSE_ENOMEM, LSE_EBUDGET, LSE_ENUMERIC, LSE_ENOTCONV, LSE_ETIMEOUT, LSE_ECUDA, LSE_ECAPACITY = range(9)
LSE_PREC_FP64, LSE_PREC_MIXED, LSE_PREC_MIXED_DF = 0, 1, 2
LSE_F32, LSE_F64 = 0, 1
LSE_FLAG_NO_AUTOTUNE, LSE_FLAG_NO_CLUSTER, LSE_FLAG_LEVINSON, LSE_FLAG_DIRECT_SUMS, LSE_FLAG_LBFGS = 1, 2, 4, 8, 16

c_double_p = ctypes.POINTER(ctypes.c_double)
c_int32_p = ctypes.POINTER(ctypes.c_int32)
c_int64_p = ctypes.POINTER(ctypes.c_int64)
c_float_p = ctypes.POINTER(ctypes.c_float)


class lse_config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("precision", ctypes.c_int32), ("hbm_budget_bytes", ctypes.c_uint64),
                ("grid_size", ctypes.c_int32), ("tau", ctypes.c_double), ("max_outer", ctypes.c_int32),
                ("max_inner", ctypes.c_int32), ("approx_activation_iters", ctypes.c_int32),
                ("flags", ctypes.c_uint64)]


class lse_result(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int32), ("K_cap", ctypes.c_int32), ("theta", c_double_p), ("alpha", c_double_p),
                ("gamma", c_double_p), ("beta", ctypes.c_double), ("objective", ctypes.c_double),
                ("iters", ctypes.c_int32), ("n_evals", ctypes.c_int32), ("n_grid", ctypes.c_int32)]


class lse_serve_result(ctypes.Structure):
    _fields_ = [("request_id", ctypes.c_int64), ("status", ctypes.c_int32), ("N", ctypes.c_int32),
                ("K", ctypes.c_int32), ("K_cap", ctypes.c_int32), ("theta", c_double_p), ("gamma", c_double_p),
                ("alpha", c_double_p), ("beta", ctypes.c_double), ("objective", ctypes.c_double),
                ("iters", ctypes.c_int32), ("n_evals", ctypes.c_int32)]


class lse_batch_out(ctypes.Structure):
    _fields_ = [("theta", ctypes.c_void_p), ("gamma", ctypes.c_void_p), ("alpha", ctypes.c_void_p),
                ("K", ctypes.c_void_p), ("beta", ctypes.c_void_p), ("objective", ctypes.c_void_p),
                ("iters", ctypes.c_void_p), ("n_evals", ctypes.c_void_p), ("n_grid", ctypes.c_void_p),
                ("status", ctypes.c_void_p)]


EXPORTS = ["lse_config_default", "lse_create", "lse_destroy", "lse_strerror", "lse_last_error", "lse_fit",
           "lse_fit_batch", "lse_fit_batch_d", "lse_eval_grid", "lse_eval_grid_batch_d", "lse_kernel_time",
           "lse_plan_fit", "lse_plan_launch", "lse_plan_graph_launch", "lse_plan_destroy", "lse_serve_create",
           "lse_serve_submit", "lse_serve_poll", "lse_serve_in_flight", "lse_serve_device_bytes", "lse_serve_destroy",
           "lse_fit_mmv", "lse_fit_mmv_batch_d", "lse_serve_reserve", "lse_eval_semifast_batch_d",
           "lse_fit_incomplete", "lse_fit_incomplete_batch_d"]

_lib = None


def load(path: str = LIB_PATH):
    """Load liblse.so and declare the C signatures (raises if it is absent)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} (run __graft_entry__.build())")
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    sig = {
        "lse_config_default": (None, [ctypes.POINTER(lse_config)]),
        "lse_create": (ctypes.c_int, [ctypes.POINTER(lse_config), ctypes.POINTER(P)]),
        "lse_destroy": (None, [P]),
        "lse_strerror": (ctypes.c_char_p, [ctypes.c_int]),
        "lse_last_error": (ctypes.c_char_p, [P]),
        "lse_fit": (ctypes.c_int, [P, c_float_p, ctypes.c_int32, ctypes.POINTER(lse_result)]),
        "lse_fit_batch": (ctypes.c_int, [P, c_float_p, c_int64_p, ctypes.c_int32, ctypes.POINTER(lse_result),
                                         c_int32_p]),
        "lse_fit_batch_d": (ctypes.c_int, [P, P, c_int64_p, ctypes.c_int32, ctypes.POINTER(lse_batch_out), P]),
        "lse_fit_mmv": (ctypes.c_int, [P, c_float_p, ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(lse_result)]),
        "lse_fit_mmv_batch_d": (ctypes.c_int, [P, P, c_int64_p, ctypes.c_int32, ctypes.c_int32,
                                               ctypes.POINTER(lse_batch_out), P]),
        "lse_eval_grid": (ctypes.c_int, [P, c_float_p, ctypes.c_int32, c_double_p, c_double_p, ctypes.c_int32,
                                         ctypes.c_double, ctypes.c_int32, ctypes.c_int32, P, P, P, P, P, P]),
        "lse_eval_grid_batch_d": (ctypes.c_int, [P, P, c_int64_p, ctypes.c_int32, P, P, c_int64_p, P, c_int32_p,
                                                 ctypes.c_int32, P, P, P, P, P, P, P]),
        "lse_kernel_time": (ctypes.c_int, [P, ctypes.c_int32, c_double_p, c_int64_p]),
        "lse_plan_fit": (ctypes.c_int, [P, c_int64_p, ctypes.c_int32, ctypes.POINTER(P)]),
        "lse_plan_launch": (ctypes.c_int, [P, P, ctypes.POINTER(lse_batch_out), P]),
        "lse_plan_graph_launch": (ctypes.c_int, [P, P, ctypes.POINTER(lse_batch_out), P]),
        "lse_plan_destroy": (None, [P]),
        "lse_serve_create": (ctypes.c_int, [ctypes.POINTER(lse_config), ctypes.c_int32, ctypes.c_int32,
                                            ctypes.POINTER(P)]),
        "lse_serve_submit": (ctypes.c_int, [P, c_float_p, ctypes.c_int32, ctypes.c_int64]),
        "lse_serve_poll": (ctypes.c_int32, [P, ctypes.POINTER(lse_serve_result), ctypes.c_int32]),
        "lse_serve_in_flight": (ctypes.c_int32, [P]),
        "lse_serve_device_bytes": (ctypes.c_uint64, [P]),
        "lse_serve_destroy": (None, [P]),
        "lse_serve_reserve": (ctypes.c_int, [P, ctypes.c_int32]),
        "lse_fit_incomplete": (ctypes.c_int, [P, c_float_p, c_int32_p, ctypes.c_int32, ctypes.c_int32,
                                              ctypes.POINTER(lse_result)]),
        "lse_fit_incomplete_batch_d": (ctypes.c_int, [P, P, P, c_int64_p, ctypes.c_int32, c_int32_p,
                                                      ctypes.POINTER(lse_batch_out), P]),
        "lse_eval_semifast_batch_d": (ctypes.c_int, [P, P, P, c_int64_p, ctypes.c_int32, c_int32_p, P, P, c_int64_p,
                                                     P, c_int32_p, ctypes.c_int32, P, P, P, P, P, P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


class LseError(RuntimeError):
    def __init__(self, status: int, detail: str = ""):
        self.status = status
        msg = load().lse_strerror(status).decode()
        super().__init__(f"lse status {status} ({msg}){': ' + detail if detail else ''}")


def _check(ctx, st):
    if st != LSE_OK:
        detail = load().lse_last_error(ctx).decode() if ctx else ""
        raise LseError(st, detail)


def _ptr(a: np.ndarray, t):
    return a.ctypes.data_as(t)


# ------------------------------------------------------------ C functions ---

def lse_config_default(**overrides) -> lse_config:
    cfg = lse_config()
    load().lse_config_default(ctypes.byref(cfg))
    for k, v in overrides.items():
        setattr(cfg, k, v)
    return cfg


def lse_create(cfg: lse_config | None = None):
    h = ctypes.c_void_p()
    st = load().lse_create(ctypes.byref(cfg) if cfg is not None else None, ctypes.byref(h))
    _check(None, st)
    return h


def lse_destroy(ctx) -> None:
    load().lse_destroy(ctx)


def lse_strerror(status: int) -> str:
    return load().lse_strerror(status).decode()


def _c64(y) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(y, dtype=np.complex64))


def lse_fit(ctx, y, K_cap: int | None = None) -> dict:
    """Fit one instance; returns dict(theta, alpha, gamma, beta, objective, iters, n_evals, status)."""
    y = _c64(y)
    r = lse_fit_batch(ctx, [y], K_cap=K_cap)[0]
    _check(ctx, r["status"] if r["status"] not in (LSE_ENOTCONV,) else LSE_OK)
    return r


def lse_fit_batch(ctx, ys, K_cap: int | None = None) -> list:
    """Fit a list of instances (possibly different N) in one launch."""
    ys = [_c64(y) for y in ys]
    B = len(ys)
    offsets = np.zeros(B + 1, np.int64)
    offsets[1:] = np.cumsum([y.shape[0] for y in ys])
    ycat = np.ascontiguousarray(np.concatenate(ys))
    res = (lse_result * B)()
    bufs = []
    for b, y in enumerate(ys):
        cap = y.shape[0] if K_cap is None else K_cap
        th = np.zeros(cap)
        ga = np.zeros(cap)
        al = np.zeros(2 * cap)
        bufs.append((th, ga, al))
        res[b].K_cap = cap
        res[b].theta = _ptr(th, c_double_p)
        res[b].gamma = _ptr(ga, c_double_p)
        res[b].alpha = _ptr(al, c_double_p)
    per = np.zeros(B, np.int32)
    st = load().lse_fit_batch(ctx, ycat.view(np.float32).ctypes.data_as(c_float_p), _ptr(offsets, c_int64_p), B, res,
                              _ptr(per, c_int32_p))
    _check(ctx, st)
    out = []
    for b in range(B):
        K = res[b].K
        th, ga, al = bufs[b]
        ok = per[b] != LSE_ECAPACITY
        out.append(dict(K=K, theta=th[:K].copy() if ok else None, gamma=ga[:K].copy() if ok else None,
                        alpha=(al[0:2 * K:2] + 1j * al[1:2 * K:2]) if ok else None, beta=res[b].beta,
                        objective=res[b].objective, iters=res[b].iters, n_evals=res[b].n_evals,
                        n_grid=res[b].n_grid, status=int(per[b])))
    return out


def lse_fit_batch_d(ctx, y_d, offsets: np.ndarray, out: dict, stream=None) -> None:
    """Device batched fit: y_d a torch complex64 CUDA tensor (concatenated
    instances), offsets a host int64 array [B+1], out a dict of torch CUDA
    tensors (theta, gamma, alpha [complex128], K, beta, objective, iters,
    n_evals, status) as in lse_batch_out."""
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    bo = lse_batch_out(out["theta"].data_ptr(), out["gamma"].data_ptr(), out["alpha"].data_ptr(),
                       out["K"].data_ptr(), out["beta"].data_ptr(), out["objective"].data_ptr(),
                       out["iters"].data_ptr(), out["n_evals"].data_ptr(), out["n_grid"].data_ptr(),
                       out["status"].data_ptr())
    s = ctypes.c_void_p(stream.cuda_stream) if stream is not None else None
    st = load().lse_fit_batch_d(ctx, ctypes.c_void_p(y_d.data_ptr()), _ptr(offsets, c_int64_p), len(offsets) - 1,
                                ctypes.byref(bo), s)
    _check(ctx, st)


def lse_fit_mmv(ctx, Y, K_cap: int | None = None) -> dict:
    """Fit one instance of G snapshots (Sec. V): Y a G x N complex array
    (snapshot g = Y[g]); returns dict(theta, gamma, alpha [K x G], beta, ...)."""
    Y = np.ascontiguousarray(np.asarray(Y, dtype=np.complex64))
    if Y.ndim == 1:
        Y = Y[None, :]
    G, N = Y.shape
    cap = N if K_cap is None else K_cap
    th = np.zeros(cap)
    ga = np.zeros(cap)
    al = np.zeros(2 * cap * G)
    r = lse_result()
    r.K_cap = cap
    r.theta = _ptr(th, c_double_p)
    r.gamma = _ptr(ga, c_double_p)
    r.alpha = _ptr(al, c_double_p)
    st = load().lse_fit_mmv(ctx, Y.view(np.float32).ctypes.data_as(c_float_p), N, G, ctypes.byref(r))
    if st not in (LSE_OK, LSE_ENOTCONV):
        _check(ctx, st)
    K = r.K
    a = (al[0::2] + 1j * al[1::2]).reshape(G, cap)[:, :K].T.copy()
    return dict(K=K, theta=th[:K].copy(), gamma=ga[:K].copy(), alpha=a, beta=r.beta, objective=r.objective,
                iters=r.iters, n_evals=r.n_evals, n_grid=r.n_grid, status=int(st))


def lse_fit_mmv_batch_d(ctx, y_d, offsets: np.ndarray, G: int, out: dict, stream=None) -> None:
    """Device batched fit of instances of G snapshots: y_d a torch complex64
    CUDA tensor (instance b's snapshot g at G offsets[b] + g N_b), offsets a
    host int64 array [B+1] of samples per snapshot, out as from
    alloc_batch_out(offsets, G=G)."""
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    bo = _batch_out(out)
    s = ctypes.c_void_p(stream.cuda_stream) if stream is not None else None
    st = load().lse_fit_mmv_batch_d(ctx, ctypes.c_void_p(y_d.data_ptr()), _ptr(offsets, c_int64_p),
                                    len(offsets) - 1, int(G), ctypes.byref(bo), s)
    _check(ctx, st)


def _batch_out(out: dict):
    return lse_batch_out(out["theta"].data_ptr(), out["gamma"].data_ptr(), out["alpha"].data_ptr(),
                         out["K"].data_ptr(), out["beta"].data_ptr(), out["objective"].data_ptr(),
                         out["iters"].data_ptr(), out["n_evals"].data_ptr(), out["n_grid"].data_ptr(),
                         out["status"].data_ptr())


def lse_plan_fit(ctx, offsets: np.ndarray):
    """Plan batched fits of the shape `offsets` (host int64 [B+1])."""
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    h = ctypes.c_void_p()
    _check(ctx, load().lse_plan_fit(ctx, _ptr(offsets, c_int64_p), len(offsets) - 1, ctypes.byref(h)))
    return h


def lse_plan_launch(plan, y_d, out: dict, stream=None, graph: bool = False) -> None:
    """Enqueue a planned fit (directly, or as a replay of its CUDA graph)."""
    bo = _batch_out(out)
    s = ctypes.c_void_p(stream.cuda_stream) if stream is not None else None
    f = load().lse_plan_graph_launch if graph else load().lse_plan_launch
    st = f(plan, ctypes.c_void_p(y_d.data_ptr()), ctypes.byref(bo), s)
    _check(None, st)


def lse_plan_destroy(plan) -> None:
    load().lse_plan_destroy(plan)


def alloc_batch_out(offsets: np.ndarray, device="cuda", G: int = 1):
    import torch
    tot = int(offsets[-1])
    B = len(offsets) - 1
    f64 = dict(dtype=torch.float64, device=device)
    i32 = dict(dtype=torch.int32, device=device)
    return dict(theta=torch.zeros(tot, **f64), gamma=torch.zeros(tot, **f64),
                alpha=torch.zeros(G * tot, dtype=torch.complex128, device=device), K=torch.zeros(B, **i32),
                beta=torch.zeros(B, **f64), objective=torch.zeros(B, **f64), iters=torch.zeros(B, **i32),
                n_evals=torch.zeros(B, **i32), n_grid=torch.zeros(B, **i32), status=torch.zeros(B, **i32))


def lse_eval_grid(ctx, y, theta, gamma, beta: float, L: int, f64: bool = True, want=("q", "dq", "d2q", "s", "ds", "d2s")):
    """Grid q, s and their theta-derivatives (host arrays in, numpy out)."""
    y = _c64(y)
    N = y.shape[0]
    th = np.ascontiguousarray(np.asarray(theta, np.float64))
    ga = np.ascontiguousarray(np.asarray(gamma, np.float64))
    K = th.shape[0]
    rt = np.float64 if f64 else np.float32
    ct = np.complex128 if f64 else np.complex64
    outs = {}
    ptrs = []
    for name in ("q", "dq", "d2q", "s", "ds", "d2s"):
        if name in want:
            a = np.zeros(L, ct if name in ("q", "dq", "d2q") else rt)
            outs[name] = a
            ptrs.append(a.ctypes.data_as(ctypes.c_void_p))
        else:
            ptrs.append(None)
    st = load().lse_eval_grid(ctx, y.view(np.float32).ctypes.data_as(c_float_p), N, _ptr(th, c_double_p),
                              _ptr(ga, c_double_p), K, float(beta), int(L), LSE_F64 if f64 else LSE_F32, *ptrs)
    _check(ctx, st)
    return outs


def lse_eval_grid_batch_d(ctx, y_d, y_offsets, theta_d, gamma_d, k_offsets, beta_d, L, outs: dict, f64: bool,
                          stream=None) -> None:
    """Device batched grid evaluation; outs maps q, dq, d2q, s, ds, d2s to torch
    CUDA tensors (or None)."""
    y_offsets = np.ascontiguousarray(y_offsets, dtype=np.int64)
    k_offsets = np.ascontiguousarray(k_offsets, dtype=np.int64)
    L = np.ascontiguousarray(L, dtype=np.int32)
    p = [ctypes.c_void_p(outs[n].data_ptr()) if outs.get(n) is not None else None
         for n in ("q", "dq", "d2q", "s", "ds", "d2s")]
    s = ctypes.c_void_p(stream.cuda_stream) if stream is not None else None
    st = load().lse_eval_grid_batch_d(ctx, ctypes.c_void_p(y_d.data_ptr()), _ptr(y_offsets, c_int64_p),
                                      len(y_offsets) - 1, ctypes.c_void_p(theta_d.data_ptr()),
                                      ctypes.c_void_p(gamma_d.data_ptr()), _ptr(k_offsets, c_int64_p),
                                      ctypes.c_void_p(beta_d.data_ptr()), _ptr(L, c_int32_p),
                                      LSE_F64 if f64 else LSE_F32, *p, s)
    _check(ctx, st)


def lse_fit_incomplete(ctx, y, obs, N: int, K_cap: int | None = None) -> dict:
    """Fit one instance observed at the indices obs (Sec. IV setting): y the
    observed samples (complex), obs their indices in [0, N)."""
    y = _c64(y)
    obs = np.ascontiguousarray(np.asarray(obs, dtype=np.int32))
    M = y.shape[0]
    cap = M if K_cap is None else K_cap
    th = np.zeros(cap)
    ga = np.zeros(cap)
    al = np.zeros(2 * cap)
    r = lse_result()
    r.K_cap = cap
    r.theta = _ptr(th, c_double_p)
    r.gamma = _ptr(ga, c_double_p)
    r.alpha = _ptr(al, c_double_p)
    st = load().lse_fit_incomplete(ctx, y.view(np.float32).ctypes.data_as(c_float_p), _ptr(obs, c_int32_p), M, int(N),
                                   ctypes.byref(r))
    if st not in (LSE_OK, LSE_ENOTCONV):
        _check(ctx, st)
    K = r.K
    return dict(K=K, theta=th[:K].copy(), gamma=ga[:K].copy(), alpha=al[0:2 * K:2] + 1j * al[1:2 * K:2], beta=r.beta,
                objective=r.objective, iters=r.iters, n_evals=r.n_evals, n_grid=r.n_grid, status=int(st))


def lse_fit_incomplete_batch_d(ctx, y_d, obs_d, m_offsets, N, out: dict, stream=None) -> None:
    """Device batched fit of incomplete-data instances: torch CUDA tensors
    y_d (complex64) and obs_d (int32), host m_offsets [B+1] and N [B], out
    as from alloc_batch_out(m_offsets)."""
    m_offsets = np.ascontiguousarray(m_offsets, dtype=np.int64)
    N = np.ascontiguousarray(N, dtype=np.int32)
    bo = _batch_out(out)
    s = ctypes.c_void_p(stream.cuda_stream) if stream is not None else None
    st = load().lse_fit_incomplete_batch_d(ctx, ctypes.c_void_p(y_d.data_ptr()), ctypes.c_void_p(obs_d.data_ptr()),
                                           _ptr(m_offsets, c_int64_p), len(m_offsets) - 1, _ptr(N, c_int32_p),
                                           ctypes.byref(bo), s)
    _check(ctx, st)


def lse_eval_semifast_batch_d(ctx, y_d, obs_d, m_offsets, N, theta_d, gamma_d, k_offsets, beta_d, L, scal_d, vec_d,
                              status_d, q=None, s=None, f64: bool = True, stream=None) -> None:
    """Semifast evaluation of incomplete observations (Sec. IV): torch CUDA
    tensors y_d (complex64), obs_d (int32), theta_d, gamma_d, beta_d (float64),
    scal_d (float64 [2B]), vec_d (complex128 [7 sum K]), status_d (int32 [B]),
    optional grid outputs q (complex) and s (real); host offsets, N and L."""
    m_offsets = np.ascontiguousarray(m_offsets, dtype=np.int64)
    k_offsets = np.ascontiguousarray(k_offsets, dtype=np.int64)
    N = np.ascontiguousarray(N, dtype=np.int32)
    L = np.ascontiguousarray(L, dtype=np.int32)
    ptr = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None  # noqa: E731
    st = load().lse_eval_semifast_batch_d(ctx, ptr(y_d), ptr(obs_d), _ptr(m_offsets, c_int64_p), len(m_offsets) - 1,
                                          _ptr(N, c_int32_p), ptr(theta_d), ptr(gamma_d), _ptr(k_offsets, c_int64_p),
                                          ptr(beta_d), _ptr(L, c_int32_p), LSE_F64 if f64 else LSE_F32, ptr(scal_d),
                                          ptr(vec_d), ptr(q), ptr(s), ptr(status_d),
                                          ctypes.c_void_p(stream.cuda_stream) if stream is not None else None)
    _check(ctx, st)


def lse_kernel_time(ctx, which: int):
    """(total ms, launches) of kernel `which` (0 fit, 1 factor, 2 grid) since the last call."""
    ms = ctypes.c_double()
    n = ctypes.c_int64()
    _check(ctx, load().lse_kernel_time(ctx, which, ctypes.byref(ms), ctypes.byref(n)))
    return ms.value, n.value


def lse_fit_noalloc_d(y_d, N: int, out: dict, cfg: lse_config | None = None, stream=None) -> None:
    """Single-instance fit that allocates no device memory (see include/lse.h):
    y_d a torch complex64 CUDA tensor, out a dict of torch CUDA tensors as
    from alloc_batch_out for one instance of size N."""
    lib = load()
    f = lib.lse_fit_noalloc_d
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.POINTER(lse_config), ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(lse_batch_out),
                  ctypes.c_void_p]
    bo = lse_batch_out(out["theta"].data_ptr(), out["gamma"].data_ptr(), out["alpha"].data_ptr(),
                       out["K"].data_ptr(), out["beta"].data_ptr(), out["objective"].data_ptr(),
                       out["iters"].data_ptr(), out["n_evals"].data_ptr(), out["n_grid"].data_ptr(),
                       out["status"].data_ptr())
    s = ctypes.c_void_p(stream.cuda_stream) if stream is not None else None
    st = f(ctypes.byref(cfg) if cfg is not None else None, ctypes.c_void_p(y_d.data_ptr()), int(N), ctypes.byref(bo), s)
    _check(None, st)


class Server:
    """Continuous-batching server (lse_serve_*): submit host requests, poll
    for finished results.  Results are dicts like lse_fit's plus request_id."""

    def __init__(self, cfg: lse_config | None = None, streams: int = 8, max_group: int = 19, K_cap: int = 32768):
        self.h = ctypes.c_void_p()
        _check(None, load().lse_serve_create(ctypes.byref(cfg) if cfg is not None else None, streams, max_group,
                                             ctypes.byref(self.h)))
        self.K_cap = K_cap
        self._buf = (lse_serve_result * 64)()
        self._arr = [(np.zeros(K_cap), np.zeros(K_cap), np.zeros(2 * K_cap)) for _ in range(64)]
        for i, (th, ga, al) in enumerate(self._arr):
            self._buf[i].K_cap = K_cap
            self._buf[i].theta = _ptr(th, c_double_p)
            self._buf[i].gamma = _ptr(ga, c_double_p)
            self._buf[i].alpha = _ptr(al, c_double_p)

    def submit(self, y, request_id: int) -> int:
        y = _c64(y)
        return load().lse_serve_submit(self.h, y.view(np.float32).ctypes.data_as(c_float_p), y.shape[0],
                                       int(request_id))

    def poll(self) -> list:
        out = []
        while True:
            n = load().lse_serve_poll(self.h, self._buf, 64)
            for i in range(n):
                r = self._buf[i]
                th, ga, al = self._arr[i]
                K = r.K
                ok = r.status != LSE_ECAPACITY
                out.append(dict(request_id=r.request_id, status=r.status, N=r.N, K=K,
                                theta=th[:K].copy() if ok else None, gamma=ga[:K].copy() if ok else None,
                                alpha=(al[0:2 * K:2] + 1j * al[1:2 * K:2]) if ok else None, beta=r.beta,
                                objective=r.objective, iters=r.iters, n_evals=r.n_evals))
                self._buf[i].K_cap = self.K_cap
            if n < 64:
                return out

    def reserve(self, n_max: int) -> None:
        """Grow every slot for a full group of requests of up to n_max samples."""
        _check(None, load().lse_serve_reserve(self.h, int(n_max)))

    def in_flight(self) -> int:
        return load().lse_serve_in_flight(self.h)

    def device_bytes(self) -> int:
        return load().lse_serve_device_bytes(self.h)

    def close(self) -> None:
        if self.h:
            load().lse_serve_destroy(self.h)
            self.h = ctypes.c_void_p()
