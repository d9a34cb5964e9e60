"""Python binding of libascg (include/ascg.h): argument marshalling only.

Every function has the name of the C call it wraps and passes plain pointers
and sizes. Arrays may be given as integers (raw pointers), numpy arrays (host
memory), or objects with a `data_ptr()` method such as torch tensors (device
or host memory, as the C call expects). PyTorch is not imported here; callers
use it only to own device memory and streams.

All numerical work runs in the CUDA kernels of libascg.so. If the library has
not been built, importing this package raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libascg.so")

ASCG_MAX_S = 16
ASCG_MAX_W = 2 * ASCG_MAX_S + 1

# ascg_status
ASCG_OK, ASCG_ERR_INVALID, ASCG_ERR_OOM, ASCG_ERR_CUDA = 0, 1, 2, 3
ASCG_ERR_BREAKDOWN, ASCG_NOT_CONVERGED, ASCG_ERR_TIMEOUT, ASCG_ERR_NOT_SPD = 4, 5, 6, 7
STATUS_NAMES = {0: "OK", 1: "ERR_INVALID", 2: "ERR_OOM", 3: "ERR_CUDA", 4: "ERR_BREAKDOWN",
                5: "NOT_CONVERGED", 6: "ERR_TIMEOUT", 7: "ERR_NOT_SPD"}
# ascg_method / ascg_basis / ascg_stop
ASCG_CLASSICAL, ASCG_FIXED_S, ASCG_ADAPTIVE, ASCG_VARIABLE_S = 0, 1, 2, 3
ASCG_MONOMIAL, ASCG_NEWTON, ASCG_CHEBYSHEV = 0, 1, 2
ASCG_STOP_DONE, ASCG_STOP_CONVERGED, ASCG_STOP_BREAK, ASCG_STOP_BREAKDOWN, ASCG_STOP_MAXITER = 0, 1, 2, 3, 4
ASCG_FLAG_TIMING = 1
ASCG_FLAG_GRAM_FP64 = 2
ASCG_FLAG_C_FORMULA = 4
ASCG_FLAG_MOMENT_GRAM = 8
ASCG_FLAG_TEST_GRAM_STALL = 16
ASCG_FLAG_GRAM_TC = 32
ASCG_FLAG_RECOVER_FP64 = 64


class ascg_block_info(C.Structure):
    _fields_ = [("sbar", C.c_int), ("stilde", C.c_int), ("s_k", C.c_int), ("stop", C.c_int),
                ("m", C.c_int), ("pad_", C.c_int), ("rnorm", C.c_double), ("threshold", C.c_double),
                ("gamma", C.c_double), ("sqrt_kappa", C.c_double * ASCG_MAX_S)]


class ascg_options(C.Structure):
    _fields_ = [("method", C.c_int), ("basis", C.c_int), ("s_max", C.c_int), ("s0", C.c_int),
                ("f", C.c_int), ("newton_warmup", C.c_int), ("max_iters", C.c_int),
                ("check_in_loop", C.c_int), ("flags", C.c_int), ("pad_", C.c_int),
                ("eps_target", C.c_double), ("c", C.c_double), ("lambda_min", C.c_double),
                ("lambda_max", C.c_double),
                ("res_hist", C.POINTER(C.c_double)), ("res_hist_cap", C.c_int), ("pad2_", C.c_int),
                ("block_hist", C.POINTER(ascg_block_info)), ("block_hist_cap", C.c_int), ("pad3_", C.c_int),
                ("alpha_hist", C.POINTER(C.c_double)), ("beta_hist", C.POINTER(C.c_double)),
                ("coef_hist_cap", C.c_int), ("pad4_", C.c_int),
                ("s_seq", C.POINTER(C.c_int)), ("s_seq_len", C.c_int), ("pad5_", C.c_int),
                ("kappa_A", C.c_double), ("norm_A", C.c_double), ("tc_lane_rows", C.c_int64)]


class ascg_result(C.Structure):
    _fields_ = [("status", C.c_int), ("iters", C.c_int), ("blocks", C.c_int), ("grid_reductions", C.c_int),
                ("wasted_vecs", C.c_int), ("launches", C.c_int), ("bnorm", C.c_double),
                ("rel_res_updated", C.c_double), ("rel_res_true", C.c_double),
                ("t_total_ms", C.c_double), ("t_mpk_ms", C.c_double), ("t_gram_ms", C.c_double),
                ("t_ctrl_ms", C.c_double), ("t_recover_ms", C.c_double), ("t_cg_ms", C.c_double),
                ("gram_launches", C.c_int), ("mpk_launches", C.c_int), ("gram_flops", C.c_double),
                ("gram_bytes", C.c_double), ("mpk_flops", C.c_double), ("mpk_bytes", C.c_double),
                ("recover_flops", C.c_double), ("recover_bytes", C.c_double)]


class ascg_completion(C.Structure):
    _fields_ = [("tag", C.c_int64), ("result", ascg_result), ("queue_ms", C.c_double), ("latency_ms", C.c_double),
                ("step_admitted", C.c_int64), ("step_done", C.c_int64)]


class ascg_server_stats(C.Structure):
    _fields_ = [("budget_bytes", C.c_int64), ("basis_bytes_total", C.c_int64), ("basis_bytes_used", C.c_int64),
                ("systems_running", C.c_int), ("max_systems", C.c_int), ("queued", C.c_int64),
                ("completions_pending", C.c_int64), ("steps", C.c_int64), ("launches", C.c_int64)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"libascg.so not found at {LIB_PATH}; build it with "
            "`python -m paper_1701_03989_gb300.build` (there is no CPU fallback)")
    lib = C.CDLL(LIB_PATH)
    P = C.c_void_p
    I64 = C.c_int64
    sig = {
        "ascg_options_default": (C.c_int, [C.POINTER(ascg_options)]),
        "ascg_op_create_csr": (C.c_int, [I64, I64, P, P, P, C.c_int, C.POINTER(P)]),
        "ascg_op_destroy": (C.c_int, [P]),
        "ascg_op_size": (C.c_int, [P, C.POINTER(I64), C.POINTER(I64)]),
        "ascg_solve": (C.c_int, [P, P, P, C.POINTER(ascg_options), C.POINTER(ascg_result), P]),
        "ascg_solve_host": (C.c_int, [P, P, P, C.POINTER(ascg_options), C.POINTER(ascg_result), P]),
        "ascg_solve_batch": (C.c_int, [C.c_int, C.POINTER(P), C.POINTER(P), C.POINTER(P), P,
                                       C.POINTER(ascg_options), C.POINTER(ascg_result), P]),
        "ascg_spmv": (C.c_int, [P, P, P, P]),
        "ascg_matrix_powers": (C.c_int, [P, C.c_int, P, P, P, P, I64, P]),
        "ascg_gram": (C.c_int, [I64, C.c_int, P, I64, P, P]),
        "ascg_gram_noalloc": (C.c_int, [I64, C.c_int, P, I64, P, P]),
        "ascg_gram_moments": (C.c_int, [I64, C.c_int, P, I64, P, P]),
        "ascg_block_step": (C.c_int, [C.c_int, P, C.c_int, P, P, P, I64, C.c_double, C.c_double, C.c_int,
                                      C.c_int, C.c_double, P, C.POINTER(ascg_block_info), P, P]),
        "ascg_recover": (C.c_int, [I64, C.c_int, P, I64, P, P, P, P, P]),
        "ascg_recover_tc": (C.c_int, [I64, C.c_int, P, I64, P, P, P, P, P]),
        "ascg_newton_shifts": (C.c_int, [P, P, C.c_int, C.c_int, P, P]),
        "ascg_server_create": (C.c_int, [C.POINTER(ascg_options), I64, C.c_int, P, C.POINTER(P)]),
        "ascg_server_submit": (C.c_int, [P, P, P, P, C.c_double, I64]),
        "ascg_server_step": (C.c_int, [P, C.POINTER(ascg_completion), C.c_int, C.POINTER(C.c_int),
                                       C.POINTER(C.c_int), C.POINTER(C.c_int)]),
        "ascg_server_info": (C.c_int, [P, C.POINTER(ascg_server_stats)]),
        "ascg_server_set_policy": (C.c_int, [P, C.c_int, C.c_int, C.c_int]),
        "ascg_server_destroy": (C.c_int, [P]),
        "ascg_tune_gram_schedule": (C.c_int, [C.c_int, C.POINTER(I64), P, C.c_int, C.POINTER(C.c_int), P]),
        "ascg_last_error": (C.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_lib = _load()


class AscgError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {last_error()}")


def _ptr(a):
    """Raw address of an array-like: int, numpy array, or object with data_ptr()."""
    if a is None:
        return None
    if isinstance(a, int):
        return a
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    raise TypeError(f"cannot take the address of {type(a)}")


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream  # torch.cuda.Stream


def _check(status, where, ok=(ASCG_OK,)):
    if status not in ok:
        raise AscgError(status, where)
    return status


def last_error() -> str:
    return _lib.ascg_last_error().decode()


def ascg_options_default() -> ascg_options:
    o = ascg_options()
    _check(_lib.ascg_options_default(C.byref(o)), "ascg_options_default")
    return o


def ascg_op_create_csr(n, nnz, rowptr, colind, val, on_device=0):
    """Returns an opaque operator handle (int). rowptr int64, colind int32, val float64."""
    h = C.c_void_p()
    _check(_lib.ascg_op_create_csr(int(n), int(nnz), _ptr(rowptr), _ptr(colind), _ptr(val), int(on_device),
                                   C.byref(h)), "ascg_op_create_csr")
    return h.value


def ascg_op_destroy(op):
    _check(_lib.ascg_op_destroy(op), "ascg_op_destroy")


def ascg_op_size(op):
    n, nnz = C.c_int64(), C.c_int64()
    _check(_lib.ascg_op_size(op, C.byref(n), C.byref(nnz)), "ascg_op_size")
    return n.value, nnz.value


def ascg_solve(op, b, x, opts=None, stream=None, raise_on=(ASCG_OK, ASCG_NOT_CONVERGED)):
    """b, x: device arrays. Returns the ascg_result struct."""
    res = ascg_result()
    st = _lib.ascg_solve(op, _ptr(b), _ptr(x), C.byref(opts) if opts is not None else None, C.byref(res),
                         _stream(stream))
    _check(st, "ascg_solve", raise_on)
    return res


def ascg_solve_batch(ops, bs, xs, opts, eps_targets=None, stream=None,
                     raise_on=(ASCG_OK, ASCG_NOT_CONVERGED, ASCG_ERR_BREAKDOWN)):
    """ops: list of operators; bs, xs: lists of device arrays (x: start in, solution
    out); eps_targets: per-system relative targets or None. Returns the list of
    per-system ascg_result structs and the call's status."""
    count = len(ops)
    if not (len(bs) == len(xs) == count) or count < 1:
        raise ValueError("ops, bs and xs must have the same positive length")
    oa = (C.c_void_p * count)(*[C.c_void_p(o) if isinstance(o, int) else o for o in ops])
    ba = (C.c_void_p * count)(*[_ptr(b) for b in bs])
    xa = (C.c_void_p * count)(*[_ptr(x) for x in xs])
    eps = None
    if eps_targets is not None:
        eps_arr = np.ascontiguousarray(np.asarray(eps_targets, dtype=np.float64))
        if eps_arr.shape != (count,):
            raise ValueError("eps_targets must have one entry per system")
        eps = eps_arr.ctypes.data
    res = (ascg_result * count)()
    st = _lib.ascg_solve_batch(count, oa, ba, xa, eps, C.byref(opts), res, _stream(stream))
    _check(st, "ascg_solve_batch", raise_on)
    return list(res), st


def ascg_server_create(opts, hbm_budget, max_systems, stream=None):
    """A solve server (continuous batching); returns its handle."""
    h = C.c_void_p()
    _check(_lib.ascg_server_create(C.byref(opts), int(hbm_budget), int(max_systems), _stream(stream), C.byref(h)),
           "ascg_server_create")
    return h.value


def ascg_server_submit(srv, op, b, x, eps_target, tag):
    """Queues A x = b (device arrays; x holds x_1 and receives the solution)."""
    _check(_lib.ascg_server_submit(srv, op, _ptr(b), _ptr(x), float(eps_target), int(tag)), "ascg_server_submit")


def ascg_server_step(srv, cap=64):
    """One server step. Returns (completions, nactive, npending)."""
    buf = (ascg_completion * max(int(cap), 1))()
    nd, na, npd = C.c_int(), C.c_int(), C.c_int()
    _check(_lib.ascg_server_step(srv, buf, int(cap), C.byref(nd), C.byref(na), C.byref(npd)), "ascg_server_step")
    return [buf[i] for i in range(nd.value)], na.value, npd.value


ASCG_ADMIT_FIFO, ASCG_ADMIT_SHORTEST_FIRST = 0, 1


def ascg_server_set_policy(srv, admit_order, large_class_cap=0, yield_large=False):
    _check(_lib.ascg_server_set_policy(srv, int(admit_order), int(large_class_cap), 1 if yield_large else 0),
           "ascg_server_set_policy")


def ascg_server_info(srv):
    st = ascg_server_stats()
    _check(_lib.ascg_server_info(srv, C.byref(st)), "ascg_server_info")
    return st


def ascg_tune_gram_schedule(s_max, stream=None):
    """Measured Gram schedule threshold for batched solves: returns (tc_lane_rows,
    table as a list of (n, fp64_us, tensor_us))."""
    thr = C.c_int64()
    buf = np.zeros((16, 3))
    rows = C.c_int()
    _check(_lib.ascg_tune_gram_schedule(int(s_max), C.byref(thr), buf.ctypes.data, 16, C.byref(rows), _stream(stream)),
           "ascg_tune_gram_schedule")
    return thr.value, [tuple(buf[i]) for i in range(rows.value)]


def ascg_server_destroy(srv):
    _check(_lib.ascg_server_destroy(srv), "ascg_server_destroy")


def ascg_solve_host(op, b, x, opts=None, stream=None, raise_on=(ASCG_OK, ASCG_NOT_CONVERGED)):
    """b, x: host arrays (x holds x_1 and receives the solution)."""
    res = ascg_result()
    st = _lib.ascg_solve_host(op, _ptr(b), _ptr(x), C.byref(opts) if opts is not None else None, C.byref(res),
                              _stream(stream))
    _check(st, "ascg_solve_host", raise_on)
    return res


def ascg_spmv(op, x, y, stream=None):
    _check(_lib.ascg_spmv(op, _ptr(x), _ptr(y), _stream(stream)), "ascg_spmv")


def ascg_matrix_powers(op, s, theta, sigma, gamma, Y, ldY, stream=None):
    th = np.ascontiguousarray(theta, dtype=np.float64)
    sg = np.ascontiguousarray(sigma, dtype=np.float64)
    gm = np.ascontiguousarray(gamma, dtype=np.float64)
    _check(_lib.ascg_matrix_powers(op, int(s), _ptr(th), _ptr(sg), _ptr(gm), _ptr(Y), int(ldY), _stream(stream)),
           "ascg_matrix_powers")


def ascg_gram(n, w, Y, ldY, G, stream=None):
    _check(_lib.ascg_gram(int(n), int(w), _ptr(Y), int(ldY), _ptr(G), _stream(stream)), "ascg_gram")


def ascg_gram_moments(n, s, Y, ldY, G, stream=None):
    """Gram matrix of a monomial basis of size s from its 6s moments (see include/ascg.h)."""
    _check(_lib.ascg_gram_moments(int(n), int(s), _ptr(Y), int(ldY), _ptr(G), _stream(stream)), "ascg_gram_moments")


def ascg_gram_noalloc(n, w, Y, ldY, G, stream=None):
    """As ascg_gram, but with no device allocation (static scratch; see include/ascg.h).
    Enqueues only: synchronise the stream before reading G."""
    _check(_lib.ascg_gram_noalloc(int(n), int(w), _ptr(Y), int(ldY), _ptr(G), _stream(stream)),
           "ascg_gram_noalloc")


def ascg_block_step(sbar, G, method, theta, sigma, gamma, nrows, eps_star, c, check_in_loop, max_steps, bnorm,
                    coords, stream=None):
    """Returns (ascg_block_info, hist ndarray [s_k, 3] of alpha, beta, relres)."""
    th = np.ascontiguousarray(theta, dtype=np.float64)
    sg = np.ascontiguousarray(sigma, dtype=np.float64)
    gm = np.ascontiguousarray(gamma, dtype=np.float64)
    info = ascg_block_info()
    hist = np.zeros(3 * ASCG_MAX_S)
    _check(_lib.ascg_block_step(int(sbar), _ptr(G), int(method), _ptr(th), _ptr(sg), _ptr(gm), int(nrows),
                                float(eps_star), float(c), int(check_in_loop), int(max_steps), float(bnorm),
                                _ptr(coords), C.byref(info), _ptr(hist), _stream(stream)), "ascg_block_step")
    return info, hist[: 3 * max(info.s_k, 0)].reshape(-1, 3)


def ascg_recover(n, w, Y, ldY, coords, x, r, p, stream=None):
    _check(_lib.ascg_recover(int(n), int(w), _ptr(Y), int(ldY), _ptr(coords), _ptr(x), _ptr(r), _ptr(p),
                             _stream(stream)), "ascg_recover")


def ascg_recover_tc(n, w, Y, ldY, coords, x, r, p, stream=None):
    _check(_lib.ascg_recover_tc(int(n), int(w), _ptr(Y), int(ldY), _ptr(coords), _ptr(x), _ptr(r), _ptr(p),
                                _stream(stream)), "ascg_recover_tc")


def ascg_newton_shifts(alphas, betas, k, s, stream=None):
    al = np.ascontiguousarray(alphas, dtype=np.float64)
    be = np.ascontiguousarray(betas if len(betas) else [0.0], dtype=np.float64)
    out = np.zeros(s)
    _check(_lib.ascg_newton_shifts(_ptr(al), _ptr(be), int(k), int(s), _ptr(out), _stream(stream)),
           "ascg_newton_shifts")
    return out


# --- convenience: options from keywords -------------------------------------

_METHODS = {"classical": ASCG_CLASSICAL, "fixed": ASCG_FIXED_S, "adaptive": ASCG_ADAPTIVE,
            "variable": ASCG_VARIABLE_S}
_BASES = {"monomial": ASCG_MONOMIAL, "newton": ASCG_NEWTON, "chebyshev": ASCG_CHEBYSHEV}


def make_options(method="adaptive", basis="monomial", s_max=8, s0=None, f=None, eps_target=1e-10, c=1.0,
                 lam=None, newton_warmup=0, max_iters=100000, check_in_loop=True, timing=False,
                 res_hist=None, block_hist=None, alpha_hist=None, beta_hist=None,
                 gram_fp64=False, s_seq=None, c_formula=None, moment_gram=False,
                 tc_lane_rows=0, test_gram_stall=False, gram_tc=False, recover_fp64=False) -> ascg_options:
    """ascg_options filled from keywords. History arrays are numpy (float64) or a
    ctypes array of ascg_block_info; the caller keeps them alive for the call.
    s_seq (method "variable"): the block sizes s_0, s_1, ... (the last repeats);
    the options object keeps its own copy alive. c_formula = (kappa(A), ||A||):
    c_{k,j} = 6 N_k j kappa(A) instead of the constant c. moment_gram: G from
    the monomial basis' moments (ascg_gram_moments). recover_fp64: the recovery by
    FP64 FMAs even where the Gram took the tensor cores."""
    o = ascg_options_default()
    o.method = _METHODS[method] if isinstance(method, str) else int(method)
    o.basis = _BASES[basis] if isinstance(basis, str) else int(basis)
    o.s_max = int(s_max)
    o.s0 = int(s_max if s0 is None else s0)
    o.f = int(s_max if f is None else f)
    o.eps_target = float(eps_target)
    o.c = float(c)
    if lam is not None:
        o.lambda_min, o.lambda_max = float(lam[0]), float(lam[1])
    o.newton_warmup = int(newton_warmup)
    o.max_iters = int(max_iters)
    o.check_in_loop = 1 if check_in_loop else 0
    o.flags = (ASCG_FLAG_TIMING if timing else 0) | (ASCG_FLAG_GRAM_FP64 if gram_fp64 else 0)
    o.tc_lane_rows = int(tc_lane_rows)
    if moment_gram:
        o.flags |= ASCG_FLAG_MOMENT_GRAM
    if test_gram_stall:
        o.flags |= ASCG_FLAG_TEST_GRAM_STALL
    if gram_tc:
        o.flags |= ASCG_FLAG_GRAM_TC
    if recover_fp64:
        o.flags |= ASCG_FLAG_RECOVER_FP64
    if c_formula is not None:
        o.flags |= ASCG_FLAG_C_FORMULA
        o.kappa_A, o.norm_A = float(c_formula[0]), float(c_formula[1])
    if res_hist is not None:
        o.res_hist = res_hist.ctypes.data_as(C.POINTER(C.c_double))
        o.res_hist_cap = len(res_hist)
    if block_hist is not None:
        o.block_hist = C.cast(block_hist, C.POINTER(ascg_block_info))
        o.block_hist_cap = len(block_hist)
    if alpha_hist is not None and beta_hist is not None:
        o.alpha_hist = alpha_hist.ctypes.data_as(C.POINTER(C.c_double))
        o.beta_hist = beta_hist.ctypes.data_as(C.POINTER(C.c_double))
        o.coef_hist_cap = min(len(alpha_hist), len(beta_hist))
    if s_seq is not None:
        arr = (C.c_int * len(s_seq))(*[int(v) for v in s_seq])
        o._s_seq_keep = arr
        o.s_seq = C.cast(arr, C.POINTER(C.c_int))
        o.s_seq_len = len(s_seq)
    return o


def block_infos(count: int):
    """A ctypes array of ascg_block_info for options.block_hist."""
    return (ascg_block_info * count)()


EXPORTED = ["ascg_options_default", "ascg_op_create_csr", "ascg_op_destroy", "ascg_op_size", "ascg_solve",
            "ascg_solve_host", "ascg_solve_batch", "ascg_spmv", "ascg_matrix_powers", "ascg_gram", "ascg_gram_noalloc", "ascg_gram_moments",
            "ascg_block_step", "ascg_recover", "ascg_recover_tc",
            "ascg_newton_shifts", "ascg_server_create", "ascg_server_submit", "ascg_server_step",
            "ascg_server_info", "ascg_server_set_policy", "ascg_server_destroy", "ascg_tune_gram_schedule",
            "ascg_last_error"]
