"""ctypes binding of libfde (include/fde.h): argument marshalling only.

Every function here has the name of the C entry point it calls and forwards
its arguments.  Device arrays are passed as torch CUDA tensors (float64,
contiguous, n2 x n1 or flat) and handed to C as raw pointers; PyTorch only
provides the memory and the stream.  There is no CPU fallback: if
``libfde.so`` is missing or fails to load, ``lib()`` raises.
"""
import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfde.so")

FDE_OK, FDE_ERR_ARG, FDE_ERR_NOT_CONVERGED, FDE_ERR_NONFINITE = 0, 1, 2, 3
FDE_ERR_CUDA, FDE_ERR_TIMEOUT, FDE_ERR_UNSUPPORTED = 4, 5, 6
FDE_PRECOND_NONE, FDE_PRECOND_MG_SG, FDE_PRECOND_MG_REDISC, FDE_PRECOND_P2 = 0, 1, 2, 3
FDE_PRECOND_MG_EXACT = 4
FDE_PREC_FP64, FDE_PREC_FP32, FDE_PREC_BF16, FDE_PREC_FP16, FDE_PREC_BF16X3 = 0, 1, 2, 3, 4
FDE_PATH_AUTO, FDE_PATH_GEMM, FDE_PATH_FFT, FDE_PATH_DIRECT, FDE_PATH_TUNE = 0, 1, 2, 3, 4
FDE_OUTER_FP64, FDE_OUTER_DF32 = 0, 1
FDE_SOLVER_FGMRES, FDE_SOLVER_MG = 0, 1
FDE_COEF_NEW, FDE_COEF_OLD = 0, 1
FDE_KCLASS_OUTER_APPLY, FDE_KCLASS_LEVEL_APPLY, FDE_KCLASS_KRYLOV, FDE_KCLASS_MG_OTHER = 0, 1, 2, 3
FDE_KCLASS_OUTER_FP32, FDE_KCLASS_TC_GEMM, FDE_KCLASS_COUNT = 4, 5, 6


class fde_params(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_double), ("beta", ctypes.c_double),
                ("qx", ctypes.c_int), ("qy", ctypes.c_int),
                ("a1", ctypes.c_double), ("b1", ctypes.c_double),
                ("a2", ctypes.c_double), ("b2", ctypes.c_double),
                ("n1", ctypes.c_int), ("n2", ctypes.c_int),
                ("dt", ctypes.c_double), ("rtol", ctypes.c_double),
                ("restart", ctypes.c_int), ("maxit", ctypes.c_int),
                ("precond", ctypes.c_int), ("nu_pre", ctypes.c_int), ("nu_post", ctypes.c_int),
                ("omega", ctypes.c_double), ("coarsest_n", ctypes.c_int),
                ("precision", ctypes.c_int), ("toeplitz_path", ctypes.c_int),
                ("outer", ctypes.c_int), ("cycles", ctypes.c_int), ("relax", ctypes.c_int),
                ("solver", ctypes.c_int), ("warm", ctypes.c_int)]


class fde_stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("restarts", ctypes.c_int),
                ("converged", ctypes.c_int), ("rel_residual", ctypes.c_double),
                ("relaxed", ctypes.c_int)]


_lib = None
_VP, _DP, _IP = ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)

# C entry points: name -> (restype, argtypes)
SIGNATURES = {
    "fde_default_params": (None, [ctypes.POINTER(fde_params)]),
    "fde_create": (ctypes.c_int, [ctypes.POINTER(fde_params), _VP, ctypes.POINTER(_VP)]),
    "fde_destroy": (None, [_VP]),
    "fde_last_error": (ctypes.c_char_p, [_VP]),
    "fde_set_coefficients": (ctypes.c_int, [_VP, ctypes.c_int, _DP, _DP, _DP, _DP]),
    "fde_rhs": (ctypes.c_int, [_VP, _DP, _DP, _DP]),
    "fde_apply": (ctypes.c_int, [_VP, _DP, _DP]),
    "fde_vcycle": (ctypes.c_int, [_VP, _DP, _DP]),
    "fde_level_apply": (ctypes.c_int, [_VP, ctypes.c_int, _DP, _DP]),
    "fde_levels": (ctypes.c_int, [_VP, _IP, _IP, _IP]),
    "fde_level_path": (ctypes.c_int, [_VP, ctypes.c_int]),
    "fde_weights": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.c_int]),
    "fde_solve": (ctypes.c_int, [_VP, _DP, _DP, ctypes.POINTER(fde_stats)]),
    "fde_step": (ctypes.c_int, [_VP, _DP, _DP, _DP, ctypes.POINTER(fde_stats)]),
    "fde_step_host": (ctypes.c_int, [_VP, _DP, _DP, _DP, ctypes.POINTER(fde_stats)]),
    "fde_get_state": (ctypes.c_int, [_VP, _IP, _DP]),
    "fde_set_state": (ctypes.c_int, [_VP, ctypes.c_int]),
    "fde_wait_selftest": (ctypes.c_int, [_VP, ctypes.c_int]),
    "fde_conversion_selftest": (ctypes.c_int, [ctypes.c_longlong, ctypes.POINTER(ctypes.c_longlong)]),
    "fde_profile_enable": (ctypes.c_int, [_VP, ctypes.c_int]),
    "fde_profile_query": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.POINTER(ctypes.c_longlong),
                                         ctypes.POINTER(ctypes.c_double)]),
    "fde_launch_count": (ctypes.c_longlong, [_VP]),
    "fde_apply_noalloc": (ctypes.c_int, [ctypes.POINTER(fde_params), _DP, _DP, _DP, _DP, _DP,
                                         _DP, _VP]),
    "fde_batch_create": (ctypes.c_int, [ctypes.POINTER(fde_params), ctypes.c_int, _VP,
                                        ctypes.POINTER(_VP)]),
    "fde_batch_destroy": (None, [_VP]),
    "fde_batch_size": (ctypes.c_int, [_VP]),
    "fde_batch_handle": (_VP, [_VP, ctypes.c_int]),
    "fde_batch_step": (ctypes.c_int, [_VP, ctypes.POINTER(_VP), ctypes.POINTER(_VP),
                                      ctypes.POINTER(_VP), ctypes.POINTER(fde_stats)]),
    "fde_batch_status": (ctypes.c_int, [_VP, ctypes.c_int]),
    "fde_batch_engine": (ctypes.c_int, [_VP]),
    "fde_batch_engine_note": (ctypes.c_char_p, [_VP]),
    "fde_batch_launch_count": (ctypes.c_longlong, [_VP]),
}


def lib():
    """Load libfde.so (raises OSError if it is missing: there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise OSError(f"{LIB_PATH} is missing: run __graft_entry__.build() first")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype, f.argtypes = res, args
        _lib = L
    return _lib


class FDEError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libfde status {code}: {msg}")
        self.code = code


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if hasattr(t, "data_ptr"):
        if t.is_cuda:
            assert t.is_contiguous(), "device arrays must be contiguous"
        return t.data_ptr()
    if hasattr(t, "ctypes"):  # numpy (host arrays for the *_host calls)
        return t.ctypes.data
    raise TypeError(type(t))


def _check(h, rc, ok=(FDE_OK,)):
    if rc not in ok:
        raise FDEError(rc, fde_last_error(h))
    return rc


# ---------------------------------------------------------------- same names as C

def fde_default_params():
    p = fde_params()
    lib().fde_default_params(ctypes.byref(p))
    return p


def fde_create(params, stream=0):
    h = _VP()
    rc = lib().fde_create(ctypes.byref(params), ctypes.c_void_p(stream), ctypes.byref(h))
    if rc != FDE_OK:
        raise FDEError(rc, lib().fde_last_error(None).decode())
    return h


def fde_destroy(h):
    lib().fde_destroy(h)


def fde_last_error(h):
    m = lib().fde_last_error(h)
    return m.decode() if m else ""


def fde_set_coefficients(h, which, dp, dm, ep, em):
    return _check(h, lib().fde_set_coefficients(h, which, _ptr(dp), _ptr(dm), _ptr(ep), _ptr(em)))


def fde_rhs(h, u_prev, v_half, b):
    return _check(h, lib().fde_rhs(h, _ptr(u_prev), _ptr(v_half), _ptr(b)))


def fde_apply(h, x, y):
    return _check(h, lib().fde_apply(h, _ptr(x), _ptr(y)))


def fde_vcycle(h, r, z):
    return _check(h, lib().fde_vcycle(h, _ptr(r), _ptr(z)))


def fde_level_apply(h, level, x, y):
    return _check(h, lib().fde_level_apply(h, level, _ptr(x), _ptr(y)))


def fde_levels(h):
    n = ctypes.c_int()
    lib().fde_levels(h, ctypes.byref(n), None, None)
    a = (ctypes.c_int * n.value)()
    b = (ctypes.c_int * n.value)()
    _check(h, lib().fde_levels(h, None, a, b))
    return list(zip(list(a), list(b)))


def fde_weights(h, axis, count):
    buf = (ctypes.c_double * count)()
    _check(h, lib().fde_weights(h, axis, buf, count))
    return list(buf)


def fde_solve(h, b, x, allow_not_converged=False):
    st = fde_stats()
    ok = (FDE_OK, FDE_ERR_NOT_CONVERGED) if allow_not_converged else (FDE_OK,)
    _check(h, lib().fde_solve(h, _ptr(b), _ptr(x), ctypes.byref(st)), ok)
    return st


def fde_step(h, u_prev, v_half, u_next, allow_not_converged=False):
    st = fde_stats()
    ok = (FDE_OK, FDE_ERR_NOT_CONVERGED) if allow_not_converged else (FDE_OK,)
    _check(h, lib().fde_step(h, _ptr(u_prev), _ptr(v_half), _ptr(u_next), ctypes.byref(st)), ok)
    return st


def fde_step_host(h, u_prev, v_half, u_next, allow_not_converged=False):
    st = fde_stats()
    ok = (FDE_OK, FDE_ERR_NOT_CONVERGED) if allow_not_converged else (FDE_OK,)
    _check(h, lib().fde_step_host(h, _ptr(u_prev), _ptr(v_half), _ptr(u_next),
                                  ctypes.byref(st)), ok)
    return st


def fde_get_state(h, u_out=None):
    m = ctypes.c_int()
    _check(h, lib().fde_get_state(h, ctypes.byref(m), _ptr(u_out)))
    return m.value


def fde_set_state(h, m):
    return _check(h, lib().fde_set_state(h, m))


def fde_wait_selftest(h, complete):
    return _check(h, lib().fde_wait_selftest(h, int(complete)))


def fde_conversion_selftest(n):
    bad = ctypes.c_longlong()
    _check(None, lib().fde_conversion_selftest(int(n), ctypes.byref(bad)))
    return bad.value


def fde_profile_enable(h, on):
    return _check(h, lib().fde_profile_enable(h, 1 if on else 0))


def fde_profile_query(h, kclass):
    n, ms = ctypes.c_longlong(), ctypes.c_double()
    _check(h, lib().fde_profile_query(h, kclass, ctypes.byref(n), ctypes.byref(ms)))
    return n.value, ms.value


def fde_launch_count(h):
    return lib().fde_launch_count(h)


def fde_apply_noalloc(params, dp, dm, ep, em, x, y, stream=0):
    rc = lib().fde_apply_noalloc(ctypes.byref(params), _ptr(dp), _ptr(dm), _ptr(ep), _ptr(em),
                                 _ptr(x), _ptr(y), ctypes.c_void_p(stream))
    if rc != FDE_OK:
        raise FDEError(rc, fde_last_error(None))
    return rc


# ---------------------------------------------------------------- convenience

def params(**kw):
    """fde_params with defaults overridden by keyword arguments."""
    p = fde_default_params()
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


# ---------------------------------------------------------------- batches

def fde_batch_create(params_list, stream=0):
    """One batch over a list of fde_params (copied)."""
    n = len(params_list)
    arr = (fde_params * n)(*params_list)
    b = _VP()
    rc = lib().fde_batch_create(arr, n, ctypes.c_void_p(stream), ctypes.byref(b))
    if rc != FDE_OK:
        raise FDEError(rc, lib().fde_last_error(None).decode())
    return b


def fde_batch_destroy(b):
    lib().fde_batch_destroy(b)


def fde_batch_size(b):
    return lib().fde_batch_size(b)


def fde_batch_handle(b, i):
    h = lib().fde_batch_handle(b, i)
    if not h:
        raise FDEError(FDE_ERR_ARG, f"no problem {i} in the batch")
    return _VP(h)


def fde_batch_status(b, i):
    return lib().fde_batch_status(b, i)


def fde_batch_step(b, u_prev, v_half, u_next, allow_not_converged=False):
    """Step every problem: u_prev, v_half, u_next are sequences of device
    arrays (one per problem). Returns the list of fde_stats."""
    n = fde_batch_size(b)
    if not (len(u_prev) == len(v_half) == len(u_next) == n):
        raise FDEError(FDE_ERR_ARG, f"expected {n} arrays per argument")
    P = lambda xs: (_VP * n)(*[_ptr(x) for x in xs])
    st = (fde_stats * n)()
    rc = lib().fde_batch_step(b, P(u_prev), P(v_half), P(u_next), st)
    ok = (FDE_OK, FDE_ERR_NOT_CONVERGED) if allow_not_converged else (FDE_OK,)
    if rc not in ok:
        raise FDEError(rc, lib().fde_last_error(None).decode())
    return list(st)


def fde_level_path(h, level):
    return lib().fde_level_path(h, level)


def fde_batch_engine(b):
    return lib().fde_batch_engine(b)


def fde_batch_engine_note(b):
    m = lib().fde_batch_engine_note(b)
    return m.decode() if m else ""


def fde_batch_launch_count(b):
    return lib().fde_batch_launch_count(b)
