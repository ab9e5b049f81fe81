"""ctypes binding of ``libsvgp.so`` (the C-ABI declared in include/svgp.h).

Argument marshalling only: every computation runs in the CUDA library.  Device
tensors are passed as raw pointers (``tensor.data_ptr()``).  Loading fails
loudly when the library has not been built; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, byref, c_char_p, c_double, c_float, c_int, c_void_p

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsvgp.so")

SVGP_OK = 0
SVGP_ERR_INVALID_ARG = 1
SVGP_ERR_CUDA = 2
SVGP_ERR_OOM = 3
SVGP_ERR_NONFINITE = 4
SVGP_ERR_NOT_CONVERGED = 5
SVGP_ERR_TIMEOUT = 6
SVGP_ERR_UNSUPPORTED = 7

SVGP_LIK_GAUSSIAN = 0
SVGP_LIK_BERNOULLI_PROBIT = 1
SVGP_FP32 = 0
SVGP_BF16 = 1
SVGP_BF16X3 = 2
SVGP_BF16X3K = 3

TERMS = ["F", "E", "KL", "trKT", "trPKuu", "quad", "logdetT", "sqerr", "sumvar", "logdetS", "nclamp"]
SVGP_NTERMS = len(TERMS)

EXPORTED = [
    "svgp_create", "svgp_destroy", "svgp_set_stream", "svgp_bound", "svgp_backward",
    "svgp_ng_update_T", "svgp_train_step", "svgp_predict", "svgp_adam_step", "svgp_param_count",
    "svgp_sync_status", "svgp_last_error", "svgp_status_string", "svgp_has_tensor_cores",
    "svgp_gauss_hermite", "svgp_variance_gap", "svgp_ng_update_T_gap", "svgp_bound_hutchinson",
]


class svgp_config(ctypes.Structure):
    _fields_ = [("M", c_int), ("D", c_int), ("B_max", c_int), ("lik", c_int), ("prec", c_int),
                ("cuda_stream", c_void_p), ("gh_points", c_int), ("unpreconditioned", c_int)]


class svgp_params(ctypes.Structure):
    _fields_ = [(n, c_void_p) for n in ("Z", "ell", "sf2", "noise", "m", "s", "L")]


class svgp_batch(ctypes.Structure):
    _fields_ = [("X", c_void_p), ("y", c_void_p), ("B", c_int), ("N", c_double)]


class svgp_grads(ctypes.Structure):
    _fields_ = [(n, c_void_p) for n in ("dZ", "dell", "dsf2", "dnoise", "dm", "ds")]


class SvgpError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"svgp status {status}: {msg}")
        self.status = status


_lib = None


def load(path: str = LIB_PATH):
    """Load the shared library (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} not found: build it with `python -m paper_2604_00697_gb300.build` "
                           "(there is no CPU fallback)")
    lib = ctypes.CDLL(path)
    H = c_void_p
    lib.svgp_create.argtypes = [POINTER(svgp_config), POINTER(H)]
    lib.svgp_destroy.argtypes = [H]
    lib.svgp_destroy.restype = None
    lib.svgp_set_stream.argtypes = [H, c_void_p]
    lib.svgp_bound.argtypes = [H, POINTER(svgp_params), POINTER(svgp_batch), c_void_p]
    lib.svgp_backward.argtypes = [H, POINTER(svgp_params), POINTER(svgp_batch), c_void_p, POINTER(svgp_grads)]
    lib.svgp_ng_update_T.argtypes = [H, POINTER(svgp_params), c_void_p, c_void_p, c_int, c_double, c_void_p,
                                     c_void_p]
    lib.svgp_train_step.argtypes = [H, POINTER(svgp_params), POINTER(svgp_batch), c_void_p, c_void_p, c_int,
                                    c_double, c_void_p, c_void_p, c_void_p, POINTER(svgp_grads)]
    lib.svgp_predict.argtypes = [H, POINTER(svgp_params), c_void_p, c_int, c_void_p, c_void_p, c_int]
    lib.svgp_adam_step.argtypes = [H, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                   c_void_p]
    lib.svgp_param_count.argtypes = [H]
    lib.svgp_param_count.restype = c_int
    lib.svgp_sync_status.argtypes = [H]
    lib.svgp_last_error.argtypes = [H]
    lib.svgp_last_error.restype = c_char_p
    lib.svgp_status_string.argtypes = [c_int]
    lib.svgp_status_string.restype = c_char_p
    lib.svgp_has_tensor_cores.argtypes = []
    lib.svgp_has_tensor_cores.restype = c_int
    lib.svgp_gauss_hermite.argtypes = [c_int, POINTER(c_double), POINTER(c_double)]
    lib.svgp_variance_gap.argtypes = [H, POINTER(svgp_params), POINTER(svgp_batch), c_double, c_void_p]
    lib.svgp_bound_hutchinson.argtypes = [H, POINTER(svgp_params), POINTER(svgp_batch), c_void_p, c_int, c_void_p]
    lib.svgp_ng_update_T_gap.argtypes = [H, POINTER(svgp_params), POINTER(svgp_batch), c_void_p, c_void_p, c_int,
                                         c_double, c_double, c_void_p, c_void_p]
    lib.svgp_gauss_hermite.restype = c_int
    for name in ("svgp_create", "svgp_set_stream", "svgp_bound", "svgp_backward", "svgp_ng_update_T",
                 "svgp_train_step", "svgp_predict", "svgp_adam_step", "svgp_sync_status", "svgp_variance_gap",
                 "svgp_ng_update_T_gap", "svgp_bound_hutchinson"):
        getattr(lib, name).restype = c_int
    _lib = lib
    return lib


def _check(h, status):
    if status != SVGP_OK:
        lib = load()
        msg = lib.svgp_last_error(h).decode() if h else lib.svgp_status_string(status).decode()
        raise SvgpError(status, msg or lib.svgp_status_string(status).decode())


def svgp_create(M, D, B_max, prec=SVGP_BF16, lik=SVGP_LIK_GAUSSIAN, cuda_stream=None, gh_points=0,
                unpreconditioned=False):
    lib = load()
    cfg = svgp_config(M, D, B_max, lik, prec, cuda_stream, gh_points, int(bool(unpreconditioned)))
    h = c_void_p()
    st = lib.svgp_create(byref(cfg), byref(h))
    if st != SVGP_OK:
        raise SvgpError(st, lib.svgp_status_string(st).decode())
    return h


def svgp_gauss_hermite(n):
    """Nodes and weights (lists of n floats) of the Gauss-Hermite rule for exp(-t^2)."""
    t, w = (c_double * max(n, 1))(), (c_double * max(n, 1))()
    st = load().svgp_gauss_hermite(n, t, w)
    if st != SVGP_OK:
        raise SvgpError(st, "svgp_gauss_hermite: n out of [1, 64]")
    return list(t), list(w)


def svgp_destroy(h):
    load().svgp_destroy(h)


def svgp_set_stream(h, stream_ptr):
    _check(h, load().svgp_set_stream(h, c_void_p(stream_ptr)))


def svgp_bound(h, params, batch, terms_ptr):
    _check(h, load().svgp_bound(h, byref(params), byref(batch), c_void_p(terms_ptr)))


def svgp_backward(h, params, batch, terms_ptr, grads):
    _check(h, load().svgp_backward(h, byref(params), byref(batch), c_void_p(terms_ptr), byref(grads)))


def svgp_ng_update_T(h, params, L_ptr, gamma_ptr, max_iters, eps, iters_ptr=None, resid_ptr=None):
    _check(h, load().svgp_ng_update_T(h, byref(params), c_void_p(L_ptr), c_void_p(gamma_ptr), max_iters,
                                      c_double(eps), c_void_p(iters_ptr), c_void_p(resid_ptr)))


def svgp_train_step(h, params, batch, L_ptr, gamma_ptr, max_iters, eps, iters_ptr, resid_ptr, terms_ptr, grads):
    _check(h, load().svgp_train_step(h, byref(params), byref(batch), c_void_p(L_ptr), c_void_p(gamma_ptr),
                                     max_iters, c_double(eps), c_void_p(iters_ptr), c_void_p(resid_ptr),
                                     c_void_p(terms_ptr), byref(grads)))


SVGP_HUTCH_KMAX = 256


def svgp_bound_hutchinson(h, params, batch, probes_ptr, K, terms_ptr):
    _check(h, load().svgp_bound_hutchinson(h, byref(params), byref(batch), c_void_p(probes_ptr), K,
                                           c_void_p(terms_ptr)))


def svgp_variance_gap(h, params, batch, sigma2, gap_ptr):
    _check(h, load().svgp_variance_gap(h, byref(params), byref(batch), c_double(sigma2), c_void_p(gap_ptr)))


def svgp_ng_update_T_gap(h, params, batch, L_ptr, gamma_ptr, max_iters, eps, sigma2, iters_ptr, gap_ptr):
    _check(h, load().svgp_ng_update_T_gap(h, byref(params), byref(batch), c_void_p(L_ptr), c_void_p(gamma_ptr),
                                          max_iters, c_double(eps), c_double(sigma2), c_void_p(iters_ptr),
                                          c_void_p(gap_ptr)))


def svgp_predict(h, params, Xs_ptr, Ns, mean_ptr, var_ptr, include_noise=False):
    _check(h, load().svgp_predict(h, byref(params), c_void_p(Xs_ptr), Ns, c_void_p(mean_ptr),
                                  c_void_p(var_ptr), int(bool(include_noise))))


def svgp_adam_step(h, raw_ptr, cons_ptr, grad_ptr, m1_ptr, m2_ptr, step_ptr, hyper_ptr, zbeta1_ptr=None):
    _check(h, load().svgp_adam_step(h, c_void_p(raw_ptr), c_void_p(cons_ptr), c_void_p(grad_ptr),
                                    c_void_p(m1_ptr), c_void_p(m2_ptr), c_void_p(step_ptr),
                                    c_void_p(hyper_ptr), c_void_p(zbeta1_ptr)))


def svgp_param_count(h):
    return load().svgp_param_count(h)


def svgp_sync_status(h):
    return load().svgp_sync_status(h)


def svgp_last_error(h):
    return load().svgp_last_error(h).decode()


def svgp_has_tensor_cores():
    return bool(load().svgp_has_tensor_cores())


def svgp_status_string(status):
    return load().svgp_status_string(int(status)).decode()


PROF_KINDS = ["vt", "sym", "lupd", "ls", "out", "psi", "w"]
SVGP_PROF_NKINDS = len(PROF_KINDS)
EXPORTED += ["svgp_profile_enable", "svgp_profile_read"]


def svgp_profile_enable(h, enable=True):
    lib = load()
    lib.svgp_profile_enable.argtypes = [c_void_p, c_int]
    lib.svgp_profile_enable.restype = c_int
    _check(h, lib.svgp_profile_enable(h, int(bool(enable))))


def svgp_profile_read(h):
    """Per-kind (total ms, launch count) over the recorded launches."""
    lib = load()
    lib.svgp_profile_read.argtypes = [c_void_p, POINTER(c_float), POINTER(c_int)]
    lib.svgp_profile_read.restype = c_int
    ms = (c_float * SVGP_PROF_NKINDS)()
    cnt = (c_int * SVGP_PROF_NKINDS)()
    _check(h, lib.svgp_profile_read(h, ms, cnt))
    return {k: (ms[i], cnt[i]) for i, k in enumerate(PROF_KINDS)}


EXPORTED += ["svgp_launch_count"]


def svgp_launch_count(h=None):
    lib = load()
    lib.svgp_launch_count.argtypes = [c_void_p]
    lib.svgp_launch_count.restype = ctypes.c_longlong
    return int(lib.svgp_launch_count(h))


EXPORTED += ["svgp_set_split", "svgp_get_split", "svgp_split_candidates"]


def svgp_set_split(h, kind, kmin):
    """Split-K threshold of a contraction kind (see svgp.h); kind: PROF_KINDS index."""
    lib = load()
    lib.svgp_set_split.argtypes = [c_void_p, c_int, c_int]
    lib.svgp_set_split.restype = c_int
    _check(h, lib.svgp_set_split(h, int(kind), int(kmin)))


def svgp_get_split(h, kind):
    lib = load()
    lib.svgp_get_split.argtypes = [c_void_p, c_int]
    lib.svgp_get_split.restype = c_int
    return int(lib.svgp_get_split(h, int(kind)))


def svgp_split_candidates(h, kind):
    lib = load()
    lib.svgp_split_candidates.argtypes = [c_void_p, c_int, POINTER(c_int), c_int]
    lib.svgp_split_candidates.restype = c_int
    buf = (c_int * 16)()
    n = lib.svgp_split_candidates(h, int(kind), buf, 16)
    return [int(buf[i]) for i in range(min(n, 16))]


EXPORTED += ["svgp_check_wait_timeout"]


def svgp_check_wait_timeout(h):
    """Launch the probe whose bounded device wait runs out (see svgp.h)."""
    lib = load()
    lib.svgp_check_wait_timeout.argtypes = [c_void_p]
    lib.svgp_check_wait_timeout.restype = c_int
    _check(h, lib.svgp_check_wait_timeout(h))


EXPORTED += ["svgp_predict_noalloc"]


def svgp_predict_noalloc(params, M, D, Xs_ptr, Ns, mean_ptr, var_ptr, include_noise=False, cuda_stream=None):
    """Prediction without a handle or any device allocation (fixed scratch)."""
    lib = load()
    fn = lib.svgp_predict_noalloc
    fn.argtypes = [POINTER(svgp_params), c_int, c_int, c_void_p, c_int, c_void_p, c_void_p, c_int, c_void_p]
    fn.restype = c_int
    st = fn(byref(params), M, D, c_void_p(Xs_ptr), Ns, c_void_p(mean_ptr), c_void_p(var_ptr),
            int(bool(include_noise)), c_void_p(cuda_stream))
    if st != SVGP_OK:
        raise SvgpError(st, lib.svgp_status_string(st).decode())
