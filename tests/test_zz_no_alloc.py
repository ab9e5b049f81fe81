"""svgp_predict_noalloc: prediction for callers that cannot allocate device
memory (graph-capturing frameworks, fixed-budget plug-ins).  It must give the
same mean and variance as svgp_predict on an FP32 handle, call after call,
while using only the library's fixed scratch array.

This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes when run alone.
"""
import ctypes

import numpy as np
import pytest

from _helpers import f32, rel, small_case

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _noalloc(lib, params, M, D, Xd, Ns, mean, var, stream):
    fn = lib.svgp_predict_noalloc
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                   ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
    fn.restype = ctypes.c_int
    return fn(ctypes.addressof(params), M, D, Xd.data_ptr(), Ns, mean.data_ptr(), var.data_ptr(), 1, stream)


def test_predict_noalloc_matches_predict_call_after_call():
    """Calls in a row on one device, alternating inducing-point counts whose
    padded sizes differ (M <= 128 and 129..256), each checked against
    svgp_predict on an FP32 handle and against the oracle's predictive
    moments."""
    from oracle import rsvgp as O
    from paper_2604_00697_gb300 import _lib
    from paper_2604_00697_gb300.model import RSVGP

    lib = _lib.load()
    D, Ns = 3, 300
    stream = torch.cuda.current_stream().cuda_stream
    for call, M in enumerate((150, 100, 200, 100, 256)):
        p, _, _, _ = small_case(M, D, 4, 9 + call, state="chol")
        m = RSVGP(M, D, Ns, prec="fp32")
        m.set_state(p["Z"], p["ell"], p["sf2"], p["noise"], p["m"], p["s"], p["L"])
        Xs = f32(np.random.default_rng(40 + call).normal(size=(Ns, D)))
        Xd = torch.tensor(Xs, dtype=torch.float32, device="cuda")
        ref_mean, ref_var = m.predict(Xd, include_noise=True)
        mean = torch.full((Ns,), float("nan"), device="cuda")
        var = torch.full((Ns,), float("nan"), device="cuda")
        st = _noalloc(lib, m.params, M, D, Xd, Ns, mean, var, stream)
        torch.cuda.synchronize()
        assert st == _lib.SVGP_OK
        gm, gv = mean.double().cpu().numpy(), var.double().cpu().numpy()
        assert rel(gm, ref_mean.double().cpu().numpy()) <= 1e-4, (M, call)
        assert rel(gv, ref_var.double().cpu().numpy()) <= 1e-4, (M, call)
        om, ov = O.predict(p, Xs, include_noise=True)
        assert rel(gm, om) <= 1e-4 and rel(gv, ov) <= 1e-4, (M, call, rel(gm, om), rel(gv, ov))
        m.close()


def test_predict_noalloc_rejects_sizes_beyond_its_limit():
    from paper_2604_00697_gb300 import _lib

    lib = _lib.load()
    M, D, Ns = 257, 2, 10
    p, _, _, _ = small_case(M, D, 4, 1)
    dev = {k: torch.tensor(np.reshape(v, -1), dtype=torch.float32, device="cuda") for k, v in p.items()}
    params = _lib.svgp_params(*[dev[k].data_ptr() for k in ("Z", "ell", "sf2", "noise", "m", "s", "L")])
    Xd = torch.zeros(Ns, D, device="cuda")
    mean = torch.zeros(Ns, device="cuda")
    var = torch.zeros(Ns, device="cuda")
    assert _noalloc(lib, params, M, D, Xd, Ns, mean, var, None) == _lib.SVGP_ERR_INVALID_ARG
    assert _noalloc(lib, params, 16, D, Xd, 4097, mean, var, None) == _lib.SVGP_ERR_INVALID_ARG
