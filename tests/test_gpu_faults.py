"""Failure detection without a GPU fault.

Invalid inputs are made on the host (NaN in y or L, s~ <= 0, a zero on the
diagonal of L, a diverging NG step size); each call must return, with the
device error word reporting SVGP_ERR_NONFINITE, and the handle must stay
usable: the error word is cleared by reading it and a valid call that
follows gives the oracle's bound.  The timeout path is checked with the
probe whose bounded wait runs out on an mbarrier nothing arrives on.
"""
import numpy as np
import pytest

from _helpers import TOL, small_case

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.tensor(np.asarray(a), dtype=torch.float32, device="cuda")


def _model(p, prec, B):
    from paper_2604_00697_gb300 import _lib
    from paper_2604_00697_gb300.model import RSVGP

    if prec != "fp32" and not _lib.svgp_has_tensor_cores():
        pytest.fail("tensor-core path not available on this device")
    M, D = p["Z"].shape
    m = RSVGP(M, D, B, prec=prec)
    m.set_state(p["Z"], p["ell"], p["sf2"], p["noise"], p["m"], p["s"], p["L"])
    return m


def _clean_bound(p, prec, X, y, N):
    m = _model(p, prec, X.shape[0])
    F = float(m.bound(_dev(X), _dev(y), N)[0])
    assert m.sync_status() == 0
    m.close()
    return F


def _recovers(m, p, X, y, N, F_clean, prec):
    """After an error the handle computes what a fresh handle computes, up to
    the order of the atomic sums (within the precision's bound tolerance)."""
    m.set_state(p["Z"], p["ell"], p["sf2"], p["noise"], p["m"], p["s"], p["L"])
    F = float(m.bound(_dev(X), _dev(y), N)[0])
    assert m.sync_status() == 0
    assert abs(F - F_clean) <= TOL[prec]["bound"] * abs(F_clean)


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
@pytest.mark.parametrize("fault", ["nan_y", "nan_L", "zero_s", "negative_s", "zero_L_diag"])
def test_invalid_input_reports_nonfinite(prec, fault):
    from paper_2604_00697_gb300 import _lib

    p, X, y, N = small_case(150, 3, 200, 11, state="chol")
    q = {k: (np.array(v, copy=True) if isinstance(v, np.ndarray) else v) for k, v in p.items()}
    yq = np.array(y, copy=True)
    if fault == "nan_y":
        yq[17] = np.nan
    elif fault == "nan_L":
        q["L"][40, 3] = np.nan
    elif fault == "zero_s":
        q["s"][5] = 0.0
    elif fault == "negative_s":
        q["s"][5] = -0.1
    elif fault == "zero_L_diag":
        q["L"][9, 9] = 0.0
    F_clean = _clean_bound(p, prec, X, y, N)
    m = _model(q, prec, X.shape[0])
    m.backward(_dev(X), _dev(yq), N)
    assert m.sync_status() == _lib.SVGP_ERR_NONFINITE
    assert m.sync_status() == _lib.SVGP_OK          # cleared after reading
    _recovers(m, p, X, y, N, F_clean, prec)
    m.close()


@pytest.mark.parametrize("prec", ["fp32", "bf16", "bf16x3"])
def test_diverging_ng_step_size_is_reported(prec):
    """gamma = 40 makes the NG iteration of Prop. 1 blow up: the loop stops at
    the first non-finite residual (no further updates) and reports it."""
    from paper_2604_00697_gb300 import _lib

    p, X, y, N = small_case(130, 3, 100, 12, state="chol")
    F_clean = _clean_bound(p, prec, X, y, N)
    m = _model(p, prec, X.shape[0])
    m.ng_update(max_iters=60, eps=0.0, gammas=[40.0] * 60)
    assert m.sync_status() == _lib.SVGP_ERR_NONFINITE
    assert int(m.iters[0]) < 60
    assert not np.isfinite(float(m.resid[0]))
    _recovers(m, p, X, y, N, F_clean, prec)
    m.close()


def test_bounded_wait_timeout_is_reported():
    """The bounded device wait gives up, the error word says so, and the
    handle keeps working."""
    from paper_2604_00697_gb300 import _lib

    p, X, y, N = small_case(130, 3, 100, 13, state="chol")
    F_clean = _clean_bound(p, "bf16x3", X, y, N)
    m = _model(p, "bf16x3", X.shape[0])
    _lib.svgp_check_wait_timeout(m.h)
    assert m.sync_status() == _lib.SVGP_ERR_TIMEOUT
    assert m.sync_status() == _lib.SVGP_OK
    _recovers(m, p, X, y, N, F_clean, "bf16x3")
    m.close()
