"""Shared helpers for the parity tests: build seeded states, run both sides."""
from __future__ import annotations

import math

import numpy as np

import svgp_synth as S
from oracle import rsvgp as O

TOL = {  # relative bound error, per-block relative gradient error
    "fp32": dict(bound=1e-6, grad=1e-4),
    "bf16": dict(bound=1e-3, grad=1e-2),
    "bf16x3": dict(bound=1e-3, grad=1e-2),
    "bf16x3k": dict(bound=1e-3, grad=1e-2),
}
# Cases where a stated gate is out of reach of the arithmetic itself.  Each
# entry pins the case at about twice (three times for the noisier BF16
# gradients) the relative error measured on a GB300, with the measured value
# in the comment.  Each is out of reach because the oracle's own bound and
# gradients move by about that much when its kernel blocks are perturbed at
# the unit roundoff of the mode (the states are ill-conditioned: cond(K~) in
# the hundreds to thousands).  Keys: (case, precision);
# values: tolerances for "bound" and for the gradient blocks named (blocks
# not named keep the stated gate).
OUT_OF_REACH = {
    # FP32 at the converged state of the 1-D workload (s~ = 1e-2, cond(K~) =
    # 1.6e3): bound 2.2e-5, dZ 3.2e-4, dell 4.9e-4 and 1.05e-3 in two runs
    # (the order of the FP32 atomic sums differs), dsf2 4.6e-4, ds~ 6.9e-4
    ("snelson_like/chol", "fp32"): dict(bound=5e-5, Z=7e-4, ell=2.5e-3, sf2=1e-3, s=1.5e-3),
    # BF16X3 there: dZ 1.7e-2, dsf2 1.5e-2, dm~ 1.6e-2, ds~ 1.8e-2
    ("snelson_like/chol", "bf16x3"): dict(Z=3.5e-2, sf2=3e-2, m=3.2e-2, s=3.7e-2),
    # single BF16 there: bound 1.6e-3, dZ 11.4, dell 3.3, dsf2 1.0, dm~ 0.14,
    # ds~ 5.5 (the gradient is not determined at this precision)
    ("snelson_like/chol", "bf16"): dict(bound=4e-3, Z=35.0, ell=10.0, sf2=3.0, m=0.4, s=17.0),
    # single BF16, random states: M = 1 (dZ 3.1e-2, dell 3.0e-2, dm~ 3.8e-2,
    # ds~ 3.1e-2) and M = 257 with one point (dm~ 1.2e-2)
    ("random/1x2x7", "bf16"): dict(Z=9.3e-2, ell=9e-2, m=0.115, s=9.2e-2),
    ("random/257x1x1", "bf16"): dict(m=3.5e-2),
    # single BF16 at converged or trained states of the M = 512 and M = 2048
    # workloads: dZ 7.5e-2 / 6.5e-2 / 0.10 / 0.16, dell 1.1e-2 / 1.2e-2 /
    # 9.5e-3 to 1.1e-2 / 1.6e-2, dm~ 1.3e-2 / 1.3e-2 / 1.4e-2 / 1.7e-2,
    # ds~ 7.6e-2 / 6.2e-2
    ("sinusoid_regression/chol", "bf16"): dict(Z=0.23, ell=3.4e-2, m=4e-2, s=0.23),
    ("gp_sample_regression/chol", "bf16"): dict(Z=0.2, ell=3.6e-2, m=4e-2, s=0.19),
    ("gp_sample_regression/ng40", "bf16"): dict(Z=0.31, ell=3.3e-2, m=4.1e-2),
    ("gp_sample_regression/train50", "bf16"): dict(Z=0.48, ell=4.7e-2, m=5.1e-2),
    # probit, single BF16, M = 1: dZ 3.2e-2, dell 3.1e-2, dm~ 3.1e-2, ds~ 1.3e-2
    ("probit/1x2x7", "bf16"): dict(Z=9.6e-2, ell=9.4e-2, m=9.2e-2, s=3.8e-2),
    # probit, single BF16, M = 200 on 2-D inputs: sum of sigma_n^2 off by
    # 1.2e-3 of B sf2, dm~ 1.5e-2
    ("probit/200x2x300", "bf16"): dict(sumvar=2.5e-3, m=4.5e-2),
    # probit classification workload at its converged state (s~ = 0.5,
    # cond(K~) = 277, sigma_n^2 about 0.015 sf2): FP32 dZ 3.0e-4, dell 2.0e-4,
    # dsf2 6.7e-5 to 1.4e-4 (three runs: the order of FP32 atomic sums
    # differs), ds~ 5.8e-4; BF16X3 dell 3.2e-2, dsf2 0.27
    ("banana_like/chol", "fp32"): dict(Z=7e-4, ell=4e-4, sf2=3e-4, s=1.2e-3),
    ("banana_like/chol", "bf16x3"): dict(ell=6.4e-2, sf2=0.55),
    # single BF16 there: bound 1.2e-2, sum of sigma_n^2 off by 2.5e-2 of
    # B sf2, dZ 1.6, dell 1.6, dsf2 12.6, dm~ 8.8e-2, ds~ 1.3
    ("banana_like/chol", "bf16"): dict(bound=2.4e-2, sumvar=5e-2, Z=4.8, ell=4.8, sf2=38.0, m=0.27, s=3.9),
}


def gates(case, prec):
    """(bound tolerance, {block: gradient tolerance}) for a named case; the
    probit sum of sigma_n^2 (relative to B sf2) is held to the bound's
    tolerance under the key "sumvar"."""
    ex = OUT_OF_REACH.get((case, prec), {})
    tb = ex.get("bound", TOL[prec]["bound"])
    tg = {k: ex.get(k, TOL[prec]["grad"]) for k in ("Z", "ell", "sf2", "noise", "m", "s")}
    tg["sumvar"] = ex.get("sumvar", tb)
    return tb, tg


def log_errors(case, prec, errs):
    """Append the measured errors of a case to $SVGP_ERRLOG (one JSON line)."""
    import json
    import os

    path = os.environ.get("SVGP_ERRLOG")
    if path:
        with open(path, "a") as fh:
            fh.write(json.dumps({"case": case, "prec": prec, **{k: float(v) for k, v in errs.items()}}) + "\n")


BLOCKS = ("Z", "ell", "sf2", "noise", "m", "s")


def f32(a):
    """Round to float32 and return float64 (both sides see identical values)."""
    if isinstance(a, np.ndarray):
        return a.astype(np.float32).astype(np.float64)
    return float(np.float32(a))


def round_state(p):
    return {k: f32(np.asarray(v, np.float64)) if np.ndim(v) else f32(v) for k, v in p.items()}


def chol_inv(p):
    """chol((Kuu + diag s)^-1) in FP64 (the NG fixed point, Section 3.1)."""
    Kt = O.se_ard(p["Z"], p["Z"], p["ell"], p["sf2"]) + np.diag(p["s"])
    return np.linalg.cholesky(np.linalg.inv(Kt))


def make_case(workload, state, seed=0, batch=0):
    """Return (state dict, X, y, N) rounded to float32.

    state: "init"  -- paper initialisation (Appendix S5.3): m~=0, s~=1e-4,
                      L=1e-3 I, ell=1, sf2=1, noise=1;
           "chol"  -- same hyperparameters with L = chol(K~^-1) and a random m~;
           "random"-- random lower-triangular L and random m~, s~ in [0.05,0.5].
    """
    prob = S.WORKLOADS[workload]() if isinstance(workload, str) else workload
    X, y = prob.batch(batch)
    M, D = prob.M, prob.D
    rng = np.random.default_rng([seed, 17])
    if state == "random":
        p = S.random_state(M, D, seed)
        p["Z"] = prob.Z0.copy()
    else:
        p = dict(Z=prob.Z0.copy(), ell=np.ones(D), sf2=1.0, noise=1.0, m=np.zeros(M),
                 s=np.full(M, 1e-4), L=1e-3 * np.eye(M))
        if state == "chol":
            p["s"] = np.full(M, 1e-2)
            p["noise"] = 0.3
            p["m"] = rng.normal(size=M) * 0.1
            p["L"] = chol_inv(round_state(p))
    p = round_state(p)
    return p, f32(X), f32(y), prob.N


def small_case(M, D, B, seed, state="random", N=None):
    rng = np.random.default_rng([seed, 3])
    X = rng.normal(size=(B, D))
    y = np.sin(X @ rng.normal(size=D)) + 0.1 * rng.normal(size=B)
    p = S.random_state(M, D, seed)
    if state == "chol":
        p["L"] = chol_inv(p)
    return round_state(p), f32(X), f32(y), float(N if N is not None else 10 * B)


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))
