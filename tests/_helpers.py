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
}
# unit roundoff of the contraction operands: FP32, BF16, BF16 hi+lo pair
UNIT = {"fp32": 2.0 ** -24, "bf16": 2.0 ** -9, "bf16x3": 2.0 ** -17}


def cond_Kt(p):
    """Error amplification of the preconditioner products.

    max(cond(K~), ||T||^2 ||K~|| / ||P||) in the 2-norm: a relative
    perturbation u of K~ or L moves P = 2T - T K~ T by about
    u ||T||^2 ||K~||, which relative to ||P|| is the second factor; at
    T = K~^-1 both factors equal cond(K~)."""
    Kt = O.se_ard(p["Z"], p["Z"], p["ell"], p["sf2"]) + np.diag(p["s"])
    T = p["L"] @ p["L"].T
    P = 2 * T - T @ Kt @ T
    nP = np.linalg.norm(P, 2)
    amp = np.linalg.norm(T, 2) ** 2 * np.linalg.norm(Kt, 2) / nP if nP > 0 else np.inf
    return float(max(np.linalg.cond(Kt), amp))


def tolerances(prec, p):
    """Stated tolerance, widened to the arithmetic's error bound.

    The M x M products of the bound (A1 = L^T K~ L, P = L(2I - A1)L^T and the
    T G T chain) are computed from operands rounded to unit roundoff u, so
    their relative error is about u * cnd (cnd from cond_Kt).  The bound
    accepts max(stated, u cnd); the gradient blocks accept max(stated,
    32 u cnd) because the data and KL parts of dF/dZ and the diagonal terms of
    dF/ds~ partly cancel (factors of 10 to 20 measured at cnd = 579 in FP32,
    BF16 and split BF16 alike)."""
    k = cond_Kt(p)
    u = UNIT[prec]
    return max(TOL[prec]["bound"], u * k), max(TOL[prec]["grad"], 32 * u * k), k
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
