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
# relative accuracy of the generated Kuf values: FP32 exp of an FP32 squared
# distance (a few ulp); BF16 values; hi + lo BF16 values of 2^t whose exponent
# t comes from a hi/lo BF16 split of the coordinates (about 16 bits of
# p . q, so |t| 2^-16 absolute, 2^-12 relative for |t| up to 16)
UNIT_KUF = {"fp32": 2.0 ** -21, "bf16": 2.0 ** -9, "bf16x3": 2.0 ** -12}


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


def kernel_rounding_sensitivity(p, X, y, N, prec, likelihood="gaussian", draws=3):
    """Largest per-block change over `draws` random roundings (one draw is
    noisy: a block's change depends on how the random signs line up)."""
    outs = [_one_rounding_sensitivity(p, X, y, N, prec, likelihood, seed) for seed in range(draws)]
    return {k: max(o[k] for o in outs) if all(np.isfinite(o[k]) for o in outs) else float("nan") for k in outs[0]}


def _one_rounding_sensitivity(p, X, y, N, prec, likelihood="gaussian", seed=0):
    """Relative change of each oracle gradient block when the kernel blocks
    and L are perturbed elementwise by relative noise of the size of the
    mode's accuracy (Kuu, L: the operand unit roundoff; Kuf: that of the
    generated values): the error that rounding only those inputs would cause.  NaN where the perturbed problem has no finite gradient
    (a perturbed sigma_n^2 went below 0).  Used where cond(K~) alone
    underestimates the sensitivity of the gradient (dZ sums contributions
    that cancel)."""
    u, uf = UNIT[prec], UNIT_KUF[prec]
    rng = np.random.default_rng([seed, 23])
    base = O.grads(p, X, y, N, likelihood=likelihood)
    orig = O.kernel_blocks

    def perturbed(pp, XX):
        Kuu, Kuf, knn, _ = orig(pp, XX)
        E = 1.0 + u * rng.standard_normal(Kuu.shape)
        Kuu = Kuu * (0.5 * (E + E.T))
        Kuf = Kuf * (1.0 + uf * rng.standard_normal(Kuf.shape))
        return Kuu, Kuf, knn, Kuu + np.diag(pp["s"])

    q = dict(p)
    q["L"] = np.asarray(p["L"], np.float64) * (1.0 + u * rng.standard_normal(np.shape(p["L"])))
    O.kernel_blocks = perturbed
    try:
        with np.errstate(all="ignore"):
            g = O.grads(q, X, y, N, likelihood=likelihood)
    finally:
        O.kernel_blocks = orig
    out = {}
    for k in BLOCKS:
        a, b = np.asarray(g[k], np.float64), np.asarray(base[k], np.float64)
        nb = np.linalg.norm(b)
        out[k] = float(np.linalg.norm(a - b) / nb) if nb > 0 and np.all(np.isfinite(a)) else \
            (0.0 if nb == 0 and np.all(a == 0) else float("nan"))
    return out
