"""FP64 CPU oracle for the preconditioned inverse-free SVGP (R-SVGP) step.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  The GPU library never
calls it and shares no code with it.

Everything here is plain NumPy in float64, written as the paper states it:

* SE-ARD ("ARD RBF") kernel blocks Kuu, Kuf, k_nn (Section 2, M-SVGP
  paragraph; Section 4 uses the ARD RBF kernel), built from per-dimension
  differences, never from a norm expansion.
* K~ = Kuu + S~ (Section 2, L-SVGP paragraph), T = L L^T (Section 3.1).
* Preconditioner P = 2T - T K~ T (Section 3.2, P^(R)).
* Predictive moments mu_n = k_nu P m~, sigma_n^2 = k_nn - k_nu P k_un and the
  KL upper bound, Eq. (7) (preconditioned R-SVGP bound).
* Gaussian expected log-likelihood (Appendix S3, closed form), summed over a
  minibatch and scaled by N/B (stochastic SVGP, Section 1 / Eq. (1)).
* Bernoulli likelihood with probit link (the classification experiments of
  Section 4.1; GPflow's Bernoulli, Appendix S5.3): expected log-likelihood
  by 20-point Gauss-Hermite quadrature, and its derivatives with respect to
  the predictive mean and variance taken from the same quadrature rule.
* Natural-gradient step on L, Prop. 1 / Eq. (6), with the Frobenius stopping
  residual of Eq. (8), taken in the order of Section 3.1 ("Alternating
  Optimisation") and Section 3.3.
* Analytic gradients of the bound with T held fixed (the paper differentiates
  with TensorFlow; the formulas below are derived from Eq. (7) by the chain
  rule and are pinned to central finite differences in the tests).
* Prediction with the same moments (Eq. (7) form) and a small training driver
  (NG step then Adam step, Section 3.1; schedule of Section 3.4).

Parity status: every function here is pinned by tests in
``tests/test_oracle_pins.py``.  For ``train`` the pins fix its two halves
(with Adam off the NG half reaches the fixed point of Prop. 1; with the NG
half off one Adam step ascends by the first-order amount) and its progress
on the 1-D workload; the trajectory as a whole is parity unpinned, since the
paper prints no worked values for it.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "se_ard",
    "kernel_blocks",
    "preconditioner",
    "bound",
    "grads",
    "probit_terms",
    "ng_residual",
    "ng_step",
    "ng_solve",
    "variance_gap",
    "hutchinson_traces",
    "ng_solve_gap",
    "gamma_schedule",
    "predict",
    "softplus",
    "softplus_inv",
    "adam_update",
    "train",
]


def se_ard(A, B, ell, sf2):
    """SE-ARD kernel k(a, b) = sf2 * exp(-1/2 sum_d (a_d - b_d)^2 / ell_d^2).

    "ARD RBF" kernel of Section 4 (after Williams & Rasmussen).  Built from
    per-dimension differences (no ||a||^2 + ||b||^2 - 2 a.b expansion).
    """
    A = np.asarray(A, np.float64)
    B = np.asarray(B, np.float64)
    r2 = np.zeros((A.shape[0], B.shape[0]))
    for d in range(A.shape[1]):
        diff = (A[:, d][:, None] - B[:, d][None, :]) / ell[d]
        r2 += diff * diff
    return sf2 * np.exp(-0.5 * r2)


def kernel_blocks(p, X):
    """Kuu = k(Z, Z), Kuf = k(Z, X), k_nn = k(x_n, x_n), K~ = Kuu + diag(s~).

    Section 2 (M-SVGP paragraph for Kuu, k_un, k_nn; L-SVGP paragraph for K~).
    No jitter is added: S~ lower-bounds the eigenvalues of K~ (Section 2).
    """
    Kuu = se_ard(p["Z"], p["Z"], p["ell"], p["sf2"])
    Kuf = se_ard(p["Z"], X, p["ell"], p["sf2"])
    knn = np.full(X.shape[0], float(p["sf2"]))
    Kt = Kuu + np.diag(p["s"])
    return Kuu, Kuf, knn, Kt


def preconditioner(L, Kt):
    """T = L L^T and the inverse-free preconditioner P = 2T - T K~ T.

    Section 3.1 (T parameterised by its Cholesky-like factor L) and Section 3.2
    (P^(R) = 2T - T K~ T, one Newton-Schulz step from T).
    """
    T = L @ L.T
    P = 2.0 * T - T @ Kt @ T
    return T, P


def _gauss_expected_loglik(y, mu, var, noise):
    """E_{N(mu, var)}[log N(y | f, noise)] for each point (Appendix S3)."""
    return -0.5 * np.log(2 * math.pi * noise) - ((y - mu) ** 2 + var) / (2 * noise)


def hutchinson_traces(p, probes):
    """Hutchinson estimates (Section 3.4) of the two cubic KL traces.

    With K probe vectors z_k (columns of ``probes``, M x K, entries +-1):
      tr(K~ T)  ~ (1/K) sum_k z_k^T L^T K~ L z_k
      tr(P Kuu) ~ (1/K) sum_k z_k^T P Kuu z_k
    Each is unbiased for Rademacher probes; the average over all 2^M sign
    patterns is exact.
    """
    Zp = np.asarray(probes, np.float64)
    K = Zp.shape[1]
    L = np.asarray(p["L"], np.float64)
    Kuu = se_ard(p["Z"], p["Z"], p["ell"], p["sf2"])
    Kt = Kuu + np.diag(p["s"])
    T, P = preconditioner(L, Kt)
    trKT = float(np.sum(Zp * (L.T @ (Kt @ (L @ Zp))))) / K
    trPKuu = float(np.sum(Zp * (P @ (Kuu @ Zp)))) / K
    return trKT, trPKuu


def bound(p, X, y, N=None, likelihood="gaussian", precond=True, probes=None):
    """Preconditioned R-SVGP bound, Eq. (7), on one minibatch.

    F = (N/B) sum_n E_{N(mu_n, sigma_n^2)}[log p(y_n | f_n)] - KL_R with

      mu_n       = k_nu P m~
      sigma_n^2  = k_nn - k_nu P k_un
      KL_R       = 1/2 ( -tr(P Kuu) + tr(K~ T) - M + m~^T P Kuu P m~
                         - log|T| - log|S~| )

    Returns a dict holding F and its terms.  ``N`` defaults to the batch size
    (full-batch ELBO, Eq. (1)).

    ``precond=False`` gives the R-SVGP bound without the mean preconditioner
    (Section 2, inverse-free parameterisation, with m = Kuu m~): mu_n =
    k_nu m~ and the quadratic KL term m~^T Kuu m~ (the KL bound of Section 2);
    sigma_n^2 and the trace terms are unchanged.

    With ``probes`` (M x K, entries +-1) the two cubic traces tr(K~ T) and
    tr(P Kuu) of the KL bound are the Hutchinson estimates of
    ``hutchinson_traces`` (Section 3.4); every other term is exact.
    """
    X = np.asarray(X, np.float64)
    y = np.asarray(y, np.float64)
    B = X.shape[0]
    N = float(B if N is None else N)
    L = np.asarray(p["L"], np.float64)
    M = L.shape[0]
    Kuu, Kuf, knn, Kt = kernel_blocks(p, X)
    T, P = preconditioner(L, Kt)
    # per-point moments (Eq. (7), first line)
    Pm = P @ p["m"] if precond else np.asarray(p["m"], np.float64)
    mu = np.array([Kuf[:, n] @ Pm for n in range(B)]) if B <= 64 else Kuf.T @ Pm
    if B <= 64:
        var = np.array([knn[n] - Kuf[:, n] @ P @ Kuf[:, n] for n in range(B)])
    else:
        var = knn - np.einsum("in,in->n", Kuf, P @ Kuf)
    if likelihood == "gaussian":
        En = _gauss_expected_loglik(y, mu, var, float(p["noise"]))
    elif likelihood == "probit":
        En = probit_expected_loglik(y, mu, var)
    else:
        raise ValueError(likelihood)
    E = (N / B) * En.sum()
    # KL upper bound (Eq. (7), second and third lines); each trace as a product
    if probes is None:
        tr_PKuu = np.trace(P @ Kuu)
        tr_KtT = np.trace(Kt @ T)
    else:
        tr_KtT, tr_PKuu = hutchinson_traces(p, probes)
    quad = Pm @ Kuu @ Pm
    # log|T| with T = L L^T: for the lower-triangular L of the parameterisation
    # (kept lower triangular by the NG update of Prop. 1) the product rule
    # gives 2 sum_i log|L_ii| exactly; forming T first and factorising it loses
    # accuracy once cond(T) nears 1/eps (random triangular L at M = 300)
    if np.all(np.triu(L, 1) == 0.0):
        logdetT = 2.0 * np.sum(np.log(np.abs(np.diag(L))))
    else:
        sign, logdetT = np.linalg.slogdet(T)
    logdetS = np.sum(np.log(p["s"]))
    KL = 0.5 * (-tr_PKuu + tr_KtT - M + quad - logdetT - logdetS)
    return dict(F=E - KL, E=E, KL=KL, tr_PKuu=tr_PKuu, tr_KtT=tr_KtT, quad=quad,
                logdetT=logdetT, logdetS=logdetS, mu=mu, var=var, En=En, P=P, T=T)


def probit_expected_loglik(y, mu, var, n_gh=20):
    """E_{N(mu, var)}[log Phi(s f)], s = 2y - 1, by Gauss-Hermite quadrature.

    Bernoulli likelihood with probit link (GPflow's Bernoulli, Appendix S5.3);
    20 nodes from numpy's hermgauss.  log Phi via scipy's log_ndtr.
    """
    return probit_terms(y, mu, var, n_gh)[0]


def probit_terms(y, mu, var, n_gh=20):
    """Per-point probit terms (E_n, g_n, h_n) of the quadrature rule.

    With nodes t_k and weights w_k of the rule for exp(-t^2) (numpy's
    hermgauss), s_n = 2 y_n - 1, sd_n = sqrt(max(var_n, 0)) and
    f_nk = mu_n + sqrt(2) sd_n t_k:

      E_n = sum_k w_k / sqrt(pi) log Phi(s_n f_nk)
      g_n = dE_n / dmu_n      = sum_k w_k / sqrt(pi) s_n r(s_n f_nk)
      h_n = dE_n / dsigma_n^2 = sum_k w_k / sqrt(pi) s_n r(s_n f_nk) t_k / (sqrt(2) sd_n)

    where r = phi / Phi is the inverse Mills ratio (the derivative of
    log Phi).  h_n is the derivative of the rule itself, so it is what finite
    differences of ``bound(..., likelihood="probit")`` give.
    """
    from scipy.special import log_ndtr

    t, w = np.polynomial.hermite.hermgauss(n_gh)
    s = 2.0 * np.asarray(y, np.float64) - 1.0
    mu = np.asarray(mu, np.float64)
    sd = np.sqrt(np.maximum(np.asarray(var, np.float64), 0.0))
    f = mu[:, None] + math.sqrt(2.0) * sd[:, None] * t[None, :]
    a = s[:, None] * f
    logPhi = log_ndtr(a)
    r = np.exp(-0.5 * a * a - 0.5 * math.log(2.0 * math.pi) - logPhi)
    wk = w[None, :] / math.sqrt(math.pi)
    En = (wk * logPhi).sum(axis=1)
    g = (wk * s[:, None] * r).sum(axis=1)
    h = (wk * s[:, None] * r * t[None, :]).sum(axis=1) / (math.sqrt(2.0) * sd)
    return En, g, h


def grads(p, X, y, N=None, likelihood="gaussian", precond=True):
    """Gradient of the bound of Eq. (7) with T held fixed.

    T is a separate variational parameter optimised by natural gradients
    (Section 3.1, alternating optimisation), so the Adam step on
    xi = {theta, Z, m~, S~} differentiates with L fixed.  Gradients are w.r.t.
    the constrained values Z, ell, sf2, noise, m~, s~.

    Derivation (c = N/B, g_n = dE_n/dmu_n, h_n = dE_n/dsigma_n^2, v = P m~,
    w = Kuu v, dP = -T dK~ T):

      G_Kuf = c (v g^T - 2 P Kuf diag(h))
      G_P   = c ((Kuf g) m~^T - Kuf diag(h) Kuf^T) - 1/2 (-Kuu + m~ w^T + w m~^T)
      G_K~  = -T sym(G_P) T - T/2
      G_Kuu = G_K~ + P/2 - v v^T / 2
      ds~   = diag(G_K~) + 1/(2 s~)
      dm~   = c P Kuf g - P w
      then the SE-ARD chain rule for Z, ell, sf2.

    Without the preconditioner (``precond=False``: mu = Kuf^T m~, quadratic
    term m~^T Kuu m~) v = m~, the m~ terms leave G_P and dm~ = c Kuf g - Kuu m~.

    Gaussian likelihood: g_n = (y_n - mu_n) / noise, h_n = -1 / (2 noise).
    Probit (``likelihood="probit"``): g_n, h_n from ``probit_terms``; the
    bound does not depend on the noise variance, whose gradient is 0.
    """
    X = np.asarray(X, np.float64)
    y = np.asarray(y, np.float64)
    B = X.shape[0]
    N = float(B if N is None else N)
    c = N / B
    Z, ell, sf2, noise = p["Z"], p["ell"], float(p["sf2"]), float(p["noise"])
    m, s, L = p["m"], p["s"], p["L"]
    Kuu, Kuf, knn, Kt = kernel_blocks(p, X)
    T, P = preconditioner(L, Kt)
    v = P @ m if precond else np.asarray(m, np.float64)
    w = Kuu @ v
    mu = Kuf.T @ v
    var = knn - np.einsum("in,in->n", Kuf, P @ Kuf)
    if likelihood == "gaussian":
        g = (y - mu) / noise
        h = np.full(B, -0.5 / noise)
    elif likelihood == "probit":
        _, g, h = probit_terms(y, mu, var)
    else:
        raise ValueError(likelihood)
    Kg = Kuf @ g
    G_Kuf = c * (np.outer(v, g) - 2.0 * (P @ Kuf) * h[None, :])
    if precond:
        G_P = c * (np.outer(Kg, m) - (Kuf * h[None, :]) @ Kuf.T) \
            - 0.5 * (-Kuu + np.outer(m, w) + np.outer(w, m))
    else:
        G_P = -c * (Kuf * h[None, :]) @ Kuf.T + 0.5 * Kuu
    G_Psym = 0.5 * (G_P + G_P.T)
    G_Kt = -T @ G_Psym @ T - 0.5 * T
    G_Kuu = G_Kt + 0.5 * P - 0.5 * np.outer(v, v)
    ds = np.diag(G_Kt) + 0.5 / s
    dm = c * (P @ Kg) - P @ w if precond else c * Kg - w
    # SE-ARD chain rule
    A_f = G_Kuf * Kuf                      # M x B
    A_u = G_Kuu * Kuu                      # M x M (symmetric)
    dZ = np.zeros_like(Z)
    dell = np.zeros_like(ell)
    for d in range(Z.shape[1]):
        df = X[:, d][None, :] - Z[:, d][:, None]      # x_nd - z_id
        du = Z[:, d][None, :] - Z[:, d][:, None]      # z_jd - z_id
        dZ[:, d] = (A_f * df).sum(1) / ell[d] ** 2 + 2.0 * (A_u * du).sum(1) / ell[d] ** 2
        dell[d] = ((A_f * df * df).sum() + (A_u * du * du).sum()) / ell[d] ** 3
    dsf2 = c * h.sum() + (A_f.sum() + A_u.sum()) / sf2
    if likelihood == "gaussian":
        Q = (y - mu) ** 2 + var
        dnoise = c * np.sum(-0.5 / noise + Q / (2 * noise ** 2))
    else:
        dnoise = 0.0
    return dict(Z=dZ, ell=dell, sf2=dsf2, noise=dnoise, m=dm, s=ds)


def ng_residual(A):
    """Normalised residual ||A - I||_F / sqrt(M) with A = L^T K~ L, Eq. (8)."""
    M = A.shape[0]
    return float(np.linalg.norm(A - np.eye(M), "fro") / math.sqrt(M))


def ng_step(L, Kt, gamma):
    """One natural-gradient step on L for the auxiliary objective, Prop. 1.

    A = L^T K~ L;  natural gradient = L [tril(A) - 1/2 (I + diag(A))]
    (tril keeps the diagonal, diag returns a diagonal matrix; Appendix S1);
    L <- L - gamma * natural gradient.  Returns (L_new, residual(A)).
    """
    M = L.shape[0]
    A = L.T @ Kt @ L
    r = ng_residual(A)
    nat = L @ (np.tril(A) - 0.5 * (np.eye(M) + np.diag(np.diag(A))))
    return L - gamma * nat, r


def ng_solve(L, Kt, gammas, eps=0.0, max_iters=None):
    """Run NG steps with the Frobenius stopping rule of Section 3.3.

    For t = 0, 1, ...: compute A(L_t) and r_t = ||A - I||_F/sqrt(M); stop
    (without updating) when r_t < eps; otherwise L_{t+1} = NG step with
    gamma_t.  At most ``max_iters`` updates are applied.  Returns
    (L, number of updates applied, last residual computed).
    """
    gammas = list(gammas)
    max_iters = len(gammas) if max_iters is None else max_iters
    r = float("nan")
    it = 0
    for it in range(max_iters):
        A = L.T @ Kt @ L
        r = ng_residual(A)
        if eps > 0 and r < eps:
            return L, it, r
        L, _ = ng_step(L, Kt, gammas[it])
    return L, max_iters, r


def variance_gap(p, X, sigma2=None):
    """Per-point gap G_n = U_n - L_n of Prop. 3 (Section 3.3).

    With the split S~ = S~' + sigma^2 I (S~' diagonal, sigma2 defaults to
    min_i s~_i), U_n is the R-SVGP predictive variance and L_n the lower
    bound of Prop. 3 on the L-SVGP variance; their difference is
      G_n = ||(I - K~ T) k_un||^2 / sigma^2.
    The Gaussian stopping rule stops the NG iterations once
    sum_n G_n <= 2 noise eps.
    """
    Kuu, Kuf, knn, Kt = kernel_blocks(p, np.asarray(X, np.float64))
    L = np.asarray(p["L"], np.float64)
    T = L @ L.T
    if sigma2 is None:
        sigma2 = float(np.min(p["s"]))
    R = Kuf - Kt @ (T @ Kuf)
    return (R * R).sum(axis=0) / sigma2


def ng_solve_gap(p, X, gammas, eps, sigma2=None, max_iters=None):
    """NG steps on p["L"] with the Prop. 3 gap stopping rule of Section 3.3.

    For t = 0, 1, ...: G_t = sum_n G_n(L_t); stop (without updating) when
    G_t <= 2 noise eps; otherwise L_{t+1} = NG step with gamma_t.  Returns
    (L, number of updates applied, last gap computed).
    """
    q = dict(p)
    Kt = kernel_blocks(q, np.asarray(X, np.float64))[3]
    gammas = list(gammas)
    max_iters = len(gammas) if max_iters is None else max_iters
    L = np.asarray(q["L"], np.float64)
    G = float("nan")
    for it in range(max_iters):
        q["L"] = L
        G = float(variance_gap(q, X, sigma2).sum())
        if G <= 2.0 * float(q["noise"]) * eps:
            return L, it, G
        L, _ = ng_step(L, Kt, gammas[it])
    return L, max_iters, G


def gamma_schedule(t, gamma0=1e-5, gammaT=1.0, ramp=10):
    """Log-linear NG step-size schedule of Section 3.4 / Appendix S5.4.

    gamma_t = gamma0 * (gammaT / gamma0)^(t / ramp) for t <= ramp, then gammaT,
    with t the global NG-update counter.
    """
    if t >= ramp:
        return gammaT
    return gamma0 * (gammaT / gamma0) ** (t / ramp)


def predict(p, Xs, include_noise=False):
    """Predictive mean and variance at test inputs, same form as Eq. (7)."""
    Kuu, Ksu, kss, Kt = kernel_blocks(p, Xs)
    T, P = preconditioner(p["L"], Kt)
    mean = Ksu.T @ (P @ p["m"])
    var = kss - np.einsum("in,in->n", Ksu, P @ Ksu)
    if include_noise:
        var = var + float(p["noise"])
    return mean, var


def softplus(x):
    return np.logaddexp(0.0, x)


def softplus_inv(y):
    y = np.asarray(y, np.float64)
    return y + np.log(-np.expm1(-y))


_POSITIVE = ("ell", "sf2", "noise", "s")


def adam_update(raw, grad_c, state, lr, b1=0.9, b2=0.999, eps=1e-8, lr_scale=None):
    """One Adam ascent step (Kingma & Ba) on unconstrained parameters.

    ``raw`` holds unconstrained values (softplus for the positive ones);
    ``grad_c`` gradients w.r.t. constrained values; the chain rule through
    softplus multiplies by sigmoid(raw).  Ascent because F is maximised.
    """
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    out = {}
    for k, x in raw.items():
        g = np.asarray(grad_c[k], np.float64)
        if k in _POSITIVE:
            g = g / (1.0 + np.exp(-np.asarray(x)))
        mom = state.setdefault("m_" + k, np.zeros_like(np.asarray(x, np.float64)))
        vel = state.setdefault("v_" + k, np.zeros_like(np.asarray(x, np.float64)))
        mom[...] = b1 * mom + (1 - b1) * g
        vel[...] = b2 * vel + (1 - b2) * g * g
        mhat = mom / (1 - b1 ** t)
        vhat = vel / (1 - b2 ** t)
        rate = lr * (1.0 if lr_scale is None else lr_scale.get(k, 1.0))
        out[k] = x + rate * mhat / (np.sqrt(vhat) + eps)
    return out


def constrain(raw):
    return {k: (softplus(v) if k in _POSITIVE else np.asarray(v, np.float64))
            for k, v in raw.items()}


def train(p0, batches, N, steps, lr=5e-3, gamma=None, train_Z=True, eps=0.0,
          max_ng=1, ng_counts=None):
    """Alternating optimisation of Section 3.1: NG step(s) on L, then Adam on xi.

    ``gamma`` is a callable t -> gamma_t over the global NG counter (default:
    gamma = 1, the fixed-Z setting of Section 3.4).  Returns the final state
    and the list of bound values recorded after each Adam step; the number of
    NG updates of each step is appended to ``ng_counts`` when given.
    """
    gamma = gamma or (lambda t: 1.0)
    raw = {k: (softplus_inv(p0[k]) if k in _POSITIVE else np.array(p0[k], np.float64))
           for k in ("Z", "ell", "sf2", "noise", "m", "s")}
    L = np.array(p0["L"], np.float64)
    state = {}
    trace = []
    t_ng = 0
    for step in range(steps):
        X, y = batches(step)
        c = constrain(raw)
        _, _, _, Kt = kernel_blocks(c, X[:1])
        n_ng = 0
        for _ in range(max_ng):
            A = L.T @ Kt @ L
            if eps > 0 and ng_residual(A) < eps:
                break
            L, _ = ng_step(L, Kt, gamma(t_ng))
            t_ng += 1
            n_ng += 1
        if ng_counts is not None:
            ng_counts.append(n_ng)
        c["L"] = L
        gr = grads(c, X, y, N)
        trace.append(bound(c, X, y, N)["F"])
        if not train_Z:
            gr = dict(gr)
            gr["Z"] = np.zeros_like(gr["Z"])
        raw = adam_update(raw, gr, state, lr)
    out = constrain(raw)
    out["L"] = L
    return out, trace
