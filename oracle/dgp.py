"""FP64 CPU oracle of a deep GP whose layers are R-SVGPs (Section 4.2, "Deep GPs").

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  The GPU library never
calls it and shares no code with it.

The model, as Section 4.2 and the deep-regression set-up of the appendix fix
it:

* L layers.  Layer l has its own inducing locations Z^(l) (M x D_l) and
  SE-ARD hyper-parameters (ell^(l), sf2^(l)) shared by its Q_l outputs, one
  diagonal S~^(l) shared by those outputs (so one K~^(l) and one
  T^(l) = L^(l) L^(l)T, one NG loop per layer), and one mean vector m~^(l,q)
  per output (the columns of an M x Q_l matrix).
* The variational posterior factorises over layers; the ELBO is a Monte
  Carlo estimate of the expected log-likelihood through the latent layers
  minus the sum of the layers' KL terms.  Every layer is an R-SVGP with the
  preconditioned moments and KL upper bound of Eq. (7): for output q,
  mu_nq = k_n^T P m~_q, and sigma_n^2 = k_nn - k_n^T P k_n is the same for
  all outputs of the layer.

Readings where the paper defers to the library it used:

* hidden layers have width Q_l equal to their input width and the identity
  mean function; the output layer (Q = 1) has zero mean;
* propagation is doubly stochastic with one draw per point and layer from
  the marginal N(mu_nq, sigma_n^2) by reparameterisation:
  h_nq = h_prev,nq + mu_nq + sigma_n eps_nq, the standard normal draws eps
  being inputs of the oracle (so both sides of a parity test use the same
  draws); sigma_n = sqrt(max(sigma_n^2, 0));
* the output layer's expectation under its Gaussian marginal is the closed
  form of Appendix S3 (Gaussian likelihood), scaled by N / B as in Eq. (1).

Gradients are taken with every T^(l) held fixed (Section 3.1, alternating
optimisation), with respect to the constrained values.  The multi-output
layer gradient generalises the single-layer derivation of ``rsvgp.grads``
(which it reproduces for one output); it is pinned to central differences
of ``elbo`` in the tests.
"""
from __future__ import annotations

import numpy as np

from . import rsvgp as R

__all__ = ["layer_forward", "layer_backward", "elbo", "grads"]


def layer_forward(lp, H):
    """Moments and KL bound of one layer at inputs H (B x D_in), Eq. (7).

    ``lp``: Z (M x D_in), ell (D_in), sf2, s (M), L (M x M), m (M x Q).
    Returns mu (B x Q), var (B), KL (sum over the Q outputs) and the blocks
    the backward pass reuses.
    """
    H = np.asarray(H, np.float64)
    m = np.asarray(lp["m"], np.float64).reshape(len(lp["s"]), -1)
    Q = m.shape[1]
    Kuu, Kuf, knn, Kt = R.kernel_blocks(lp, H)
    L = np.asarray(lp["L"], np.float64)
    M = L.shape[0]
    T, P = R.preconditioner(L, Kt)
    V = P @ m                                     # M x Q
    mu = Kuf.T @ V                                # B x Q
    var = knn - np.einsum("in,in->n", Kuf, P @ Kuf)
    # KL bound of each output: the trace and log-det terms are shared, the
    # quadratic term is m~_q^T P Kuu P m~_q
    if np.all(np.triu(L, 1) == 0.0):
        logdetT = 2.0 * np.sum(np.log(np.abs(np.diag(L))))
    else:
        logdetT = np.linalg.slogdet(T)[1]
    shared = -np.trace(P @ Kuu) + np.trace(Kt @ T) - M - logdetT - np.sum(np.log(lp["s"]))
    quad = np.einsum("iq,iq->", V, Kuu @ V)
    KL = 0.5 * (Q * shared + quad)
    return dict(mu=mu, var=var, KL=KL, Kuu=Kuu, Kuf=Kuf, Kt=Kt, T=T, P=P, V=V, m=m, Q=Q)


def layer_backward(lp, H, fw, gmu, gvar):
    """Gradient of (data term) - KL of one layer, T held fixed.

    ``gmu`` (B x Q) and ``gvar`` (B) are the derivatives of the data term with
    respect to the layer's mu and sigma^2.  With v = P m~ (M x Q),
    w = Kuu v:

      G_Kuf = v gmu^T - 2 (P Kuf) diag(gvar)
      G_P   = (Kuf gmu) m~^T - Kuf diag(gvar) Kuf^T + Q Kuu / 2 - (m~ w^T + w m~^T) / 2
      G_K~  = -T sym(G_P) T - Q T / 2
      G_Kuu = G_K~ + Q P / 2 - v v^T / 2
      ds~   = diag(G_K~) + Q / (2 s~),   dm~ = P Kuf gmu - P w
      dsf2  = sum_n gvar_n + (<G_Kuf, Kuf> + <G_Kuu, Kuu>) / sf2

    then the SE-ARD chain rule for Z and ell, and for the inputs
    dH_nd = sum_i (G_Kuf o Kuf)_in (z_id - h_nd) / ell_d^2.
    """
    H = np.asarray(H, np.float64)
    Z, ell, sf2, s = lp["Z"], lp["ell"], float(lp["sf2"]), lp["s"]
    Kuu, Kuf, T, P, V, m, Q = fw["Kuu"], fw["Kuf"], fw["T"], fw["P"], fw["V"], fw["m"], fw["Q"]
    gmu = np.asarray(gmu, np.float64).reshape(H.shape[0], Q)
    gvar = np.asarray(gvar, np.float64)
    W = Kuu @ V
    Kg = Kuf @ gmu                                                    # M x Q
    G_Kuf = V @ gmu.T - 2.0 * (P @ Kuf) * gvar[None, :]
    G_P = Kg @ m.T - (Kuf * gvar[None, :]) @ Kuf.T + 0.5 * Q * Kuu - 0.5 * (m @ W.T + W @ m.T)
    G_Psym = 0.5 * (G_P + G_P.T)
    G_Kt = -T @ G_Psym @ T - 0.5 * Q * T
    G_Kuu = G_Kt + 0.5 * Q * P - 0.5 * V @ V.T
    ds = np.diag(G_Kt) + 0.5 * Q / s
    dm = P @ Kg - P @ W
    A_f = G_Kuf * Kuf
    A_u = G_Kuu * Kuu
    dZ = np.zeros_like(np.asarray(Z, np.float64))
    dell = np.zeros(len(ell))
    dH = np.zeros_like(H)
    for d in range(Z.shape[1]):
        df = H[:, d][None, :] - Z[:, d][:, None]      # h_nd - z_id
        du = Z[:, d][None, :] - Z[:, d][:, None]      # z_jd - z_id
        dZ[:, d] = (A_f * df).sum(1) / ell[d] ** 2 + 2.0 * (A_u * du).sum(1) / ell[d] ** 2
        dell[d] = ((A_f * df * df).sum() + (A_u * du * du).sum()) / ell[d] ** 3
        dH[:, d] = -(A_f * df).sum(0) / ell[d] ** 2
    dsf2 = gvar.sum() + (A_f.sum() + A_u.sum()) / sf2
    return dict(Z=dZ, ell=dell, sf2=dsf2, m=dm.reshape(np.shape(lp["m"])), s=ds), dH


def _propagate(layers, X, eps):
    H = np.asarray(X, np.float64)
    Hs, fws = [H], []
    for l, lp in enumerate(layers):
        fw = layer_forward(lp, H)
        fws.append(fw)
        if l < len(layers) - 1:
            sig = np.sqrt(np.maximum(fw["var"], 0.0))
            H = H + fw["mu"] + sig[:, None] * np.asarray(eps[l], np.float64)
            Hs.append(H)
    return Hs, fws


def elbo(layers, X, y, N, noise, eps):
    """Doubly stochastic ELBO of the deep GP for one minibatch and one set of
    draws: (N/B) sum_n E_{N(mu_n, sigma_n^2)}[log N(y_n | f, noise)] at the
    output layer, minus the KL bounds of every layer.

    ``layers``: list of layer dicts (``layer_forward``), hidden layers first;
    ``eps``: one B x Q_l array of standard normal draws per hidden layer.
    """
    y = np.asarray(y, np.float64)
    B = y.shape[0]
    Hs, fws = _propagate(layers, X, eps)
    out = fws[-1]
    En = R._gauss_expected_loglik(y, out["mu"][:, 0], out["var"], float(noise))
    return (float(N) / B) * En.sum() - sum(fw["KL"] for fw in fws)


def grads(layers, X, y, N, noise, eps):
    """Gradient of ``elbo`` for every layer's Z, ell, sf2, m~, s~ and for the
    noise variance, all T^(l) held fixed.  Returns (list of per-layer dicts,
    dnoise).  A hidden layer's output h = h_prev + mu + sigma eps passes the
    incoming gradient G on as gmu = G, gvar_n = sum_q G_nq eps_nq / (2 sigma_n),
    and G plus the layer's input gradient to the layer below."""
    y = np.asarray(y, np.float64)
    B = y.shape[0]
    c = float(N) / B
    noise = float(noise)
    Hs, fws = _propagate(layers, X, eps)
    out = fws[-1]
    mu = out["mu"][:, 0]
    g = c * (y - mu) / noise
    h = np.full(B, -0.5 * c / noise)
    dnoise = c * np.sum(-0.5 / noise + ((y - mu) ** 2 + out["var"]) / (2 * noise ** 2))
    res = [None] * len(layers)
    res[-1], G = layer_backward(layers[-1], Hs[-1], out, g[:, None], h)
    for l in range(len(layers) - 2, -1, -1):
        fw = fws[l]
        sig = np.sqrt(np.maximum(fw["var"], 0.0))
        e = np.asarray(eps[l], np.float64)
        gvar = np.where(sig > 0, (G * e).sum(1) / (2.0 * np.where(sig > 0, sig, 1.0)), 0.0)
        res[l], dH = layer_backward(layers[l], Hs[l], fw, G, gvar)
        G = G + dH
    return res, dnoise
