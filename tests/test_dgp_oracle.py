"""Pins of the deep-GP oracle (Section 4.2, "Deep GPs") on the CPU.

The deep-GP oracle composes R-SVGP layers; each test checks it against
something other than itself: the pinned single-layer oracle it must reduce
to, the additivity of the KL bound over a layer's outputs, and central
differences of its own ELBO for the analytic gradients (every T held fixed).
"""
import copy

import numpy as np
import pytest

from oracle import dgp as G
from oracle import rsvgp as R

M, D, B = 6, 2, 7


def _layer(Q, Din, seed, scale=0.3):
    r = np.random.default_rng([seed, 5])
    Z = r.normal(size=(M, Din))
    lp = dict(Z=Z, ell=r.uniform(0.7, 1.5, Din), sf2=r.uniform(0.5, 1.5), s=r.uniform(0.05, 0.3, M),
              m=scale * r.normal(size=(M, Q)))
    Kt = R.se_ard(Z, Z, lp["ell"], lp["sf2"]) + np.diag(lp["s"])
    # near the NG fixed point chol(K~^-1), not on it
    lp["L"] = np.linalg.cholesky(np.linalg.inv(Kt)) * (1.0 + 0.05 * np.tril(r.normal(size=(M, M))))
    return lp


def _data(seed):
    r = np.random.default_rng([seed, 6])
    return r.normal(size=(B, D)), r.normal(size=B)


def test_one_layer_is_the_rsvgp_bound():
    """With only the output layer the deep-GP ELBO and its gradients are the
    single-layer bound of Eq. (7) and its gradients."""
    X, y = _data(0)
    lp = _layer(1, D, 1)
    p = dict(lp, m=lp["m"][:, 0], noise=0.4)
    assert G.elbo([lp], X, y, 50, 0.4, []) == pytest.approx(R.bound(p, X, y, 50)["F"], rel=1e-13)
    g, dn = G.grads([lp], X, y, 50, 0.4, [])
    ref = R.grads(p, X, y, 50)
    for k in ("Z", "ell", "sf2", "s"):
        np.testing.assert_allclose(g[0][k], ref[k], rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(g[0]["m"][:, 0], ref["m"], rtol=1e-10, atol=1e-12)
    assert dn == pytest.approx(ref["noise"], rel=1e-12)


def test_kl_adds_over_a_layers_outputs():
    """Outputs sharing Z, the kernel, S~ and T: with Q identical mean columns
    the layer's KL bound is Q times the single-output bound and the Q moment
    columns coincide."""
    X, _ = _data(1)
    lp = _layer(1, D, 2)
    Q = 3
    lq = dict(lp, m=np.repeat(lp["m"], Q, axis=1))
    f1, fq = G.layer_forward(lp, X), G.layer_forward(lq, X)
    assert fq["KL"] == pytest.approx(Q * f1["KL"], rel=1e-12)
    for q in range(Q):
        np.testing.assert_allclose(fq["mu"][:, q], f1["mu"][:, 0], rtol=1e-13)
    np.testing.assert_allclose(fq["var"], f1["var"], rtol=1e-13)


def test_zero_draws_and_zero_hidden_mean_pass_the_inputs_through():
    """A hidden layer with m~ = 0 and zero draws outputs its inputs unchanged
    (identity mean, mu = 0): the two-layer ELBO is the output layer's bound
    at X minus the hidden layer's KL, and the output layer's gradients are
    those of the single-layer bound."""
    X, y = _data(2)
    hid = dict(_layer(D, D, 3), m=np.zeros((M, D)))
    out = _layer(1, D, 4)
    p = dict(out, m=out["m"][:, 0], noise=0.3)
    eps = [np.zeros((B, D))]
    F = G.elbo([hid, out], X, y, 40, 0.3, eps)
    assert F == pytest.approx(R.bound(p, X, y, 40)["F"] - G.layer_forward(hid, X)["KL"], rel=1e-12)
    g, _ = G.grads([hid, out], X, y, 40, 0.3, eps)
    ref = R.grads(p, X, y, 40)
    for k in ("Z", "ell", "sf2", "s"):
        np.testing.assert_allclose(g[1][k], ref[k], rtol=1e-10, atol=1e-12)


def _fd(layers, X, y, N, noise, eps, l, k, h=1e-6):
    base = np.asarray(layers[l][k], np.float64)
    out = np.zeros(base.size)
    for idx in range(base.size):
        vals = []
        for sgn in (1.0, -1.0):
            lp = copy.deepcopy(layers)
            a = base.reshape(-1).copy()
            a[idx] += sgn * h
            lp[l][k] = a.reshape(base.shape) if base.ndim else float(a[0])
            vals.append(G.elbo(lp, X, y, N, noise, eps))
        out[idx] = (vals[0] - vals[1]) / (2 * h)
    return out


@pytest.mark.parametrize("depth,seed", [(2, 0), (2, 1), (3, 2)])
def test_gradients_match_central_differences(depth, seed):
    """Every gradient block of every layer (and the noise variance) against
    central differences of the ELBO at fixed draws, T held fixed; the hidden
    layers' gradients pass through the sampled outputs h = h_prev + mu +
    sigma eps."""
    X, y = _data(10 + seed)
    layers = [_layer(D, D, 20 + seed + l) for l in range(depth - 1)] + [_layer(1, D, 40 + seed)]
    r = np.random.default_rng([seed, 7])
    eps = [r.normal(size=(B, D)) for _ in range(depth - 1)]
    N, noise = 60.0, 0.35
    g, dn = G.grads(layers, X, y, N, noise, eps)
    for l in range(depth):
        for k in ("Z", "ell", "sf2", "m", "s"):
            fd = _fd(layers, X, y, N, noise, eps, l, k)
            an = np.asarray(g[l][k], np.float64).reshape(-1)
            assert np.linalg.norm(an - fd) <= 2e-6 * np.linalg.norm(fd), (l, k)
    h = 1e-6
    fdn = (G.elbo(layers, X, y, N, noise + h, eps) - G.elbo(layers, X, y, N, noise - h, eps)) / (2 * h)
    assert dn == pytest.approx(fdn, rel=1e-7)
