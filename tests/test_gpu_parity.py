"""GPU parity: the CUDA path (through the C-ABI) against the FP64 oracle.

Bound, gradients, NG update, prediction and Adam are compared on the same
seeded float32 inputs.  Tolerances: relative bound error <= 1e-6 (FP32 SIMT)
and <= 1e-3 (BF16 tensor cores); per-block relative gradient error <= 1e-4
(FP32) and <= 1e-2 (BF16).
"""
import math

import numpy as np
import pytest

from _helpers import BLOCKS, TOL, chol_inv, f32, gates, log_errors, make_case, rel, round_state, small_case
from oracle import rsvgp as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PRECS = ["fp32", "bf16", "bf16x3"]


def _model(p, M, D, B, prec, likelihood="gaussian", precond=True):
    from paper_2604_00697_gb300 import _lib
    from paper_2604_00697_gb300.model import RSVGP

    if prec != "fp32" and not _lib.svgp_has_tensor_cores():
        pytest.fail("tensor-core path not available on this device")
    m = RSVGP(M, D, B, prec=prec, likelihood=likelihood, precond=precond)
    m.set_state(p["Z"], p["ell"], p["sf2"], p["noise"], p["m"], p["s"], p["L"])
    return m


def _dev(a):
    return torch.tensor(np.asarray(a), dtype=torch.float32, device="cuda")


def _check_bound_and_grads(case, p, X, y, N, prec, grads=True, likelihood="gaussian", precond=True):
    """Bound and per-block gradients of the C-ABI path against the oracle at
    the stated gates (bound 1e-6 / 1e-3, gradients 1e-4 / 1e-2 for FP32 /
    BF16 forms) unless the case is listed as out of reach.  Every
    exceedance of the case is reported in one assertion."""
    M, D = p["Z"].shape
    B = X.shape[0]
    m = _model(p, M, D, B, prec, likelihood, precond)
    Xd, yd = _dev(X), _dev(y)
    ref = O.bound(p, X, y, N, likelihood=likelihood, precond=precond)
    if grads:
        terms = m.backward(Xd, yd, N)
    else:
        terms = m.bound(Xd, yd, N)
    torch.cuda.synchronize()
    assert m.sync_status() == 0
    t = terms.cpu().numpy()
    F = t[0]
    tb, tg = gates(case, prec)
    err = abs(F - ref["F"]) / abs(ref["F"])
    out = {"bound": err}
    bad = [] if err <= tb else [("bound", err, tb)]
    if likelihood == "probit":
        # sum_n sigma_n^2 = B sf2 - sum_n k_n^T P k_n: its rounding error scales with B sf2
        out["sumvar"] = abs(t[8] - np.maximum(ref["var"], 0.0).sum()) / (B * p["sf2"])
        if not out["sumvar"] <= tg["sumvar"]:
            bad.append(("sumvar", out["sumvar"], tg["sumvar"]))
        assert 0.0 <= t[10] <= B and t[10] == int(t[10])
    if grads:
        g = O.grads(p, X, y, N, likelihood=likelihood, precond=precond)
        for k in BLOCKS:
            gg = m.grad_of(k).double().cpu().numpy().reshape(np.shape(g[k]))
            if likelihood == "probit" and k == "noise":
                assert np.all(gg == 0.0)
                continue
            e = rel(gg, g[k])
            out[k] = e
            if not e <= tg[k]:
                bad.append((k, e, tg[k]))
    m.close()
    log_errors(case, prec, out)
    assert not bad, (case, prec, bad)
    return out


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("state", ["init", "chol"])
def test_snelson_like_bound_and_grads(prec, state):
    p, X, y, N = make_case("snelson_like", state)
    _check_bound_and_grads(f"snelson_like/{state}", p, X, y, N, prec)


@pytest.mark.parametrize("prec", PRECS + ["bf16x3k"])
@pytest.mark.parametrize("M,D,B,seed", [(200, 3, 300, 0), (130, 5, 129, 1), (1, 2, 7, 2), (257, 1, 1, 3),
                                        (300, 19, 260, 4)])
def test_ragged_random_state(prec, M, D, B, seed):
    p, X, y, N = small_case(M, D, B, seed)
    _check_bound_and_grads(f"random/{M}x{D}x{B}", p, X, y, N, prec)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("state", ["init", "chol"])
def test_sinusoid_regression_M512(prec, state):
    p, X, y, N = make_case("sinusoid_regression", state)
    _check_bound_and_grads(f"sinusoid_regression/{state}", p, X, y, N, prec)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("state", ["init", "chol"])
def test_gp_sample_full_size(prec, state):
    """M=2048, B=4096, D=16, N=1e6: the benchmark's workload."""
    p, X, y, N = make_case("gp_sample_regression", state)
    _check_bound_and_grads(f"gp_sample_regression/{state}", p, X, y, N, prec)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("lik", ["gaussian", "probit"])
@pytest.mark.parametrize("M,D,B,seed", [(200, 3, 300, 0), (57, 4, 1000, 1)])
def test_unpreconditioned_bound_and_grads(prec, lik, M, D, B, seed):
    """R-SVGP without the mean preconditioner (m = Kuu m~, Section 2)."""
    p, X, y, N = small_case(M, D, B, seed)
    if lik == "probit":
        y = _probit_labels(X, seed)
    _check_bound_and_grads(f"unprec/{lik}/{M}x{D}x{B}", p, X, y, N, prec, likelihood=lik, precond=False)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("sigma2", [0.0, 0.02])
def test_variance_gap_matches_oracle(prec, sigma2):
    """Prop. 3 gap G = sum_n ||(I - K~ T) k_un||^2 / sigma2 (sigma2 = 0: min s~)."""
    p, X, y, N = small_case(130, 3, 300, 4)
    m = _model(p, 130, 3, 300, prec)
    G = float(m.variance_gap(_dev(X), _dev(y), N, sigma2=sigma2)[0])
    assert m.sync_status() == 0
    ref = O.variance_gap(p, X, sigma2 if sigma2 > 0 else None).sum()
    tol = {"fp32": 1e-4, "bf16": 2e-2, "bf16x3": 1e-3}[prec]
    assert abs(G - ref) <= tol * ref, (G, ref)
    m.close()


@pytest.mark.parametrize("prec", PRECS)
def test_ng_update_with_gap_rule_matches_oracle(prec):
    """NG updates with the Section 3.3 gap stopping rule: same number of
    updates as the oracle for a threshold between two iterates, and L close
    to the oracle's."""
    p, X, y, N = small_case(96, 2, 200, 5)
    p["L"] = f32(0.6 * chol_inv(p))
    gam = [1.0, 1.0, 1.0, 1.0, 1.0]
    Kt = O.se_ard(p["Z"], p["Z"], p["ell"], p["sf2"]) + np.diag(p["s"])
    Gs = []
    for t in range(5):
        q = dict(p)
        q["L"] = O.ng_solve(p["L"], Kt, gam, max_iters=t)[0]
        Gs.append(O.variance_gap(q, X).sum())
    # stop at the first iterate at least 4x below the threshold's neighbour
    t_stop = next(t for t in range(1, 5) if Gs[t] < Gs[t - 1] / 16)
    eps = (Gs[t_stop] * 4.0) / (2.0 * p["noise"])
    Lr, itr, Gr = O.ng_solve_gap(p, X, gam, eps=eps)
    assert itr == t_stop
    m = _model(p, 96, 2, 200, prec)
    G = float(m.ng_update_gap(_dev(X), _dev(y), N, max_iters=5, eps=eps, gammas=gam)[0])
    assert m.sync_status() == 0
    assert int(m.iters[0]) == itr
    # three NG steps at cond(K~) = 1.3e3; in BF16 each step rounds A = L^T K~ L to
    # 2^-9 cnd, so the iterate is compared loosely (0.048 measured) -- the
    # point of the test is the stopping decision, which must match exactly
    tol = {"fp32": 1e-4, "bf16": 1e-1, "bf16x3": 1e-3}[prec]
    assert rel(m.L.double().cpu().numpy(), Lr) <= tol
    m.close()


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("K", [1, 16, 200])
def test_bound_hutchinson_matches_oracle(prec, K):
    """Bound with the KL traces estimated from K Rademacher probes (Section
    3.4): same probes on both sides, so the estimate is compared exactly."""
    M = 130
    p, X, y, N = small_case(M, 3, 300, 6)
    probes = np.where(np.random.default_rng([K, 8]).uniform(size=(M, K)) < 0.5, -1.0, 1.0)
    ref = O.bound(p, X, y, N, probes=probes)
    m = _model(p, M, 3, 300, prec)
    t = m.bound_hutchinson(_dev(X), _dev(y), N, torch.tensor(probes, dtype=torch.float32)).cpu().numpy()
    assert m.sync_status() == 0
    tb = TOL[prec]["bound"]
    assert abs(t[0] - ref["F"]) <= tb * abs(ref["F"]), (t[0], ref["F"])
    log_errors(f"hutchinson/K{K}", prec, {"bound": abs(t[0] - ref["F"]) / abs(ref["F"]),
                                          "trKT": abs(t[3] - ref["tr_KtT"]) / max(1.0, abs(ref["tr_KtT"])),
                                          "trPKuu": abs(t[4] - ref["tr_PKuu"]) / max(1.0, abs(ref["tr_PKuu"]))})
    # the estimates come from FP32 chains (FP32 handles) or from tensor-core
    # chains in the handle's operand precision: hi/lo BF16 operands carry
    # about 16 bits (relative error of order 1e-5 per product); single BF16
    # has no separate tolerance beyond the bound's
    tt = {"fp32": 1e-5, "bf16x3": 1e-4}.get(prec)
    if tt is not None:
        assert abs(t[3] - ref["tr_KtT"]) <= tt * max(1.0, abs(ref["tr_KtT"])), (t[3], ref["tr_KtT"])
        assert abs(t[4] - ref["tr_PKuu"]) <= tt * max(1.0, abs(ref["tr_PKuu"])), (t[4], ref["tr_PKuu"])
    m.close()


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
@pytest.mark.parametrize("lik,precond,B", [("probit", True, 300), ("gaussian", False, 300), ("gaussian", True, 600)])
def test_bound_hutchinson_likelihoods_and_batches(prec, lik, precond, B):
    """The P-free bound of Section 3.4 for the probit likelihood, without the
    mean preconditioner, and for a batch of more than 256 points (three
    blocks of points, the last one ragged), against the oracle's bound with
    the same probes."""
    M, K = 130, 16
    p, X, y, N = small_case(M, 3, B, 9)
    if lik == "probit":
        y = f32((y > np.median(y)).astype(np.float64))
    probes = np.where(np.random.default_rng([K, 9]).uniform(size=(M, K)) < 0.5, -1.0, 1.0)
    ref = O.bound(p, X, y, N, likelihood=lik, precond=precond, probes=probes)
    m = _model(p, M, 3, B, prec, likelihood=lik, precond=precond)
    t = m.bound_hutchinson(_dev(X), _dev(y), N, torch.tensor(probes, dtype=torch.float32)).cpu().numpy()
    assert m.sync_status() == 0
    tb = TOL[prec]["bound"]
    log_errors(f"hutchinson/{lik}/{'pre' if precond else 'unpre'}/B{B}", prec, {"bound": abs(t[0] - ref["F"]) / abs(ref["F"])})
    assert abs(t[0] - ref["F"]) <= tb * abs(ref["F"]), (t[0], ref["F"])
    m.close()


def test_bound_hutchinson_more_probes_than_padded_rows():
    """K = 200 probes with M = 100 (padded to 128): the probe block does not
    fit the transposed M x M buffers, so a BF16X3 handle takes the FP32 path;
    the result still matches the oracle with the same probes."""
    M, K = 100, 200
    p, X, y, N = small_case(M, 3, 150, 11)
    probes = np.where(np.random.default_rng([K, 11]).uniform(size=(M, K)) < 0.5, -1.0, 1.0)
    ref = O.bound(p, X, y, N, probes=probes)
    m = _model(p, M, 3, 150, "bf16x3")
    t = m.bound_hutchinson(_dev(X), _dev(y), N, torch.tensor(probes, dtype=torch.float32)).cpu().numpy()
    assert m.sync_status() == 0
    assert abs(t[0] - ref["F"]) <= TOL["bf16x3"]["bound"] * abs(ref["F"]), (t[0], ref["F"])
    m.close()


def test_bound_hutchinson_exact_terms_agree_with_bound_at_M1024():
    """At M = 1024 with 200 points, the P-free path's exact terms (sum of
    squared errors, sum of sigma_n^2, the quadratic term, log-determinants)
    equal those of svgp_bound, which forms P by the O(M^3) chain (FP32
    handle: both in FP32 arithmetic)."""
    M, D, B = 1024, 4, 200
    p, X, y, N = small_case(M, D, B, 10, state="chol")
    probes = np.where(np.random.default_rng([3, 10]).uniform(size=(M, 8)) < 0.5, -1.0, 1.0)
    m = _model(p, M, D, B, "fp32")
    Xd, yd = _dev(X), _dev(y)
    t_exact = m.bound(Xd, yd, N).cpu().numpy().copy()
    t_hut = m.bound_hutchinson(Xd, yd, N, torch.tensor(probes, dtype=torch.float32)).cpu().numpy().copy()
    assert m.sync_status() == 0
    for k in (5, 6, 7, 8, 9):              # quad, logdetT, sqerr, sumvar, logdetS
        assert abs(t_hut[k] - t_exact[k]) <= 1e-4 * max(1.0, abs(t_exact[k])), (k, t_hut[k], t_exact[k])
    m.close()


def test_group_step_matches_separate_models():
    """Several SVGPs of different M stepped together (one CUDA graph with a
    branch per member) give the results of stepping each alone."""
    from paper_2604_00697_gb300.model import RSVGPGroup

    sizes = [(40, 3, 100), (130, 3, 300), (256, 4, 512), (70, 2, 64)]
    cases = [small_case(M, D, B, 20 + k) for k, (M, D, B) in enumerate(sizes)]

    def make():
        ms = []
        for (M, D, B), (p, X, y, N) in zip(sizes, cases):
            ms.append(_model(p, M, D, B, "bf16"))
        return ms

    solo = make()
    for m, (p, X, y, N) in zip(solo, cases):
        m.train_step(_dev(X), _dev(y), N)
    torch.cuda.synchronize()
    group = RSVGPGroup(make())
    batches = [(_dev(X), _dev(y), N) for (p, X, y, N) in cases]
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        g = group.capture(batches)
    torch.cuda.current_stream().wait_stream(s)
    g.replay()
    torch.cuda.synchronize()
    assert group.sync_status() == [0] * len(sizes)
    for a, b in zip(solo, group.models):
        np.testing.assert_allclose(b.terms.cpu().numpy()[:10], a.terms.cpu().numpy()[:10], rtol=1e-6, atol=1e-9)
        np.testing.assert_allclose(b.cons.cpu().numpy(), a.cons.cpu().numpy(), rtol=1e-5, atol=1e-6)
        np.testing.assert_allclose(b.L.cpu().numpy(), a.L.cpu().numpy(), rtol=1e-5, atol=1e-7)
    for m in solo:
        m.close()
    group.close()


def _probit_labels(X, seed):
    """Binary labels from a smooth random latent function of X."""
    rng = np.random.default_rng([seed, 41])
    f = np.sin(X @ rng.normal(size=X.shape[1]) * 1.5) + 0.3 * rng.normal(size=X.shape[0])
    return (f > 0).astype(np.float64)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("M,D,B,seed", [(200, 2, 300, 0), (130, 5, 129, 1), (1, 2, 7, 2), (33, 19, 65, 3)])
def test_probit_ragged_random_state(prec, M, D, B, seed):
    """Bernoulli-probit bound and gradients (20-point Gauss-Hermite) against the
    oracle at ragged sizes; D = 19 is the largest the tensor-core generator takes."""
    p, X, _, N = small_case(M, D, B, seed)
    y = _probit_labels(X, seed)
    _check_bound_and_grads(f"probit/{M}x{D}x{B}", p, X, y, N, prec, likelihood="probit")


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("state", ["init", "chol"])
def test_probit_banana_config(prec, state):
    """M=256, B=2048, D=2, N=5e4: the probit classification workload.

    "chol" uses s~ = 0.5 (cond(K~) = 277; with the 256 inducing points on
    the 2-D crescents, s~ = 1e-2 gives cond(K~) = 1.4e4)."""
    p, X, y, N = make_case("banana_like", state)
    assert set(np.unique(y)) <= {0.0, 1.0}
    if state == "chol":
        p["s"] = f32(np.full(p["Z"].shape[0], 0.5))
        p["L"] = f32(chol_inv(p))
    _check_bound_and_grads(f"banana_like/{state}", p, X, y, N, prec, likelihood="probit")


@pytest.mark.parametrize("prec", PRECS + ["bf16x3k"])
@pytest.mark.parametrize("M,D,seed", [(16, 1, 0), (200, 3, 1), (512, 8, 2)])
def test_ng_step_matches_oracle(prec, M, D, seed):
    p, _, _, _ = small_case(M, D, 4, seed)
    p["L"] = f32(0.5 * chol_inv(p) + 0.02 * np.tril(np.random.default_rng(seed).normal(size=(M, M))) / math.sqrt(M))
    Kt = O.se_ard(p["Z"], p["Z"], p["ell"], p["sf2"]) + np.diag(p["s"])
    L1, r = O.ng_step(p["L"], Kt, 0.7)
    m = _model(p, M, D, 4, prec)
    m.ng_update(max_iters=1, eps=0.0, gammas=[0.7])
    torch.cuda.synchronize()
    Lg = m.L.double().cpu().numpy()
    tol = {"fp32": 1e-5, "bf16": 2e-2, "bf16x3": 1e-4, "bf16x3k": 1e-4}[prec]
    assert rel(Lg, L1) <= tol
    assert abs(float(m.resid[0]) - r) <= tol * max(r, 1.0)
    assert int(m.iters[0]) == 1
    assert np.all(np.triu(Lg, 1) == 0.0)
    m.close()


@pytest.mark.parametrize("prec", PRECS)
def test_ng_converges_to_fixed_point_with_stopping_rule(prec):
    M, D = 96, 2
    p, _, _, _ = small_case(M, D, 4, 7)
    p["s"] = f32(np.full(M, 0.2))
    Kt = O.se_ard(p["Z"], p["Z"], p["ell"], p["sf2"]) + np.diag(p["s"])
    Ls = np.linalg.cholesky(np.linalg.inv(Kt))
    p["L"] = f32(1e-3 * np.eye(M))
    eps = {"fp32": 1e-4, "bf16": 3e-2, "bf16x3": 1e-4}[prec]
    m = _model(p, M, D, 4, prec)
    gam = [O.gamma_schedule(t, gamma0=1e-1, ramp=5) for t in range(60)]
    m.ng_update(max_iters=60, eps=eps, gammas=gam)
    torch.cuda.synchronize()
    it, r = int(m.iters[0]), float(m.resid[0])
    assert r < eps and it < 60
    Lo, ito, ro = O.ng_solve(p["L"], Kt, gam, eps=eps, max_iters=60)
    assert abs(it - ito) <= {"fp32": 0, "bf16": 3, "bf16x3": 1}[prec]
    assert rel(m.L.double().cpu().numpy(), Ls) <= {"fp32": 1e-3, "bf16": 5e-2, "bf16x3": 1e-3}[prec]
    m.close()


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("Ns", [1, 300])
def test_predict_matches_oracle(prec, Ns):
    M, D = 150, 3
    p, _, _, _ = small_case(M, D, 4, 9, state="chol")
    Xs = f32(np.random.default_rng(4).normal(size=(Ns, D)))
    mean, var = O.predict(p, Xs, include_noise=True)
    m = _model(p, M, D, Ns, prec)
    gm, gv = m.predict(_dev(Xs), include_noise=True)
    torch.cuda.synchronize()
    em, ev = rel(gm.double().cpu().numpy(), mean), rel(gv.double().cpu().numpy(), var)
    log_errors(f"predict/Ns{Ns}", prec, {"mean": em, "var": ev})
    # no stated tolerance for the predictive moments: about 2.5 x the errors
    # measured on a GB300 (FP32 6e-6; BF16X3 3.9e-4, limited by the Kuf
    # generator's exponent; single BF16 5.7e-2)
    tol = {"fp32": 1e-4, "bf16": 0.15, "bf16x3": 1e-3}[prec]
    assert em <= tol and ev <= tol, (em, ev, tol)
    m.close()


@pytest.mark.parametrize("prec", ["fp32"])
def test_adam_step_matches_oracle(prec):
    M, D = 40, 3
    p, X, y, N = small_case(M, D, 50, 12)
    g = O.grads(p, X, y, N)
    g = {k: f32(np.asarray(v)) for k, v in g.items()}
    m = _model(p, M, D, 50, prec)
    for k in BLOCKS:
        m.grad[m.sl[k]] = _dev(np.reshape(g[k], -1))
    raw0 = m.raw.double().cpu().numpy().copy()
    m.adam_step()
    torch.cuda.synchronize()
    raw = {k: raw0[m.sl[k]].reshape(np.shape(p[k])) for k in BLOCKS}
    new = O.adam_update(raw, g, {}, 5e-3)
    cons = O.constrain(new)
    for k in BLOCKS:
        gv = m.cons[m.sl[k]].double().cpu().numpy().reshape(np.shape(p[k]))
        assert rel(gv, cons[k]) <= 1e-5, k
    assert int(m.step[0]) == 1
    m.close()


def test_short_training_trajectory_fp32():
    """20 alternating NG + Adam steps (Section 3.1) on the 1-D workload."""
    import svgp_synth as S

    prob = S.snelson_like()
    X, y = prob.batch(0)
    X, y = f32(X), f32(y)
    p0 = round_state(dict(Z=prob.Z0, ell=np.array([1.0]), sf2=1.0, noise=1.0, m=np.zeros(prob.M),
                          s=np.full(prob.M, 1e-4), L=1e-3 * np.eye(prob.M)))
    _, trace = O.train(p0, lambda t: (X, y), prob.N, steps=20, lr=5e-3, train_Z=True)
    m = _model(p0, prob.M, 1, prob.B, "fp32")
    Xd, yd = _dev(X), _dev(y)
    got = []
    for _ in range(20):
        m.ng_update(max_iters=1, gammas=[1.0])
        got.append(float(m.backward(Xd, yd, prob.N)[0]))
        m.adam_step()
    torch.cuda.synchronize()
    np.testing.assert_allclose(got, trace, rtol=1e-4)
    m.close()


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_training_with_adaptive_ng_loop(prec):
    """Alternating optimisation with the adaptive number of NG steps of
    Section 3.3 (Frobenius stopping rule, Eq. (8)) and the log-linear step-size
    schedule of Section 3.4, at the paper's Adam learning rate 5e-3 on every
    block: 30 steps on the sinusoid workload (M = 512) from the paper's initial
    state, against the oracle's training driver.  The number of NG updates of
    every step must match the oracle's, and the bound track it (BF16X3 within
    its stated bound gate; FP32 within 1e-4, as in the fixed-step trajectory
    test above)."""
    import svgp_synth as S

    prob = S.sinusoid_regression()
    X, y = prob.batch(0)
    X, y = f32(X), f32(y)
    M, D = prob.M, prob.D
    p0 = round_state(dict(Z=prob.Z0, ell=np.ones(D), sf2=1.0, noise=1.0, m=np.zeros(M),
                          s=np.full(M, 1e-4), L=1e-3 * np.eye(M)))
    steps, eps, max_ng = 30, 0.02, 4
    gam = O.gamma_schedule
    ref_counts = []
    _, trace = O.train(p0, lambda t: (X, y), prob.N, steps=steps, lr=5e-3, gamma=gam, eps=eps, max_ng=max_ng,
                       ng_counts=ref_counts)
    m = _model(p0, M, D, prob.B, prec)
    Xd, yd = _dev(X), _dev(y)
    got, counts, t_ng = [], [], 0
    for _ in range(steps):
        m.ng_update(max_iters=max_ng, eps=eps, gammas=[gam(t_ng + k) for k in range(max_ng)])
        n_it = int(m.iters.item())
        counts.append(n_it)
        t_ng += n_it
        got.append(float(m.backward(Xd, yd, prob.N)[0]))
        m.adam_step()
    torch.cuda.synchronize()
    assert m.sync_status() == 0
    assert np.all(np.isfinite(got))
    assert counts == ref_counts, (counts, ref_counts)
    assert sum(counts) > steps and min(counts) < max_ng, counts   # the rule both iterates and stops
    np.testing.assert_allclose(got, trace, rtol=TOL[prec]["bound"] if prec != "fp32" else 1e-4)
    m.close()


def test_nonfinite_input_is_reported():
    from paper_2604_00697_gb300 import _lib

    p, X, y, N = small_case(20, 2, 30, 1)
    X = X.copy()
    X[3, 1] = np.nan
    m = _model(p, 20, 2, 30, "fp32")
    m.bound(_dev(X), _dev(y), N)
    assert m.sync_status() == _lib.SVGP_ERR_NONFINITE
    assert m.sync_status() == 0      # cleared after reading
    m.close()


def test_invalid_arguments_are_rejected():
    from paper_2604_00697_gb300 import _lib

    with pytest.raises(_lib.SvgpError):
        _lib.svgp_create(0, 2, 10, _lib.SVGP_FP32)
    with pytest.raises(_lib.SvgpError):
        _lib.svgp_create(10, 33, 10, _lib.SVGP_FP32)
    p, X, y, N = small_case(20, 2, 30, 1)
    m = _model(p, 20, 2, 10, "fp32")
    with pytest.raises(_lib.SvgpError):
        m.bound(_dev(X), _dev(y), N)     # B = 30 > B_max = 10
    m.close()


def test_graph_captured_step_matches_eager():
    import svgp_synth as S

    p, X, y, N = make_case("sinusoid_regression", "init")
    M, D = p["Z"].shape
    B = X.shape[0]
    ms = []
    for _ in range(2):
        m = _model(p, M, D, B, "fp32")
        ms.append(m)
    Xd, yd = _dev(X), _dev(y)
    a, b = ms
    g = b.capture(Xd, yd, N)
    b.set_state(p["Z"], p["ell"], p["sf2"], p["noise"], p["m"], p["s"], p["L"])
    for _ in range(3):
        a.train_step(Xd, yd, N)
        g.replay()
    torch.cuda.synchronize()
    assert torch.allclose(a.cons, b.cons, rtol=1e-5, atol=1e-7) and torch.allclose(a.L, b.L, rtol=1e-5, atol=1e-9)
    assert abs(float(a.terms[0]) - float(b.terms[0])) <= 1e-9 * abs(float(a.terms[0]))
    for m in ms:
        m.close()


@pytest.mark.parametrize("prec", PRECS)
def test_fused_train_step_matches_separate_calls(prec):
    """svgp_train_step = svgp_ng_update_T followed by svgp_backward on the
    updated L (two NG iterations, so the between-iteration copies and the
    final log-determinant refresh are both exercised)."""
    p, X, y, N = make_case("sinusoid_regression", "chol")
    M, D = p["Z"].shape
    B = X.shape[0]
    a = _model(p, M, D, B, prec)
    b = _model(p, M, D, B, prec)
    Xd, yd = _dev(X), _dev(y)
    for m in (a, b):
        m.gamma[:2] = torch.tensor([0.7, 0.9], device=m.dev)
    a.ng_update(max_iters=2)
    ta = a.backward(Xd, yd, N).clone()
    tb = b.ng_backward(Xd, yd, N, t_star=2).clone()
    torch.cuda.synchronize()
    assert int(a.iters.item()) == int(b.iters.item()) == 2
    torch.testing.assert_close(a.L, b.L, rtol=0, atol=0)
    np.testing.assert_allclose(tb.cpu().numpy(), ta.cpu().numpy(), rtol=2e-6, atol=1e-9)
    np.testing.assert_allclose(b.grad.cpu().numpy(), a.grad.cpu().numpy(), rtol=1e-4,
                               atol=1e-5 * float(a.grad.abs().max()))
    a.close()
    b.close()


def test_empty_batch_and_probit_options_are_rejected():
    from paper_2604_00697_gb300 import _lib

    p, X, y, N = small_case(20, 2, 30, 1)
    m = _model(p, 20, 2, 30, "bf16")
    with pytest.raises(_lib.SvgpError):
        m.bound(_dev(X[:0]), _dev(y[:0]), N)        # B = 0
    with pytest.raises(_lib.SvgpError):
        m.bound_hutchinson(_dev(X), _dev(y), N, torch.ones(20, 257))   # K > 256
    m.close()
    with pytest.raises(_lib.SvgpError):           # gh_points > 32
        _lib.svgp_create(20, 2, 30, _lib.SVGP_BF16, lik=_lib.SVGP_LIK_BERNOULLI_PROBIT, gh_points=33)
    pm = _model(p, 20, 2, 30, "bf16", likelihood="probit")
    with pytest.raises(_lib.SvgpError):           # the gap rule is for the Gaussian likelihood
        pm.ng_update_gap(_dev(X), _dev(y), N, max_iters=1)
    pm.close()


@pytest.mark.parametrize("prec", PRECS)
def test_ng_fixed_point_at_large_M(prec):
    """M = 4096 (twice the benchmark's): at L = chol(K~^-1) the NG residual of
    Eq. (8) is only rounding, about u cond(K~), and the update leaves L there
    (a property that holds at any size, checked without an M^3 oracle run on
    the GPU's side)."""
    M, D = 4096, 4
    rng = np.random.default_rng(31)
    p = dict(Z=rng.uniform(-2, 2, size=(M, D)), ell=np.full(D, 0.8), sf2=1.0, noise=0.5,
             m=np.zeros(M), s=np.full(M, 0.5), L=np.eye(M))
    p = round_state(p)
    Kt = O.se_ard(p["Z"], p["Z"], p["ell"], p["sf2"]) + np.diag(p["s"])
    p["L"] = f32(np.linalg.cholesky(np.linalg.inv(Kt)))
    ev = np.linalg.eigvalsh(Kt)
    kappa = ev[-1] / ev[0]
    m = _model(p, M, D, 8, prec)
    m.ng_update(max_iters=1, eps=0.0, gammas=[1.0])
    torch.cuda.synchronize()
    assert m.sync_status() == 0
    r = float(m.resid[0])
    u = {"fp32": 2.0 ** -24, "bf16": 2.0 ** -9, "bf16x3": 2.0 ** -17}[prec]
    assert r <= 8 * u * kappa, (r, kappa)
    assert rel(m.L.double().cpu().numpy(), p["L"]) <= 8 * u * kappa
    m.close()


def _trajectory_states(prob, prec):
    """The benchmark's three states of the workload, produced on the GPU:
    the paper's initial state (Appendix S5.3), after 40 NG updates of L with
    gamma = 1, and after a further 50 training steps (NG update + bound +
    gradient + Adam, learning rate 1e-3, 2e-4 for Z).  Yields (name, state)
    with the state read back from the device as float64."""
    M, D = prob.M, prob.D
    p = round_state(dict(Z=prob.Z0, ell=np.ones(D), sf2=1.0, noise=1.0, m=np.zeros(M),
                         s=np.full(M, 1e-4), L=1e-3 * np.eye(M)))
    m = _model(p, M, D, prob.B, prec)
    yield "init", dict(p)
    m.ng_update(max_iters=40, gammas=[1.0] * 40)
    torch.cuda.synchronize()
    p["L"] = m.L.double().cpu().numpy()
    yield "ng40", dict(p)
    m.hyper[0] = 1e-3
    m.hyper[4] = 0.2
    for k in range(50):
        Xk, yk = prob.batch(1 + k)
        m.train_step(_dev(Xk), _dev(yk), prob.N)
    torch.cuda.synchronize()
    assert m.sync_status() == 0
    q = {k: m.get(k).double().cpu().numpy() for k in ("Z", "ell", "m", "s")}
    q["sf2"] = float(m.get("sf2")[0])
    q["noise"] = float(m.get("noise")[0])
    q["L"] = m.L.double().cpu().numpy()
    m.close()
    yield "train50", q


@pytest.mark.parametrize("prec", PRECS)
def test_gp_sample_trajectory_states(prec):
    """M=2048, B=4096, D=16, N=1e6 at the benchmark's three states: bound and
    every gradient block against the oracle at the state the GPU reached."""
    import svgp_synth as S

    prob = S.gp_sample_regression()
    X, y = prob.batch(0)
    X, y = f32(X), f32(y)
    for name, p in _trajectory_states(prob, prec):
        _check_bound_and_grads(f"gp_sample_regression/{name}", p, X, y, prob.N, prec)


@pytest.mark.parametrize("prec", PRECS)
def test_autograd_function_matches_oracle(prec):
    """F.backward() through the autograd Function fills every parameter's
    .grad with the library's gradient (T held fixed, Section 3.1), scaled by
    the incoming gradient; the no-grad forward gives the same bound."""
    from paper_2604_00697_gb300.autograd import RSVGPModule

    case = "sinusoid_regression/chol"
    p, X, y, N = make_case("sinusoid_regression", "chol")
    M, D = p["Z"].shape
    mod = RSVGPModule(M, D, X.shape[0], prec=prec)
    mod.set_state(p["Z"], p["ell"], p["sf2"], p["noise"], p["m"], p["s"], p["L"])
    Xd, yd = _dev(X), _dev(y)
    mod.zero_grad()
    F, terms = mod(Xd, yd, N)
    assert F.requires_grad and not terms.requires_grad
    (2.0 * F).backward()
    torch.cuda.synchronize()
    assert mod.core.sync_status() == 0
    ref = O.bound(p, X, y, N)
    g = O.grads(p, X, y, N)
    tb, tg = gates(case, prec)
    assert abs(float(F.detach()) - ref["F"]) <= tb * abs(ref["F"])
    for k in BLOCKS:
        gg = getattr(mod, k).grad.double().cpu().numpy().reshape(np.shape(g[k])) / 2.0
        assert rel(gg, g[k]) <= tg[k], (k, rel(gg, g[k]))
    # the .grad tensors alias the flat gradient the library's Adam reads
    assert mod.Z.grad.data_ptr() == mod.core.grad.data_ptr()
    torch.testing.assert_close(mod.core.grad_of("m"), mod.m.grad, rtol=0, atol=0)
    with torch.no_grad():
        F2, _ = mod(Xd, yd, N)
    # same forward pass; only the order of the FP64 atomic sums differs
    assert abs(float(F2) - float(F.detach())) <= 1e-8 * abs(float(F.detach()))
    # gradients accumulate over backward passes until zero_grad()
    g1 = mod.s.grad.clone()
    F3, _ = mod(Xd, yd, N)
    F3.backward()
    # (the second pass repeats the first up to the order of atomic sums; ds~,
    # the most cancellation-sensitive block, moved by 3.3e-5 between passes)
    assert rel(mod.s.grad.double().cpu().numpy(), 1.5 * g1.double().cpu().numpy()) <= 1e-3
    mod.zero_grad()
    assert float(mod.core.grad.abs().max()) == 0.0
    mod.close()


def test_split_schedules_agree_and_autotune_restores_state():
    """Every split-K threshold of the triangular products gives the bound and
    gradients of the whole-tile schedule (up to the order of the FP32 sums);
    the measured tuner picks a listed candidate per kind and leaves the
    model's state as it found it; invalid settings are rejected."""
    from paper_2604_00697_gb300 import _lib

    p, X, y, N = make_case("gp_sample_regression", "chol")
    M, D = p["Z"].shape
    m = _model(p, M, D, X.shape[0], "bf16x3")
    Xd, yd = _dev(X), _dev(y)
    kinds = {"sym": 1, "lupd": 2, "out": 4}
    cands = {k: _lib.svgp_split_candidates(m.h, i) for k, i in kinds.items()}
    assert all(c[0] == 0 and len(c) > 2 for c in cands.values())
    assert _lib.svgp_split_candidates(m.h, 0) == [0]            # VT keeps whole tiles
    ref_t, ref_g = None, None
    for c in range(max(len(v) for v in cands.values())):
        for k, i in kinds.items():
            _lib.svgp_set_split(m.h, i, cands[k][min(c, len(cands[k]) - 1)])
        t = m.backward(Xd, yd, N).cpu().numpy().copy()
        g = m.grad.double().cpu().numpy().copy()
        assert m.sync_status() == 0
        if ref_t is None:
            ref_t, ref_g = t, g
            continue
        # the schedules differ only in the order of the FP32 sums (1.2e-6
        # measured on the bound, against 9e-6 error of the form itself)
        assert abs(t[0] - ref_t[0]) <= 1e-5 * abs(ref_t[0]), (c, t[0], ref_t[0])
        assert rel(g, ref_g) <= 1e-4, (c, rel(g, ref_g))
    cons0, L0 = m.cons.clone(), m.L.clone()
    tuned = m.autotune_split(Xd, yd, N, reps=1)
    assert set(tuned) == set(kinds)
    for k, i in kinds.items():
        assert tuned[k]["kmin"] in cands[k] and _lib.svgp_get_split(m.h, i) == tuned[k]["kmin"]
    torch.testing.assert_close(m.cons, cons0, rtol=0, atol=0)
    torch.testing.assert_close(m.L, L0, rtol=0, atol=0)
    with pytest.raises(_lib.SvgpError):
        _lib.svgp_set_split(m.h, 0, 12)                          # a full product
    with pytest.raises(_lib.SvgpError):
        _lib.svgp_set_split(m.h, 1, 1)                           # below the smallest candidate
    _lib.svgp_set_split(m.h, 1, -1)                              # back to the cost model
    assert _lib.svgp_get_split(m.h, 1) in cands["sym"]
    m.close()


def _errors_at(p, X, y, N, prec):
    M, D = p["Z"].shape
    m = _model(p, M, D, X.shape[0], prec)
    F = float(m.backward(_dev(X), _dev(y), N)[0])
    torch.cuda.synchronize()
    assert m.sync_status() == 0
    ref = O.bound(p, X, y, N)["F"]
    g = O.grads(p, X, y, N)
    out = {"bound": abs(F - ref) / abs(ref)}
    for k in BLOCKS:
        out[k] = rel(m.grad_of(k).double().cpu().numpy().reshape(np.shape(g[k])), g[k])
    m.close()
    return out


def test_three_plane_kuu_at_an_ill_conditioned_state():
    """SVGP_BF16X3K against SVGP_BF16X3 where the rounding of Kuu in L^T K~
    dominates dZ: the largest member of the 64-SVGP group workload at its
    converged state (M = 2048 inducing points at the batch's own points,
    D = 8, cond(K~) about 3e3).  The CPU rounding study of the chain puts
    dZ at 7.0e-3 -> 1.2e-3; measured on a GB300, 8.4e-3 -> 2.3e-3 (two
    runs).  The other gradient blocks are not asserted here: dell is
    1.6e-2 in both forms, an error the chain's rounding does not explain
    (the CPU study gives 3.5e-4 for it)."""
    import svgp_synth as S

    prob = S.sinusoid_regression(seed=100, B=2048, M=2048, D=8)
    X, y = prob.batch(0)
    M, D = 2048, 8
    p = round_state(dict(Z=prob.Z0, ell=np.ones(D), sf2=1.0, noise=1.0,
                         m=0.1 * np.random.default_rng(1).normal(size=M), s=np.full(M, 1e-4), L=np.eye(M)))
    p["L"] = f32(chol_inv(p))
    X, y = f32(X), f32(y)
    e3 = _errors_at(p, X, y, prob.N, "bf16x3")
    e5 = _errors_at(p, X, y, prob.N, "bf16x3k")
    log_errors("group_member_2048/chol", "bf16x3", e3)
    log_errors("group_member_2048/chol", "bf16x3k", e5)
    assert e5["bound"] <= 1e-3
    assert e5["Z"] <= 5e-3 and e5["Z"] < e3["Z"] / 2, (e3, e5)
