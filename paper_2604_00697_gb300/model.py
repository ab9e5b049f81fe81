"""Device state and training step of one R-SVGP model on top of the C-ABI.

PyTorch supplies device memory, streams and CUDA-graph capture; every step of
the computation runs in ``libsvgp.so``.  The training step follows the
alternating optimisation of Section 3.1: natural-gradient update(s) of L given
K~, then one Adam step on xi = {Z, ell, sf2, noise, m~, s~} with L fixed.
"""
from __future__ import annotations

import math

import torch

from . import _lib as C

PREC = {"fp32": C.SVGP_FP32, "bf16": C.SVGP_BF16, "bf16x3": C.SVGP_BF16X3, "bf16x3k": C.SVGP_BF16X3K}


def _softplus_inv(x: torch.Tensor) -> torch.Tensor:
    x = x.double()
    return (x + torch.log(-torch.expm1(-x))).float()


class RSVGP:
    """One model: flat constrained/raw parameter vectors, L, Adam moments.

    Flat layout (shared with svgp_adam_step): [Z (M*D) | ell (D) | sf2 | noise |
    m~ (M) | s~ (M)].  ``params`` points into the constrained vector.
    """

    def __init__(self, M: int, D: int, B_max: int, prec: str = "bf16", device: str = "cuda",
                 likelihood: str = "gaussian", gh_points: int = 20, precond: bool = True):
        if not torch.cuda.is_available():
            raise RuntimeError("RSVGP needs a CUDA device (no CPU fallback)")
        self.M, self.D, self.B_max = M, D, B_max
        self.prec = prec
        self.likelihood = likelihood
        self.dev = torch.device(device)
        lik = {"gaussian": C.SVGP_LIK_GAUSSIAN, "probit": C.SVGP_LIK_BERNOULLI_PROBIT}[likelihood]
        self.h = C.svgp_create(M, D, B_max, PREC[prec], lik=lik, cuda_stream=torch.cuda.current_stream().cuda_stream,
                               gh_points=gh_points, unpreconditioned=not precond)
        self.n = C.svgp_param_count(self.h)
        f32 = dict(device=self.dev, dtype=torch.float32)
        self.cons = torch.zeros(self.n, **f32)
        self.raw = torch.zeros(self.n, **f32)
        self.grad = torch.zeros(self.n, **f32)
        self.m1 = torch.zeros(self.n, **f32)
        self.m2 = torch.zeros(self.n, **f32)
        self.step = torch.zeros(1, device=self.dev, dtype=torch.int32)
        self.hyper = torch.tensor([5e-3, 0.9, 0.999, 1e-8, 1, 1, 1, 1, 1, 1], **f32)
        self.L = torch.zeros(M, M, **f32)
        self.gamma = torch.ones(64, **f32)
        self.terms = torch.zeros(C.SVGP_NTERMS, device=self.dev, dtype=torch.float64)
        self.iters = torch.zeros(1, device=self.dev, dtype=torch.int32)
        self.resid = torch.zeros(1, device=self.dev, dtype=torch.float64)
        o = 0
        self.sl = {}
        for name, size in (("Z", M * D), ("ell", D), ("sf2", 1), ("noise", 1), ("m", M), ("s", M)):
            self.sl[name] = slice(o, o + size)
            o += size
        self.params = C.svgp_params(*[self.cons[self.sl[k]].data_ptr() for k in ("Z", "ell", "sf2", "noise", "m", "s")],
                                    self.L.data_ptr())
        self.grads = C.svgp_grads(*[self.grad[self.sl[k]].data_ptr() for k in ("Z", "ell", "sf2", "noise", "m", "s")])

    def close(self):
        if self.h:
            C.svgp_destroy(self.h)
            self.h = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass

    # -- state ---------------------------------------------------------------
    def set_state(self, Z, ell, sf2, noise, m, s, L):
        def t(x):
            return torch.as_tensor(x, dtype=torch.float32).reshape(-1).to(self.dev)

        for k, v in (("Z", Z), ("ell", ell), ("sf2", [sf2]), ("noise", [noise]), ("m", m), ("s", s)):
            self.cons[self.sl[k]] = t(v)
        self.L.copy_(torch.as_tensor(L, dtype=torch.float32).reshape(self.M, self.M))
        raw = self.cons.clone()
        for k in ("ell", "sf2", "noise", "s"):
            raw[self.sl[k]] = _softplus_inv(self.cons[self.sl[k]])
        self.raw.copy_(raw)
        self.m1.zero_()
        self.m2.zero_()
        self.step.zero_()

    def get(self, name):
        v = self.cons[self.sl[name]]
        return v.reshape(self.M, self.D) if name == "Z" else v

    def grad_of(self, name):
        v = self.grad[self.sl[name]]
        return v.reshape(self.M, self.D) if name == "Z" else v

    def _sync_stream(self):
        C.svgp_set_stream(self.h, torch.cuda.current_stream().cuda_stream)

    @staticmethod
    def batch(X: torch.Tensor, y: torch.Tensor, N: float):
        return C.svgp_batch(X.data_ptr(), y.data_ptr(), X.shape[0], float(N))

    # -- entry points ----------------------------------------------------------
    def bound(self, X, y, N):
        self._sync_stream()
        C.svgp_bound(self.h, self.params, self.batch(X, y, N), self.terms.data_ptr())
        return self.terms

    def backward(self, X, y, N):
        self._sync_stream()
        C.svgp_backward(self.h, self.params, self.batch(X, y, N), self.terms.data_ptr(), self.grads)
        return self.terms

    def ng_update(self, max_iters=1, eps=0.0, gammas=None):
        self._sync_stream()
        if gammas is not None:
            g = torch.as_tensor(gammas, dtype=torch.float32)
            self.gamma[: g.numel()] = g.to(self.dev)
        if max_iters > self.gamma.numel():
            raise ValueError("max_iters larger than the gamma buffer")
        C.svgp_ng_update_T(self.h, self.params, self.L.data_ptr(), self.gamma.data_ptr(), max_iters, eps,
                           self.iters.data_ptr(), self.resid.data_ptr())

    def bound_hutchinson(self, X, y, N, probes):
        """Bound with the KL traces estimated from the probe columns (M x K, +-1)."""
        self._sync_stream()
        pr = probes.to(self.dev, torch.float32).contiguous()
        C.svgp_bound_hutchinson(self.h, self.params, self.batch(X, y, N), pr.data_ptr(), pr.shape[1],
                                self.terms.data_ptr())
        return self.terms

    def variance_gap(self, X, y, N, sigma2=0.0):
        """Prop. 3 gap G = sum_n ||(I - K~ T) k_un||^2 / sigma2 (sigma2 <= 0: min s~)."""
        self._sync_stream()
        gap = torch.zeros(1, device=self.dev, dtype=torch.float64)
        C.svgp_variance_gap(self.h, self.params, self.batch(X, y, N), sigma2, gap.data_ptr())
        return gap

    def ng_update_gap(self, X, y, N, max_iters=1, eps=0.0, gammas=None, sigma2=0.0):
        """NG updates of L with the Prop. 3 gap stopping rule (Section 3.3)."""
        self._sync_stream()
        if gammas is not None:
            g = torch.as_tensor(gammas, dtype=torch.float32)
            self.gamma[: g.numel()] = g.to(self.dev)
        if max_iters > self.gamma.numel():
            raise ValueError("max_iters larger than the gamma buffer")
        gap = torch.zeros(1, device=self.dev, dtype=torch.float64)
        C.svgp_ng_update_T_gap(self.h, self.params, self.batch(X, y, N), self.L.data_ptr(), self.gamma.data_ptr(),
                               max_iters, eps, sigma2, self.iters.data_ptr(), gap.data_ptr())
        return gap

    def predict(self, Xs, include_noise=False):
        self._sync_stream()
        mean = torch.empty(Xs.shape[0], device=self.dev)
        var = torch.empty(Xs.shape[0], device=self.dev)
        C.svgp_predict(self.h, self.params, Xs.data_ptr(), Xs.shape[0], mean.data_ptr(), var.data_ptr(),
                       include_noise)
        return mean, var

    def adam_step(self):
        self._sync_stream()
        C.svgp_adam_step(self.h, self.raw.data_ptr(), self.cons.data_ptr(), self.grad.data_ptr(),
                         self.m1.data_ptr(), self.m2.data_ptr(), self.step.data_ptr(), self.hyper.data_ptr())

    def ng_backward(self, X, y, N, t_star=1, eps=0.0):
        """NG update(s) of L given K~ (Prop. 1), then bound + gradient, in one
        call (svgp_train_step: the preparation is shared by both parts)."""
        self._sync_stream()
        if t_star > self.gamma.numel():
            raise ValueError("t_star larger than the gamma buffer")
        C.svgp_train_step(self.h, self.params, self.batch(X, y, N), self.L.data_ptr(), self.gamma.data_ptr(),
                          t_star, eps, self.iters.data_ptr(), self.resid.data_ptr(), self.terms.data_ptr(),
                          self.grads)
        return self.terms

    def train_step(self, X, y, N, t_star=1, eps=0.0):
        """NG update(s) of L given K~ (Prop. 1), then bound + gradient + Adam."""
        self.ng_backward(X, y, N, t_star=t_star, eps=eps)
        self.adam_step()
        return self.terms

    def capture(self, X, y, N, t_star=1, eps=0.0):
        """Capture one training step on (X, y) into a CUDA graph."""
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.train_step(X, y, N, t_star=t_star, eps=eps)
        self._sync_stream()
        return g

    def sync_status(self):
        return C.svgp_sync_status(self.h)

    # -- schedule tuning --------------------------------------------------------
    SPLIT_KINDS = {"sym": 1, "lupd": 2, "out": 4}   # SVGP_PROF_* of the triangular products

    def autotune_split(self, X, y, N, reps=4):
        """Measured choice of the split-K threshold of each triangular
        contraction kind (svgp_set_split): for every candidate the library
        lists, `reps` eager training steps from the same saved state with
        timing events around each contraction; each kind keeps its fastest
        candidate.  The state is restored afterwards; graphs captured on this
        model before the call must be captured again.  Returns
        {kind: {"kmin": chosen, "ms_per_step": {kmin: ms}}}."""
        if self.prec == "fp32":
            return {}
        state = (self.cons, self.raw, self.L, self.m1, self.m2, self.step)
        snap = [t.clone() for t in state]

        def restore():
            for dst, src in zip(state, snap):
                dst.copy_(src)

        cands = {k: C.svgp_split_candidates(self.h, i) for k, i in self.SPLIT_KINDS.items()}
        ms = {k: {} for k in self.SPLIT_KINDS}
        for c in range(max(len(v) for v in cands.values())):
            pick = {k: v[min(c, len(v) - 1)] for k, v in cands.items()}
            for k, i in self.SPLIT_KINDS.items():
                C.svgp_set_split(self.h, i, pick[k])
            restore()
            self.train_step(X, y, N)
            torch.cuda.synchronize()
            C.svgp_profile_enable(self.h, True)
            for _ in range(reps):
                self.train_step(X, y, N)
            torch.cuda.synchronize()
            prof = C.svgp_profile_read(self.h)
            C.svgp_profile_enable(self.h, False)
            for k in self.SPLIT_KINDS:
                ms[k][pick[k]] = prof[k][0] / reps
        out = {}
        for k, i in self.SPLIT_KINDS.items():
            best = min(ms[k], key=ms[k].get)
            C.svgp_set_split(self.h, i, best)
            out[k] = {"kmin": best, "ms_per_step": {int(a): round(b, 4) for a, b in ms[k].items()}}
        restore()
        torch.cuda.synchronize()
        return out


def paper_init(M, D, Z0, sf2=1.0, noise=1.0, ell=1.0, alpha=1e-4, beta=1e-3):
    """Initial state of Appendix S5.3: m~ = 0, s~ = alpha 1, L = beta I."""
    import numpy as np

    return dict(Z=np.asarray(Z0, np.float64), ell=np.full(D, ell), sf2=sf2, noise=noise,
                m=np.zeros(M), s=np.full(M, alpha), L=beta * np.eye(M))


class RSVGPGroup:
    """Many independent SVGPs (possibly of different M) trained together.

    One training step of the group is one step of every member.  ``capture``
    records all members' steps into ONE CUDA graph whose branches run on
    separate streams forked from the capturing stream, so kernels of
    different members overlap on the GPU (a small member's launches fill the
    SMs a large member leaves idle) and the whole group step replays as a
    single graph launch.
    """

    def __init__(self, models):
        self.models = list(models)
        self.streams = [torch.cuda.Stream() for _ in self.models]

    def train_step(self, batches, t_star=1, eps=0.0):
        """Eager group step: batches[i] = (X, y, N) for member i."""
        cur = torch.cuda.current_stream()
        for m, s, (X, y, N) in zip(self.models, self.streams, batches):
            s.wait_stream(cur)
            with torch.cuda.stream(s):
                m.train_step(X, y, N, t_star=t_star, eps=eps)
        for s in self.streams:
            cur.wait_stream(s)

    def capture(self, batches, t_star=1, eps=0.0):
        """Capture one group step on fixed input buffers into a CUDA graph."""
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.train_step(batches, t_star=t_star, eps=eps)
        for m in self.models:
            m._sync_stream()
        return g

    def sync_status(self):
        return [m.sync_status() for m in self.models]

    def close(self):
        for m in self.models:
            m.close()
