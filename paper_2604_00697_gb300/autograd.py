"""PyTorch autograd over the library's bound and hand-written backward.

``SVGPBound`` is a ``torch.autograd.Function`` whose forward is the bound F of
Eq. (7) and whose backward is the library's gradient of F with T held fixed:
T is a separate variational parameter optimised by natural gradients
(Section 3.1, alternating optimisation), which is the gradient Prop. 2 is
about.  L is therefore an input without a gradient.

When any parameter needs a gradient, the forward calls ``svgp_backward``
(bound and all gradients in one pass, sharing the forward intermediates and
regenerating Kuf on chip) and keeps the gradients; the backward returns them
times the incoming gradient of F.  Without gradients the forward calls
``svgp_bound``.  Every computation of the method runs in ``libsvgp.so``; this
module only marshals tensors (the product with the incoming gradient is
autograd's chain rule).

``RSVGPModule`` is an ``nn.Module`` whose parameters (constrained values of
Z, ell, sf2, noise, m~, s~) alias the flat parameter vector of an ``RSVGP``
model, with L as a buffer updated by ``ng_update`` (Prop. 1) and ``step``
the library's Adam on the same vector.
"""
from __future__ import annotations

import torch

from . import _lib as C
from .model import RSVGP

_BLOCKS = ("Z", "ell", "sf2", "noise", "m", "s")


def _ptr(t: torch.Tensor, name: str) -> int:
    if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
        raise ValueError(f"{name}: expected a contiguous float32 CUDA tensor")
    return t.data_ptr()


class SVGPBound(torch.autograd.Function):
    """F(Z, ell, sf2, noise, m~, s~; L, X, y) of Eq. (7), T = L L^T held fixed."""

    @staticmethod
    def forward(ctx, model: RSVGP, X, y, N, Z, ell, sf2, noise, m, s, L):
        M, D = model.M, model.D
        shapes = {"Z": (M, D), "ell": (D,), "sf2": (1,), "noise": (1,), "m": (M,), "s": (M,)}
        vals = dict(zip(_BLOCKS, (Z, ell, sf2, noise, m, s)))
        for k, t in vals.items():
            if tuple(t.shape) != shapes[k]:
                raise ValueError(f"{k}: shape {tuple(t.shape)}, expected {shapes[k]}")
        if tuple(L.shape) != (M, M):
            raise ValueError(f"L: shape {tuple(L.shape)}, expected {(M, M)}")
        params = C.svgp_params(*[_ptr(vals[k], k) for k in _BLOCKS], _ptr(L, "L"))
        batch = C.svgp_batch(_ptr(X, "X"), _ptr(y, "y"), X.shape[0], float(N))
        model._sync_stream()
        terms = torch.empty(C.SVGP_NTERMS, dtype=torch.float64, device=Z.device)
        if any(ctx.needs_input_grad[4:10]):
            grads = [torch.empty_like(vals[k]) for k in _BLOCKS]
            gs = C.svgp_grads(*[g.data_ptr() for g in grads])
            C.svgp_backward(model.h, params, batch, terms.data_ptr(), gs)
            ctx.save_for_backward(*grads)
        else:
            C.svgp_bound(model.h, params, batch, terms.data_ptr())
        ctx.mark_non_differentiable(terms)
        return terms[0].clone(), terms

    @staticmethod
    def backward(ctx, gF, _gterms):
        grads = ctx.saved_tensors
        scale = gF.to(torch.float32)
        out = [None] * 4 + [None if not ctx.needs_input_grad[4 + i] else g * scale for i, g in enumerate(grads)]
        return tuple(out) + (None,)


def svgp_bound(model: RSVGP, X, y, N, Z, ell, sf2, noise, m, s, L):
    """F (0-dim float64 tensor) and the term vector (float64[SVGP_NTERMS])."""
    return SVGPBound.apply(model, X, y, N, Z, ell, sf2, noise, m, s, L)


class RSVGPModule(torch.nn.Module):
    """R-SVGP as an ``nn.Module``: ``forward(X, y, N)`` returns the bound F
    (to maximise) and the term vector; ``F.backward()`` fills the parameters'
    ``.grad`` through the library's backward.

    The parameters alias the model's flat constrained vector and their
    ``.grad`` tensors alias its flat gradient vector (autograd accumulates
    into an existing ``.grad`` in place), so ``step()`` -- one library Adam
    step with the softplus chain rule for the positive blocks -- reads the
    gradient autograd produced.  ``zero_grad()`` clears that vector in place.
    Mixing ``step()`` with an external optimiser is not supported: the
    library keeps the unconstrained vector that Adam updates.
    """

    def __init__(self, M: int, D: int, B_max: int, prec: str = "bf16x3", likelihood: str = "gaussian",
                 precond: bool = True):
        super().__init__()
        self.core = RSVGP(M, D, B_max, prec=prec, likelihood=likelihood, precond=precond)
        for k in _BLOCKS:
            view = self.core.cons[self.core.sl[k]]
            if k == "Z":
                view = view.view(M, D)
            self.register_parameter(k, torch.nn.Parameter(view))
        self.register_buffer("L", self.core.L, persistent=True)
        self._alias_grads()

    def _alias_grads(self):
        for k in _BLOCKS:
            g = self.core.grad[self.core.sl[k]]
            getattr(self, k).grad = g.view(self.core.M, self.core.D) if k == "Z" else g

    def set_state(self, Z, ell, sf2, noise, m, s, L):
        self.core.set_state(Z, ell, sf2, noise, m, s, L)

    def forward(self, X, y, N):
        return SVGPBound.apply(self.core, X, y, N, self.Z, self.ell, self.sf2, self.noise, self.m, self.s, self.L)

    def zero_grad(self, set_to_none: bool = False):
        self.core.grad.zero_()
        self._alias_grads()

    def ng_update(self, max_iters=1, eps=0.0, gammas=None):
        """NG update(s) of L given K~ (Prop. 1, Eq. (8) stopping rule)."""
        with torch.no_grad():
            self.core.ng_update(max_iters=max_iters, eps=eps, gammas=gammas)

    def step(self):
        """One Adam ascent step on the flat vector from the current ``.grad``."""
        with torch.no_grad():
            self.core.adam_step()

    def close(self):
        self.core.close()
