"""Randomized K-FAC preconditioning of a PyTorch model's linear layers (the
training-loop integration of Alg. 1 with Alg. 4/5, on the amortised schedule
of Sec. 5).

Every arithmetic step runs in libkfac through the C ABI (kfac.py): the EA
updates of both K-factors from the layer inputs and output gradients
(kfac_ea_update_rows), their randomized inversion (kfac_rsvd_invert_grouped:
SREVD, Alg. 3 / SRE-KFAC, or RSVD's V~, Alg. 2 / RS-KFAC) and the damped
Kronecker apply to every layer's gradient (kfac_precondition_grouped). This
module only captures tensors with autograd hooks, keeps the per-layer state,
picks the seeds of the Gaussian test matrices (the library draws them on the
device, omega_seed below) and copies the gradient in and out of the
Mat(g) = [dW | db] layout.

Schedule (Sec. 5): the factors are updated every `t_update` steps (T_KU) and
inverted every `t_invert` steps (T_KI); the preconditioner is applied every
step with the latest inverse. damping, rank and oversampling may be numbers or
callables of the step index (the paper's lambda / r / r_l schedules)."""
from __future__ import annotations

import torch

from . import kfac


def omega_seed(seed: int, inversion: int, factor: int) -> int:
    """Generator key of one factor's test matrix: the optimiser's seed in the
    high 32 bits, then the inversion count (20 bits) and the factor's position in
    the grouped call (12 bits), so every inversion of every factor draws a fresh
    matrix (up to 2^20 inversions of 4096 factors)."""
    return ((seed & 0xFFFFFFFF) << 32) | ((inversion & 0xFFFFF) << 12) | (factor & 0xFFF)


def _value(v, step):
    return v(step) if callable(v) else v


class _Layer:
    def __init__(self, mod: torch.nn.Linear, dev):
        self.mod = mod
        self.has_bias = mod.bias is not None
        self.d_in = mod.in_features + int(self.has_bias)
        self.d_out = mod.out_features
        z = lambda r, c: torch.zeros(r, (c + 3) // 4 * 4, device=dev)[:, :c]   # 16-byte row strides
        self.FA = z(self.d_in, self.d_in)
        self.FG = z(self.d_out, self.d_out)
        self.J = z(self.d_out, self.d_in)
        self.S = z(self.d_out, self.d_in)
        self.a = None   # last captured input (n x in_features)
        self.g = None   # last captured output gradient (n x out_features)
        self.inv = None  # ((U_A, D_A, c_A), (U_G, D_G, c_G)) of the latest inversion


class RandomizedKFAC:
    """Randomized K-FAC preconditioner for the nn.Linear layers of a model.

    Call `step()` after `loss.backward()` and before the base optimizer's
    step: it replaces every tracked layer's weight/bias gradient by the
    preconditioned one, S = (G + lambda I)^-1 [dW | db] (A + lambda I)^-1
    through the low-rank inverses of Eq. (13).

    grad_scale: multiplies the captured output gradients before the G factor
    update; the default "batch" (the batch size) turns the gradients of a
    batch-mean loss into per-sample gradients."""

    def __init__(self, model: torch.nn.Module, rank=220, oversample=10, power_iters=1, damping=0.1, rho=0.95,
                 t_update=10, t_invert=50, method: str = "srevd", prec: str = "fp32", grad_scale="batch",
                 seed: int = 0, ctx: kfac.Context | None = None):
        mods = [m for m in model.modules() if isinstance(m, torch.nn.Linear)]
        if not mods:
            raise ValueError("no nn.Linear layer to precondition")
        dev = next(model.parameters()).device
        if dev.type != "cuda":
            raise ValueError("the model must live on a CUDA device")
        self.ctx = ctx if ctx is not None else kfac.Context(dev.index if dev.index is not None else 0)
        kfac.kfac_set_option(self.ctx, "invert_method", {"srevd": 0, "rsvd": 1}[method])
        self.layers = [_Layer(m, dev) for m in mods]
        self.rank, self.oversample, self.power_iters = rank, oversample, power_iters
        self.damping, self.rho, self.prec, self.grad_scale = damping, rho, prec, grad_scale
        self.t_update, self.t_invert = int(t_update), int(t_invert)
        self.seed = int(seed)
        self.inversions = 0
        self.steps = 0
        self._hooks = []
        for L in self.layers:
            self._hooks.append(L.mod.register_forward_pre_hook(self._capture_input(L)))
            self._hooks.append(L.mod.register_full_backward_hook(self._capture_grad(L)))

    # ---- hooks -----------------------------------------------------------------
    def _capture_input(self, L):
        def hook(mod, args):
            if mod.training and self._due(self.t_update):
                L.a = args[0].detach().reshape(-1, mod.in_features)
        return hook

    def _capture_grad(self, L):
        def hook(mod, gin, gout):
            if mod.training and self._due(self.t_update):
                L.g = gout[0].detach().reshape(-1, mod.out_features)
        return hook

    def _due(self, period):
        return self.steps % period == 0

    def remove(self):
        for h in self._hooks:
            h.remove()
        self._hooks = []

    # ---- one optimisation step -----------------------------------------------------
    @torch.no_grad()
    def step(self):
        lam = float(_value(self.damping, self.steps))
        stream = self.ctx.stream
        if self._due(self.t_update):
            for L in self.layers:
                if L.a is None or L.g is None:
                    raise RuntimeError("no captured activations/gradients: run forward and backward in train mode")
                n = L.a.shape[0]
                scale = float(n) if self.grad_scale == "batch" else float(self.grad_scale)
                kfac.kfac_ea_update_rows(self.ctx, L.a.contiguous(), L.FA, self.rho, append_one=L.has_bias,
                                         prec=self.prec)
                kfac.kfac_ea_update_rows(self.ctx, L.g.contiguous(), L.FG, self.rho, scale=scale, prec=self.prec)
                L.a = L.g = None
        if self._due(self.t_invert) or self.layers[0].inv is None:
            r, p = int(_value(self.rank, self.steps)), int(_value(self.oversample, self.steps))
            items = []
            for L in self.layers:
                for F in (L.FA, L.FG):
                    d = F.shape[0]
                    items.append(dict(F=F, rank=min(r, d), oversample=p, power_iters=self.power_iters, lam=lam,
                                      omega=None, seed=omega_seed(self.seed, self.inversions, len(items)),
                                      prec=self.prec))
            outs = kfac.kfac_rsvd_invert_grouped(self.ctx, items)
            self.inversions += 1
            for i, L in enumerate(self.layers):
                L.inv = (outs[2 * i], outs[2 * i + 1])
                L.lam = lam
        pitems = []
        for L in self.layers:
            w = L.mod.weight.grad
            if w is None:
                continue
            with torch.cuda.stream(stream):
                L.J[:, :L.mod.in_features].copy_(w)
                if L.has_bias:
                    L.J[:, L.d_in - 1].copy_(L.mod.bias.grad)
            (Ua, _, ca), (Ug, _, cg) = L.inv
            pitems.append((L, dict(J=L.J, U_a=Ua, coef_a=ca, U_g=Ug, coef_g=cg, lam=L.lam, prec=self.prec, out=L.S)))
        if pitems:
            kfac.kfac_precondition_grouped(self.ctx, [it for _, it in pitems])
            with torch.cuda.stream(stream):
                for L, _ in pitems:
                    L.mod.weight.grad.copy_(L.S[:, :L.mod.in_features])
                    if L.has_bias:
                        L.mod.bias.grad.copy_(L.S[:, L.d_in - 1])
        torch.cuda.current_stream().wait_stream(stream)
        self.steps += 1

    def status(self):
        """(status code, flags) of the library since the last call (synchronises)."""
        return kfac.kfac_get_status(self.ctx)
