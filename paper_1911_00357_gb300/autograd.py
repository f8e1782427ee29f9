"""torch.autograd.Function wrappers of the library's hand-written backward passes.

The network's gradient is written out by hand in CUDA (the heads, back-propagation
through time over the LSTM, the GroupNorm ResNet encoder; Sec. 4 "Training"; App. "Agent
Design") and so is the PPO loss's (Eq. 2 with the value and entropy terms). These
Functions put each forward/backward pair of the C ABI behind PyTorch's autograd, so a
PyTorch program can compose them and call .backward():

  EncoderFunction   obs -> features          ddppo_encoder_forward / _backward
  LSTMFunction      LSTM input -> output     ddppo_lstm_forward / _backward
  PolicyFunction    observations -> (logits, values)
                                             ddppo_policy_evaluate / ddppo_policy_backward
  PPOLossFunction   (logits, values) -> loss ddppo_ppo_loss (its exact gradient)

Each takes the flat FP32 parameter vector as its first input, so its gradient arrives in
params.grad. The library keeps its own copy of the parameters: a forward pushes `params`
into the worker (ddppo_set_params, which also clears the worker's Adam state) whenever the
tensor is not the one last pushed (another tensor, or the same one modified in place).
Everything else is argument marshalling: every forward and backward runs in the CUDA
library; the only PyTorch operation is multiplying a gradient by its upstream factor
when that factor is not 1 (the chain rule across the Function's boundary).

The library keeps one set of activations per context: a backward must run before the
next forward of the same context (the library answers E_STATE otherwise), which is what
a plain forward-then-backward does.
"""
from __future__ import annotations

import torch

from . import binding as B


class _Sync:
    """Pushes a parameter tensor into a worker when it is not the one last pushed. The last
    pushed tensor is held, so that no new tensor can reuse its memory and pass for it."""

    def __init__(self):
        self._last = {}

    def __call__(self, h, params: torch.Tensor):
        hk = h.value if hasattr(h, "value") else int(h)
        last = self._last.get(hk)
        if last is None or last[0] is not params or last[1] != params._version:
            B.ddppo_set_params(h, params.detach())
            self._last[hk] = (params, params._version)

    def forget(self, h):
        """Drop the record of a worker (call before destroying it)."""
        self._last.pop(h.value if hasattr(h, "value") else int(h), None)


sync_params = _Sync()


def _scaled(g: torch.Tensor, up: torch.Tensor) -> torch.Tensor:
    if up.numel() == 1 and float(up) == 1.0:
        return g
    return g * up


class EncoderFunction(torch.autograd.Function):
    """features [N, F] (channel-major, the order of vis.w's columns) of obs [N, 1, h, w]."""

    @staticmethod
    def forward(ctx, params, obs, h, F):
        sync_params(h, params)
        N = obs.shape[0]
        feat = torch.empty(N, F, device=obs.device)
        B.ddppo_encoder_forward(h, N, obs.contiguous(), feat)
        ctx.h = h
        ctx.P = params.numel()
        return feat

    @staticmethod
    def backward(ctx, dfeat):
        grad = torch.empty(ctx.P, device=dfeat.device)
        B.ddppo_encoder_backward(ctx.h, dfeat.float().contiguous(), grad)
        return grad, None, None, None


class LSTMFunction(torch.autograd.Function):
    """Top-layer output y [T, E, H] of the LSTM layers for input x [T, E, In_0]."""

    @staticmethod
    def forward(ctx, params, x, masks, h0, c0, h, hidden):
        sync_params(h, params)
        T, E = x.shape[0], x.shape[1]
        y = torch.empty(T, E, hidden, device=x.device)
        B.ddppo_lstm_forward(h, T, E, x.float().contiguous(), masks.contiguous(), h0.contiguous(),
                             c0.contiguous(), y)
        ctx.h = h
        ctx.P = params.numel()
        ctx.xshape = x.shape
        return y

    @staticmethod
    def backward(ctx, dy):
        grad = torch.empty(ctx.P, device=dy.device)
        dx = torch.empty(ctx.xshape, device=dy.device)
        B.ddppo_lstm_backward(ctx.h, dy.float().contiguous(), dx, grad)
        return grad, dx, None, None, None, None, None


class PolicyFunction(torch.autograd.Function):
    """(logits [T, E, 4], values [T, E]) of the whole agent over a [T, E] segment."""

    @staticmethod
    def forward(ctx, params, obs, goal, prev_a, masks, h0, c0, h):
        sync_params(h, params)
        T, E = prev_a.shape
        logits = torch.empty(T, E, 4, device=goal.device)
        values = torch.empty(T, E, device=goal.device)
        B.ddppo_policy_evaluate(h, T, E, obs.contiguous(), goal.contiguous(), prev_a.contiguous(),
                                masks.contiguous(), h0.contiguous(), c0.contiguous(), logits, values)
        ctx.h = h
        ctx.P = params.numel()
        ctx.TE = (T, E)
        return logits, values

    @staticmethod
    def backward(ctx, dlogits, dvalues):
        T, E = ctx.TE
        dev = dlogits.device if dlogits is not None else dvalues.device
        grad = torch.empty(ctx.P, device=dev)
        dl = dlogits if dlogits is not None else torch.zeros(T, E, 4, device=dev)
        dv = dvalues if dvalues is not None else torch.zeros(T, E, device=dev)
        B.ddppo_policy_backward(ctx.h, dl.float().contiguous(), dv.float().contiguous(), grad)
        return grad, None, None, None, None, None, None, None


class PPOLossFunction(torch.autograd.Function):
    """Scalar PPO loss (Eq. 2 + c_v value loss - c_e entropy) of logits [..., 4] and values
    [...]; the eight statistics of ddppo_ppo_loss go to stats_out [8] when it is given."""

    @staticmethod
    def forward(ctx, logits, values, actions, logp_old, adv, ret, clip, value_coef, entropy_coef,
                stats_out=None):
        n = values.numel()
        stats = torch.empty(B.NSTATS, device=values.device) if stats_out is None else stats_out
        dl = torch.empty(n, 4, device=values.device)
        dv = torch.empty(n, device=values.device)
        B.ddppo_ppo_loss(n, logits.float().contiguous(), values.float().contiguous(),
                         actions.int().contiguous(), logp_old.float().contiguous(),
                         adv.float().contiguous(), ret.float().contiguous(), clip, value_coef,
                         entropy_coef, stats, dl, dv)
        ctx.save_for_backward(dl.view(logits.shape), dv.view(values.shape))
        return stats[0].clone()

    @staticmethod
    def backward(ctx, up):
        dl, dv = ctx.saved_tensors
        return (_scaled(dl, up), _scaled(dv, up), None, None, None, None, None, None, None, None)
