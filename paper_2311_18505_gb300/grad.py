"""Differentiable synthesis: a ``torch.autograd.Function`` over the C-ABI
tape (``sfd_tape_*``).

``synthesize(theta, strings, n_samples)`` renders the strings with the
parameters of ``theta`` (one row per string: kappa, alpha, sigma0, sigma1,
amplitude -- the pluck amplitude in metres, the hammer or the bow velocity
in m/s; strings may be f0-modulated and read on either output channel)
and returns the audio ``(n, n_samples)`` on the GPU; ``backward`` runs the
hand-written discrete adjoint kernel (checkpoints every ``checkpoint_every``
samples, each segment recomputed from its checkpoint).  Gradients hold each
string's grid (N_t, N_l) fixed at the one its parameters give.

Marshalling only: the synthesis and the adjoint run in the CUDA library.
"""

from __future__ import annotations

import copy

import numpy as np
import torch

from . import sfd

PARAM_NAMES = sfd.GRAD_PARAM_NAMES


def params_of(d: dict) -> list[float]:
    """The differentiable parameters of a string dictionary, in PARAM_NAMES order."""
    ex = d["excitation"]
    amp = ex["amp"] if ex["kind"] == "pluck" else ex["vel"]
    return [d["kappa"], d["alpha"], d["sigma0"], d["sigma1"], amp]


def with_params(d: dict, row) -> dict:
    """Copy of string dictionary `d` with the parameters of `row`."""
    out = copy.deepcopy(d)
    out["kappa"], out["alpha"], out["sigma0"], out["sigma1"] = (float(v) for v in row[:4])
    ex = out["excitation"]
    ex["amp" if ex["kind"] == "pluck" else "vel"] = float(row[4])
    return out


class _Tape:
    """Owns a library tape; destroyed with the autograd graph."""

    def __init__(self, handle: int, n: int):
        self.handle, self.n = handle, n

    def __del__(self):
        if self.handle:
            try:
                sfd.sfd_tape_destroy(self.handle)
            except Exception:
                pass
            self.handle = 0


class StringSynthesis(torch.autograd.Function):
    @staticmethod
    def forward(fctx, theta, strings, n_samples, checkpoint_every, ctx, device):
        rows = theta.detach().cpu().double().numpy()
        dicts = [with_params(d, r) for d, r in zip(strings, rows)]
        tape = _Tape(sfd.sfd_tape_create(ctx, dicts, n_samples, checkpoint_every), len(dicts))
        y = torch.empty(len(dicts), n_samples, device=device, dtype=torch.float32)
        torch.cuda.current_stream(device).synchronize()
        sfd.sfd_tape_forward(tape.handle, y)
        fctx.tape = tape
        fctx.theta_meta = (theta.dtype, theta.device)
        return y

    @staticmethod
    def backward(fctx, dy):
        dy = dy.contiguous().to(torch.float32)
        torch.cuda.current_stream(dy.device).synchronize()
        g = sfd.sfd_tape_backward(fctx.tape.handle, dy, fctx.tape.n)
        dtype, dev = fctx.theta_meta
        return torch.from_numpy(g).to(dtype=dtype, device=dev), None, None, None, None, None


def synthesize(theta: torch.Tensor, strings: list[dict], n_samples: int, ctx: int,
               checkpoint_every: int = 1024, device=None) -> torch.Tensor:
    """Audio of `strings` with parameters `theta` (n x 5), differentiable in theta."""
    device = device or torch.device("cuda", torch.cuda.current_device())
    return StringSynthesis.apply(theta, strings, n_samples, checkpoint_every, ctx, device)


def theta_of(strings: list[dict]) -> np.ndarray:
    return np.array([params_of(d) for d in strings], dtype=np.float64)
