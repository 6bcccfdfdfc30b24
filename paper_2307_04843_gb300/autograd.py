"""torch.autograd.Function over the hand-written discrete adjoint.

``mean_final_gamma(params, pulses, particles, ...)`` returns, for every pulse
set s, J_s = (1/N_s) sum_i gamma_i(T) after the push, as a differentiable
function of params[s] = (a0, w0, z_focus[, beta_f]) (beta_f: closed-form
flying focus).  The forward runs
``ap_push_adjoint`` (its forward pass with checkpoints, then the reverse sweep
through the Boris steps and the analytic fields), keeps dJ/dparams, and the
backward returns grad_J[:, None] * dJ/dparams.  All arithmetic runs in the
library's kernels; the initial particle state is left unchanged.
"""
import torch

from . import _lib

PARAM_NAMES = ("a0", "w0", "z_focus", "beta_f")


def _sets_from(params, pulses):
    p = params.detach().double().cpu().numpy()
    if p.ndim != 2 or p.shape[0] != len(pulses) or p.shape[1] not in (3, 4):
        raise ValueError("params must be [n_sets, 3] or [n_sets, 4]")
    out = []
    for s, base in enumerate(pulses):
        d = dict(base)
        for k, name in enumerate(PARAM_NAMES[:p.shape[1]]):
            d[name] = float(p[s, k])
        out.append(d)
    return out


def adjoint(pulses, particles, set_offsets, t0, dt, n_steps, ckpt_every=100, precision="fp32",
            grid=None, stream=None):
    """Run ap_push_adjoint; returns (J [n_sets], dJ [n_sets, 4]) as float64
    CUDA tensors (columns a0, w0, z_focus, beta_f)."""
    with _lib.Handle(pulses) as h:
        n = particles["x"].numel()
        nbytes = _lib.ap_adjoint_workspace_bytes(h.h, n, n_steps, ckpt_every)
        if nbytes == 0:
            raise ValueError("invalid adjoint arguments (n_steps >= 1, 1 <= ckpt_every <= 256)")
        ws = torch.empty((nbytes + 255) // 256 * 64, dtype=torch.float32, device="cuda")
        S = len(pulses)
        dJ = torch.zeros((S, _lib.AP_NPARAM), dtype=torch.float64, device="cuda")
        J = torch.zeros(S, dtype=torch.float64, device="cuda")
        _lib.ap_push_adjoint(h.h, particles, set_offsets, grid, t0, dt, n_steps, ckpt_every, precision,
                             dJ, J, ws, stream)
        st = h.status(stream)
        if st != 0:
            raise _lib.APError("ap_push_adjoint", st)
    return J, dJ


class MeanFinalGamma(torch.autograd.Function):
    @staticmethod
    def forward(ctx, params, pulses, particles, set_offsets, t0, dt, n_steps, ckpt_every, precision, grid):
        sets = _sets_from(params, pulses)
        J, dJ = adjoint(sets, particles, set_offsets, t0, dt, n_steps, ckpt_every, precision, grid)
        ctx.save_for_backward(dJ[:, :params.shape[1]].to(params.device, params.dtype))
        return J.to(params.device, params.dtype)

    @staticmethod
    def backward(ctx, gJ):
        (dJ,) = ctx.saved_tensors
        return (gJ[:, None] * dJ,) + (None,) * 9


def mean_final_gamma(params, pulses, particles, set_offsets=None, t0=0.0, dt=0.02, n_steps=100,
                     ckpt_every=100, precision="fp32", grid=None):
    """Differentiable per-set mean final gamma.  params: [n_sets, 3] tensor of
    (a0, w0, z_focus), or [n_sets, 4] with beta_f appended; pulses: list of
    base pulse dicts (other parameters);
    particles: dict of CUDA tensors (initial state, unchanged)."""
    return MeanFinalGamma.apply(params, list(pulses), particles, set_offsets, float(t0), float(dt),
                                int(n_steps), int(ckpt_every), precision, grid)
