"""torch.autograd.Function over pflb_adjoint: the droplet objective J of the
final state as a differentiable function of the initial velocity field and
of M, sigma and W (argument marshalling only; forward and reverse sweeps run
in the CUDA library)."""

import torch

from . import pflb


class PFLBObjective(torch.autograd.Function):
    """J = w_vol V_s + sum_k w_cen[k] c_k after ``nsteps`` steps from the
    equilibrium state of (phi0, u0). One call of pflb_adjoint computes J and
    every derivative; backward scales them by the incoming gradient."""

    @staticmethod
    def forward(ctx, u0, M, sigma, W, params, phi0, nsteps, weights, checkpoint_every):
        P = dict(params, M=float(M), sigma=float(sigma), W=float(W), storage=pflb.FP32)
        stream = torch.cuda.current_stream(u0.device)
        sim = pflb.Sim(P, stream=stream)
        try:
            u = u0.detach().to(torch.float32).contiguous()
            sim.init(phi0.detach().to(torch.float32).contiguous(), u)
            du0 = torch.empty_like(u)
            g = sim.adjoint(nsteps, du0=du0, checkpoint_every=checkpoint_every, **(weights or {}))
        finally:
            sim.close()
        ctx.save_for_backward(du0)
        ctx.dparams = (g["dJ_dM"], g["dJ_dsigma"], g["dJ_dW"])
        ctx.u0_dtype = u0.dtype
        return torch.tensor(g["J"], dtype=torch.float64, device=u0.device)

    @staticmethod
    def backward(ctx, gJ):
        (du0,) = ctx.saved_tensors
        dM, ds, dW = ctx.dparams
        gu = (gJ.to(du0.dtype) * du0).to(ctx.u0_dtype) if ctx.needs_input_grad[0] else None
        dev = gJ.device
        gM = gJ * torch.tensor(dM, dtype=torch.float64, device=dev) if ctx.needs_input_grad[1] else None
        gs = gJ * torch.tensor(ds, dtype=torch.float64, device=dev) if ctx.needs_input_grad[2] else None
        gW = gJ * torch.tensor(dW, dtype=torch.float64, device=dev) if ctx.needs_input_grad[3] else None
        return gu, gM, gs, gW, None, None, None, None, None


def droplet_objective(params, phi0, u0, M, sigma, W, nsteps, weights=None, checkpoint_every=0):
    """Differentiable J(u0, M, sigma, W) (see PFLBObjective). M, sigma, W:
    0-d float64 tensors (or floats); phi0 (field) and u0 (d, field): CUDA
    tensors."""
    as_t = lambda v: v if torch.is_tensor(v) else torch.tensor(float(v), dtype=torch.float64)
    return PFLBObjective.apply(u0, as_t(M), as_t(sigma), as_t(W), params, phi0, int(nsteps), weights,
                               int(checkpoint_every))
