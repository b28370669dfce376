"""The converged free energy as a differentiable function of beta for
torch.autograd.

forward: the FP64 form of the library runs Algorithm 3 of arXiv:2004.08669 to
its fixed point at beta and returns f = -ln(kappa) / (2 beta) (the growth
factor of the normalised half-row tensor).
backward: d f / d beta by implicit differentiation of the converged fixed
point on the device (ctm_step_backward: the linear fixed-point equation of
the gauge-fixed step, solved by GMRES with the GPU tangent step).

Both directions run in the CUDA library; this module only marshals beta in
and f and its derivative out.  The derivative is computed in the forward
pass, while the converged handle is alive, when beta requires a gradient.
"""
from __future__ import annotations

import torch


def _library():
    from paper_2004_08669_gb300 import ctm
    return ctm


class FreeEnergy(torch.autograd.Function):
    """f(beta) per spin of the CTMRG fixed point with a fixed boundary spin;
    beta is a 0-d tensor, spins the q x dim table, m the bond dimension."""

    @staticmethod
    def forward(ctx, beta, spins, m, max_steps=5000, device="cuda:0"):
        ctm = _library()
        b = float(beta.detach().cpu())
        g = ctm.CTMRG(spins, int(m), b, device=device)
        try:
            g.run(int(max_steps))
            o = g.observables()
            if not o["converged"]:
                raise RuntimeError(f"CTMRG did not converge in {max_steps} steps at beta = {b}")
            df = g.df_dbeta() if ctx.needs_input_grad[0] else 0.0
        finally:
            g.close()
        ctx.save_for_backward(torch.tensor(df, dtype=beta.dtype))
        return beta.new_tensor(o["f"])

    @staticmethod
    @torch.autograd.function.once_differentiable
    def backward(ctx, grad_f):
        # First derivative only: a double backward (d2f/dbeta2) is not
        # available here.  The specific heat and dM/dT come from
        # ctm_step_backward with the gradient of u or M (ctm.ctm_step_backward).
        (df,) = ctx.saved_tensors
        return grad_f * df.to(grad_f.device), None, None, None, None


def free_energy(beta: torch.Tensor, spins, m: int, max_steps: int = 5000, device: str = "cuda:0") -> torch.Tensor:
    return FreeEnergy.apply(beta, spins, m, max_steps, device)
