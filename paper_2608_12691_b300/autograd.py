"""torch.autograd.Function over the C-ABI: U(lambda) and dU/dlambda as
functions of the solute atoms' charges and Lennard-Jones sigma / epsilon.

The forward pass loads the parameters into the system (``lfe_set_solute_params``)
and evaluates Eq. 4 at lambda (``lfe_eval``); the backward pass is the
hand-written FP64 parameter-gradient kernel (``lfe_param_grad``), which
recomputes each solute atom's interactions at the current positions instead of
keeping per-pair state from the forward pass.  Both outputs are
differentiable:

    dL/dp_i = dL/dU * dU/dp_i + dL/d(dU/dlambda) * d2U/(dlambda dp_i).

lambda and the positions are inputs held fixed (no gradient flows to them),
and the system must not move between the forward and the backward pass.
CUDA tensors are passed to the library as device pointers on torch's current
stream; CPU tensors go through host buffers.  Everything that is computed
runs in the CUDA library: this module only marshals arguments.
"""
import torch

from . import lfe


def _f64(t):
    return t.detach().to(torch.float64).contiguous()


def _load_params(system, charge, sigma, epsilon):
    if charge.is_cuda:
        stream = torch.cuda.current_stream(charge.device)
        system.set_solute_params_device(charge.data_ptr(), sigma.data_ptr(), epsilon.data_ptr(), stream=stream)
    else:
        system.set_solute_params(charge.numpy(), sigma.numpy(), epsilon.numpy())


class LambdaNonbonded(torch.autograd.Function):
    """(U, dU/dlambda) = LambdaNonbonded.apply(charge_u, sigma_u, epsilon_u, system, lam)."""

    @staticmethod
    def forward(ctx, charge, sigma, epsilon, system, lam):
        q, s, e = _f64(charge), _f64(sigma), _f64(epsilon)
        n_u = system.n_solute
        for t in (q, s, e):
            if t.shape != (n_u,):
                raise ValueError(f"solute parameters must have shape ({n_u},), got {tuple(t.shape)}")
        _load_params(system, q, s, e)
        if q.is_cuda:
            terms = torch.zeros(lfe.NTERMS, dtype=torch.float64, device=q.device)
            system.eval_device(lam, None, terms.data_ptr(), stream=torch.cuda.current_stream(q.device))
        else:
            t, _ = system.eval(lam, forces=False)
            terms = torch.tensor([t[k] for k in lfe.TERM_NAMES], dtype=torch.float64)
        ctx.system = system
        ctx.lam = float(lam)
        ctx.save_for_backward(q, s, e)
        return terms[0].clone().to(charge.dtype), terms[1].clone().to(charge.dtype)

    @staticmethod
    def backward(ctx, g_U, g_dUdl):
        q, s, e = ctx.saved_tensors
        system = ctx.system
        n_u = q.shape[0]
        _load_params(system, q, s, e)
        if q.is_cuda:
            dU = torch.empty(n_u, 3, dtype=torch.float64, device=q.device)
            d2 = torch.empty(n_u, 3, dtype=torch.float64, device=q.device)
            system.param_grad_device(ctx.lam, dU.data_ptr(), d2.data_ptr(),
                                     stream=torch.cuda.current_stream(q.device))
        else:
            a, b, _ = system.param_grad(ctx.lam)
            dU, d2 = torch.from_numpy(a), torch.from_numpy(b)
        g = g_U.to(torch.float64) * dU + g_dUdl.to(torch.float64) * d2
        return g[:, 0], g[:, 1], g[:, 2], None, None


def lambda_nonbonded(system, lam, charge, sigma, epsilon):
    """U(lambda) and dU/dlambda of `system` with the given solute parameters."""
    return LambdaNonbonded.apply(charge, sigma, epsilon, system, lam)
