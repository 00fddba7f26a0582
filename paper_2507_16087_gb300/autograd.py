"""torch.autograd over the Born solver: fields of several sources as a
differentiable function of sound speed and density.

Forward: one solver (Algorithm 1 preprocessing) for the medium, one
solve_forward per source.  Backward: for each source the adjoint field lambda
solves A^H lambda = g with g the incoming gradient of the fields (torch's
convention for a real loss L of complex X: dL = Re<g, dX>), and
medium_gradient adds Re<lambda, db/dm - dA/dm X> (Sec. 2.3: A^H is accretive
for alpha >= 0, so the adjoint uses the same iteration).  All compute runs in
the CUDA library; this module only orders the calls.

Checkpointing: with checkpoint=True the forward fields are not kept; the
backward pass recomputes each source's field before its adjoint solve (one
extra forward solve per source, C*N*16 bytes saved per source).
"""
from __future__ import annotations

import torch

from . import cbs


class _HelmholtzFields(torch.autograd.Function):
    @staticmethod
    def forward(ctx, c0, rho, alpha, sources, opts):
        s = cbs.solver_create(c0.detach().contiguous(), rho.detach().contiguous(), alpha.detach().contiguous(),
                              **opts["create"])
        fields = torch.empty_like(sources)
        infos = []
        for k in range(sources.shape[0]):
            infos.append(s.solve_forward(sources[k], fields[k]))
        ctx.solver = s
        ctx.checkpoint = bool(opts.get("checkpoint", False))
        ctx.infos = infos
        opts.setdefault("infos", []).extend(infos)
        if ctx.checkpoint:
            ctx.save_for_backward(c0.detach(), rho.detach(), alpha.detach(), sources)
        else:
            ctx.save_for_backward(c0.detach(), rho.detach(), alpha.detach(), sources, fields.detach())
        return fields

    @staticmethod
    def backward(ctx, grad_fields):
        saved = ctx.saved_tensors
        c0, rho, alpha, sources = saved[:4]
        s = ctx.solver
        gc = torch.zeros_like(c0)
        gr = torch.zeros_like(rho)
        field = torch.empty_like(sources[0])
        lam = torch.empty_like(sources[0])
        for k in range(sources.shape[0]):
            if ctx.checkpoint:
                s.solve_forward(sources[k], field)
                X = field
            else:
                X = saved[4][k]
            g = grad_fields[k].contiguous()
            if not torch.any(g != 0):
                continue
            s.solve_adjoint(g, lam)
            s.medium_gradient(c0, rho, alpha, sources[k], X, lam, gc, gr, accumulate=True)
        s.destroy()
        ctx.solver = None
        return gc, gr, None, None, None


def helmholtz_fields(c0, rho, alpha, sources, dx, omega, nabs, gamma_max, power=2.0, precision="fp32_refine",
                     tol=1e-8, checkpoint=False, infos=None, **kw):
    """Physical fields (S, D+1, *shape) for physical sources (S, D+1, *shape); differentiable in c0 and rho."""
    opts = {"create": dict(dx=dx, omega=omega, nabs=nabs, gamma_max=gamma_max, power=power, precision=precision,
                           tol=tol, **kw), "checkpoint": checkpoint}
    if infos is not None:
        opts["infos"] = infos
    return _HelmholtzFields.apply(c0, rho, alpha, sources, opts)


def receiver_misfit(fields, data, rec_idx):
    """J = 1/2 sum_s sum_r |p_s(x_r) - d_s(r)|^2 with rec_idx a tuple of index tensors into the grid."""
    D = fields.shape[1] - 1
    p = fields[:, D][(slice(None),) + tuple(rec_idx)]
    return 0.5 * torch.sum(torch.abs(p - data) ** 2)
