"""torch.autograd interface of the FIDS march.

FidsSolve.apply(kappa, f, solver, phi) returns u^M of the FIDS time march
for a time-independent diffusivity kappa(x) and source f(x); its backward
pass runs the discrete adjoint sweep on the GPU (tsfde_adjoint) and returns
dJ/dkappa and dJ/df for whatever scalar J the caller built on u^M.  With a
solver made with ckpt_stride != 0 no trajectory is kept: the sweep marches
each segment again from the solver's checkpoints.
"""
from __future__ import annotations

import numpy as np


def _fids_solve_class():
    import torch

    class FidsSolve(torch.autograd.Function):
        """u^M = FidsSolve.apply(kappa, f, solver, phi).

        kappa, f, phi: CUDA float64 tensors of n entries (kappa > 0).
        solver: a paper_2002_11978_gb300.Solver set up for the mesh; its
        problem is replaced by (phi, kappa, f) in forward and again in
        backward, so one solver can serve several graphs."""

        @staticmethod
        def forward(ctx, kappa, f, solver, phi):
            kappa = kappa.detach().contiguous()
            f = f.detach().contiguous()
            phi = phi.detach().contiguous()
            ones = np.ones(solver.M + 1)
            solver.set_problem(phi, kappa, None, None, F=[f], G=[ones])
            uM = torch.empty(solver.n, dtype=torch.float64, device=kappa.device)
            ctx.solver = solver
            if solver.ckpt_stride:
                # the solver keeps checkpoints of the march: no trajectory here
                solver.solve(uM)
                ctx.token = solver.problem_token
                ctx.save_for_backward(kappa, f, phi)
            else:
                U = torch.empty((solver.M + 1, solver.n), dtype=torch.float64, device=kappa.device)
                solver.solve(uM, U)
                ctx.token = None
                ctx.save_for_backward(kappa, f, phi, U)
            return uM.clone()

        @staticmethod
        def backward(ctx, g):
            solver = ctx.solver
            kappa, f, phi = ctx.saved_tensors[:3]
            gk = torch.empty_like(kappa)
            gf = torch.empty_like(f)
            gd = g.detach().contiguous().to(torch.float64)
            if ctx.token is not None:
                if solver.problem_token is not ctx.token or solver.m != solver.M:
                    # the solver served another problem since: march this one again
                    solver.set_problem(phi, kappa, None, None, F=[f], G=[np.ones(solver.M + 1)])
                    solver.solve(torch.empty_like(kappa))
                solver.adjoint(None, gd, gk, gf)
            else:
                solver.set_problem(phi, kappa, None, None, F=[f], G=[np.ones(solver.M + 1)])
                solver.adjoint(ctx.saved_tensors[3], gd, gk, gf)
            return gk, gf, None, None

    return FidsSolve


_CLS = None


def fids_solve(kappa, f, solver, phi):
    """u^M as a differentiable function of kappa and f (see FidsSolve)."""
    global _CLS
    if _CLS is None:
        _CLS = _fids_solve_class()
    return _CLS.apply(kappa, f, solver, phi)
