"""torch.autograd wrappers with hand-written adjoints over the libpd C entry points.

* ``matvec(grid, u)``: y = K u.  K is symmetric, so the adjoint is K again.
* ``static_solve(grid, b, E)``: u = (P K(E) P)^-1 P b by CG.  The adjoint of the
  solve is a second solve with the same symmetric operator,
  lam = (P K P)^-1 P du; dL/db = lam and
  dL/dE_r = -1/2 sum_{q intact} (lam_q - lam_r)^T C1(q - r) (u_q - u_r)
  for the bond modulus (E_p + E_q)/2 (pd_grad_modulus).
* ``verlet_run(grid, E, u0, v0, ...)``: the velocity-Verlet crack loop
  (Algorithm 2).  The forward keeps (u, v) every ``checkpoint_every`` steps and
  the step at which every bond broke; the backward replays each segment from
  its checkpoint and sweeps it in reverse (pd_step_adjoint), holding the
  recorded bond history fixed (breaking itself is not differentiable).

Every step runs in the library's kernels; this module only orders the calls and
keeps the tensors the backward needs.  Calls change the grid's material (the
modulus field) and, for ``verlet_run``, its bond state, like the underlying
C calls do.
"""
from __future__ import annotations

import torch

from . import (PD_CG_F64, PD_CG_MIXED, PD_PROJECT, pd_cg_solve, pd_grad_modulus, pd_step, pd_step_adjoint)


class _Matvec(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u, grid, flags):
        ctx.grid, ctx.flags = grid, flags
        return grid.matvec(u.contiguous(), flags=flags)

    @staticmethod
    def backward(ctx, gy):
        return ctx.grid.matvec(gy.contiguous(), flags=ctx.flags), None, None


def matvec(grid, u, flags: int = 0):
    """y = K u (P K P u with PD_PROJECT) with autograd support for u."""
    return _Matvec.apply(u, grid, flags)


def _set_modulus(grid, E):
    if E is not None:
        grid.set_material(E=1.0, rho=grid.rho, thickness=grid.thickness, s0=grid.s0, E_field=E.detach().contiguous())


class _StaticSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, b, E, grid, rtol, mode, max_iter):
        _set_modulus(grid, E)
        u = torch.zeros_like(b)
        pd_cg_solve(grid.handle, b.detach().contiguous(), u, rtol, max_iter, mode)
        ctx.grid, ctx.rtol, ctx.mode, ctx.max_iter = grid, rtol, mode, max_iter
        ctx.save_for_backward(u, E if E is not None else torch.empty(0))
        ctx.has_E = E is not None
        return u

    @staticmethod
    def backward(ctx, ubar):
        u, E = ctx.saved_tensors
        grid = ctx.grid
        if ctx.has_E:
            _set_modulus(grid, E)
        lam = torch.zeros_like(u)
        pd_cg_solve(grid.handle, ubar.contiguous(), lam, ctx.rtol, ctx.max_iter, ctx.mode)
        grad_b = lam if ctx.needs_input_grad[0] else None
        grad_E = None
        if ctx.has_E and ctx.needs_input_grad[1]:
            grad_E = torch.zeros_like(E)
            pd_grad_modulus(grid.handle, u, lam, -0.5, grad_E)
        return grad_b, grad_E, None, None, None, None


def static_solve(grid, b, E=None, rtol: float = 1e-10, mode: int = PD_CG_MIXED, max_iter: int = 1_000_000):
    """u solving P K(E) P u = P b; differentiable in b and in the modulus field E."""
    return _StaticSolve.apply(b, E, grid, rtol, mode, max_iter)


class _VerletRun(torch.autograd.Function):
    @staticmethod
    def forward(ctx, E, u0, v0, grid, b, v_prescribed, nsteps, dt, every):
        _set_modulus(grid, E)
        mask0 = grid.bond_mask().clone()
        bstep = torch.zeros(grid.N * grid.nnb, dtype=torch.int32, device=u0.device)
        u, v = u0.detach().clone(), v0.detach().clone()
        starts, states = [], []
        s = 0
        while s < nsteps:
            n = min(every, nsteps - s)
            starts.append((s, n))
            states.append((u.clone(), v.clone()))
            pd_step(grid.handle, u, v, b, n, dt, v_prescribed, bstep, s)
            s += n
        ctx.grid, ctx.b, ctx.vp, ctx.dt, ctx.starts = grid, b, v_prescribed, dt, starts
        flat = [t for pair in states for t in pair]
        ctx.save_for_backward(E, mask0, bstep, *flat)
        ctx.final_v = v
        return u

    @staticmethod
    def backward(ctx, ubar):
        E, mask0, bstep, *flat = ctx.saved_tensors
        grid = ctx.grid
        _set_modulus(grid, E)
        ub = ubar.contiguous().clone()
        vb = torch.zeros_like(ub)
        ab = torch.zeros_like(ub)
        gE = torch.zeros_like(E)
        for i in reversed(range(len(ctx.starts))):
            s0, n = ctx.starts[i]
            uc, vc = flat[2 * i], flat[2 * i + 1]
            pd_step_adjoint(grid.handle, uc, vc, ctx.b, n, ctx.dt, ctx.vp, mask0, bstep, s0, ub, vb, ab,
                            gE if ctx.needs_input_grad[0] else None)
        return (gE if ctx.needs_input_grad[0] else None, ub if ctx.needs_input_grad[1] else None,
                vb if ctx.needs_input_grad[2] else None, None, None, None, None, None, None)


def verlet_run(grid, E, u0, v0, nsteps: int, dt: float, b=None, v_prescribed=None, checkpoint_every: int = 45):
    """Final displacement after ``nsteps`` Verlet steps (with bond breaking);
    differentiable in the modulus field E and the initial state (u0, v0)."""
    return _VerletRun.apply(E, u0, v0, grid, b, v_prescribed, nsteps, dt, checkpoint_every)
