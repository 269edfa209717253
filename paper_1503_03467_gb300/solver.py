"""Differentiable gamblet solve: log a (one value per fine cell) -> u.

Forward: the library assembles the fine operator's values from exp(log a)
(gamblet_assemble_cells), builds the hierarchy (gamblet_setup) and solves
A u = g (gamblet_solve).  The hierarchy either stays alive for the backward
pass (keep_hierarchy=True) or is released after the forward solve and
recomputed level by level in the backward pass from the saved operator
values (keep_hierarchy=False: between the two passes only the fine values,
8 bytes per stored entry, are held instead of every level's operators and
interpolation rows).  Backward: for an upstream gradient G = dL/du the
adjoint system A lambda = G is solved with the same hierarchy and the
per-cell contraction dL/dlog a_c = -a_c lambda_c^T K_ref u_c runs in the
library's adjoint kernel (gamblet_grad with u_obs = u - G, so that its
right-hand side u - u_obs is G).  The paper has no adjoint; this is the
discrete adjoint of the system of Sec. 5.1.

gamblet_one_pass differentiates the one-pass localized map itself
(Algorithm 2 without refinement) through its setup, with respect to log a
and g.
"""
from __future__ import annotations

import torch

from . import native as nv


class _Handle:
    """Owns a library handle; destroyed with the Python object."""

    def __init__(self, h: int):
        self.h = h

    def __del__(self):
        if self.h:
            nv.gamblet_destroy(self.h)
            self.h = 0


class Q1Mesh:
    """Device-resident description of a Q1 mesh: CSR pattern of the fine
    operator, level-q cells of the unknowns, corner unknowns of each cell
    and the reference element matrix."""

    def __init__(self, rowptr, colind, cells, cell_nodes, K_ref, q, device="cuda"):
        dev = torch.device(device)
        t = lambda a, dt: torch.as_tensor(a, dtype=dt).to(dev).contiguous()
        self.rowptr = t(rowptr, torch.int32)
        self.colind = t(colind, torch.int32)
        self.cells = t(cells, torch.int32)
        self.cell_nodes = t(cell_nodes, torch.int32)
        self.K_ref = t(K_ref, torch.float64).reshape(16)
        self.q = int(q)
        self.n = int(self.rowptr.numel()) - 1
        self.ncell = int(self.cell_nodes.shape[0])


class GambletSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, log_a, g, mesh: Q1Mesh, opts, keep_hierarchy=True):
        stream = torch.cuda.current_stream(log_a.device).cuda_stream
        log_a = log_a.detach().contiguous()
        val = torch.empty(mesh.colind.numel(), dtype=torch.float64, device=log_a.device)
        a = torch.empty_like(log_a)
        nv.gamblet_assemble_cells(mesh.rowptr, mesh.colind, mesh.cell_nodes, log_a, mesh.K_ref,
                                  val, a, stream)
        o = nv.Opts.from_buffer_copy(opts) if opts is not None else nv.gamblet_default_opts()
        o.stream = stream
        handle = _Handle(nv.gamblet_setup(mesh.rowptr, mesh.colind, val, mesh.q, mesh.cells, o))
        g = g.detach().contiguous()
        u = torch.empty_like(g)
        nv.gamblet_solve(handle.h, g, u)
        ctx.mesh = mesh
        ctx.opts = o
        if keep_hierarchy:
            ctx.handle = handle
        else:  # released now, recomputed in backward
            nv.gamblet_destroy(handle.h)
            handle.h = 0
            ctx.handle = None
            ctx.val = val
        ctx.save_for_backward(a, u)
        return u

    @staticmethod
    def backward(ctx, grad_u):
        a, u = ctx.saved_tensors
        mesh = ctx.mesh
        handle = ctx.handle
        if handle is None:
            o = ctx.opts
            o.stream = torch.cuda.current_stream(grad_u.device).cuda_stream
            handle = _Handle(nv.gamblet_setup(mesh.rowptr, mesh.colind, ctx.val, mesh.q,
                                              mesh.cells, o))
        u_obs = (u - grad_u.contiguous()).contiguous()
        dlog_a = torch.empty_like(a)
        nv.gamblet_grad(handle.h, mesh.cell_nodes, a, mesh.K_ref, u, u_obs, dlog_a)
        return dlog_a, None, None, None, None


class GambletOnePass(torch.autograd.Function):
    """u_loc(log a, g): the one-pass localized transform (Algorithm 2 with the
    handle's patch and level solves, no outer refinement), differentiable
    through the localized setup.  Backward: gamblet_grad_onepass with
    u_obs = u_loc - G, so that its misfit is the upstream gradient G; it
    returns dL/dlog a and dL/dg = G_loc G."""

    @staticmethod
    def forward(ctx, log_a, g, mesh: Q1Mesh, opts):
        stream = torch.cuda.current_stream(log_a.device).cuda_stream
        log_a = log_a.detach().contiguous()
        val = torch.empty(mesh.colind.numel(), dtype=torch.float64, device=log_a.device)
        a = torch.empty_like(log_a)
        nv.gamblet_assemble_cells(mesh.rowptr, mesh.colind, mesh.cell_nodes, log_a, mesh.K_ref,
                                  val, a, stream)
        # a copy: the caller's options keep their refinement settings
        o = nv.Opts.from_buffer_copy(opts) if opts is not None else nv.gamblet_default_opts()
        o.stream = stream
        o.refine_max_iter = 0  # the one-pass output
        handle = _Handle(nv.gamblet_setup(mesh.rowptr, mesh.colind, val, mesh.q, mesh.cells, o))
        g = g.detach().contiguous()
        u = torch.empty_like(g)
        nv.gamblet_solve(handle.h, g, u)
        ctx.mesh = mesh
        ctx.handle = handle
        ctx.save_for_backward(a, g, u)
        return u

    @staticmethod
    def backward(ctx, grad_u):
        a, g, u = ctx.saved_tensors
        mesh = ctx.mesh
        u_obs = (u - grad_u.contiguous()).contiguous()
        dlog_a = torch.empty_like(a)
        dg = torch.empty_like(g)
        nv.gamblet_grad_onepass(ctx.handle.h, mesh.cell_nodes, a, mesh.K_ref, g, u_obs, dlog_a,
                                dJ_dg=dg)
        return dlog_a, dg, None, None


def gamblet_one_pass(log_a: torch.Tensor, g: torch.Tensor, mesh: Q1Mesh,
                     opts=None) -> torch.Tensor:
    """u_loc(log a, g) of the one-pass localized transform, differentiable
    with respect to log_a and g (float64 handle: opts.precision = 0, and
    patch_tol >= 0)."""
    return GambletOnePass.apply(log_a, g, mesh, opts)


def gamblet_solve(log_a: torch.Tensor, g: torch.Tensor, mesh: Q1Mesh, opts=None,
                  keep_hierarchy: bool = True) -> torch.Tensor:
    """u(log a) for the mesh, differentiable with respect to log_a.  With
    keep_hierarchy=False the hierarchy is released after the forward solve
    and recomputed in the backward pass."""
    return GambletSolve.apply(log_a, g, mesh, opts, keep_hierarchy)
