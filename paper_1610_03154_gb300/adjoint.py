"""Differentiation through the root-node AMG solve.

``AMGSolve`` is a ``torch.autograd.Function`` for x = A(values)^{-1} b on a
fixed CSR pattern.  Forward builds a hierarchy for A (rn_setup) and solves;
backward solves the adjoint system A^T lambda = dL/dx (with the same
hierarchy when A is symmetric, else with one built for A^T) and forms the
gradient with respect to A's stored values on the GPU, dL/dA_ij =
-lambda_i x_j (rn_adjoint_grad); dL/db = lambda.  Gradients with respect to
parameters the values depend on follow by torch's own chain rule.

``VarCoefFV`` assembles the cell-centred finite-volume operator of
-div(exp(theta) grad u) = f (unit square, Dirichlet u = 0, harmonic-mean face
coefficients, boundary faces at half distance) from theta with torch
operations on a pattern fixed once, so the values are differentiable in theta.
Every solve and the gradient scatter run in the library's CUDA kernels; torch
holds the tensors and the chain rule through the assembly.
"""
import numpy as np
import torch

from . import rn


class VarCoefFV:
    """CSR pattern of the m x m cell-centred 5-point operator and the maps from
    faces to stored entries; ``values(theta)`` is differentiable in theta."""

    def __init__(self, m: int, device):
        self.m = m
        n = m * m
        idx = np.arange(n).reshape(m, m)
        # interior faces (a, b): x-faces then y-faces
        a = np.concatenate([idx[:, :-1].ravel(), idx[:-1, :].ravel()])
        b = np.concatenate([idx[:, 1:].ravel(), idx[1:, :].ravel()])
        # CSR pattern: row i holds its neighbours and itself, sorted
        rows = np.concatenate([a, b, np.arange(n)])
        cols = np.concatenate([b, a, np.arange(n)])
        order = np.lexsort((cols, rows))
        rows, cols = rows[order], cols[order]
        rowptr = np.zeros(n + 1, np.int64)
        np.add.at(rowptr, rows + 1, 1)
        rowptr = np.cumsum(rowptr)
        pos = np.empty(len(rows), np.int64)
        pos[order] = np.arange(len(rows))
        nf = len(a)
        self.n, self.nnz = n, len(rows)
        self.pos_ab = torch.from_numpy(pos[:nf]).to(device)
        self.pos_ba = torch.from_numpy(pos[nf:2 * nf]).to(device)
        self.pos_diag = torch.from_numpy(pos[2 * nf:]).to(device)  # entry (i, i) of row i
        self.fa = torch.from_numpy(a).to(device)
        self.fb = torch.from_numpy(b).to(device)
        nbnd = np.zeros((m, m))
        nbnd[:, 0] += 1
        nbnd[:, -1] += 1
        nbnd[0, :] += 1
        nbnd[-1, :] += 1
        self.nbnd = torch.from_numpy(nbnd.ravel()).to(device)  # boundary faces per cell
        self.rowptr = torch.from_numpy(rowptr.astype(np.int32)).to(device)
        self.col = torch.from_numpy(cols.astype(np.int32)).to(device)
        self.device = device

    def values(self, theta: torch.Tensor) -> torch.Tensor:
        k = torch.exp(theta)
        ka, kb = k[self.fa], k[self.fb]
        kf = 2.0 * ka * kb / (ka + kb)
        v = torch.zeros(self.nnz, dtype=k.dtype, device=k.device)
        v = v.index_add(0, self.pos_ab, -kf).index_add(0, self.pos_ba, -kf)
        diag = torch.zeros(self.n, dtype=k.dtype, device=k.device)
        diag = diag.index_add(0, self.fa, kf).index_add(0, self.fb, kf) + 2.0 * k * self.nbnd
        return v.index_add(0, self.pos_diag, diag)


def transpose_map(rowptr: np.ndarray, col: np.ndarray):
    """CSR pattern of A^T and the permutation perm with vals_T = vals[perm]."""
    n = len(rowptr) - 1
    rows = np.repeat(np.arange(n), np.diff(rowptr))
    order = np.lexsort((rows, col))
    rt = np.zeros(n + 1, np.int64)
    np.add.at(rt, col + 1, 1)
    return np.cumsum(rt).astype(np.int32), rows[order].astype(np.int32), order


class AMGSolve(torch.autograd.Function):
    """x = A^{-1} b with A given by (rowptr, col, values); differentiable in values and b."""

    @staticmethod
    def forward(ctx, values, b, rowptr, col, params, rtol, maxit, symmetric, tmap):
        B = torch.ones(rowptr.shape[0] - 1, dtype=torch.float64, device=values.device)
        Bh = None if params.symmetric else B  # candidates for A^T when R is built from A^T
        h = rn.Hierarchy(rowptr, col, values.detach().contiguous(), B, Bh, params=params)
        x = torch.zeros_like(b)
        h.solve(b.detach().contiguous(), x, rtol=rtol, maxit=maxit)
        ctx.h = h
        ctx.rowptr, ctx.col, ctx.params, ctx.rtol, ctx.maxit = rowptr, col, params, rtol, maxit
        ctx.symmetric, ctx.tmap = symmetric, tmap
        ctx.save_for_backward(values, x)
        return x

    @staticmethod
    def backward(ctx, gx):
        values, x = ctx.saved_tensors
        lam = torch.zeros_like(x)
        if ctx.symmetric:
            ctx.h.solve(gx.contiguous(), lam, rtol=ctx.rtol, maxit=ctx.maxit)
        else:  # a hierarchy for A^T
            rpt, colt, perm = ctx.tmap
            B = torch.ones_like(x)
            ht = rn.Hierarchy(rpt, colt, values.detach()[perm].contiguous(), B, None if ctx.params.symmetric else B,
                              params=ctx.params)
            ht.solve(gx.contiguous(), lam, rtol=ctx.rtol, maxit=ctx.maxit)
            ht.close()
        ctx.h.close()
        grad = torch.empty_like(values)
        rn.adjoint_grad(ctx.rowptr, ctx.col, lam, x, grad)
        return grad, lam, None, None, None, None, None, None, None


def solve(values, b, rowptr, col, params=None, rtol=1e-14, maxit=2000, symmetric=True):
    """Differentiable x = A^{-1} b (see AMGSolve).  For symmetric=False the
    adjoint uses a hierarchy built for A^T."""
    if params is None:
        params = rn.default_params()
    tmap = None
    if not symmetric:
        rpt, colt, perm = transpose_map(rowptr.cpu().numpy(), col.cpu().numpy())
        dev = values.device
        tmap = (torch.from_numpy(rpt).to(dev), torch.from_numpy(colt).to(dev), torch.from_numpy(perm).to(dev))
    return AMGSolve.apply(values, b, rowptr, col, params, rtol, maxit, symmetric, tmap)
