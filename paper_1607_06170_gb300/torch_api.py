"""PyTorch-facing layer: the PSF projector as a differentiable op and the MLEM
driver.  Every arithmetic step runs in libpsf.so; torch provides the tensors
and the stream."""
from __future__ import annotations

import torch

from . import psf


class PSFProject(torch.autograd.Function):
    """y = A x with A the PSF system matrix; the backward pass is the
    hand-written PSF back-projector A^T (psf_back)."""

    @staticmethod
    def forward(ctx, x, matrix):
        ctx.matrix = matrix
        return matrix.forward(x.contiguous())

    @staticmethod
    def backward(ctx, grad_y):
        return ctx.matrix.back(grad_y.contiguous()), None


def project(x, matrix):
    return PSFProject.apply(x, matrix)


def sensitivity(matrix, n_rows: int, device="cuda"):
    """A^T 1 through psf_sensitivity (n_rows kept for the call's signature)."""
    del n_rows
    return matrix.sensitivity(device=device)


def mlem(matrix, y, iters: int = 10, x0=None, sens=None, graph: bool = False):
    """MLEM (Sec. 3): sens = A^T 1; x <- x * A^T(y / A x) / sens.

    Voxels with sens < 1e-12 * max(sens) are held at zero, and 0/0 in the
    ratio is zero.  All steps are library kernels (psf_forward, psf_em_ratio,
    psf_back, psf_em_update).  With graph=True the `iters` iterations are
    captured once in a CUDA graph (after one uncaptured iteration on a copy,
    which sets up the kernels' launch attributes) and replayed as one launch.
    """
    yhat = torch.empty_like(y)
    ratio = torch.empty_like(y)
    if sens is None and x0 is None and iters > 0:
        # first iteration from an image of ones: its forward projection equals
        # that of ones on the voxels the scanner sees (the others' columns are
        # zero), so sens = A^T 1 comes with the first back-projection
        # (psf_back_sens, one pass over the rows)
        x = torch.ones(matrix.n_cols, dtype=torch.float32, device=y.device)
        matrix.forward(x, out=yhat)
        psf.em_ratio(y, yhat, out=ratio)
        bp, sens = matrix.back_sens(ratio)
        floor = 1e-12 * float(sens.max())
        psf.em_update(x, bp, sens, floor)
        iters -= 1
    else:
        if sens is None:
            sens = sensitivity(matrix, y.numel(), y.device)
        floor = 1e-12 * float(sens.max())
        if x0 is None:
            x = torch.ones_like(sens)
            psf.em_update(x, sens, sens, floor)  # 1 on voxels the scanner sees, 0 elsewhere
        else:
            x = x0.clone()
        bp = torch.empty_like(sens)

    def iteration(xi):
        matrix.forward(xi, out=yhat)
        psf.em_ratio(y, yhat, out=ratio)
        matrix.back(ratio, out=bp)
        psf.em_update(xi, bp, sens, floor)

    if not graph:
        for _ in range(iters):
            iteration(x)
        return x
    if iters == 0:
        return x
    iteration(x.clone())  # uncaptured warm-up on a scratch copy
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, capture_error_mode="relaxed"):
        for _ in range(iters):
            iteration(x)
    g.replay()
    return x


def listmode_osem(matrix, rows, n_subsets: int, iters: int = 1, x0=None, sens=None,
                  sparse_adjoint: bool = True):
    """List-mode OSEM over events (the next step named in Sec. 5, with the
    subsets of Sec. 3): the events (their set rows, psf_event_rows) are split
    into n_subsets consecutive subsets, and each sub-iteration is
      x <- x * sum_{e in subset} A_e^T / (A_e x) / (A^T 1 / n_subsets),
    formed as the MLEM update on the subset's counts weighted by n_subsets
    (psf_histogram, psf_forward_masked -- the projection only on the LORs the
    subset's events hit --, psf_em_ratio, psf_back, psf_em_update).
    Voxels with sens < 1e-12 * max(sens) are held at zero.  With top-N spreads
    and sparse_adjoint, the plan's transpose of S is built once so that S^T of
    a subset's counts and ratios scatters from their nonzero entries."""
    n_ev = rows.numel()
    if sparse_adjoint and matrix.topn > 0:
        matrix.build_sparse_adjoint()
    if sens is None:
        sens = matrix.sensitivity(device=rows.device)
    floor = 1e-12 * float(sens.max())
    if x0 is None:
        x = torch.ones_like(sens)
        psf.em_update(x, sens, sens, floor)  # 1 on voxels the scanner sees
    else:
        x = x0.clone()
    counts = torch.empty(matrix.n_rows, dtype=torch.float32, device=rows.device)
    yhat = torch.empty_like(counts)
    ratio = torch.empty_like(counts)
    bp = torch.empty_like(sens)
    bounds = [n_ev * j // n_subsets for j in range(n_subsets + 1)]
    for _ in range(iters):
        for j in range(n_subsets):
            psf.histogram(rows[bounds[j]:bounds[j + 1]], matrix.n_rows, float(n_subsets),
                          out=counts)
            matrix.forward_masked(x, counts, out=yhat)
            psf.em_ratio(counts, yhat, out=ratio)
            matrix.back(ratio, out=bp)
            psf.em_update(x, bp, sens, floor)
    return x

