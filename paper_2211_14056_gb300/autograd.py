"""The cross-section estimate as a differentiable PyTorch function.

arXiv:2211.14056 (Sec. 2) builds the integrand from framework operations so
that it is differentiable, and notes that its custom matrix-element operator
has no derivative yet.  ``cross_section(theta, ...)`` is one Vegas iteration's
estimate I(theta) for theta = (g_s, m_t, Gamma_t); its backward pass uses the
forward-mode derivatives of ``mf_grad`` (dual numbers through the sampling and
amplitude kernels), so ``torch.autograd`` sees an ordinary scalar function.

Forward and backward run in the CUDA library only.  The Vegas grid, seed,
iteration and event count are fixed inputs (no derivative).
"""
import torch

from .binding import Process


class _CrossSection(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, process_id, edges, seed, it, n, kwargs):
        g_s, m_t, w_t = (float(v) for v in theta.detach().cpu().tolist())
        proc = Process(process_id, gs=g_s, mt=m_t, wt=w_t, **kwargs)
        grid = proc.grid(edges.shape[1] - 1)
        grid.set(edges)
        sigma, ds = proc.grad(grid, seed, it, n)
        grid.close()
        proc.close()
        ctx.save_for_backward(torch.tensor(ds, dtype=torch.float64))
        return theta.new_tensor(sigma)

    @staticmethod
    def backward(ctx, g):
        (ds,) = ctx.saved_tensors
        return g * ds.to(device=g.device, dtype=g.dtype), None, None, None, None, None, None


def cross_section(theta, process_id, edges, seed, it, n, **kwargs):
    """I(theta) of iteration `it` over events 0..n-1 on the grid `edges`
    (numpy [ndim, nbins+1]); theta = tensor([g_s, m_t, Gamma_t]); kwargs are the
    remaining ``Process`` parameters (sqrt_s, lumi, cuts, precision)."""
    if theta.shape != (3,):
        raise ValueError("theta must be (g_s, m_t, Gamma_t)")
    return _CrossSection.apply(theta, process_id, edges, seed, it, n, kwargs)
