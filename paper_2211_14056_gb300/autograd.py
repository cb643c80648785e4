"""The estimate and the event weights as differentiable PyTorch functions.

arXiv:2211.14056 (Sec. 2) builds the integrand from framework operations so
that it is differentiable, and notes that its custom matrix-element operator
has no derivative yet.  Here the derivatives come from the CUDA library's
reverse-mode pass (``mf_grad``: a hand-written adjoint sweep of |M|^2 that
recomputes every current, with forward tangents through the sampler), so
``torch.autograd`` sees ordinary functions:

* ``cross_section(theta, ...)``: one Vegas iteration's estimate I(theta), a
  scalar, for theta = (g_s, m_t, Gamma_t); backward = dI/dtheta.
* ``event_weights(theta, y, ...)``: the per-event weights w[n] of the same
  iteration as a function of theta and of the events' uniforms y[ndim, n];
  backward = the vector-Jacobian products sum_e g_e dw_e/dtheta and
  g_e dw_e/dy_je.  The uniforms are those of the library's Philox stream
  (``binding.uniforms``) and are checked against it: the weights are defined
  at those points only; y carries their derivative.

Forward and backward run in the CUDA library only; the derivative pass runs
only when an input requires a gradient.  The Vegas grid, seed, iteration and
event count are fixed inputs (no derivative).  Processes and grids are cached
per parameter set, so repeated evaluations do not re-create them.
"""
import functools

import torch

from .binding import Process, uniforms

@functools.lru_cache(maxsize=16)
def _process(process_id, g_s, m_t, w_t, kw_items):
    return Process(process_id, gs=g_s, mt=m_t, wt=w_t, **dict(kw_items))


@functools.lru_cache(maxsize=16)
def _grid(process_id, g_s, m_t, w_t, kw_items, nbins):
    return _process(process_id, g_s, m_t, w_t, kw_items).grid(nbins)


def _setup(theta, process_id, edges, kwargs):
    g_s, m_t, w_t = (float(v) for v in theta.detach().cpu().tolist())
    key = (process_id, g_s, m_t, w_t, tuple(sorted(kwargs.items())))
    proc = _process(*key)
    grid = _grid(*key, edges.shape[1] - 1)
    grid.set(edges)
    grid.reset()
    return proc, grid


class _CrossSection(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, process_id, edges, seed, it, n, kwargs):
        proc, grid = _setup(theta, process_id, edges, kwargs)
        if ctx.needs_input_grad[0]:
            sigma, ds = proc.grad(grid, seed, it, n)
        else:
            sigma, ds = proc.vegas_iterate(grid, seed, it, n, refine=False)["I_k"], [0.0, 0.0, 0.0]
        ctx.save_for_backward(torch.tensor(ds, dtype=torch.float64))
        return theta.new_tensor(sigma)

    @staticmethod
    def backward(ctx, g):
        (ds,) = ctx.saved_tensors
        return g * ds.to(device=g.device, dtype=g.dtype), None, None, None, None, None, None


class _EventWeights(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, y, process_id, edges, seed, it, kwargs):
        proc, grid = _setup(theta, process_id, edges, kwargs)
        ndim, n = y.shape
        if ndim != proc.ndim:
            raise ValueError(f"y must have shape ({proc.ndim}, n)")
        if not torch.equal(y, uniforms(seed, it, n, ndim)):
            raise ValueError("y must be the library's uniforms of these events (binding.uniforms(seed, it, n, ndim))")
        w = torch.empty(n, dtype=torch.float64, device="cuda")
        if ctx.needs_input_grad[0] or ctx.needs_input_grad[1]:
            th = torch.empty((3, n), dtype=torch.float64, device="cuda")
            dy = torch.empty((ndim, n), dtype=torch.float64, device="cuda")
            proc.grad(grid, seed, it, n, dw_dtheta=th, dw_dy=dy)
            ctx.save_for_backward(th, dy)
        ctx.theta_device = theta.device
        proc.vegas_accumulate(grid, seed, it, 0, n, weights=w)
        return w

    @staticmethod
    def backward(ctx, g):
        th, dy = ctx.saved_tensors
        g = g.to(dtype=torch.float64)
        gt = (th @ g).to(ctx.theta_device) if ctx.needs_input_grad[0] else None
        gy = dy * g[None, :] if ctx.needs_input_grad[1] else None
        return gt, gy, None, None, None, None, None


def cross_section(theta, process_id, edges, seed, it, n, **kwargs):
    """I(theta) of iteration `it` over events 0..n-1 on the grid `edges`
    (numpy [ndim, nbins+1]); theta = tensor([g_s, m_t, Gamma_t]); kwargs are the
    remaining ``Process`` parameters (sqrt_s, lumi, cuts, precision)."""
    if theta.shape != (3,):
        raise ValueError("theta must be (g_s, m_t, Gamma_t)")
    return _CrossSection.apply(theta, process_id, edges, seed, it, n, kwargs)


def event_weights(theta, y, process_id, edges, seed, it, **kwargs):
    """w[n] (device, float64) of iteration `it` over events 0..n-1 on the grid
    `edges`, differentiable in theta = tensor([g_s, m_t, Gamma_t]) and in the
    events' uniforms y = binding.uniforms(seed, it, n, ndim) (a device tensor
    [ndim, n], possibly with requires_grad)."""
    if theta.shape != (3,):
        raise ValueError("theta must be (g_s, m_t, Gamma_t)")
    return _EventWeights.apply(theta, y, process_id, edges, seed, it, kwargs)
