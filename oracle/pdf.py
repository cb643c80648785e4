"""Parton densities on a grid: log-bicubic (Hermite) interpolation.

Test infrastructure (see ``oracle/__init__``).

arXiv:2211.14056 (Sec. 1) feeds its integrand with parton densities from
PDFFlow, the GPU port of the LHAPDF interpolation: x f(x, Q^2) is tabulated
per flavour on nodes in ln x and ln Q^2 and interpolated cubically in both
logarithms.  The scheme written out here (the paper prints none; this is the
LHAPDF/PDFFlow log-bicubic family, a reading):

  * nodes t_k = ln x_min + k (ln x_max - ln x_min) / (nx - 1), k = 0..nx-1, and
    s_l likewise in ln Q^2 (uniform in both logarithms);
  * a query outside [x_min, x_max] x [Q2_min, Q2_max] is clamped to the edge;
  * the cell: i = floor((t - t_0) / dt) clamped to [0, nx - 2], u = (t - t_i) / dt;
    j, v likewise in ln Q^2;
  * 1-D cubic Hermite on a cell [t_i, t_i+1] of width h:
        f(u) = h00(u) f_i + h10(u) h m_i + h01(u) f_i+1 + h11(u) h m_i+1,
        h00 = 2u^3 - 3u^2 + 1, h10 = u^3 - 2u^2 + u, h01 = -2u^3 + 3u^2, h11 = u^3 - u^2,
    with node slopes m_k from finite differences: the mean of the two
    neighbouring difference quotients inside, the one-sided quotient at the
    first and last node;
  * in 2-D: the rows l = j-1 .. j+2 (those that exist) are interpolated in
    ln x at t (each with its own x-slopes), giving g_l; then the Hermite step
    in ln Q^2 on [s_j, s_j+1] uses g_j, g_j+1 and slopes from the same finite
    differences of the g_l (one-sided where the grid ends).

The grid is an input (``xf[flavour][l][k]`` = x f at x_k, Q^2_l); this module
only interpolates it.
"""
import numpy as np


def _hermite(u, h, f0, f1, m0, m1):
    """Cubic Hermite on one cell of width h at local coordinate u in [0, 1]."""
    u2, u3 = u * u, u * u * u
    h00 = 2 * u3 - 3 * u2 + 1
    h10 = u3 - 2 * u2 + u
    h01 = -2 * u3 + 3 * u2
    h11 = u3 - u2
    return h00 * f0 + h10 * h * m0 + h01 * f1 + h11 * h * m1


def node_slopes(f, h):
    """Finite-difference slopes at every node of the last axis of f (equal
    spacing h): the mean of the two neighbouring difference quotients
    inside, the one-sided quotient at the first and last node."""
    f = np.asarray(f)
    d = np.diff(f, axis=-1) / h
    m = np.empty_like(f)
    m[..., 0] = d[..., 0]
    m[..., -1] = d[..., -1]
    m[..., 1:-1] = 0.5 * (d[..., 1:] + d[..., :-1])
    return m


def _cell(t, t0, h, n):
    """(cell index, local coordinate) of t on n nodes t0 + k h, t clamped."""
    t = np.clip(t, t0, t0 + (n - 1) * h)
    i = np.floor((t - t0) / h).astype(np.int64)
    i = np.clip(i, 0, n - 2)
    return i, (t - (t0 + i * h)) / h


class PDFGrid:
    """One tabulated set: xf[nflav][nq][nx] on uniform nodes in ln x and ln Q^2.
    dtype: the arithmetic (FP64; np.longdouble gives the same scheme with a
    wider mantissa, which the tests use to measure FP64 rounding)."""

    def __init__(self, x_min, x_max, q2_min, q2_max, xf, dtype=np.float64):
        self.dtype = dtype
        self.xf = np.asarray(xf, dtype=dtype)
        self.nflav, self.nq, self.nx = self.xf.shape
        self.t0, self.s0 = np.log(dtype(x_min)), np.log(dtype(q2_min))
        self.ht = (np.log(dtype(x_max)) - self.t0) / (self.nx - 1)
        self.hs = (np.log(dtype(q2_max)) - self.s0) / (self.nq - 1)
        self.mx = node_slopes(self.xf, self.ht)          # x-slopes of every row's nodes

    def _row(self, f, l, i, u):
        """x-interpolation of rows l (arrays) at cells i, coordinates u."""
        return _hermite(u, self.ht, self.xf[f, l, i], self.xf[f, l, i + 1], self.mx[f, l, i], self.mx[f, l, i + 1])

    def xfx(self, flavour, x, q2):
        """x f(x, Q^2) of one flavour index at arrays x, q2 (same shape)."""
        x = np.asarray(x, dtype=self.dtype)
        q2 = np.asarray(q2, dtype=self.dtype)
        shape = np.broadcast(x, q2).shape
        x, q2 = np.broadcast_to(x, shape).ravel(), np.broadcast_to(q2, shape).ravel()
        i, u = _cell(np.log(x), self.t0, self.ht, self.nx)
        j, v = _cell(np.log(q2), self.s0, self.hs, self.nq)
        nq, hs = self.nq, self.hs
        # the rows j-1 .. j+2 interpolated in ln x (a row outside the grid is
        # never used: its slope term falls back to the one-sided quotient)
        g = [self._row(flavour, np.clip(j + d, 0, nq - 1), i, u) for d in (-1, 0, 1, 2)]
        gm, g0, g1, g2 = g
        m0 = np.where(j == 0, (g1 - g0) / hs, 0.5 * ((g1 - g0) / hs + (g0 - gm) / hs))
        m1 = np.where(j + 1 == nq - 1, (g1 - g0) / hs, 0.5 * ((g2 - g1) / hs + (g1 - g0) / hs))
        return _hermite(v, hs, g0, g1, m0, m1).reshape(shape)
