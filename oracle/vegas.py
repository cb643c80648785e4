"""Vegas adaptive importance sampling: map, accumulation, refinement, combination.

Test infrastructure (see ``oracle/__init__``).

The paper (arXiv:2211.14056, Sec. 1) names Vegas (Lepage, J. Comput. Phys. 27
(1978) 192; CLNS-80/447 (1980)) as the integrator that VegasFlow tensorises
over events.  The steps below follow Lepage's separable-grid algorithm:

  map         y in [0,1)^d -> x through d piecewise-linear maps of N_b bins;
              bin i = floor(y * N_b), x = e_i + (y N_b - i)(e_{i+1} - e_i),
              Jacobian prod_j N_b (e_{i+1} - e_i).
  estimate    I_k = <w>,  sigma_k^2 = (<w^2> - I_k^2) / (N - 1).
  histogram   d_{j,b} = sum of w^2 over events whose bin in dim j is b.
  refine      smooth d (neighbour average), normalise, damp with
              r = ((1 - d) / ln(1/d))^alpha, then place new edges so that
              each new bin holds an equal share of sum(r), interpolating
              linearly inside the old bins (Lepage 1980 order: smoothing
              before damping).
  combine     inverse-variance weighted mean of the iterations, its error
              and chi^2 per degree of freedom.
"""
import numpy as np

NBINS = 50
ALPHA = 1.5


def uniform_grid(ndim, nbins=NBINS):
    """Edges e[ndim, nbins+1] of the uniform grid on [0, 1]."""
    return np.tile(np.linspace(0.0, 1.0, nbins + 1), (ndim, 1))


def vegas_map(y, edges):
    """y[d, N] -> (x[d, N], jacobian[N], bins[d, N]).

    The bin is taken from the IEEE product fl(y * N_b) and clamped to N_b - 1,
    which keeps the index inside the grid even if that product rounds up to
    N_b (it cannot for y < 1 drawn with 53 bits, but the clamp is part of the
    definition used on both sides).
    """
    y = np.asarray(y, dtype=np.float64)
    nb = edges.shape[1] - 1
    t = y * float(nb)
    bins = np.minimum(np.floor(t), nb - 1).astype(np.int64)
    lo = np.take_along_axis(edges, bins, axis=1)
    hi = np.take_along_axis(edges, bins + 1, axis=1)
    width = hi - lo
    x = lo + (t - bins) * width
    jac = np.prod(nb * width, axis=0)
    return x, jac, bins


def accumulate(w, bins, nbins=NBINS):
    """Per-iteration sums: (sum w, sum w^2, d[d, nbins] = sum w^2 per bin)."""
    w = np.asarray(w, dtype=np.float64)
    w2 = w * w
    ndim = bins.shape[0]
    hist = np.zeros((ndim, nbins))
    for j in range(ndim):
        hist[j] = np.bincount(bins[j], weights=w2, minlength=nbins)
    return float(np.sum(w)), float(np.sum(w2)), hist


def estimate(sum_w, sum_w2, n):
    """I_k and sigma_k^2 of one iteration of n events."""
    mean = sum_w / n
    var = (sum_w2 / n - mean * mean) / (n - 1)
    return mean, var


def refine_dim(edges, d, alpha=ALPHA):
    """New edges of one dimension from its histogram d (Lepage 1980).

    A dimension whose histogram is all zero keeps its edges.
    """
    nb = d.size
    if not np.any(d > 0):
        return edges.copy()
    # smoothing: neighbour average, halves at the two ends
    ds = np.empty(nb)
    ds[0] = (d[0] + d[1]) / 2.0
    ds[-1] = (d[-2] + d[-1]) / 2.0
    ds[1:-1] = (d[:-2] + d[1:-1] + d[2:]) / 3.0
    dn = ds / np.sum(ds)
    # damping; r(0) = 0 and r(1) = 1 (the 0/0 limit)
    r = np.zeros(nb)
    mid = (dn > 0) & (dn < 1)
    r[mid] = ((1.0 - dn[mid]) / np.log(1.0 / dn[mid])) ** alpha
    r[dn >= 1] = 1.0
    # equal shares of sum(r), linear inside the old bins
    cum = np.concatenate(([0.0], np.cumsum(r)))
    total = cum[-1]
    new = np.empty(nb + 1)
    new[0], new[-1] = 0.0, 1.0
    for k in range(1, nb):
        target = total * k / nb
        j = int(np.searchsorted(cum, target, side="right")) - 1
        j = min(max(j, 0), nb - 1)
        frac = (target - cum[j]) / r[j] if r[j] > 0 else 0.0
        new[k] = edges[j] + frac * (edges[j + 1] - edges[j])
    return new


def refine(edges, hist, alpha=ALPHA):
    """Refine every dimension of a grid from its per-bin sums of w^2."""
    return np.stack([refine_dim(edges[j], hist[j], alpha) for j in range(edges.shape[0])])


def combine(means, variances):
    """(I, sigma, chi2/dof) over iterations with means I_k and variances sigma_k^2.

    Every iteration is included; a zero variance makes the weights undefined
    and raises ValueError.
    """
    means = np.asarray(means, dtype=np.float64)
    variances = np.asarray(variances, dtype=np.float64)
    if np.any(variances <= 0):
        raise ValueError("an iteration has zero variance; combination undefined")
    wts = 1.0 / variances
    mean = np.sum(means * wts) / np.sum(wts)
    sigma = np.sum(wts) ** -0.5
    k = means.size
    chi2 = float(np.sum((means - mean) ** 2 * wts) / (k - 1)) if k > 1 else 0.0
    return float(mean), float(sigma), chi2
