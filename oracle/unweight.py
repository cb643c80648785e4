"""Hit-or-miss unweighting of weighted events.

Test infrastructure (see ``oracle/__init__``).

arXiv:2211.14056 computes weighted events for the integral; an event
generator turns them into unweighted events by the hit-or-miss method (the
practice of MadEvent and MadFlow; the paper states no algorithm, so this is a
reading).  For an event of weight w, a uniform r from an independent stream
(``philox.unweight_uniforms``) and a maximum weight w_max > 0:

  * the event is kept if r w_max < w (so with probability min(w, w_max)/w_max;
    events of weight <= 0 are never kept);
  * a kept event carries the weight max(1, w / w_max): 1 for an ordinary
    event, w / w_max for an overweight one (w > w_max), so that
    w_max * (sum of kept weights) / n estimates the integral without bias.
"""
import numpy as np


def unweight(w, r, w_max):
    """(kept [N] bool, weight of each event if kept [N])."""
    w = np.asarray(w, dtype=np.float64)
    r = np.asarray(r, dtype=np.float64)
    if not w_max > 0:
        raise ValueError("w_max must be > 0")
    kept = r * w_max < w
    weight = np.where(w > w_max, w / w_max, 1.0)
    return kept, weight
