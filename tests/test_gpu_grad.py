"""Derivatives of the estimate: mf_grad (reverse mode, a hand-written adjoint
sweep of |M|^2) and mf_grad_forward (forward mode, dual numbers) against
each other and against central finite differences.

What pins them:
  * the oracle's FP64 weights at y +- h e_j, at m_t +- h and at Gamma_t +- h
    (a few events, fully independent of the CUDA path), as plain central
    differences and, for a tight bar, Richardson-extrapolated;
  * the CUDA path's own FP64 weights at theta +- h (all events of the sample,
    a different code path: the plain iteration kernels with shifted
    parameters), per event, for m_t and Gamma_t, as a consistency check of
    the whole sample beside the oracle's few events;
  * g_s: I(g_s) is a homogeneous polynomial of degree 2 n_gluons, so the
    central difference of the library's own I agrees to O(h^2);
  * sigma and the per-event weights equal those of mf_vegas_iterate.

Central differences have truncation error O(h^2 w''') and rounding error
O(eps w / h); events whose cut decision or Vegas bin changes inside +- h have
no derivative there and are excluded.  The error of an event is measured
relative to max(|fd|, 1e-2 |w| / theta): a derivative far below the weight's
own scale is compared with that scale.
"""
import math

import numpy as np
import pytest
import torch

import oracle.integrate as oi
import oracle.philox as oph
from tests.inputs import random_grid

pytestmark = pytest.mark.gpu

NAMES = ["gg_ttx_1tev", "gg_ttxg_13tev", "gg_ttxgg_13tev"]


@pytest.fixture(scope="module")
def mf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2211_14056_gb300 as mf
    return mf


def _proc(mf, name, precision, **over):
    from paper_2211_14056_gb300.workloads import PROCESS_IDS, WORKLOADS, process_kwargs
    w = dict(WORKLOADS[name], **over)
    return mf.Process(PROCESS_IDS[w["process"]], **process_kwargs(w, precision)), w


def _grad(p, edges, seed, it, n):
    g = p.grid()
    g.set(edges)
    th = torch.full((3 * n,), float("nan"), dtype=torch.float64, device="cuda")
    dy = torch.full((p.ndim * n,), float("nan"), dtype=torch.float64, device="cuda")
    sigma, ds = p.grad(g, seed, it, n, dw_dtheta=th, dw_dy=dy)
    torch.cuda.synchronize()
    return sigma, ds, th.view(3, n).cpu().numpy(), dy.view(p.ndim, n).cpu().numpy()


def _grad_both(p, edges, seed, it, n):
    """(reverse, forward) results of the same derivative request."""
    out = []
    for forward in (False, True):
        g = p.grid()
        g.set(edges)
        th = torch.full((3 * n,), float("nan"), dtype=torch.float64, device="cuda")
        dy = torch.full((p.ndim * n,), float("nan"), dtype=torch.float64, device="cuda")
        sigma, ds = p.grad(g, seed, it, n, dw_dtheta=th, dw_dy=dy, forward=forward)
        torch.cuda.synchronize()
        out.append((sigma, ds, th.view(3, n).cpu().numpy(), dy.view(p.ndim, n).cpu().numpy()))
    return out


@pytest.mark.parametrize("precision,bar", [("MF_FP64", 1e-9), ("MF_FP32", 2e-3)])
@pytest.mark.parametrize("name", NAMES)
def test_reverse_mode_matches_forward_mode(mf, name, precision, bar):
    """The adjoint sweep (mf_grad) and the dual-number passes
    (mf_grad_forward) compute the same derivatives by different algorithms:
    per event and per output row they agree to rounding (relative to the
    row's largest entry; FP32 rounding of two different operation orders)."""
    p, w = _proc(mf, name, getattr(mf, precision))
    n = 3001
    edges = random_grid(p.ndim, seed=31)
    (sr, dr, tr, yr), (sf, df, tf, yf) = _grad_both(p, edges, 17, 2, n)
    assert np.isfinite(tr).all() and np.isfinite(yr).all()
    rows = [("w", tr[0], tf[0]), ("dm_t", tr[1], tf[1]), ("dGamma_t", tr[2], tf[2])]
    rows += [(f"dy{j}", yr[j], yf[j]) for j in range(p.ndim)]
    # rows whose exact value vanishes (d/dGamma_t at Gamma_t = 0, d/dphi of a
    # 2 -> 2 process) hold rounding noise in both modes: each row is measured
    # against max(its largest entry, floor * the largest weight)
    floor = 1e-5 if precision == "MF_FP64" else 1e-3
    wmax = np.max(np.abs(tf[0]))           # dw/dg_s = (2 n_gluons / g_s) w: the weights' scale
    worst = 0.0
    for label, a, b in rows:
        scale = max(np.max(np.abs(b)), floor * wmax)
        err = np.max(np.abs(a - b)) / scale
        print(f"{name} {precision} {label}: max |rev - fwd| / scale = {err:.2e}")
        worst = max(worst, err)
    assert worst < bar
    assert sr == pytest.approx(sf, rel=1e-12 if precision == "MF_FP64" else 1e-6)
    for k in range(3):
        assert dr[k] == pytest.approx(df[k], rel=10 * bar, abs=floor * abs(df[0]))


def _weights(mf, name, edges, seed, it, n, **over):
    p, _ = _proc(mf, name, mf.MF_FP64, **over)
    g = p.grid()
    g.set(edges)
    wt = torch.empty(n, dtype=torch.float64, device="cuda")
    r = p.vegas_iterate(g, seed=seed, it=it, n=n, refine=False, weights=wt)
    return wt.cpu().numpy(), r


def _fd_error(ad, wp, wm, w0, h, theta):
    fd = (wp - wm) / (2 * h)
    scale = np.maximum(np.abs(fd), 1e-2 * np.abs(w0) / theta)
    return np.abs(ad - fd) / scale


def _report(label, err):
    print(f"{label}: {err.size} events, median {np.median(err):.2e}, p99 {np.quantile(err, 0.99):.2e}, "
          f"max {err.max():.2e}")


@pytest.mark.parametrize("name,n", [("gg_ttx_1tev", 20000), ("gg_ttxg_13tev", 6000), ("gg_ttxgg_13tev", 1500)])
def test_theta_derivatives_match_central_differences(mf, name, n):
    seed, it = 21, 2
    p, w = _proc(mf, name, mf.MF_FP64, wt=1.5)
    edges = random_grid(p.ndim, seed=5)
    sigma, ds, th, dy = _grad(p, edges, seed, it, n)
    w0, r0 = _weights(mf, name, edges, seed, it, n, wt=1.5)
    # the estimate and the weights are those of the iteration
    assert sigma == pytest.approx(r0["I_k"], rel=1e-12)
    ng = p.ngluons
    wg = th[0] * w["gs"] / (2 * ng)
    nz = w0 > 0
    np.testing.assert_array_equal(wg > 0, nz)
    rel = np.abs(wg[nz] / w0[nz] - 1)
    assert np.mean(rel <= 1e-12) >= 0.99 and rel.max() <= 1e-10
    # sigma and its derivatives are the means of the per-event rows
    assert ds[0] == pytest.approx(2 * ng * sigma / w["gs"], rel=1e-14)
    assert ds[1] == pytest.approx(th[1].mean(), rel=1e-10, abs=1e-14 * abs(sigma))
    assert ds[2] == pytest.approx(th[2].mean(), rel=1e-10, abs=1e-14 * abs(sigma))
    assert np.all(np.isfinite(th)) and np.all(np.isfinite(dy))
    assert np.all(th[:, ~nz] == 0) and np.all(dy[:, ~nz] == 0)
    for row, key, h_rel in ((1, "mt", 1e-6), (2, "wt", 1e-5)):
        theta = w[key]
        h = h_rel * theta
        wp, _ = _weights(mf, name, edges, seed, it, n, **{"wt": 1.5, key: theta + h})
        wm, _ = _weights(mf, name, edges, seed, it, n, **{"wt": 1.5, key: theta - h})
        keep = nz & (wp > 0) & (wm > 0)
        assert keep.sum() >= 0.9 * nz.sum()
        err = _fd_error(th[row][keep], wp[keep], wm[keep], w0[keep], h, theta)
        _report(f"{name} dw/d{key}", err)
        assert np.mean(err <= 1e-5) >= 0.99
        assert err.max() <= 1e-2


def test_g_s_law_against_the_estimate(mf):
    """dI/dg_s against the central difference of the library's own estimate."""
    name, n, seed = "gg_ttxg_13tev", 4000, 8
    p, w = _proc(mf, name, mf.MF_FP64)
    edges = random_grid(p.ndim, seed=6)
    sigma, ds, _, _ = _grad(p, edges, seed, 0, n)
    h = 1e-4 * w["gs"]
    _, rp = _weights(mf, name, edges, seed, 0, n, gs=w["gs"] + h)
    _, rm = _weights(mf, name, edges, seed, 0, n, gs=w["gs"] - h)
    fd = (rp["I_k"] - rm["I_k"]) / (2 * h)
    # truncation: I ~ g^6, (I(g+h) - I(g-h))/(2h) = I'(g) (1 + 10/6 (h/g)^2 + ...)
    assert ds[0] == pytest.approx(fd, rel=1e-7)


def _oracle_setup(w, amplitude="bg", **over):
    from paper_2211_14056_gb300.workloads import oracle_cfg
    cfg = dict(oracle_cfg(w), **over)
    return oi.Setup(cfg, amplitude=amplitude)


@pytest.mark.parametrize("name,k", [("gg_ttx_1tev", 40), ("gg_ttxg_13tev", 30), ("gg_ttxgg_13tev", 20)])
def test_uniform_and_mass_derivatives_match_oracle_differences(mf, name, k):
    """dw/dy_j and dw/dm_t of the first k events passing the cuts against
    central differences of the oracle's weights (its own Vegas map, phase
    space and amplitudes).  gg_ttxg has an odd Vegas dimension (7): the last
    uniform rides alone in its tangent pass."""
    seed, it, n = 33, 1, 256
    p, w = _proc(mf, name, mf.MF_FP64)
    edges = random_grid(p.ndim, seed=9)
    _, _, th, dy = _grad(p, edges, seed, it, n)
    amp = "feynman" if name == "gg_ttx_1tev" else "bg"
    st = _oracle_setup(w, amp)
    ev = np.arange(n, dtype=np.uint64)
    y = oph.uniforms(seed, it, ev, st.ndim)
    w0, b0 = st.weights(y, edges)
    sel = np.flatnonzero(w0 > 0)[:k]
    assert sel.size == k
    ys = y[:, sel]
    hy = 1e-7
    errs = []
    for j in range(st.ndim):
        yp, ym = ys.copy(), ys.copy()
        yp[j] += hy
        ym[j] -= hy
        wp, bp = st.weights(yp, edges)
        wm, bm = st.weights(ym, edges)
        keep = (wp > 0) & (wm > 0) & np.all(bp == b0[:, sel], axis=0) & np.all(bm == b0[:, sel], axis=0)
        errs.append(_fd_error(dy[j, sel][keep], wp[keep], wm[keep], w0[sel][keep], hy, 1.0))
    err = np.concatenate(errs)
    _report(f"{name} dw/dy vs oracle", err)
    assert err.size >= 0.8 * k * st.ndim
    assert np.mean(err <= 1e-5) >= 0.95 and err.max() <= 1e-3
    mt = w["mt"]
    hm = 1e-6 * mt
    wp, _ = _oracle_setup(w, amp, mt=mt + hm).weights(ys, edges)
    wm, _ = _oracle_setup(w, amp, mt=mt - hm).weights(ys, edges)
    keep = (wp > 0) & (wm > 0)
    err = _fd_error(th[1, sel][keep], wp[keep], wm[keep], w0[sel][keep], hm, mt)
    _report(f"{name} dw/dmt vs oracle", err)
    assert keep.sum() >= k - 1
    assert np.mean(err <= 1e-5) >= 0.9 and err.max() <= 1e-3


def _richardson(f, h):
    """Derivative at 0 from central differences at h and h/2, extrapolated
    (Richardson): truncation O(h^4), rounding O(eps / h)."""
    d1 = (f(h) - f(-h)) / (2 * h)
    d2 = (f(h / 2) - f(-h / 2)) / h
    return (4 * d2 - d1) / 3


@pytest.mark.parametrize("name,k", [("gg_ttx_1tev", 40), ("gg_ttxg_13tev", 30), ("gg_ttxgg_13tev", 20)])
def test_derivatives_match_extrapolated_oracle_differences(mf, name, k):
    """FP64 dw/dy_j and dw/dm_t against the oracle's Richardson-extrapolated
    central differences (h = 1e-4 in y, 1e-3 m_t in m_t), accurate to ~1e-10
    (the oracle's extrapolations at h and 2h agree to a median of 1e-11).
    Events whose bins or cut decision change within +-h are excluded; events
    with a large fourth derivative inside +-h (a few near-singular ones) are
    the tail the 99% bar leaves out."""
    seed, it, n = 33, 1, 256
    p, w = _proc(mf, name, mf.MF_FP64)
    edges = random_grid(p.ndim, seed=9)
    _, _, th, dy = _grad(p, edges, seed, it, n)
    amp = "feynman" if name == "gg_ttx_1tev" else "bg"
    st = _oracle_setup(w, amp)
    y = oph.uniforms(seed, it, np.arange(n, dtype=np.uint64), st.ndim)
    w0, b0 = st.weights(y, edges)
    sel = np.flatnonzero(w0 > 0)[:k]
    ys = y[:, sel]
    errs = []
    for j in range(st.ndim):
        def f(h, j=j):
            yy = ys.copy()
            yy[j] += h
            ww, bb = st.weights(yy, edges)
            return np.where((ww > 0) & np.all(bb == b0[:, sel], axis=0), ww, np.nan)
        ref = _richardson(f, 1e-4)
        ok = np.isfinite(ref)
        scale = np.maximum(np.abs(ref[ok]), 1e-2 * np.abs(w0[sel][ok]))
        errs.append(np.abs(dy[j, sel][ok] - ref[ok]) / scale)
    err = np.concatenate(errs)
    _report(f"{name} dw/dy vs extrapolated oracle", err)
    assert err.size >= 0.8 * k * st.ndim
    assert np.median(err) < 1e-9 and np.quantile(err, 0.95) < 1e-7 and np.mean(err < 1e-6) >= 0.99
    mt = w["mt"]
    def fm(h):
        ww, _ = _oracle_setup(w, amp, mt=mt + h).weights(ys, edges)
        return np.where(ww > 0, ww, np.nan)
    ref = _richardson(fm, 1e-3 * mt)
    ok = np.isfinite(ref)
    scale = np.maximum(np.abs(ref[ok]), 1e-2 * np.abs(w0[sel][ok]) / mt)
    err = np.abs(th[1, sel][ok] - ref[ok]) / scale
    _report(f"{name} dw/dmt vs extrapolated oracle", err)
    assert ok.sum() >= k - 1 and err.max() < 1e-8


@pytest.mark.parametrize("name,k", [("gg_ttx_1tev", 40), ("gg_ttxg_13tev", 30), ("gg_ttxgg_13tev", 20)])
def test_width_derivative_matches_extrapolated_oracle_differences(mf, name, k):
    """FP64 dw/dGamma_t at Gamma_t = 1.5 GeV against Richardson-extrapolated
    central differences of the oracle's weights at Gamma_t +- h (h = 1e-2
    GeV, its own Vegas map, phase space and amplitudes; a different algorithm
    from the adjoint sweep).  Gamma_t enters only the internal top propagators
    1/(P^2 - m_t^2 + i m_t Gamma_t), smooth on the scale Gamma_t, so the
    extrapolation's O(h^4) truncation is ~(h/Gamma_t)^4 ~ 2e-9 relative and the
    rounding ~eps w / h ~ 1e-14 w.  Cuts and bins do not depend on Gamma_t:
    every event that passes is compared.  The forward-mode pass
    (mf_grad_forward) is held to the same reference."""
    seed, it, n = 41, 1, 256
    wt = 1.5
    p, w = _proc(mf, name, mf.MF_FP64, wt=wt)
    edges = random_grid(p.ndim, seed=19)
    _, _, th, _ = _grad(p, edges, seed, it, n)
    (_, _, _, _), (_, _, thf, _) = _grad_both(p, edges, seed, it, n)
    amp = "feynman" if name == "gg_ttx_1tev" else "bg"
    w1 = dict(w, wt=wt)
    st = _oracle_setup(w1, amp)
    y = oph.uniforms(seed, it, np.arange(n, dtype=np.uint64), st.ndim)
    w0, _ = st.weights(y, edges)
    sel = np.flatnonzero(w0 > 0)[:k]
    assert sel.size == k
    ys = y[:, sel]

    def f(h):
        ww, _ = _oracle_setup(w1, amp, wt=wt + h).weights(ys, edges)
        return ww

    ref = _richardson(f, 1e-2)
    # the weight's own scale per unit Gamma_t is w / Gamma_t; a derivative far
    # below it (an event with no near-resonant internal top) is compared there
    scale = np.maximum(np.abs(ref), 1e-2 * np.abs(w0[sel]) / wt)
    for label, got in (("reverse", th[2, sel]), ("forward", thf[2, sel])):
        err = np.abs(got - ref) / scale
        _report(f"{name} dw/dGamma_t ({label}) vs extrapolated oracle", err)
        assert np.median(err) < 1e-8 and err.max() < 1e-6
    # with a final-state gluon an internal top (t + g) can come near its pole:
    # there Gamma_t moves the weights visibly (for g g -> t tbar the internal
    # tops are space-like and the derivative is ~1e-6 w / Gamma_t)
    if name != "gg_ttx_1tev":
        assert np.max(np.abs(ref) * wt / np.abs(w0[sel])) > 1e-4


@pytest.mark.parametrize("name,n", [("gg_ttxg_13tev", 20000), ("gg_ttxgg_13tev", 4000)])
def test_fp32_derivatives_against_fp64(mf, name, n):
    """FP32 kinematics and amplitudes (FP64 weights): the error of the
    single-precision derivatives of the estimate.  dI/dm_t and dI/dGamma_t
    are sums of terms of both signs (the width term changes sign across the
    internal top resonance), so their error is measured against the mean
    |per-event derivative|, the scale of the terms summed.  A near-resonant
    internal top propagator, P^2 - m_t^2 formed from FP32 momenta of size E,
    carries a relative error ~ 6e-8 E^2 / |P^2 - m_t^2|: a few such events
    dominate the FP32 Gamma_t sum of gg -> t tbar g g (up to ~6e-3 per event)."""
    edges = random_grid(_proc(mf, name, mf.MF_FP64)[0].ndim, seed=12)
    s64, d64, t64, _ = _grad(_proc(mf, name, mf.MF_FP64, wt=1.5)[0], edges, 4, 0, n)
    s32, d32, t32, _ = _grad(_proc(mf, name, mf.MF_FP32, wt=1.5)[0], edges, 4, 0, n)
    rel = [abs(s32 / s64 - 1), abs(d32[0] / d64[0] - 1)]
    # events whose cut decision is the same in both precisions
    both = (t64[0] != 0) & (t32[0] != 0)
    flips = int(np.sum((t64[0] != 0) != (t32[0] != 0)))
    for k in (1, 2):
        scale = np.mean(np.abs(t64[k]))
        rel.append(abs(np.sum(t32[k][both] - t64[k][both])) / n / scale)
        ev = np.abs(t32[k][both] - t64[k][both]) / np.maximum(np.abs(t64[k][both]), 1e-2 * scale)
        print(f"{name} FP32 per-event d/d{'m_t' if k == 1 else 'Gamma_t'}: median {np.median(ev):.1e} "
              f"p99 {np.quantile(ev, 0.99):.1e} max {ev.max():.1e}")
        assert np.median(ev) < 1e-4
    print(f"{name} FP32 vs FP64: sigma {rel[0]:.2e}, dg_s {rel[1]:.2e}; common events ({flips} cut flips): "
          f"dm_t {rel[2]:.2e}, dGamma_t {rel[3]:.2e} of the mean |term|")
    assert rel[0] < 1e-4 and rel[1] < 1e-4 and rel[2] < 1e-4 and rel[3] < 3e-3


def test_sizes_and_arguments(mf):
    """One event, a ragged count, derivative rows optional, bad arguments."""
    p, w = _proc(mf, "gg_ttxg_13tev", mf.MF_FP64)
    edges = random_grid(p.ndim, seed=3)
    g = p.grid()
    g.set(edges)
    s_all, d_all, th, _ = _grad(p, edges, 2, 0, 333)
    s_row, d_row = p.grad(g, 2, 0, 333)               # no per-event rows
    # the sums follow the list of passing events, whose order comes from the
    # sampling kernel's atomics: equal up to summation order
    assert s_row == pytest.approx(s_all, rel=1e-13)
    np.testing.assert_allclose(d_row, d_all, rtol=1e-12)
    s1, d1, th1, _ = _grad(p, edges, 2, 0, 1)
    assert th1[1, 0] == th[1, 0] and s1 == pytest.approx(th[0, 0] * w["gs"] / 6, rel=1e-15, abs=0)
    with pytest.raises(mf.MFError):
        p.grad(g, 2, 0, 0)
    with pytest.raises(mf.MFError):
        p.grad(g, 2, -1, 10)
    q, _ = _proc(mf, "gg_ttxgg_13tev", mf.MF_FP64)
    with pytest.raises(mf.MFError):
        q.grad(g, 2, 0, 10)


def test_autograd_cross_section(mf):
    """torch.autograd through the estimate: backward returns mf_grad's
    derivatives, and a step along the gradient changes I to first order."""
    from paper_2211_14056_gb300.autograd import cross_section
    from paper_2211_14056_gb300.workloads import PROCESS_IDS, WORKLOADS, process_kwargs
    name, n, seed = "gg_ttxg_13tev", 3000, 5
    w = dict(WORKLOADS[name], wt=1.5)
    kw = process_kwargs(w, mf.MF_FP64)
    for key in ("gs", "mt", "wt"):
        kw.pop(key)
    p, _ = _proc(mf, name, mf.MF_FP64, wt=1.5)
    edges = random_grid(p.ndim, seed=4)
    theta = torch.tensor([w["gs"], w["mt"], w["wt"]], dtype=torch.float64, requires_grad=True)
    I = cross_section(theta, PROCESS_IDS[w["process"]], edges, seed, 0, n, **kw)
    I.backward()
    sigma, ds, _, _ = _grad(p, edges, seed, 0, n)
    assert I.item() == pytest.approx(sigma, rel=1e-13)              # summation order
    np.testing.assert_allclose(theta.grad.numpy(), np.array(ds), rtol=1e-12)
    step = 1e-6 * theta.detach() * torch.sign(theta.grad)
    I2 = cross_section(theta.detach() + step, PROCESS_IDS[w["process"]], edges, seed, 0, n, **kw)
    pred = float((theta.grad * step).sum())
    assert (I2.item() - sigma) == pytest.approx(pred, rel=1e-2)
    assert math.isfinite(I2.item())


def test_autograd_event_weights(mf):
    """torch.autograd through the per-event weights w(theta, y): the forward
    values equal mf_vegas_iterate's weights, backward gives the
    vector-Jacobian products of mf_grad's per-event derivatives for theta and
    for the uniforms, and the uniforms are the library's Philox stream
    (checked against the oracle's Philox bit for bit)."""
    from paper_2211_14056_gb300.autograd import event_weights
    from paper_2211_14056_gb300.workloads import PROCESS_IDS, WORKLOADS, process_kwargs
    name, n, seed, it = "gg_ttxgg_13tev", 777, 6, 1
    w = WORKLOADS[name]
    kw = process_kwargs(w, mf.MF_FP64)
    for key in ("gs", "mt", "wt"):
        kw.pop(key)
    p, _ = _proc(mf, name, mf.MF_FP64)
    edges = random_grid(p.ndim, seed=8)
    y = mf.uniforms(seed, it, n, p.ndim)
    yo = oph.uniforms(seed, it, np.arange(n, dtype=np.uint64), p.ndim)
    np.testing.assert_array_equal(y.cpu().numpy(), yo)
    y.requires_grad_(True)
    theta = torch.tensor([w["gs"], w["mt"], w["wt"]], dtype=torch.float64, requires_grad=True)
    wts = event_weights(theta, y, PROCESS_IDS[w["process"]], edges, seed, it, **kw)
    w0, _ = _weights(mf, name, edges, seed, it, n)
    np.testing.assert_array_equal(wts.detach().cpu().numpy(), w0)
    gvec = torch.linspace(-1.0, 2.0, n, dtype=torch.float64, device="cuda")
    (wts * gvec).sum().backward()
    _, _, th, dy = _grad(p, edges, seed, it, n)
    gv = gvec.cpu().numpy()
    np.testing.assert_allclose(theta.grad.numpy(), th @ gv, rtol=1e-12)
    np.testing.assert_allclose(y.grad.cpu().numpy(), dy * gv[None, :], rtol=1e-12, atol=0)
    with pytest.raises(ValueError):
        event_weights(theta, torch.rand(p.ndim, n, dtype=torch.float64, device="cuda"),
                      PROCESS_IDS[w["process"]], edges, seed, it, **kw)


def test_fp32_derivatives_finite_near_the_luminosity_edge(mf):
    """2^20 events on the uniform grid include one with x_1 within an FP32 ulp
    of 1 (its weight is ~1e-33 pb): ln(1 - x_1) comes from expm1, so the
    FP32 weight and every derivative stay finite."""
    p, w = _proc(mf, "gg_ttxgg_13tev", mf.MF_FP32)
    g = p.grid()
    n = 2 ** 20
    th = torch.empty(3 * n, dtype=torch.float64, device="cuda")
    dy = torch.empty(p.ndim * n, dtype=torch.float64, device="cuda")
    sigma, ds = p.grad(g, w["seed"], 5001, n, th, dy)
    torch.cuda.synchronize()
    assert math.isfinite(sigma) and all(math.isfinite(x) for x in ds)
    assert torch.isfinite(th).all().item() and torch.isfinite(dy).all().item()
