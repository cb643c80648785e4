"""GPU parity: the CUDA library (through its C ABI) against the FP64 oracle.

Bars (FP64 path): bins bit-exact; momenta and phase-space weights within
1e-12 relative; I_k, sigma_k and refined edges within 1e-12 relative; per-event
|M|^2 and event weights within 1e-12 relative, except events on which the
oracle's own FP64 algorithms disagree (``assert_fp64_parity``): there the
GPU value must lie within four times that disagreement of the reference, and
every event within 1e-10.  FP32 path: per-event |M|^2 within 2e-4 relative,
its error statistics printed.

Why the per-event |M|^2 bar has a tail: input momenta conserve momentum only
to ~1e-14 relative (rounding in the phase-space map), and a propagator whose
invariant is small against the energies (a top nearly collinear with a gluon,
E^2 / (P^2 - m^2) ~ 10^2..10^3) turns the routing-dependent part of that
violation into ~1e-11 of |M|^2: the value of |M|^2 on such inputs is only
defined to that level.  Likewise a helicity spinor of a momentum within a
degree of the -z axis forms |p| + p_z with a cancellation (the oracle writes it
as such; the GPU uses the cancellation-free form), worth ~1e-12 of |M|^2.  The
oracle's evaluations (Feynman diagrams with the internal momenta summed from
the tree's root, the same diagrams re-rooted at the antitop, the same in a
rotated frame, and the colour-ordered recursion) measure that ambiguity event
by event, and each tail event is held to it.  A wrong term would show at
O(1), far above 1e-10.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import integrate as oi, philox as oph, vegas as ov  # noqa: E402
from oracle.processes import Process as OracleProcess  # noqa: E402
from tests.inputs import event_sample, random_grid  # noqa: E402


@pytest.fixture(scope="module")
def mf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2211_14056_gb300 as mf
    return mf


def _rotated(p, axis=(1.0, 1.0, 1.0), angle=1.0):
    """All momenta rotated by `angle` about `axis` (|M|^2 is invariant)."""
    a = np.asarray(axis) / np.linalg.norm(axis)
    K = np.array([[0.0, -a[2], a[1]], [a[2], 0.0, -a[0]], [-a[1], a[0], 0.0]])
    R = np.eye(3) + np.sin(angle) * K + (1.0 - np.cos(angle)) * (K @ K)
    q = np.array(p, dtype=np.float64, copy=True)
    q[..., 1:] = q[..., 1:] @ R.T
    return q


def oracle_spread(setup, p):
    """Relative spread of |M|^2 over the oracle's independent FP64 evaluations
    of the same events: Feynman diagrams routed from the last leg (the
    reference), Feynman diagrams re-rooted at the antitop (every internal
    momentum summed from the other side of the tree), the reference in a
    rotated frame (helicity spinors of a momentum near the -z axis cancel in
    |p| + p_z, by ~1e-12 for a top within a degree of the beam; a rotation
    moves every momentum off the axis) and, for a heavy quark pair plus
    gluons, the colour-ordered recursion."""
    from oracle.berends_giele import QQbarGluons
    from oracle.feynman import Amplitude, DiagramSet
    from oracle.processes import outgoing_flavours
    proc = setup.proc
    p = np.asarray(p)
    vals = [proc.me2(p)]
    ds = DiagramSet(outgoing_flavours(proc.name), root=list(proc.particles).index("t~"))
    amp = Amplitude(ds, proc.mass, proc.amp.widths, {"gs": proc.gs, "e": proc.ee})
    ext, q = proc.external(p)
    vals.append(amp.summed_squared(ext, q) / proc.average)
    vals.append(proc.me2(_rotated(p)))
    if all(x in ("g", "t", "t~") for x in proc.particles):
        vals.append(QQbarGluons(proc).me2(p))
    v = np.stack(vals)
    return (v.max(axis=0) - v.min(axis=0)) / np.abs(v[0])


def assert_fp64_parity(got, ref, core=1e-12, tail=1e-10, frac=0.99, momenta=None, setup=None, extra=None):
    """Per-event FP64 parity.  With the events' momenta and oracle set-up
    given, every event outside ``core`` is arbitrated: the oracle evaluates it
    with each of its algorithms (``oracle_spread``), and the GPU value must
    lie within core |ref| + 4 * (their spread) of the reference (relative
    deviations of weights equal those of |M|^2 up to the weight factor's own
    rounding, ~1e-15; ``extra(indices)``, if given, adds the relative rounding
    spread of another factor of the weight, e.g. an interpolated luminosity).
    Without momenta the blanket fraction ``frac`` applies instead.  Returns
    the relative deviation each event was allowed (core, or its arbitrated
    bound), from which sums of the values can be bounded."""
    got, ref = np.asarray(got), np.asarray(ref)
    assert got.shape == ref.shape
    rel = np.abs(got - ref) / np.abs(ref)
    inside = rel <= core
    print(f"FP64 parity: {np.mean(inside):.4f} of {rel.size} within {core:g}, max {rel.max():.2e}")
    assert rel.max() <= tail
    allowed = np.full(rel.shape, core)
    if momenta is None:
        assert np.mean(inside) >= frac
        allowed[~inside] = tail
        return allowed
    out = np.flatnonzero(~inside)
    if out.size == 0:
        return allowed
    spread = oracle_spread(setup, np.asarray(momenta)[out])
    if extra is not None:
        spread = spread + extra(out)
    ratio = rel[out] / np.maximum(spread, core)
    print(f"  {out.size} tail events: GPU deviation / oracle spread: median {np.median(ratio):.2f}, "
          f"max {ratio.max():.2f}; spread median {np.median(spread):.1e}, max {spread.max():.1e}")
    assert np.all(rel[out] <= core + 4 * spread)
    allowed[out] = core + 4 * spread
    return allowed


def _proc(mf, name, precision, **over):
    from paper_2211_14056_gb300.workloads import PROCESS_IDS, WORKLOADS, process_kwargs
    w = dict(WORKLOADS[name], **over)
    return mf.Process(PROCESS_IDS[w["process"]], **process_kwargs(w, precision)), w


def _oracle_setup(w, amplitude="feynman"):
    from paper_2211_14056_gb300.workloads import oracle_cfg
    return oi.Setup(oracle_cfg(w), amplitude=amplitude)


def _soa_to_aos(t, n_ext, n):
    return t.view(n_ext, 4, n).permute(2, 0, 1).cpu().numpy()


def _aos_to_soa(p):
    return torch.tensor(np.ascontiguousarray(np.transpose(p, (1, 2, 0))), dtype=torch.float64, device="cuda")


NAMES = ["gg_ttx_1tev", "gg_ttxg_13tev", "gg_ttxgg_13tev"]


@pytest.mark.parametrize("name", NAMES)
def test_sample_matches_oracle(mf, name):
    p, w = _proc(mf, name, mf.MF_FP64)
    g = p.grid()
    edges = random_grid(p.ndim, seed=11)
    g.set(edges)
    n = 3001                                  # ragged: not a multiple of any tile
    mom = torch.empty(p.n_ext * 4 * n, dtype=torch.float64, device="cuda")
    wps = torch.empty(n, dtype=torch.float64, device="cuda")
    bins = torch.empty(p.ndim * n, dtype=torch.uint8, device="cuda")
    p.sample(g, seed=77, it=3, n=n, momenta=mom, weight_ps=wps, bins=bins)
    torch.cuda.synchronize()
    st = _oracle_setup(w)
    y = oph.uniforms(77, 3, np.arange(n, dtype=np.uint64), st.ndim)
    po, wk, bo, cut = st.kinematics(y, edges)
    np.testing.assert_array_equal(bins.view(p.ndim, n).cpu().numpy(), bo)
    pg = _soa_to_aos(mom, p.n_ext, n)
    scale = po[:, 0, 0][:, None, None] * 2
    assert np.max(np.abs(pg - po) / scale) < 1e-12
    wg = wps.cpu().numpy()
    np.testing.assert_array_equal(wg > 0, wk > 0)
    nz = wk > 0
    np.testing.assert_allclose(wg[nz], wk[nz], rtol=1e-12)


def _cut_events(st, seed, nev):
    """Momenta of events that pass the workload's cuts (the population the
    fused path evaluates), from the oracle's own phase-space map."""
    y = oph.uniforms(seed, 0, np.arange(4 * nev, dtype=np.uint64), st.ndim)
    po, _, _, cut = st.kinematics(y, ov.uniform_grid(st.ndim))
    return po[cut][:nev]


@pytest.mark.parametrize("name,nev", [("gg_ttx_1tev", 1000), ("gg_ttxg_13tev", 500), ("gg_ttxgg_13tev", 200)])
def test_matrix_element_fp64_matches_feynman_oracle(mf, name, nev):
    p, w = _proc(mf, name, mf.MF_FP64)
    st = _oracle_setup(w)
    po = _cut_events(st, 5, nev)
    ref = st.proc.me2_batched(po)
    out = torch.empty(len(po), dtype=torch.float64, device="cuda")
    p.matrix_element(len(po), _aos_to_soa(po), out)
    torch.cuda.synchronize()
    assert_fp64_parity(out.cpu().numpy(), ref, momenta=po, setup=st)


@pytest.mark.parametrize("tc", [False, True])
@pytest.mark.parametrize("name,nev", [("gg_ttx_1tev", 1000), ("gg_ttxg_13tev", 500), ("gg_ttxgg_13tev", 200)])
def test_matrix_element_fp32_error(mf, name, nev, tc):
    """FP32 amplitudes (colour sum on the FMA pipes, or on the tensor cores
    with the TF32 hi/lo split): the error statement of the single-precision
    path."""
    p, w = _proc(mf, name, mf.MF_FP32_TC if tc else mf.MF_FP32)
    st = _oracle_setup(w)
    po = _cut_events(st, 6, nev)
    ref = st.proc.me2_batched(po)
    out = torch.empty(len(po), dtype=torch.float64, device="cuda")
    p.matrix_element(len(po), _aos_to_soa(po), out)
    torch.cuda.synchronize()
    rel = np.abs(out.cpu().numpy() / ref - 1)
    print(f"{name} FP32{'/TC' if tc else ''} |M|^2 rel. error: max {rel.max():.2e} p99 {np.quantile(rel, 0.99):.2e} "
          f"median {np.median(rel):.2e}")
    assert np.median(rel) < 1e-5 and np.quantile(rel, 0.99) < 1e-4 and rel.max() < 5e-3


@pytest.mark.parametrize("name,nev", [("gg_ttx_1tev", 4096), ("gg_ttxg_13tev", 4096), ("gg_ttxgg_13tev", 2048)])
def test_tensor_core_colour_sum_matches_fma(mf, name, nev):
    """Same FP32 amplitudes, colour sum on the tensor cores vs on the FMA
    pipes: the difference is the colour sum's own rounding (TF32 hi/lo split
    of J, FP32 accumulation in another order), ~1e-7 relative."""
    p32, w = _proc(mf, name, mf.MF_FP32)
    ptc, _ = _proc(mf, name, mf.MF_FP32_TC)
    st = _oracle_setup(w)
    po = _cut_events(st, 7, nev)
    a = torch.empty(len(po), dtype=torch.float64, device="cuda")
    b = torch.empty(len(po), dtype=torch.float64, device="cuda")
    mom = _aos_to_soa(po)
    p32.matrix_element(len(po), mom, a)
    ptc.matrix_element(len(po), mom, b)
    torch.cuda.synchronize()
    rel = (b / a - 1).abs().cpu().numpy()
    print(f"{name} TC vs FMA colour sum: median {np.median(rel):.2e} max {rel.max():.2e}")
    assert np.median(rel) < 1e-6 and rel.max() < 1e-5


def test_tensor_core_iteration_sigma_error(mf):
    """One iteration of gg -> t tbar g g on a frozen random grid in FP64, FP32
    and FP32/TC on identical events: the arithmetic error of sigma."""
    name, n = "gg_ttxgg_13tev", 1 << 16
    res = {}
    for prec in (mf.MF_FP64, mf.MF_FP32, mf.MF_FP32_TC):
        p, _ = _proc(mf, name, prec)
        g = p.grid()
        g.set(random_grid(p.ndim, seed=13))
        res[prec] = p.vegas_iterate(g, seed=17, it=0, n=n, refine=False)
    e32 = abs(res[mf.MF_FP32]["I_k"] / res[mf.MF_FP64]["I_k"] - 1)
    etc = abs(res[mf.MF_FP32_TC]["I_k"] / res[mf.MF_FP64]["I_k"] - 1)
    print(f"sigma rel. error: FP32 {e32:.2e}, FP32/TC {etc:.2e}")
    assert etc < 1e-5 and e32 < 1e-5
    assert res[mf.MF_FP32_TC]["n_pass"] == res[mf.MF_FP32]["n_pass"]


def test_matrix_element_edge_cases(mf):
    """A top exactly along +z or -z (the limiting helicity spinors), n = 0,
    n = 1, and a count that fills no lane group evenly."""
    p, w = _proc(mf, "gg_ttxg_13tev", mf.MF_FP64)
    st = _oracle_setup(w)
    N = 7
    po = np.zeros((N, 5, 4))
    m = 173.0
    for e in range(N):
        sgn = 1 if e % 2 else -1
        pt_ = np.array([0.0, 0.0, sgn * (120.0 + 15 * e)])          # top on the z axis
        k = np.array([60.0 + 5 * e, -40.0, 25.0 * sgn])             # gluon off the axes
        ptb = -(pt_ + k)
        po[e, 2] = [math.sqrt(m * m + pt_ @ pt_), *pt_]
        po[e, 4] = [math.sqrt(k @ k), *k]
        po[e, 3] = [math.sqrt(m * m + ptb @ ptb), *ptb]
        tot = po[e, 2:, 0].sum()
        po[e, 0] = [tot / 2, 0, 0, tot / 2]
        po[e, 1] = [tot / 2, 0, 0, -tot / 2]
    ref = st.proc.me2(po)
    assert np.all(np.isfinite(ref))
    out = torch.empty(N, dtype=torch.float64, device="cuda")
    p.matrix_element(N, _aos_to_soa(po), out)
    torch.cuda.synchronize()
    assert_fp64_parity(out.cpu().numpy(), ref)
    p.matrix_element(0, torch.empty(0, dtype=torch.float64, device="cuda"),
                     torch.empty(0, dtype=torch.float64, device="cuda"))
    one = torch.empty(1, dtype=torch.float64, device="cuda")
    p.matrix_element(1, _aos_to_soa(po[:1]), one)
    torch.cuda.synchronize()
    assert_fp64_parity(one.cpu().numpy(), ref[:1])


@pytest.mark.parametrize("name,n,amp", [("gg_ttx_1tev", 20000, "feynman"), ("gg_ttxg_13tev", 4000, "bg"),
                                        ("gg_ttxgg_13tev", 700, "bg")])
def test_vegas_iterations_match_oracle(mf, name, n, amp):
    """Two iterations with refinement: weights, I_k, sigma_k and the refined
    grid against the oracle's (colour-ordered recursion for the big processes,
    itself pinned to the Feynman-diagram oracle).  Each iteration is compared
    on the GPU's own current edges: the refined edges agree with the oracle's
    refinement to 1e-12 absolute, and a narrow bin would turn that rounding
    into ~1e-11 of an event's Vegas Jacobian, which is not the arithmetic
    under test."""
    p, w = _proc(mf, name, mf.MF_FP64)
    g = p.grid()
    st = _oracle_setup(w, amplitude=amp)
    edges = ov.uniform_grid(st.ndim)
    wt = torch.empty(n, dtype=torch.float64, device="cuda")
    for it in range(2):
        np.testing.assert_allclose(g.get(), edges, rtol=0, atol=1e-12)
        edges = g.get()
        r = p.vegas_iterate(g, seed=9, it=it, n=n, refine=True, weights=wt)
        ro = oi.iteration(st, 9, it, n, edges)
        wg = wt.cpu().numpy()
        np.testing.assert_array_equal(wg > 0, ro["w"] > 0)
        nz = ro["w"] > 0
        pk = st.kinematics(oph.uniforms(9, it, np.arange(n, dtype=np.uint64), st.ndim), edges)[0]
        assert_fp64_parity(wg[nz], ro["w"][nz], momenta=pk[nz], setup=st)
        assert r["I_k"] == pytest.approx(ro["I"], rel=1e-12)
        assert r["sigma_k"] == pytest.approx(math.sqrt(ro["var"]), rel=1e-11)
        assert r["n_pass"] == int(nz.sum())
        edges = ov.refine(edges, ro["hist"])
    np.testing.assert_allclose(g.get(), edges, rtol=0, atol=1e-12)
    assert r["iterations"] == 2


def test_full_size_sampled_weights_and_determinism(mf):
    """The FP64 fused kernel at the full 2^22-event workload: sampled events'
    weights against the oracle, I_k = mean of all weights, and a bitwise
    identical rerun."""
    p, w = _proc(mf, "gg_ttxgg_13tev", mf.MF_FP64)
    n = w["events"]
    g = p.grid()
    wt = torch.empty(n, dtype=torch.float64, device="cuda")
    r = p.vegas_iterate(g, seed=w["seed"], it=0, n=n, refine=False, weights=wt)
    wall = wt.cpu().numpy()
    assert r["I_k"] == pytest.approx(wall.mean(), rel=1e-12)
    idx = event_sample(n, 48, seed=4)
    st = _oracle_setup(w, amplitude="feynman")
    y = oph.uniforms(w["seed"], 0, idx, st.ndim)
    wo, _ = st.weights(y, ov.uniform_grid(st.ndim))
    nz = wo > 0
    np.testing.assert_array_equal(wall[idx.astype(np.int64)] > 0, nz)
    pk = st.kinematics(y, ov.uniform_grid(st.ndim))[0]
    assert_fp64_parity(wall[idx.astype(np.int64)][nz], wo[nz], momenta=pk[nz], setup=st)
    g2 = p.grid()
    wt2 = torch.empty(n, dtype=torch.float64, device="cuda")
    p.vegas_iterate(g2, seed=w["seed"], it=0, n=n, refine=False, weights=wt2)
    assert torch.equal(wt, wt2)


def test_iterate_rejects_bad_sizes(mf):
    p, w = _proc(mf, "gg_ttx_1tev", mf.MF_FP64)
    g = p.grid()
    with pytest.raises(mf.MFError):
        p.vegas_iterate(g, 1, 0, 1)
    p2, _ = _proc(mf, "gg_ttxg_13tev", mf.MF_FP64)
    with pytest.raises(mf.MFError):
        p2.vegas_iterate(g, 1, 0, 100)       # grid of another process
