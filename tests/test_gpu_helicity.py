"""GPU: helicity sampling against the oracle (oracle.helicity).

* mf_matrix_element_hel in FP64: |M_h|^2 of given configurations within
  1e-12 relative of oracle.helicity.me2_helicity, except events on which the
  oracle's own FP64 evaluations of that configuration disagree (colour-ordered
  recursion, the same in a rotated frame, Feynman diagrams): there the GPU
  value lies within four times their spread, every event within 1e-10 (the
  summed path's bar and reasoning, test_gpu_parity);
* completeness on the GPU: the 2^(NG+1) configurations sum to
  mf_matrix_element (FP64 1e-12, FP32 1e-5 median);
* FP32: the error statement of the summed path (median 1e-5, p99 1e-4);
* an iteration with sampling on: the per-event weights are the oracle's
  sampled weights for the draws of the third Philox stream (FP64 parity as
  above, the arbitration adding the weight's conditioning at FP64 rounding:
  the GPU's sampler reaches the oracle's momenta to a few ulps, which some
  events' |M_h|^2 amplifies ~10^4-fold), and I_k, sigma_k follow from them;
* unbiasedness: sampled and summed iterations agree within their errors;
* edge cases: n = 0, one event, bits above NG + 1 ignored; the combinations
  that are not covered raise;
* the two-quark-line channels of p p -> t t~ g g (one event per thread):
  per configuration in FP64 against the oracle's Feynman diagrams, the 32
  configurations summing to the summed kernel, a sampled iteration of
  u u~ -> t t~ g g against the oracle, and sampled against summed estimates.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import helicity as oh, integrate as oi, philox as oph, vegas as ov  # noqa: E402
from tests.inputs import random_grid  # noqa: E402
from tests.test_gpu_parity import _aos_to_soa, _cut_events, _oracle_setup, _proc, _rotated  # noqa: E402

NAMES = [("gg_ttx_1tev", 1200), ("gg_ttxg_13tev", 800), ("gg_ttxgg_13tev", 400)]


@pytest.fixture(scope="module")
def mf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2211_14056_gb300 as mf
    return mf


def hel_spread(proc, p, h):
    """Relative spread of me2_helicity over the oracle's FP64 evaluations of
    the same configurations: the colour-ordered recursion, the same in a
    rotated frame, the Feynman diagrams routed from the last leg and the same
    diagrams re-rooted at the antitop (every internal momentum summed from the
    other side of the tree: the routing-dependent rounding that test_gpu_parity
    describes)."""
    from oracle.feynman import Amplitude, DiagramSet
    from oracle.processes import outgoing_flavours
    ds = DiagramSet(outgoing_flavours(proc.name), root=list(proc.particles).index("t~"))
    rerooted = Amplitude(ds, proc.mass, proc.amp.widths, {"gs": proc.gs, "e": proc.ee})
    alg = "bg" if all(x in ("g", "t", "t~") for x in proc.particles) else "feynman"
    v = np.stack([oh.me2_helicity(proc, p, h, alg), oh.me2_helicity(proc, _rotated(p), h, alg),
                  oh.me2_helicity(proc, p, h, "feynman"), oh.me2_helicity(proc, p, h, "feynman", amp=rerooted)])
    scale = np.maximum(np.abs(v[0]), 1e-300)
    return (v.max(axis=0) - v.min(axis=0)) / scale


def kin_spread(st, y, edges, p, h):
    """Conditioning of an iteration's weight at FP64 rounding, from the oracle
    alone, per event: the relative change of the oracle's weight factor when
    one uniform moves by one ulp (largest over the dimensions and both
    directions), the synthetic luminosity's own rounding (its FP64 value
    against extended precision), plus that of its |M_h|^2 when the momenta's components are
    multiplied by 1 + 2^-51 u, u uniform in [-1, 1] (two seeded draws): the
    GPU's sampler reaches the same momenta to a few ulps only (on the events
    this arbitrates, ~4e-16 of the beam energy), and where |M_h|^2 amplifies
    that ~10^4-fold its value is defined to ~1e-12 only."""
    _, wk0, _, _ = st.kinematics(y, edges)
    dwk = np.zeros(y.shape[1])
    for j in range(y.shape[0]):
        for sgn in (-1.0, 1.0):
            yp = y.copy()
            yp[j] = yp[j] + sgn * np.spacing(yp[j])
            _, wkp, _, _ = st.kinematics(yp, edges)
            dwk = np.maximum(dwk, np.abs(wkp / wk0 - 1))
    if st.lumi is True:
        # the synthetic luminosity's own FP64 rounding (the oracle forms 1 - x
        # as written, which for x near 1 costs ~1e-16 / (1 - x) relative, to
        # the power b): its value against the same map in extended precision
        from oracle import phase_space as ps
        x, _, _ = ov.vegas_map(y, edges)
        c = st.cfg
        S = c["sqrt_s"] ** 2
        tau0 = sum(st.masses) ** 2 / S
        args = (c.get("lumi_N", 1.0), c.get("lumi_a", -1.1), c.get("lumi_b", 5.0))
        L64 = ps.luminosity_map(x[0], x[1], tau0, S, *args)[3]
        Lx = ps.luminosity_map(np.asarray(x[0], dtype=np.longdouble), np.asarray(x[1], dtype=np.longdouble),
                               np.longdouble(tau0), np.longdouble(S), *args)[3]
        dwk = dwk + np.asarray(np.abs(L64 / Lx - 1), dtype=np.float64)
    rng = np.random.default_rng(35)
    alg = "bg" if st.bg is not None else "feynman"
    m0 = oh.me2_helicity(st.proc, p, h, alg)
    dme = np.zeros(p.shape[0])
    for _ in range(2):
        pp = p * (1 + 2.0 ** -51 * rng.uniform(-1, 1, p.shape))
        dme = np.maximum(dme, np.abs(oh.me2_helicity(st.proc, pp, h, alg) / m0 - 1))
    return dwk + dme


def assert_hel_parity(got, ref, proc, p, h, core=1e-12, tail=1e-10, kin=None):
    """Per-event FP64 parity with arbitration; returns the allowed relative
    deviation of every event.  kin = (setup, y, edges) of the events (an
    iteration's weights): the arbitration adds the weight's conditioning at
    FP64 rounding (kin_spread)."""
    rel = np.abs(got - ref) / np.abs(ref)
    print(f"FP64 parity: {np.mean(rel <= core):.4f} of {rel.size} within {core:g}, max {rel.max():.2e}")
    assert rel.max() <= tail
    allowed = np.full(rel.shape, core)
    out = np.flatnonzero(rel > core)
    if out.size:
        spread = hel_spread(proc, p[out], h[out])
        if kin is not None:
            st, y, edges = kin
            spread = spread + kin_spread(st, y[:, out], edges, p[out], h[out])
        print(f"  {out.size} tail events: deviation / spread max {np.max(rel[out] / np.maximum(spread, core)):.2f}, "
              f"deviation / bound max {np.max(rel[out] / (core + 4 * spread)):.2f}")
        assert np.all(rel[out] <= core + 4 * spread)
        allowed[out] = core + 4 * spread
    return allowed


def _hel_me(p, po, hel):
    out = torch.full((len(po),), float("nan"), dtype=torch.float64, device="cuda")
    p.matrix_element_hel(len(po), _aos_to_soa(po), torch.tensor(hel, dtype=torch.int32, device="cuda"), out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("name,nev", NAMES)
def test_configuration_fp64_matches_oracle(mf, name, nev):
    p, w = _proc(mf, name, mf.MF_FP64)
    st = _oracle_setup(w, amplitude="bg")
    po = _cut_events(st, 8, nev)
    nc = oh.n_configs(st.proc)
    hel = (np.arange(len(po)) * 7 + 3) % nc                # every configuration, several times
    ref = oh.me2_helicity(st.proc, po, hel, "bg")
    got = _hel_me(p, po, hel)
    assert_hel_parity(got, ref, st.proc, po, hel)


@pytest.mark.parametrize("name,nev", NAMES)
def test_configurations_sum_to_the_summed_kernel(mf, name, nev):
    for prec, bar in ((mf.MF_FP64, 1e-12), (mf.MF_FP32, 1e-5)):
        p, w = _proc(mf, name, prec)
        st = _oracle_setup(w)
        po = _cut_events(st, 9, nev // 4)
        nc = oh.n_configs(st.proc)
        m = len(po)
        rep = np.repeat(po, nc, axis=0)
        v = _hel_me(p, rep, np.tile(np.arange(nc), m)).reshape(m, nc).sum(axis=1)
        tot = torch.empty(m, dtype=torch.float64, device="cuda")
        p.matrix_element(m, _aos_to_soa(po), tot)
        torch.cuda.synchronize()
        rel = np.abs(v / tot.cpu().numpy() - 1)
        print(f"{name} prec {prec}: sum of configurations vs summed kernel: median {np.median(rel):.2e} "
              f"max {rel.max():.2e}")
        assert np.median(rel) < bar and rel.max() < 100 * bar


@pytest.mark.parametrize("name,nev", NAMES)
def test_configuration_fp32_error(mf, name, nev):
    p, w = _proc(mf, name, mf.MF_FP32)
    st = _oracle_setup(w, amplitude="bg")
    po = _cut_events(st, 10, nev)
    hel = np.arange(len(po)) % oh.n_configs(st.proc)
    ref = oh.me2_helicity(st.proc, po, hel, "bg")
    rel = np.abs(_hel_me(p, po, hel) / ref - 1)
    print(f"{name} FP32 |M_h|^2 rel. error: max {rel.max():.2e} p99 {np.quantile(rel, 0.99):.2e} "
          f"median {np.median(rel):.2e}")
    assert np.median(rel) < 1e-5 and np.quantile(rel, 0.99) < 1e-4 and rel.max() < 5e-3


@pytest.mark.parametrize("name,n", [("gg_ttxg_13tev", 3001), ("gg_ttxgg_13tev", 1501)])
def test_sampled_iteration_matches_oracle(mf, name, n):
    p, w = _proc(mf, name, mf.MF_FP64)
    p.set_helicity_sampling(True)
    g = p.grid()
    edges = random_grid(p.ndim, seed=31)
    g.set(edges)
    seed, it = 41, 2
    wt = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
    r = p.vegas_iterate(g, seed, it, n, refine=False, weights=wt)
    st = _oracle_setup(w, amplitude="bg")
    ev = np.arange(n, dtype=np.uint64)
    y = oph.uniforms(seed, it, ev, st.ndim)
    wo, bins, hel = oh.sampled_weights(st, y, edges, seed, it, ev)
    wg = wt.cpu().numpy()
    np.testing.assert_array_equal(wg == 0, wo == 0)
    nz = np.flatnonzero(wo != 0)
    po = st.kinematics(y[:, nz], edges)[0]
    allowed = np.zeros(n)
    allowed[nz] = assert_hel_parity(wg[nz], wo[nz], st.proc, po, hel[nz], kin=(st, y[:, nz], edges))
    sw, sw2, _ = ov.accumulate(wo, bins, edges.shape[1] - 1)
    I, var = ov.estimate(sw, sw2, n)
    dI = np.sum(allowed * np.abs(wo)) / n + 1e-12 * abs(I)
    assert abs(r["I_k"] - I) <= dI
    # var = (sum w^2 / n - I^2) / (n - 1): its deviation from the weights' allowances
    dvar = (2 * np.sum(allowed * wo ** 2) / n + 2 * abs(I) * dI) / (n - 1) + 1e-11 * var
    assert abs(r["sigma_k"] ** 2 - var) <= dvar
    assert r["n_pass"] == nz.size


def test_sampling_is_unbiased(mf):
    """FP32, g g -> t t~ g g, on a grid adapted by three summed iterations and
    then frozen: four sampled and four summed iterations of 2^20 events each
    agree within their combined errors (the variance ratio is printed; its
    estimates are too heavy-tailed at this size for a bound)."""
    name, n = "gg_ttxgg_13tev", 1 << 20
    ps, _ = _proc(mf, name, mf.MF_FP32)
    pu, _ = _proc(mf, name, mf.MF_FP32)
    ps.set_helicity_sampling(True)
    gu = pu.grid()
    for it in range(3):
        pu.vegas_iterate(gu, 50, it, n, refine=True)
    edges = gu.get()
    gs = ps.grid()
    est = {}
    for label, p, g in (("sampled", ps, gs), ("summed", pu, gu)):
        Is, Vs = [], []
        for it in range(4):
            g.set(edges)
            r = p.vegas_iterate(g, 51, 10 + it, n, refine=False)
            Is.append(r["I_k"])
            Vs.append(r["sigma_k"] ** 2)
        Is, Vs = np.array(Is), np.array(Vs)
        est[label] = (np.sum(Is / Vs) / np.sum(1 / Vs), 1 / np.sqrt(np.sum(1 / Vs)), Vs.mean())
    (I_s, s_s, v_s), (I_u, s_u, v_u) = est["sampled"], est["summed"]
    print(f"sampled {I_s:.6g} +- {s_s:.2g}, summed {I_u:.6g} +- {s_u:.2g}; variance ratio {v_s / v_u:.2f}")
    assert abs(I_s - I_u) < 5 * np.hypot(s_s, s_u)


def test_edge_cases_and_errors(mf):
    p, w = _proc(mf, "gg_ttxg_13tev", mf.MF_FP64)
    st = _oracle_setup(w, amplitude="bg")
    po = _cut_events(st, 11, 1)
    # one event; the bits above NG + 1 are not read
    a = _hel_me(p, po, np.array([5]))
    b = _hel_me(p, po, np.array([5 | (1 << 9) | (1 << 30)]))
    assert a[0] == b[0]
    np.testing.assert_allclose(a, oh.me2_helicity(st.proc, po, np.array([5]), "bg"), rtol=1e-12)
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    p.matrix_element_hel(0, _aos_to_soa(po), torch.zeros(1, dtype=torch.int32, device="cuda"), out)
    # not covered
    ptc, _ = _proc(mf, "gg_ttxg_13tev", mf.MF_FP32_TC)
    with pytest.raises(mf.MFError):
        ptc.set_helicity_sampling(True)
    pee, _ = _proc(mf, "epem_mupmum_100gev", mf.MF_FP64)
    with pytest.raises(mf.MFError):
        pee.set_helicity_sampling(True)
    p.set_helicity_sampling(True)
    g = p.grid()
    with pytest.raises(mf.MFError):
        mf.Mixed([p], [g], [1000])
    p.set_helicity_sampling(False)
    r = p.vegas_iterate(g, 1, 0, 4096, refine=False)
    assert r["I_k"] > 0


# ---------------------------------------------------------------------------
# the adapted draw (mf_set_helicity_sampling(proc, 2), mf_grid_set_helicity)

@pytest.mark.parametrize("name,n", [("gg_ttxg_13tev", 3001), ("gg_ttxgg_13tev", 1501)])
def test_adapted_draw_and_refinement_match_oracle(mf, name, n):
    """A non-uniform table set through the ABI: the GPU's thresholds are the
    oracle's, the draws and per-event weights f_h / p_h are the oracle's (FP64
    parity as above), the per-configuration sums of squared weights in the
    totals are the oracle's within what their events were allowed, and the
    table refined on the device (refine bit 2, edges untouched) is the
    oracle's refinement of those sums (the sums differ in summation order,
    so a threshold may move by one step of 2^-32)."""
    from paper_2211_14056_gb300.sharding import totals_tensor
    p, w = _proc(mf, name, mf.MF_FP64)
    p.set_helicity_sampling("adaptive")
    g = p.grid()
    edges = random_grid(p.ndim, seed=33)
    g.set(edges)
    H = g.n_configs
    rng = np.random.default_rng(34)
    prob = rng.uniform(0.3, 3.0, H)
    prob /= prob.sum()
    g.set_helicity(prob)
    T = oh.thresholds(prob)
    np.testing.assert_array_equal(g.helicity(), oh.probabilities(T))
    seed, it = 43, 5
    wt = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
    p.vegas_accumulate(g, seed, it, 0, n, weights=wt)
    torch.cuda.synchronize()
    st = _oracle_setup(w, amplitude="bg")
    ev = np.arange(n, dtype=np.uint64)
    y = oph.uniforms(seed, it, ev, st.ndim)
    wo, bins, hel, So = oh.adapted_weights(st, y, edges, seed, it, ev, T)
    wg = wt.cpu().numpy()
    np.testing.assert_array_equal(wg == 0, wo == 0)
    nz = np.flatnonzero(wo != 0)
    po = st.kinematics(y[:, nz], edges)[0]
    allowed = np.zeros(n)
    allowed[nz] = assert_hel_parity(wg[nz], wo[nz], st.proc, po, hel[nz], kin=(st, y[:, nz], edges))
    tot = totals_tensor(g).cpu().numpy()
    assert tot.size == 2 + p.ndim * g.nbins + 2 + H
    Sg = tot[-H:]
    dS = np.zeros(H)
    np.add.at(dS, hel, 2 * allowed * wo ** 2)
    assert np.all(np.abs(Sg - So) <= dS + 1e-12 * So)
    r = p.vegas_finish(g, n, refine="helicities")
    np.testing.assert_array_equal(g.get(), edges)
    p_ref = oh.probabilities(oh.refine(T, So))
    p_gpu = g.helicity()
    assert np.max(np.abs(p_gpu - p_ref)) <= 2.0 ** -31
    assert abs(p_gpu.sum() - 1) < 1e-15 and p_gpu.min() >= oh.REFINE_FLOOR / H - 2.0 ** -32
    print(f"{name}: refined table max |GPU - oracle| = {np.max(np.abs(p_gpu - p_ref)):.2e}, I_k {r['I_k']:.5g}")


def test_adaptation_lowers_the_variance_and_stays_unbiased(mf):
    """FP32 g g -> t t~ g g on a grid adapted by three summed iterations and
    frozen: five adapting iterations of 2^20 events refine the helicity table
    only; then four iterations each with the adapted and the uniform table.
    The adapted estimate agrees with the summed one within the combined
    errors, and its variance per event is below the uniform draw's."""
    name, n = "gg_ttxgg_13tev", 1 << 20
    pu, _ = _proc(mf, name, mf.MF_FP32)
    gu = pu.grid()
    for it in range(3):
        pu.vegas_iterate(gu, 60, it, n, refine=True)
    edges = gu.get()
    pa, _ = _proc(mf, name, mf.MF_FP32)
    pa.set_helicity_sampling("adaptive")
    ga = pa.grid()
    ga.set(edges)
    for it in range(5):
        pa.vegas_iterate(ga, 61, it, n, refine="helicities")
    np.testing.assert_array_equal(ga.get(), edges)
    table = ga.helicity()
    assert table.max() > 2.0 / 32                        # adapted away from uniform
    est = {}
    pn, _ = _proc(mf, name, mf.MF_FP32)
    pn.set_helicity_sampling(True)
    gn = pn.grid()
    for label, p, g in (("adapted", pa, ga), ("uniform", pn, gn), ("summed", pu, gu)):
        Is, Vs = [], []
        for it in range(4):
            g.set(edges)
            r = p.vegas_iterate(g, 62, 10 + it, n, refine=False)
            Is.append(r["I_k"])
            Vs.append(r["sigma_k"] ** 2)
        Is, Vs = np.array(Is), np.array(Vs)
        est[label] = (np.sum(Is / Vs) / np.sum(1 / Vs), 1 / np.sqrt(np.sum(1 / Vs)), Vs.mean())
    np.testing.assert_array_equal(ga.helicity(), table)   # refine=False keeps the table
    (I_a, s_a, v_a), (I_n, s_n, v_n), (I_u, s_u, v_u) = est["adapted"], est["uniform"], est["summed"]
    print(f"adapted {I_a:.6g} +- {s_a:.2g}, uniform {I_n:.6g} +- {s_n:.2g}, summed {I_u:.6g} +- {s_u:.2g}; "
          f"variance adapted / uniform {v_a / v_n:.2f}, adapted / summed {v_a / v_u:.2f}")
    assert abs(I_a - I_u) < 5 * np.hypot(s_a, s_u)
    assert v_a < v_n


def test_helicity_table_arguments_and_checkpoint(mf):
    p, _ = _proc(mf, "gg_ttx_1tev", mf.MF_FP64)
    g = p.grid()
    assert g.n_configs == 8
    np.testing.assert_array_equal(g.helicity(), np.full(8, 1 / 8))
    with pytest.raises(mf.MFError):
        g.set_helicity(np.full(4, 0.25))                 # wrong count
    with pytest.raises(mf.MFError):
        g.set_helicity(np.array([0.0] + [1 / 7] * 7))   # a configuration never drawn
    with pytest.raises(mf.MFError):
        g.set_helicity(np.full(8, 0.2))                  # does not sum to 1
    prob = np.arange(1, 9, dtype=float) / 36
    g.set_helicity(prob)
    state = g.checkpoint()
    g2 = p.grid()
    g2.restore(state)
    np.testing.assert_array_equal(g2.helicity(), g.helicity())
    pe, _ = _proc(mf, "epem_mupmum_100gev", mf.MF_FP64)
    ge = pe.grid()
    assert ge.n_configs == 0 and ge.helicity() is None
    pu, _ = _proc(mf, "uux_ttxgg_13tev", mf.MF_FP64)
    assert pu.grid().n_configs == 32
    with pytest.raises(mf.MFError):
        p.vegas_finish(g, 100, refine=4)



# ---------------------------------------------------------------------------
# the two-quark-line channels

TWO_LINE = ["uux_ttxgg_13tev", "pp_ttxgg_qxq", "pp_ttxgg_qg", "pp_ttxgg_gq", "pp_ttxgg_qxg", "pp_ttxgg_gqx"]


@pytest.mark.parametrize("name", TWO_LINE)
def test_two_line_configuration_fp64_matches_oracle(mf, name):
    """|M_h|^2 of given configurations (the synthetic luminosity's events; the
    amplitude does not depend on it) against the oracle's Feynman diagrams,
    and every configuration summed against the summed kernel (FP64, FP32)."""
    p, w = _proc(mf, name, mf.MF_FP64, lumi=True)
    st = _oracle_setup(w)
    po = _cut_events(st, 12, 40)
    hel = (np.arange(len(po)) * 11 + 7) % 32
    ref = oh.me2_helicity(st.proc, po, hel)
    got = _hel_me(p, po, hel)
    nz = ref > 1e-20 * ref.max()
    assert np.all(np.abs(got[~nz]) <= 1e-20 * ref.max())     # the light line's chirality zeros
    assert_hel_parity(got[nz], ref[nz], st.proc, po[nz], hel[nz])
    m = 6
    rep = np.repeat(po[:m], 32, axis=0)
    for prec, bar in ((mf.MF_FP64, 1e-12), (mf.MF_FP32, 1e-5)):
        q, _ = _proc(mf, name, prec, lumi=True)
        v = _hel_me(q, rep, np.tile(np.arange(32), m)).reshape(m, 32).sum(axis=1)
        tot = torch.empty(m, dtype=torch.float64, device="cuda")
        q.matrix_element(m, _aos_to_soa(po[:m]), tot)
        torch.cuda.synchronize()
        rel = np.abs(v / tot.cpu().numpy() - 1)
        assert np.median(rel) < bar and rel.max() < 100 * bar


def test_two_line_sampled_iteration_matches_oracle(mf):
    name, n = "uux_ttxgg_13tev", 1201
    p, w = _proc(mf, name, mf.MF_FP64)
    p.set_helicity_sampling(True)
    g = p.grid()
    edges = random_grid(p.ndim, seed=36)
    g.set(edges)
    seed, it = 44, 3
    wt = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
    r = p.vegas_iterate(g, seed, it, n, refine=False, weights=wt)
    st = _oracle_setup(w)
    ev = np.arange(n, dtype=np.uint64)
    y = oph.uniforms(seed, it, ev, st.ndim)
    wo, bins, hel = oh.sampled_weights(st, y, edges, seed, it, ev)
    wg = wt.cpu().numpy()
    tiny = 1e-20 * np.abs(wo).max()
    nz = np.flatnonzero(np.abs(wo) > tiny)
    zero = np.flatnonzero(np.abs(wo) <= tiny)
    assert np.all(np.abs(wg[zero]) <= tiny)                 # cuts and the chirality zeros
    po = st.kinematics(y[:, nz], edges)[0]
    allowed = np.zeros(n)
    allowed[nz] = assert_hel_parity(wg[nz], wo[nz], st.proc, po, hel[nz], kin=(st, y[:, nz], edges))
    sw, sw2, _ = ov.accumulate(wo, bins, edges.shape[1] - 1)
    I, var = ov.estimate(sw, sw2, n)
    dI = np.sum(allowed * np.abs(wo)) / n + 1e-12 * abs(I)
    assert abs(r["I_k"] - I) <= dI


@pytest.mark.parametrize("name", ["uux_ttxgg_13tev", "pp_ttxgg_qg"])
def test_two_line_sampling_is_unbiased(mf, name):
    """FP32, 2^18 events per iteration on a grid adapted by three summed
    iterations, then frozen: four uniform-draw and four summed iterations
    agree within their combined errors; the adapted draw likewise."""
    from paper_2211_14056_gb300.workloads import PROCESS_IDS, WORKLOADS, process_kwargs
    w = WORKLOADS[name]
    pdf = mf.PDFSet.from_dict(__import__("paper_2211_14056_gb300.pdfgrid", fromlist=["x"]).synthetic_set()) \
        if w["lumi"] == "pdf" else None
    mk = lambda: mf.Process(PROCESS_IDS[w["process"]], **process_kwargs(w, mf.MF_FP32, pdf=pdf))
    n = 1 << 18
    pu = mk()
    gu = pu.grid()
    for it in range(3):
        pu.vegas_iterate(gu, 70, it, n, refine=True)
    edges = gu.get()
    ps, pa = mk(), mk()
    ps.set_helicity_sampling(True)
    pa.set_helicity_sampling("adaptive")
    gs, ga = ps.grid(), pa.grid()
    ga.set(edges)
    for it in range(3):
        pa.vegas_iterate(ga, 71, it, n, refine="helicities")
    est = {}
    for label, p, g in (("sampled", ps, gs), ("adapted", pa, ga), ("summed", pu, gu)):
        Is, Vs = [], []
        for it in range(4):
            g.set(edges)
            r = p.vegas_iterate(g, 72, 10 + it, n, refine=False)
            Is.append(r["I_k"])
            Vs.append(r["sigma_k"] ** 2)
        Is, Vs = np.array(Is), np.array(Vs)
        est[label] = (np.sum(Is / Vs) / np.sum(1 / Vs), 1 / np.sqrt(np.sum(1 / Vs)), Vs.mean())
    (I_s, s_s, v_s), (I_a, s_a, v_a), (I_u, s_u, v_u) = est["sampled"], est["adapted"], est["summed"]
    print(f"{name}: sampled {I_s:.6g} +- {s_s:.2g}, adapted {I_a:.6g} +- {s_a:.2g}, summed {I_u:.6g} +- {s_u:.2g}; "
          f"variance / summed: sampled {v_s / v_u:.2f}, adapted {v_a / v_u:.2f}")
    assert abs(I_s - I_u) < 5 * np.hypot(s_s, s_u)
    assert abs(I_a - I_u) < 5 * np.hypot(s_a, s_u)


def test_adapted_sums_over_several_chunks(mf):
    """2^21 + 3 FP32 events (three record chunks): the per-configuration sums
    of squared weights in the totals equal the sums of the returned weights
    squared over the events that drew each configuration (draws from the
    oracle's Philox and thresholds), so the chunks' partial sums add up."""
    from paper_2211_14056_gb300.sharding import totals_tensor
    p, _ = _proc(mf, "gg_ttxgg_13tev", mf.MF_FP32)
    p.set_helicity_sampling("adaptive")
    g = p.grid()
    rng = np.random.default_rng(39)
    prob = rng.uniform(0.5, 2.0, 32)
    prob /= prob.sum()
    g.set_helicity(prob)
    n = (1 << 21) + 3
    wt = torch.empty(n, dtype=torch.float64, device="cuda")
    p.vegas_accumulate(g, 45, 1, 7, n, weights=wt)
    S = totals_tensor(g).cpu().numpy()[-32:]
    torch.cuda.synchronize()
    w = wt.cpu().numpy()
    h = oh.draw(oph.helicity_words(45, 1, np.arange(7, 7 + n, dtype=np.uint64)), oh.thresholds(prob))
    want = np.bincount(h, weights=w * w, minlength=32)
    np.testing.assert_allclose(S, want, rtol=1e-10)
