"""CPU-side checks of the C ABI: the library loads, exports every symbol the
header declares, rejects bad descriptions before touching the device, and the
generated device header is current."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "madflow_gb300.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mf_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2211_14056_gb300 import binding
    if not os.path.exists(binding.library_path()):
        from paper_2211_14056_gb300 import build
        build.build()
    return binding.load_library()


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert "mf_vegas_iterate" in names and "mf_matrix_element" in names
    for n in names:
        assert hasattr(lib, n), n
    from paper_2211_14056_gb300 import binding
    assert set(names) == set(binding.EXPORTS)


def test_rejects_bad_descriptions_without_device(lib):
    from paper_2211_14056_gb300 import binding as B
    h = C.c_void_p()
    assert lib.mf_init_process(None, C.byref(h)) == B.MF_ERR_ARG
    assert b"null" in lib.mf_last_error()
    masses = (C.c_double * 4)(0, 0, 173, 173)
    num, den = B.colour_matrix(2)
    cnum = (C.c_int64 * 4)(*num)
    base = dict(process_id=1, n_ext=4, masses=masses, top_width=0.0, g_s=1.2, n_flow=2, colour_num=cnum,
                colour_den=den, sqrt_s=1000.0, lumi=0, lumi_N=1, lumi_a=-1.1, lumi_b=5, pt_cut_g=0,
                dr_cut_gg=0, precision=0)
    cases = [
        (dict(process_id=99), B.MF_ERR_UNSUPPORTED),
        (dict(n_ext=5), B.MF_ERR_ARG),
        (dict(g_s=-1.0), B.MF_ERR_ARG),
        (dict(sqrt_s=300.0), B.MF_ERR_ARG),
        (dict(n_flow=6), B.MF_ERR_COLOUR),
        (dict(colour_den=7), B.MF_ERR_COLOUR),
        (dict(precision=7), B.MF_ERR_ARG),
        (dict(lumi=3), B.MF_ERR_ARG),
    ]
    for change, status in cases:
        d = B.ProcessDesc(**{**base, **change})
        assert lib.mf_init_process(C.byref(d), C.byref(h)) == status, change
    bad = (C.c_int64 * 4)(16, -2, -3, 16)      # asymmetric
    d = B.ProcessDesc(**{**base, "colour_num": bad})
    assert lib.mf_init_process(C.byref(d), C.byref(h)) == B.MF_ERR_COLOUR
    wrong_m = (C.c_double * 4)(0, 0, 173, 172)
    d = B.ProcessDesc(**{**base, "masses": wrong_m})
    assert lib.mf_init_process(C.byref(d), C.byref(h)) == B.MF_ERR_ARG
    # the uniforms' argument checks come before any device work
    assert lib.mf_uniforms(1, 0, -1, 10, 3, None, None) == B.MF_ERR_ARG
    assert lib.mf_uniforms(1, 0, 0, 10, 11, None, None) == B.MF_ERR_ARG
    assert lib.mf_uniforms(1, 0, 0, 10, 3, None, None) == B.MF_ERR_ARG
    assert lib.mf_uniforms(1, 0, 0, 0, 3, None, None) == B.MF_OK


def test_generated_header_is_current(tmp_path):
    from paper_2211_14056_gb300 import gen_tables
    assert open(gen_tables.OUT).read() == gen_tables.render()
    assert open(gen_tables.OUT_ADJ).read() == gen_tables.render_adj()


def test_product_colour_matrix_matches_oracle_brute_force():
    import numpy as np
    from oracle.colour import trace_basis_colour_matrix
    from paper_2211_14056_gb300.gen_tables import colour_matrix_exact
    for n in (2, 3, 4):
        orders, M, D = colour_matrix_exact(n)
        C_or, orders_or = trace_basis_colour_matrix(n)
        assert orders == orders_or
        np.testing.assert_allclose(np.array(M) / D, C_or, atol=1e-12)


def test_generated_uux_header_is_current():
    from paper_2211_14056_gb300 import gen_uux
    assert open(gen_uux.OUT).read() == gen_uux.render()


def test_uux_description_checks_without_device(lib):
    from paper_2211_14056_gb300 import binding as B
    h = C.c_void_p()
    masses = (C.c_double * 6)(0, 0, 173, 173, 0, 0)
    num, den = B.colour_matrix_uux()
    cnum = (C.c_int64 * 144)(*num)
    base = dict(process_id=B.MF_PROC_UUX_TTXGG, n_ext=6, masses=masses, top_width=1.5, g_s=1.2, n_flow=12,
                colour_num=cnum, colour_den=den, sqrt_s=13000.0, lumi=1, lumi_N=1, lumi_a=-1.1, lumi_b=5,
                pt_cut_g=30, dr_cut_gg=0.4, precision=0)
    # the g g -> t t~ g g matrix, or the wrong size, is not this process's
    num4, den4 = B.colour_matrix(4)
    c4 = (C.c_int64 * 576)(*num4)
    for change, status in [(dict(n_flow=24, colour_num=c4, colour_den=den4), B.MF_ERR_COLOUR),
                           (dict(colour_den=den * 5), B.MF_ERR_COLOUR),
                           (dict(precision=2), B.MF_ERR_UNSUPPORTED),
                           (dict(n_ext=5), B.MF_ERR_ARG)]:
        d = B.ProcessDesc(**{**base, **change})
        assert lib.mf_init_process(C.byref(d), C.byref(h)) == status, change


def test_uux_colour_matrix_against_oracle_brute_force():
    """The 12-structure colour matrix equals the colour sum of the structures
    built from the oracle's own SU(3) generators (an independent evaluation)."""
    import itertools
    import numpy as np
    from oracle.colour import gell_mann
    from paper_2211_14056_gb300.gen_uux import colour_matrix_exact
    M, D = colour_matrix_exact()
    T = np.asarray(gell_mann()) / 2
    I3 = np.eye(3)

    def string(seq, a5, a6):
        R = I3.astype(complex)
        for g in seq:
            R = R @ T[a5 if g == 5 else a6]
        return R

    splits = []
    for nA in range(3):
        for A in itertools.permutations((5, 6), nA):
            B = tuple(g for g in (5, 6) if g not in A)
            for Bp in itertools.permutations(B):
                splits.append((A, Bp))
    tens = []
    for kind in ("tu", "tt"):
        for A, B in splits:
            t = np.zeros((3, 3, 3, 3, 8, 8), dtype=complex)
            for a5 in range(8):
                for a6 in range(8):
                    LA, LB = string(A, a5, a6), string(B, a5, a6)
                    if kind == "tu":     # (T^A)_{c3 c1} (T^B)_{c2 c4}
                        t[..., a5, a6] = np.einsum("da,ce->acde", LA, LB)
                    else:                # (T^A)_{c3 c4} (T^B)_{c2 c1}
                        t[..., a5, a6] = np.einsum("de,ca->acde", LA, LB)
            tens.append(t)
    ref = np.array([[np.vdot(a, b).real for b in tens] for a in tens])
    np.testing.assert_allclose(np.array(M) / D, ref, atol=1e-12)


def test_ee_description_checks_without_device(lib):
    from paper_2211_14056_gb300 import binding as B
    h = C.c_void_p()
    masses = (C.c_double * 4)(0, 0, 0, 0)
    one = (C.c_int64 * 1)(1)
    base = dict(process_id=B.MF_PROC_EE_MUMU, n_ext=4, masses=masses, top_width=0.0, g_s=1.2, n_flow=1,
                colour_num=one, colour_den=1, sqrt_s=100.0, lumi=0, lumi_N=1, lumi_a=-1.1, lumi_b=5,
                pt_cut_g=0, dr_cut_gg=0, precision=0, e_qed=0.3)
    two = (C.c_int64 * 1)(2)
    massive = (C.c_double * 4)(0, 0, 0.105, 0.105)
    for change, status in [(dict(masses=massive), B.MF_ERR_ARG),
                           (dict(lumi=1), B.MF_ERR_ARG),
                           (dict(e_qed=0.0), B.MF_ERR_ARG),
                           (dict(sqrt_s=0.0), B.MF_ERR_ARG),
                           (dict(n_ext=5), B.MF_ERR_ARG),
                           (dict(precision=2), B.MF_ERR_UNSUPPORTED),
                           (dict(n_flow=2), B.MF_ERR_COLOUR),
                           (dict(colour_num=two), B.MF_ERR_COLOUR)]:
        d = B.ProcessDesc(**{**base, **change})
        assert lib.mf_init_process(C.byref(d), C.byref(h)) == status, change


def test_grid_history_null_arguments(lib):
    from paper_2211_14056_gb300 import binding as B
    n = C.c_int(0)
    assert lib.mf_grid_history(None, C.byref(n), None, None) == B.MF_ERR_ARG
    assert lib.mf_grid_set_history(None, 0, None, None) == B.MF_ERR_ARG
