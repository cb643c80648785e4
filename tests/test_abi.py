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
        (dict(process_id=9), B.MF_ERR_UNSUPPORTED),
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


def test_generated_header_is_current(tmp_path):
    from paper_2211_14056_gb300 import gen_tables
    assert open(gen_tables.OUT).read() == gen_tables.render()


def test_product_colour_matrix_matches_oracle_brute_force():
    import numpy as np
    from oracle.colour import trace_basis_colour_matrix
    from paper_2211_14056_gb300.gen_tables import colour_matrix_exact
    for n in (2, 3, 4):
        orders, M, D = colour_matrix_exact(n)
        C_or, orders_or = trace_basis_colour_matrix(n)
        assert orders == orders_or
        np.testing.assert_allclose(np.array(M) / D, C_or, atol=1e-12)
