"""Pins for oracle.colour: SU(3) algebra and the trace-basis colour matrices.

C_{ss} = C_F^n N = (4/3)^n 3; for n = 2, C = (1/3)[[16, -2], [-2, 16]], which
follows by hand from T^a T^b T^a = -T^b / (2N)."""
import itertools

import numpy as np
import pytest

from oracle import colour


def test_generators():
    T, F = colour.T, colour.F
    np.testing.assert_allclose(np.einsum("aij,bji->ab", T, T), 0.5 * np.eye(8), atol=1e-15)
    comm = np.einsum("aij,bjk->abik", T, T) - np.einsum("bij,ajk->abik", T, T)
    np.testing.assert_allclose(comm, 1j * np.einsum("abc,cik->abik", F, T), atol=1e-15)
    np.testing.assert_allclose(np.einsum("aij,ajk->ik", T, T), 4 / 3 * np.eye(3), atol=1e-15)
    assert F[0, 1, 2] == pytest.approx(1.0)
    np.testing.assert_allclose(F, -np.transpose(F, (1, 0, 2)), atol=1e-15)
    np.testing.assert_allclose(np.einsum("acd,bcd->ab", F, F), 3 * np.eye(8), atol=1e-14)


@pytest.mark.parametrize("n", [2, 3, 4])
def test_trace_basis_matrix(n):
    C, orders = colour.trace_basis_colour_matrix(n)
    assert C.shape == (len(orders),) * 2
    np.testing.assert_allclose(C, C.T, atol=1e-12)
    np.testing.assert_allclose(np.diag(C), 3 * (4 / 3) ** n, rtol=1e-13)
    # exact rationals whose denominators divide 2 * 3^(n-1); scaled to
    # integers they stay within 2^11, so they are exact in TF32
    D = 2 * 3 ** (n - 1)
    np.testing.assert_allclose(C * D, np.round(C * D), atol=1e-9)
    assert np.max(np.abs(np.round(C * D))) <= 2 ** 11
    if n == 2:
        np.testing.assert_allclose(C, np.array([[16, -2], [-2, 16]]) / 3, atol=1e-13)
