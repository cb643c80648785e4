"""SU(3) colour algebra by brute force over explicit indices.

Test infrastructure (see ``oracle/__init__``).

The paper (arXiv:2211.14056, Sec. 2) evaluates MadGraph matrix elements whose
colour sum is the quadratic form J^dagger C J over colour-flow amplitudes.  The
oracle never uses a colour identity: it builds the generators
T^a = lambda^a / 2 from the eight Gell-Mann matrices, the structure constants
f^{abc} = -2i Tr([T^a, T^b] T^c), and sums products of explicit numbers over
every external colour index.
"""
import itertools
import numpy as np

NC = 3


def gell_mann():
    lam = np.zeros((8, 3, 3), dtype=complex)
    lam[0][0, 1] = lam[0][1, 0] = 1
    lam[1][0, 1], lam[1][1, 0] = -1j, 1j
    lam[2][0, 0], lam[2][1, 1] = 1, -1
    lam[3][0, 2] = lam[3][2, 0] = 1
    lam[4][0, 2], lam[4][2, 0] = -1j, 1j
    lam[5][1, 2] = lam[5][2, 1] = 1
    lam[6][1, 2], lam[6][2, 1] = -1j, 1j
    lam[7] = np.diag([1, 1, -2]) / np.sqrt(3)
    return lam


T = gell_mann() / 2.0


def structure_constants():
    """f[a, b, c] = -2i Tr([T^a, T^b] T^c) (real, totally antisymmetric)."""
    comm = np.einsum("aij,bjk->abik", T, T) - np.einsum("bij,ajk->abik", T, T)
    f = -2j * np.einsum("abik,cki->abc", comm, T)
    return f.real


F = structure_constants()


def trace_basis_element(order):
    """c_sigma[a_1..a_n, i, j] = (T^{a_sigma1} ... T^{a_sigman})_{ij}.

    Axis k of the gluon indices belongs to gluon k (not to position k in the
    product), so elements for different orders can be compared entrywise.
    """
    n = len(order)
    out = np.zeros((8,) * n + (NC, NC), dtype=complex)
    for a in itertools.product(range(8), repeat=n):
        prod = np.eye(NC, dtype=complex)
        for g in order:
            prod = prod @ T[a[g]]
        out[a] = prod
    return out


def trace_basis_colour_matrix(n):
    """C[s, t] = sum over all colours of conj(c_s) c_t, s, t in S_n (lexicographic)."""
    orders = list(itertools.permutations(range(n)))
    c = np.stack([trace_basis_element(o).ravel() for o in orders])
    return (np.conj(c) @ c.T).real, orders
