"""Colour-ordered Berends-Giele recursion for a heavy quark pair plus n gluons.

Test infrastructure (see ``oracle/__init__``); a second, independent way to the
same |M|^2 as ``feynman`` (used to pin it, and faster for large batches).

Colour decomposition (trace basis) with T^a = lambda^a/2:
    M = sum_{sigma in S_n} (T^{a_sigma1} ... T^{a_sigman})_{i_t j_tbar} J_sigma,
    sum_colours |M|^2 = sum_{sigma,tau} conj(J_sigma) C_{sigma tau} J_tau,
with C computed by brute force in ``colour``.  The colour-ordered rules follow
from the Feynman rules of ``feynman`` by writing f^{abc} T^c = -i [T^a, T^b]
and keeping the coefficient of one ordering (F.A. Berends, W.T. Giele,
Nucl. Phys. B306 (1988) 759, recursion in their Eq. (2.x) style):
    3-gluon, inputs L, R in colour order:  -i g Gamma(k_L, k_R, k_out)
    4-gluon, inputs L, M, R in order:       i g^2 [2 (L.R) M - (L.M) R - (M.R) L]
    quark-gluon:                             i g gamma^mu
with the propagators of ``feynman``.  All legs outgoing (q = -p incoming).

Recursion:
    G(i) = external polarisation of gluon i
    G(S) = (-i / P_S^2) [ sum_{S = L R} (-i g) O3(L, R) + sum_{S = L M R} (i g^2) O4(L, M, R) ]
    R()  = v(tbar);   R(S) = S_F(P) sum_{S = B S'} (i g Gslash(B)) R(S'),  P = -(q_tbar + sum_S q)
    J_sigma = ubar(t) sum_{sigma = B S'} (i g Gslash(B)) R(S')
"""
import itertools
import numpy as np

from .wavefunctions import mdot, slash
from .colour import trace_basis_colour_matrix


class QQbarGluons:
    """Partial amplitudes of a process whose legs are gluons plus one t tbar pair."""

    def __init__(self, process):
        self.proc = process
        parts = process.particles
        self.t = parts.index("t")
        self.tb = parts.index("t~")
        self.gluons = [i for i, x in enumerate(parts) if x == "g"]
        self.n = len(self.gluons)
        self.C, self.orders = trace_basis_colour_matrix(self.n)
        self.mt = process.mass["t"]
        self.wt = process.amp.widths["t"]
        self.gs = process.gs

    def partial_amplitudes(self, p):
        """J[sigma, *helicity axes, N] for every ordering sigma of the gluons.

        sigma runs over permutations of positions in ``self.gluons``
        (lexicographic, matching ``self.orders``).
        """
        ext, q = self.proc.external(np.asarray(p, dtype=np.float64))
        g = self.gs
        G, P = {}, {}

        def gcur(S):
            if S in G:
                return G[S]
            if len(S) == 1:
                leg = self.gluons[S[0]]
                G[S], P[S] = ext[leg], q[leg]
                return G[S]
            Ps = sum(q[self.gluons[i]] for i in S)
            acc = 0
            for m in range(1, len(S)):
                L, R = S[:m], S[m:]
                GL, GR = gcur(L), gcur(R)
                k1, k2 = -P[L], -P[R]
                k3 = P[L] + P[R]
                O3 = (mdot(GL, GR)[..., None] * (k1 - k2)
                      + GR * mdot(k2 - k3, GL)[..., None]
                      + GL * mdot(k3 - k1, GR)[..., None])
                acc = acc + (-1j * g) * O3
            for a in range(1, len(S) - 1):
                for b in range(a + 1, len(S)):
                    L, M, R = S[:a], S[a:b], S[b:]
                    GL, GM, GR = gcur(L), gcur(M), gcur(R)
                    O4 = (2 * mdot(GL, GR)[..., None] * GM - mdot(GL, GM)[..., None] * GR
                          - mdot(GM, GR)[..., None] * GL)
                    acc = acc + (1j * g * g) * O4
            G[S] = (-1j / mdot(Ps, Ps))[..., None] * acc
            P[S] = Ps
            return G[S]

        Rs = {}

        def rcur(S):
            if S in Rs:
                return Rs[S]
            if len(S) == 0:
                Rs[S] = ext[self.tb]
                return Rs[S]
            acc = 0
            for m in range(1, len(S) + 1):
                B, Sp = S[:m], S[m:]
                acc = acc + np.einsum("...ab,...b->...a", 1j * g * slash(gcur(B)), rcur(Sp))
            Pf = -(q[self.tb] + sum(q[self.gluons[i]] for i in S))
            den = mdot(Pf, Pf) - self.mt ** 2 + 1j * self.mt * self.wt
            prop = 1j * (slash(Pf) + self.mt * np.eye(4)) / den[..., None, None]
            Rs[S] = np.einsum("...ab,...b->...a", prop, acc)
            return Rs[S]

        ubar = ext[self.t]
        J = []
        for order in self.orders:
            acc = 0
            for m in range(1, self.n + 1):
                B, Sp = tuple(order[:m]), tuple(order[m:])
                acc = acc + np.einsum("...a,...ab,...b->...", ubar, 1j * g * slash(gcur(B)), rcur(Sp))
            J.append(acc)
        shape = np.broadcast_shapes(*[j.shape for j in J])
        return np.stack([np.broadcast_to(j, shape) for j in J])

    def me2(self, p):
        J = self.partial_amplitudes(p)
        Jf = J.reshape(J.shape[0], -1, J.shape[-1])
        s = np.real(np.einsum("shn,st,thn->n", np.conj(Jf), self.C, Jf))
        return s / self.proc.average
