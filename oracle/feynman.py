"""Tree-level amplitudes as a plain sum of Feynman diagrams with explicit colour.

Test infrastructure (see ``oracle/__init__``).

This is the definition of the quantity the paper's device kernels evaluate
(arXiv:2211.14056, Sec. 2: "matrix element" of a process autogenerated by
MG5_aMC, Table 1 counts its diagrams):

    sum_colours |M_h|^2 = sum_colours | sum_diagrams colour_d * K_d(h) |^2
                        = sum_{d,d'} conj(K_d) Chat_{dd'} K_d',
    Chat_{dd'} = sum over every external colour index of conj(colour_d) colour_d'.

Diagrams are enumerated from the vertices {q qbar g}, {g g g}, {g g g g},
{l+ l- photon}; a four-gluon vertex carries three colour structures, so a
diagram containing it is split into separate (colour, Lorentz) terms.

Feynman rules (Peskin & Schroeder, Ch. 16; D_mu = d_mu - i g A^a_mu T^a),
all momenta flowing into a vertex:
    q qbar g     i g gamma^mu T^a_{ij}      (i on the quark leg, j on the antiquark leg)
    g g g        g f^{abc} [g^{mu nu}(k1-k2)^rho + g^{nu rho}(k2-k3)^mu + g^{rho mu}(k3-k1)^nu]
    g g g g      -i g^2 [f^{abe}f^{cde}(g^{mu rho}g^{nu sig} - g^{mu sig}g^{nu rho})
                        + f^{ace}f^{bde}(g^{mu nu}g^{rho sig} - g^{mu sig}g^{nu rho})
                        + f^{ade}f^{bce}(g^{mu nu}g^{rho sig} - g^{mu rho}g^{nu sig})]
    l l photon   -i e Q gamma^mu, Q = -1
    gluon/photon propagator  -i g_{mu nu} / P^2
    fermion propagator       i (P-slash + m) / (P^2 - m^2 + i m Gamma)
External factors: incoming vector eps, outgoing vector eps*, incoming fermion
u, outgoing fermion ubar, incoming antifermion vbar, outgoing antifermion v.

Internally every leg is treated as outgoing with momentum q (q = -p for an
incoming leg).  A sub-tree over a set S of legs "emits" a flavour into the
vertex above it; a fermion it emits is carried as a row spinor (ubar-like),
an antifermion as a column spinor (v-like), a vector as a contravariant vector.
Momentum along the fermion arrow: +sum_S q for a row spinor, -sum_S q for a
column spinor.
"""
import itertools
import numpy as np

from .wavefunctions import GAMMA, mdot, slash
from .colour import T as TGEN, F as FABC

ANTI = {"t": "t~", "t~": "t", "u": "u~", "u~": "u", "g": "g", "a": "a",
        "e-": "e+", "e+": "e-", "mu-": "mu+", "mu+": "mu-"}
ROW = {"t", "u", "e-", "mu-"}          # fermions: carried as row spinors
COL = {"t~", "u~", "e+", "mu+"}        # antifermions: carried as column spinors
VEC = {"g", "a"}
COLOUR_DIM = {"t": 3, "t~": 3, "u": 3, "u~": 3, "g": 8, "a": 1,
              "e-": 1, "e+": 1, "mu-": 1, "mu+": 1}

# all-outgoing vertex content
VERTICES = [
    ("qqg", ("t", "t~", "g")),
    ("qqg", ("u", "u~", "g")),
    ("ggg", ("g", "g", "g")),
    ("gggg", ("g", "g", "g", "g")),
    ("llA", ("e-", "e+", "a")),
    ("llA", ("mu-", "mu+", "a")),
]


def _set_partitions(items, k):
    """All partitions of the tuple ``items`` into k unordered non-empty blocks."""
    items = tuple(items)
    if k == 1:
        yield (items,)
        return
    if len(items) < k:
        return
    first, rest = items[0], items[1:]
    # first item in its own block
    for p in _set_partitions(rest, k - 1):
        yield ((first,),) + p
    # first item joins a block of a k-partition of the rest
    for p in _set_partitions(rest, k):
        for b in range(k):
            yield p[:b] + ((first,) + p[b],) + p[b + 1:]


def _multiset_minus(legs, f):
    legs = list(legs)
    if f not in legs:
        return None
    legs.remove(f)
    return tuple(legs)


class DiagramSet:
    """All tree diagrams of a process given by its outgoing-convention flavours."""

    def __init__(self, flavours, root=None):
        self.flavours = tuple(flavours)
        self.n = len(flavours)
        self.root = self.n - 1 if root is None else root
        self._memo = {}
        rest = tuple(i for i in range(self.n) if i != self.root)
        self.diagrams = self._attach(rest, self.flavours[self.root])

    def _subtrees(self, S, F):
        """Trees over legs S (sorted tuple) that emit flavour F."""
        key = (S, F)
        if key in self._memo:
            return self._memo[key]
        if len(S) == 1:
            out = [("leaf", S[0])] if self.flavours[S[0]] == F else []
        else:
            out = [("node", kind, F, ch) for kind, ch in self._vertex_options(S, ANTI[F])]
        self._memo[key] = out
        return out

    def _vertex_options(self, S, parent_leg):
        """(vertex kind, children) joining the legs S with a vertex whose
        remaining leg has flavour ``parent_leg``; children are (role flavour, tree)."""
        opts = []
        for kind, legs in VERTICES:
            others = _multiset_minus(legs, parent_leg)
            if others is None:
                continue
            k = len(others)
            for part in _set_partitions(S, k):
                seen = set()
                for assign in itertools.permutations(others):
                    if assign in seen:
                        continue
                    seen.add(assign)
                    choices = [self._subtrees(tuple(sorted(b)), fl) for b, fl in zip(part, assign)]
                    if any(len(c) == 0 for c in choices):
                        continue
                    for combo in itertools.product(*choices):
                        opts.append((kind, tuple(zip(assign, combo))))
        return opts

    def _attach(self, rest, root_flavour):
        """Root vertices: the root leg plus sub-trees over ``rest``."""
        return [(kind, ch) for kind, ch in self._vertex_options(rest, root_flavour)]


def _legs_of(tree):
    if tree[0] == "leaf":
        return (tree[1],)
    out = ()
    for _, t in tree[3]:
        out += _legs_of(t)
    return tuple(sorted(out))


class Amplitude:
    """Evaluates every diagram term of a DiagramSet on a batch of events.

    couplings: dict with 'gs' and 'e'; masses/widths per flavour via dicts.
    """

    def __init__(self, diagrams, masses, widths, couplings):
        self.ds = diagrams
        self.n = diagrams.n
        self.masses = masses
        self.widths = widths
        self.gs = couplings.get("gs", 0.0)
        self.ee = couplings.get("e", 0.0)
        self._colour_cache = {}
        self._colour_matrix = None

    # ---------------- colour ----------------
    def _leaf_colour(self, leg):
        d = COLOUR_DIM[self.ds.flavours[leg]]
        return np.eye(d, dtype=complex)

    def _vertex_colour_terms(self, kind, child_roles, parent_role):
        """Colour tensors of a vertex with legs ordered (children..., parent)."""
        if kind == "qqg":
            roles = list(child_roles) + [parent_role]
            idx = [("q" if r in ROW else "qb" if r in COL else "g") for r in roles]
            base = np.einsum("aij->ija", TGEN)          # axes (q, qbar, g)
            perm = [("q", "qb", "g").index(x) for x in idx]
            return [np.transpose(base, perm)]
        if kind == "llA":
            return [np.ones((1, 1, 1), dtype=complex)]
        if kind == "ggg":
            return [FABC.astype(complex)]
        if kind == "gggg":
            A = np.einsum("abe,cde->abcd", FABC, FABC)
            B = np.einsum("ace,bde->abcd", FABC, FABC)
            C = np.einsum("ade,bce->abcd", FABC, FABC)
            return [A.astype(complex), B.astype(complex), C.astype(complex)]
        raise ValueError(kind)

    def _colour_of(self, tree):
        """List of colour tensors (one per term): axes = sorted legs + parent line."""
        key = ("sub", tree)
        if key in self._colour_cache:
            return self._colour_cache[key]
        if tree[0] == "leaf":
            res = [self._leaf_colour(tree[1])]
        else:
            _, kind, F, children = tree
            res = self._combine_colour(kind, children, ANTI[F], keep_parent=True)
        self._colour_cache[key] = res
        return res

    def _combine_colour(self, kind, children, parent_role, keep_parent):
        n = self.n
        child_lists = [self._colour_of(t) for _, t in children]
        vterms = self._vertex_colour_terms(kind, [r for r, _ in children], parent_role)
        legs_all = tuple(sorted(sum((_legs_of(t) for _, t in children), ())))
        out = []
        for combo in itertools.product(*child_lists):
            for vt in vterms:
                ops = []
                for k, ((_, t), c) in enumerate(zip(children, combo)):
                    ops += [c, list(_legs_of(t)) + [n + k]]
                ops += [vt, [n + k for k in range(len(children))] + [n + 10]]
                out_labels = list(legs_all) + ([n + 10] if keep_parent else [])
                if not keep_parent:
                    # contract the vertex's parent leg with the root leg
                    ops += [self._leaf_colour(self.ds.root), [self.ds.root, n + 10]]
                    out_labels = sorted(list(legs_all) + [self.ds.root])
                out.append(np.einsum(*ops, out_labels, optimize=True))
        return out

    def colour_terms(self):
        """Colour tensor of every amplitude term, flattened: [terms, prod(dims)]."""
        if "root" not in self._colour_cache:
            rows = []
            for kind, children in self.ds.diagrams:
                for c in self._combine_colour(kind, children, self.ds.flavours[self.ds.root], keep_parent=False):
                    rows.append(c.ravel())
            self._colour_cache["root"] = np.stack(rows)
        return self._colour_cache["root"]

    def colour_matrix(self):
        """Chat[t, t'] = sum over all external colours of conj(c_t) c_t'."""
        if self._colour_matrix is None:
            c = self.colour_terms()
            self._colour_matrix = np.conj(c) @ c.T
        return self._colour_matrix

    # ---------------- kinematics ----------------
    def _propagator_fermion(self, P, flavour):
        m = self.masses.get(flavour, 0.0)
        w = self.widths.get(flavour, 0.0)
        den = mdot(P, P) - m * m + 1j * m * w
        num = slash(P) + m * np.eye(4)
        return 1j * num / den[..., None, None]

    def _coupling(self, kind):
        return self.gs if kind in ("qqg", "ggg", "gggg") else self.ee

    def _kin_of(self, tree, ext, q):
        key = ("kin", tree)
        if key in self._kin_cache:
            return self._kin_cache[key]
        if tree[0] == "leaf":
            res = [ext[tree[1]]]
        else:
            _, kind, F, children = tree
            amps = self._vertex_kin(kind, children, ANTI[F], ext, q)
            S = _legs_of(tree)
            Ptot = sum(q[i] for i in S)
            res = []
            for a in amps:
                if F in VEC:
                    res.append(-1j * a / mdot(Ptot, Ptot)[..., None])
                elif F in ROW:
                    Sp = self._propagator_fermion(Ptot, F)
                    res.append(np.einsum("...a,...ab->...b", a, Sp))
                else:
                    Sp = self._propagator_fermion(-Ptot, ANTI[F])
                    res.append(np.einsum("...ab,...b->...a", Sp, a))
        self._kin_cache[key] = res
        return res

    def _vertex_kin(self, kind, children, parent_role, ext, q):
        """Amputated vertex outputs (one per colour term) for the given children."""
        g = self._coupling(kind)
        kids = [(role, self._kin_of(t, ext, q), sum(q[i] for i in _legs_of(t))) for role, t in children]
        out = []
        for combo in itertools.product(*[k[1] for k in kids]):
            cur = [(role, c, P) for (role, _, P), c in zip(kids, combo)]
            if kind in ("qqg", "llA"):
                cpl = 1j * g            # i g gamma^mu  (and -i e Q gamma^mu with Q = -1)
                row = [c for r, c, _ in cur if r in ROW]
                col = [c for r, c, _ in cur if r in COL]
                vec = [c for r, c, _ in cur if r in VEC]
                if parent_role in VEC:
                    out.append(cpl * np.einsum("...a,nab,...b->...n", row[0], GAMMA, col[0]))
                elif parent_role in COL:    # children row + vector -> row output
                    out.append(cpl * np.einsum("...a,...ab->...b", row[0], slash(vec[0])))
                else:                       # children column + vector -> column output
                    out.append(cpl * np.einsum("...ab,...b->...a", slash(vec[0]), col[0]))
            elif kind == "ggg":
                (_, V1, P1), (_, V2, P2) = cur
                k1, k2, k3 = -P1, -P2, P1 + P2
                O = (mdot(V1, V2)[..., None] * (k1 - k2)
                     + V2 * mdot(k2 - k3, V1)[..., None]
                     + V1 * mdot(k3 - k1, V2)[..., None])
                out.append(g * O)
            elif kind == "gggg":
                (_, V1, _), (_, V2, _), (_, V3, _) = cur
                d12, d13, d23 = mdot(V1, V2)[..., None], mdot(V1, V3)[..., None], mdot(V2, V3)[..., None]
                A = d13 * V2 - d23 * V1
                B = d12 * V3 - d23 * V1
                C = d12 * V3 - d13 * V2
                out.extend([-1j * g * g * A, -1j * g * g * B, -1j * g * g * C])
            else:
                raise ValueError(kind)
        return out

    def amplitude_terms(self, ext, q):
        """Kinematic factor of every term: array [terms, *helicity axes, N].

        ext[i]: external wavefunction of leg i with helicity axis i;
        q[i]: outgoing-convention momentum of leg i, [N, 4].
        The term order matches colour_terms().
        """
        self._kin_cache = {}
        r = self.ds.root
        root_wf = ext[r]
        rf = self.ds.flavours[r]
        terms = []
        for kind, children in self.ds.diagrams:
            for a in self._vertex_kin(kind, children, rf, ext, q):
                if rf in VEC:
                    terms.append(mdot(a, root_wf))
                elif rf in COL:      # amputated row times column root
                    terms.append(np.einsum("...a,...a->...", a, root_wf))
                else:                # row root times amputated column
                    terms.append(np.einsum("...a,...a->...", root_wf, a))
        self._kin_cache = {}
        shape = np.broadcast_shapes(*[t.shape for t in terms])
        return np.stack([np.broadcast_to(t, shape) for t in terms])

    def summed_squared(self, ext, q):
        """sum over helicities and colours of |M|^2, per event [N]."""
        K = self.amplitude_terms(ext, q)
        nt = K.shape[0]
        Kf = K.reshape(nt, -1, K.shape[-1])
        C = self.colour_matrix()
        Y = np.einsum("st,thn->shn", C, Kf)
        return np.real(np.einsum("shn,shn->n", np.conj(Kf), Y))
