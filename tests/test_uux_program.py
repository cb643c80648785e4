"""Host-side check of the u u~ -> t t~ g g amplitude program (gen_uux).

The generator enumerates the tree diagrams, decomposes their colour factors
onto 12 structures and emits a program of primitive operations that the CUDA
kernel executes.  This test interprets the same program in numpy with
explicit 4x4 gamma matrices (chiral representation), sums helicities and
colours, and compares |M|^2 with the oracle's independent Feynman-diagram sum
with explicit colour indices (``oracle.processes``): a wrong diagram, sign,
factor of i, momentum or colour coefficient anywhere fails it, without a GPU.
"""
import numpy as np
import pytest

from oracle import integrate as oi, philox as oph
from oracle.processes import Process as OracleProcess
from paper_2211_14056_gb300.gen_uux import build

SIG = [np.array([[0, 1], [1, 0]], dtype=complex), np.array([[0, -1j], [1j, 0]]), np.array([[1, 0], [0, -1]], dtype=complex)]
Z2, I2 = np.zeros((2, 2)), np.eye(2)
GAMMA = [np.block([[Z2, I2], [I2, Z2]])] + [np.block([[Z2, s], [-s, Z2]]) for s in SIG]
METRIC = np.diag([1.0, -1.0, -1.0, -1.0])


def slash(V):
    return sum(METRIC[m, m] * V[m] * GAMMA[m] for m in range(4))


def mdot(a, b):
    return a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3]


def chi(p, lam):
    px, py, pz = p[1], p[2], p[3]
    pa = np.sqrt(px * px + py * py + pz * pz)
    s = pa + pz
    if s > 0:
        n = 1 / np.sqrt(2 * pa * s)
        return np.array([s * n, (px + 1j * py) * n]) if lam > 0 else np.array([(-px + 1j * py) * n, s * n])
    return np.array([0, 1], dtype=complex) if lam > 0 else np.array([-1, 0], dtype=complex)


def omegas(p, m):
    pa = np.sqrt(p[1] ** 2 + p[2] ** 2 + p[3] ** 2)
    wp = np.sqrt(p[0] + pa)
    return wp, (m / wp if m else 0.0)


def u_spinor(p, m, lam):
    wp, wm = omegas(p, m)
    c = chi(p, lam)
    wl, wml = (wp, wm) if lam > 0 else (wm, wp)
    return np.concatenate([wml * c, wl * c])


def v_spinor(p, m, lam):
    wp, wm = omegas(p, m)
    c = chi(p, -lam)
    wl, wml = (wp, wm) if lam > 0 else (wm, wp)
    return np.concatenate([-lam * wl * c, lam * wml * c])


def bar(s):
    return s.conj() @ GAMMA[0]


def eps_out(k, lam):
    kx, ky, kz = k[1], k[2], k[3]
    kt = np.hypot(kx, ky)
    ka = np.sqrt(kt * kt + kz * kz)
    e1, e2 = np.zeros(4), np.zeros(4)
    if kt > 0:
        e1[1:] = [kx * kz / (ka * kt), ky * kz / (ka * kt), -kt / ka]
        e2[1:] = [-ky / kt, kx / kt, 0]
    else:
        e1[1] = -1 if kz < 0 else 1
        e2[2] = 1
    return (-lam * e1 + 1j * e2) / np.sqrt(2)     # eps* of an outgoing gluon


def vvv(A, KA, C, KC):
    return mdot(A, C) * (KA - KC) + C * mdot(KA + 2 * KC, A) - A * mdot(2 * KA + KC, C)


def v4(t, A, C, D):
    if t == 1:
        return mdot(A, D) * C - mdot(C, D) * A
    if t == 2:
        return mdot(A, C) * D - mdot(C, D) * A
    return mdot(A, C) * D - mdot(A, D) * C


def me2(p, prog, diags, coefs, M, D, mt, wt, gs):
    n = len(M)
    C = np.array(M, dtype=float) / D
    Kv = {name: sum(c * p[i] for i, c in enumerate(m)) for m, name in prog.moms.items()}
    total = 0.0
    for l1 in (-1, 1):
        for l2 in (-1, 1):
            for l4 in (-1, 1):
                for l5 in (-1, 1):
                    for l6 in (-1, 1):
                        env = {"U1": u_spinor(p[0], 0.0, l1), "V2": bar(v_spinor(p[1], 0.0, l2)),
                               "VTB": v_spinor(p[3], mt, l4), "E5": eps_out(p[4], l5), "E6": eps_out(p[5], l6)}
                        for name, op, a in prog.ops:
                            g = lambda x: env[x] if x in env else Kv[x]
                            if op == "slash_col":
                                r = slash(g(a[0])) @ g(a[1])
                            elif op == "slash_row":
                                r = g(a[0]) @ slash(g(a[1]))
                            elif op == "lprop_col":
                                P = g(a[0]); r = slash(P) @ g(a[1]) / mdot(P, P)
                            elif op == "lprop_row":
                                P = g(a[1]); r = g(a[0]) @ slash(P) / mdot(P, P)
                            elif op == "hprop_col":
                                P = g(a[0])
                                r = (slash(P) + mt * np.eye(4)) @ g(a[1]) / (mdot(P, P) - mt * mt + 1j * mt * mt * wt)
                            elif op == "vcur":
                                r = np.array([g(a[0]) @ GAMMA[m] @ g(a[1]) for m in range(4)])
                            elif op == "gprop":
                                K = g(a[1]); r = g(a[0]) / mdot(K, K)
                            elif op == "vvv":
                                r = vvv(g(a[0]), g(a[1]), g(a[2]), g(a[3]))
                            else:
                                r = v4(int(op[3]), g(a[0]), g(a[1]), g(a[2]))
                            env[name] = r
                        for l3 in (-1, 1):
                            ub3 = bar(u_spinor(p[2], mt, l3))
                            J = np.zeros(n, dtype=complex)
                            for di, d in enumerate(diags):
                                amp = ub3 @ env[d["column"]]
                                k = (-d["power"]["-i"] + d["power"]["+i"]) % 4
                                amp = amp * (1j ** k)
                                for b, (cr, ci) in enumerate(coefs[di]):
                                    J[b] += complex(float(cr), float(ci)) * amp
                            total += np.real(np.conj(J) @ C @ J)
    return total * gs ** 8 / (36 * 2)


@pytest.fixture(scope="module")
def program():
    prog, diags, coefs, labels, M, D = build()
    return prog, diags, coefs, M, D


def test_program_shape(program):
    prog, diags, coefs, M, D = program
    assert len(diags) == 38 and len(M) == 12
    C = np.array(M) / D
    assert np.allclose(C, C.T) and np.all(np.linalg.eigvalsh(C) > 0)


@pytest.mark.parametrize("wt", [0.0, 1.5])
def test_program_matches_oracle(program, wt):
    prog, diags, coefs, M, D = program
    cfg = dict(process="uux_ttxgg", mt=173.0, wt=wt, gs=1.2177, sqrt_s=13000.0, lumi=True, pt_cut=30.0,
               dr_cut=0.4)
    st = oi.Setup(cfg)
    y = oph.uniforms(5, 0, np.arange(40, dtype=np.uint64), st.ndim)
    from oracle import vegas as ov
    po, _, _, cut = st.kinematics(y, ov.uniform_grid(st.ndim))
    po = po[cut][:4]
    ref = OracleProcess("uux_ttxgg", mt=173.0, wt=wt, gs=1.2177).me2(po)
    got = np.array([me2(q, prog, diags, coefs, M, D, 173.0, wt / 173.0, 1.2177) for q in po])
    np.testing.assert_allclose(got, ref, rtol=1e-11)
