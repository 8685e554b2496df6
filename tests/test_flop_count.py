"""Algorithmic FLOP count of one evaluation, counted on a plain restatement.

The roofline fractions the benchmark reports divide the per-pair and per-atom counts in
paper_2606_14073_gb300/flops.py by measured kernel times.  This test pins those counts.
It restates the method's arithmetic as plain scalar code over a number type that counts
every add, subtract, multiply and divide as one FLOP (a multiply-add is two) and every
transcendental (cos, sin, 1/sqrt, tanh) as one.  The restatement follows Sections
5.1.1-5.1.2 and 5.2.3-5.2.4: the shared Chebyshev carrier, the four pairwise magnetic
sub-terms, the angular channels in harmonic (addition-theorem) form, and the
coefficient contractions hoisted out of the pair loops, as the paper does with its
precomputed fp.dC and fp.Cv products.  Products of two constants are folded and
not counted.

Two things are checked:
  1. the restatement reproduces the oracle's descriptors, per-atom energies, forces and
     spin fields on an isolated cluster to 1e-10, so the counted code is the computation;
  2. every pair of a kind costs the same count, and flops.py equals the counts.
"""
import collections
import math
import operator

import numpy as np
import pytest

from oracle import oracle as O
from paper_2606_14073_gb300 import flops, nep_params, workloads as W

NS, NCH, NK, NH, NLM = 2, 5, 9, 30, 24
Q_R, Q_A, Q_O, Q_EX, Q_SA = 0, 5, 25, 26, 46
G_R, G_A, G_EX, G_DMI, G_ANI, G_SIA = range(6)


# ------------------------------------------------------------------ counting number
class _Tally:
    def __init__(self):
        self.bucket = None
        self.n = collections.Counter()

    def tick(self):
        if self.bucket is not None:
            self.n[self.bucket] += 1


T = _Tally()


class N:
    """A float whose arithmetic is counted in T.bucket."""
    __slots__ = ("v",)

    def __init__(self, v):
        self.v = float(v)


def _val(x):
    return x.v if isinstance(x, N) else x


def _binop(fn):
    def f(a, b):
        T.tick()
        return N(fn(_val(a), _val(b)))
    return f


def _rbinop(fn):
    def f(a, b):
        T.tick()
        return N(fn(_val(b), _val(a)))
    return f


for _name, _fn in (("add", operator.add), ("sub", operator.sub), ("mul", operator.mul),
                   ("truediv", operator.truediv)):
    setattr(N, f"__{_name}__", _binop(_fn))
    setattr(N, f"__r{_name}__", _rbinop(_fn))
N.__neg__ = lambda a: N(-a.v)   # a sign change folds into the operation that uses it


def _fn1(fn):
    def f(x):
        T.tick()
        return N(fn(_val(x)))
    return f


ncos, nsin, ntanh = _fn1(math.cos), _fn1(math.sin), _fn1(math.tanh)
nrsqrt = _fn1(lambda x: 1.0 / math.sqrt(x))


def dot(a, b):
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]


def cross(a, b):
    return (a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0])


def lincomb(c, x):
    """sum_k c[k] x[k] with Python-float coefficients: one multiply per term, one add per term after the first."""
    s = c[0] * x[0]
    for k in range(1, len(x)):
        s = s + c[k] * x[k]
    return s


# ------------------------------------------------------------------ the method, restated
def carrier(r, rc, deriv):
    """f_k = (T_k(x) + 1) f_c/2, x = 2(r/rc - 1)^2 - 1, f_c = (1 + cos(pi r/rc))/2; with deriv the
    r-derivatives via dT_k/dx = k U_{k-1}."""
    t = r * (1.0 / rc)
    a = t * math.pi
    fch = (ncos(a) + 1.0) * 0.25
    y = t - 1.0
    x = y * y * 2.0 - 1.0
    x2 = x * 2.0
    f = [fch * 2.0, x * fch + fch]
    df = None
    if deriv:
        dfch = nsin(a) * (-0.25 * math.pi / rc)
        dxf = y * (4.0 / rc) * fch
        df = [dfch * 2.0, dxf + (x * dfch + dfch)]
        um, uc = 1.0, x2
    tm, tc = 1.0, x
    for k in range(2, NK):
        tn = x2 * tc - tm
        f.append(tn * fch + fch)
        if deriv:
            df.append(uc * float(k) * dxf + (tn * dfch + dfch))
            um, uc = uc, x2 * uc - um
        tm, tc = tc, tn
    return f, df


def harmonics(x, y, z, grad):
    """The 24 real solid harmonics p_lm, l = 1..4 (homogeneous polynomials), and with grad
    their Euclidean gradients."""
    x2, y2, z2 = x * x, y * y, z * z
    xy, yz, xz = x * y, y * z, x * z
    s = x2 + y2
    r2 = s + z2
    d = x2 - y2
    a3 = x2 * 3.0 - y2          # 3x^2 - y^2
    b3 = x2 - y2 * 3.0          # x^2 - 3y^2
    c4 = z2 * 4.0 - s           # 4z^2 - x^2 - y^2
    c43 = z2 * 4.0 - s * 3.0    # 4z^2 - 3x^2 - 3y^2
    c6 = z2 * 6.0 - s           # 6z^2 - x^2 - y^2
    c2 = z2 * 2.0 - s * 3.0     # 2z^2 - 3x^2 - 3y^2
    p = [x, y, z, xy, yz, xz, d, z2 * 2.0 - s,
         y * a3, xy * z, y * c4, z * c2, x * c4, z * d, x * b3,
         xy * d, yz * a3, xy * c6, yz * c43,
         z2 * z2 * 35.0 - z2 * r2 * 30.0 + r2 * r2 * 3.0,
         xz * c43, d * c6, xz * b3, x2 * x2 - x2 * y2 * 6.0 + y2 * y2]
    if not grad:
        return p, None
    g = [None] * NLM
    g[0], g[1], g[2] = (1.0, 0.0, 0.0), (0.0, 1.0, 0.0), (0.0, 0.0, 1.0)
    g[3], g[4], g[5] = (y, x, 0.0), (0.0, z, y), (z, 0.0, x)
    g[6] = (x * 2.0, y * -2.0, 0.0)
    g[7] = (x * -2.0, y * -2.0, z * 4.0)
    g[8] = (xy * 6.0, d * 3.0, 0.0)
    g[9] = (yz, xz, xy)
    g[10] = (xy * -2.0, z2 * 4.0 - x2 - y2 * 3.0, yz * 8.0)
    g[11] = (xz * -6.0, yz * -6.0, z2 * 6.0 - s * 3.0)
    g[12] = (z2 * 4.0 - x2 * 3.0 - y2, xy * -2.0, xz * 8.0)
    g[13] = (xz * 2.0, yz * -2.0, d)
    g[14] = (d * 3.0, xy * -6.0, 0.0)
    g[15] = (y * a3, x * b3, 0.0)
    g[16] = (xy * z * 6.0, z * d * 3.0, y * a3)
    g[17] = (y * (z2 * 6.0 - x2 * 3.0 - y2), x * (z2 * 6.0 - x2 - y2 * 3.0), xy * z * 12.0)
    g[18] = (xy * z * -6.0, z * (z2 * 4.0 - x2 * 3.0 - y2 * 9.0), y * (z2 * 12.0 - s * 3.0))
    g[19] = (x * (r2 * 12.0 - z2 * 60.0), y * (r2 * 12.0 - z2 * 60.0), z * (z2 * 80.0 - r2 * 48.0))
    g[20] = (z * (z2 * 4.0 - x2 * 9.0 - y2 * 3.0), xy * z * -6.0, x * (z2 * 12.0 - s * 3.0))
    g[21] = (x * (z2 * 12.0 - x2 * 4.0), y * (y2 * 4.0 - z2 * 12.0), z * d * 12.0)
    g[22] = (z * d * 3.0, xy * z * -6.0, x * b3)
    g[23] = (x * b3 * 4.0, y * (y2 - x2 * 3.0) * 4.0, 0.0)
    return p, g


HARM_L = [1] * 3 + [2] * 5 + [3] * 7 + [4] * 9


def kappa_table():
    """kappa_lm with P_l(u.v) = sum_m kappa_lm p_lm(u) p_lm(v): 4 pi / ((2l+1) |p_lm|^2), the
    squared norms integrated exactly (Gauss-Legendre in cos(theta) times an equal-angle rule in
    phi, exact for these degrees)."""
    ct, wt = np.polynomial.legendre.leggauss(8)
    ph = np.arange(16) * (2 * np.pi / 16)
    k = np.zeros(NLM)
    for c, w in zip(ct, wt):
        st = math.sqrt(1 - c * c)
        for f in ph:
            p, _ = harmonics(st * math.cos(f), st * math.sin(f), c, False)
            k += w * (2 * np.pi / 16) * np.array([float(_val(v)) ** 2 for v in p])
    return np.array([4 * np.pi / ((2 * HARM_L[lm] + 1) * k[lm]) for lm in range(NLM)])


def geometry(pi, pj):
    dx, dy, dz = pj[0] - pi[0], pj[1] - pi[1], pj[2] - pi[2]
    d2 = dx * dx + dy * dy + dz * dz
    ir = nrsqrt(d2)
    r = d2 * ir
    return (dx, dy, dz), r, ir, (dx * ir, dy * ir, dz * ir)


class Restated:
    """Forward, network and backward of every atom of a small isolated system."""

    def __init__(self, p, pos, spin, species):
        self.c = np.asarray(p["coeffs"], dtype=float)
        self.scal, self.w0, self.b0, self.w1 = (np.asarray(p[k], dtype=float) for k in ("q_scaler", "w0", "b0", "w1"))
        self.b1, self.rcr, self.rca = float(p["b1"]), float(p["rc_rad"]), float(p["rc_ang"])
        self.kap = kappa_table()
        self.n = len(pos)
        self.pos = [tuple(N(v) for v in r) for r in pos]
        self.spin = [tuple(N(v) for v in s) for s in spin]
        self.t = [int(v) for v in species]
        self.pairs = {}   # kind -> list of per-pair counts
        self.nbr = []
        for i in range(self.n):
            row = []
            for j in range(self.n):
                if j != i:
                    d = np.asarray(pos[j]) - np.asarray(pos[i])
                    r = float(np.sqrt(d @ d))
                    if r < self.rcr:
                        row.append((j, r < self.rca))
            self.nbr.append(row)

    def _count(self, kind, fn):
        before = sum(T.n.values())
        T.bucket = kind
        out = fn()
        T.bucket = None
        self.pairs.setdefault(kind, []).append(sum(T.n.values()) - before)
        return out

    # -- forward
    def forward(self, i):
        ti, si = self.t[i], self.spin[i]
        # sums start at zero and every pair adds into them: per neighbour species the R, EX, DMI,
        # ANI, SIA basis sums over k; the angular sums B_nlm, BS_nlm
        basis = [[[N(0.0)] * NK for _ in range(5)] for _ in range(NS)]
        B = [[N(0.0)] * NLM for _ in range(NCH)]
        BS = [[N(0.0)] * NLM for _ in range(NCH)]

        def add(acc, v):
            return v if acc is None else acc + v

        for j, ang in self.nbr[i]:
            tj, sj = self.t[j], self.spin[j]

            def rad():
                _, r, _, u = geometry(self.pos[i], self.pos[j])
                f, _ = carrier(r, self.rcr, False)
                sij, siu, sju = dot(si, sj), dot(si, u), dot(sj, u)
                phi = [sij, dot(cross(si, sj), u), siu * sju, siu * siu]
                b = basis[tj]
                b[0] = [b[0][k] + f[k] for k in range(NK)]
                for g in range(4):
                    b[1 + g] = [b[1 + g][k] + f[k] * phi[g] for k in range(NK)]
                return r, u, sij

            r, u, sij = self._count("fwd_rad_pair", rad)
            if ang:
                def angular():
                    f, _ = carrier(r, self.rca, False)
                    gA = [lincomb(self.c[ti, tj, G_A, n], f) for n in range(NCH)]
                    gS = [g * sij for g in gA]
                    p, _ = harmonics(u[0], u[1], u[2], False)
                    for n in range(NCH):
                        for lm in range(NLM):
                            B[n][lm] = B[n][lm] + gA[n] * p[lm]
                            BS[n][lm] = BS[n][lm] + gS[n] * p[lm]
                self._count("fwd_ang_pair", angular)

        q = [None] * 66

        def atom_rad():
            groups = (G_R, G_EX, G_DMI, G_ANI, G_SIA)
            offs = (Q_R, Q_EX, Q_EX + 5, Q_EX + 10, Q_EX + 15)
            for tj in range(NS):   # both neighbour species are contracted, present or not
                b = basis[tj]
                for gi in range(5):
                    sums = b[gi]
                    for n in range(NCH):
                        v = lincomb(self.c[ti, tj, groups[gi], n], sums)
                        q[offs[gi] + n] = v if tj == 0 else q[offs[gi] + n] + v
            q[Q_O] = dot(si, si)

        def atom_ang():
            for src, off in ((B, Q_A), (BS, Q_SA)):
                for n in range(NCH):
                    for l in range(1, 5):
                        acc = None
                        for lm in range(NLM):
                            if HARM_L[lm] == l:
                                bv = src[n][lm]
                                v = bv * bv * float(self.kap[lm])
                                acc = add(acc, v)
                        q[off + n * 4 + l - 1] = acc

        self._count("fwd_atom_rad", atom_rad)
        self._count("fwd_atom_ang", atom_ang)
        return q, B, BS

    # -- network: E_i and Fp = dE_i/dq
    def network(self, q):
        def net():
            x = [q[v] * float(self.scal[v]) for v in range(66)]
            th = [ntanh(lincomb(self.w0[h], x) - float(self.b0[h])) for h in range(NH)]
            E = lincomb(self.w1, th) - self.b1
            dz = [(1.0 - th[h] * th[h]) * float(self.w1[h]) for h in range(NH)]
            fp = [lincomb(self.w0[:, v], dz) * float(self.scal[v]) for v in range(66)]
            return E, fp
        return self._count("network", net)

    # -- backward: dE_i/dr_ij, dE_i/dS_j per pair and dE_i/dS_i
    def backward(self, i, fp, B, BS):
        ti, si = self.t[i], self.spin[i]

        def atom_ang():
            DA = [[(B[n][lm] * float(2.0 * self.kap[lm])) * fp[Q_A + n * 4 + HARM_L[lm] - 1]
                   for lm in range(NLM)] for n in range(NCH)]
            DS = [[(BS[n][lm] * float(2.0 * self.kap[lm])) * fp[Q_SA + n * 4 + HARM_L[lm] - 1]
                   for lm in range(NLM)] for n in range(NCH)]
            return DA, DS

        def atom_rad():
            C = [[None] * 5 for _ in range(NS)]
            for tj in range(NS):
                for gi, (g, off) in enumerate(((G_R, Q_R), (G_EX, Q_EX), (G_DMI, Q_EX + 5), (G_ANI, Q_EX + 10),
                                               (G_SIA, Q_EX + 15))):
                    C[tj][gi] = [lincomb(self.c[ti, tj, g, :, k], fp[off:off + NCH]) for k in range(NK)]
            fo = fp[Q_O] * 2.0
            gii = [fo * si[0], fo * si[1], fo * si[2]]
            return C, gii

        DA, DS = self._count("bwd_atom_ang", atom_ang)
        C, gii = self._count("bwd_atom_rad", atom_rad)
        fown = [N(0.0)] * 3
        out = []
        for j, ang in self.nbr[i]:
            tj, sj = self.t[j], self.spin[j]

            def rad():
                dv, r, ir, u = geometry(self.pos[i], self.pos[j])
                f, df = carrier(r, self.rcr, True)
                Cj = C[tj]
                e0 = lincomb_n(Cj[0], df)
                h = [lincomb_n(Cj[g], f) for g in range(1, 5)]
                e = [lincomb_n(Cj[g], df) for g in range(1, 5)]
                sij, siu, sju = dot(si, sj), dot(si, u), dot(sj, u)
                w = cross(si, sj)
                wu = dot(w, u)
                rad_ = e0 + e[0] * sij + e[1] * wu + e[2] * siu * sju + e[3] * siu * siu
                cu = h[2] * sju + h[3] * 2.0 * siu
                cSi, cSj, cW = cu * ir, h[2] * siu * ir, h[1] * ir
                along = rad_ - cSi * siu - cSj * sju - cW * wu
                D = [along * u[c] + cSi * si[c] + cSj * sj[c] + cW * w[c] for c in range(3)]
                for c in range(3):
                    fown[c] = fown[c] + D[c]
                uxs = cross(u, si)
                hsiu = h[2] * siu
                G = [h[0] * si[c] + h[1] * uxs[c] + hsiu * u[c] for c in range(3)]
                sxu = cross(sj, u)
                for c in range(3):
                    gii[c] = gii[c] + (h[0] * sj[c] + h[1] * sxu[c] + cu * u[c])
                return D, G, r, ir, u, sij

            D, G, r, ir, u, sij = self._count("bwd_rad_pair", rad)
            if ang:
                def angular():
                    f, df = carrier(r, self.rca, True)
                    gA = [lincomb(self.c[ti, tj, G_A, n], f) for n in range(NCH)]
                    dgA = [lincomb(self.c[ti, tj, G_A, n], df) for n in range(NCH)]
                    p, gp = harmonics(u[0], u[1], u[2], True)
                    lir = [ir * float(l) for l in range(1, 5)]
                    accu, av3, cj = None, [None] * 3, None
                    for lm in range(NLM):
                        aA = lincomb_n([DA[n][lm] for n in range(NCH)], gA)
                        aS = lincomb_n([DS[n][lm] for n in range(NCH)], gA)
                        bA = lincomb_n([DA[n][lm] for n in range(NCH)], dgA)
                        bS = lincomb_n([DS[n][lm] for n in range(NCH)], dgA)
                        av, bv = aA + sij * aS, bA + sij * bS
                        term = p[lm] * (bv - lir[HARM_L[lm] - 1] * av)
                        accu = term if accu is None else accu + term
                        for c in range(3):
                            gc = gp[lm][c]
                            if isinstance(gc, float) and gc == 0.0:
                                continue
                            t_ = av if (isinstance(gc, float) and gc == 1.0) else av * gc
                            av3[c] = t_ if av3[c] is None else av3[c] + t_
                        t_ = aS * p[lm]
                        cj = t_ if cj is None else cj + t_
                    for c in range(3):
                        dA = accu * u[c] + ir * av3[c]
                        D[c] = D[c] + dA
                        fown[c] = fown[c] + dA
                        G[c] = G[c] + cj * si[c]
                        gii[c] = gii[c] + cj * sj[c]
                self._count("bwd_ang_pair", angular)
            out.append((j, D, G))
        return out, gii, fown


def lincomb_n(c, x):
    """sum_k c[k] x[k] with counted coefficients."""
    s = c[0] * x[0]
    for k in range(1, len(x)):
        s = s + c[k] * x[k]
    return s


def _cluster():
    """The 14 atoms nearest to one atom of the seeded 512-atom FeGe crystal, isolated in a
    non-periodic box, with seeded random unit spins."""
    wl = W.fege_small()
    pos = np.mod(wl.positions, wl.box)
    c = pos[100]
    d = pos - c
    d -= wl.box * np.rint(d / wl.box)
    idx = np.argsort(np.einsum("ij,ij->i", d, d))[:14]
    p = d[idx] + 50.0
    rng = np.random.default_rng(5)
    s = rng.normal(size=(len(idx), 3))
    s /= np.linalg.norm(s, axis=1)[:, None]
    return p, s, wl.species[idx]


@pytest.fixture(scope="module")
def counted():
    params = nep_params.load()
    pos, spin, species = _cluster()
    assert set(species.tolist()) == {0, 1}
    R = Restated(params, pos, spin, species)
    n = len(pos)
    q = np.zeros((n, 66))
    Ei = np.zeros(n)
    records = [[] for _ in range(n)]   # (dE_i/dr_ik, dE_i/dS_k) addressed to atom k
    fown, gii = [None] * n, [None] * n
    for i in range(n):
        qi, B, BS = R.forward(i)
        q[i] = [_val(v) for v in qi]
        E, fp = R.network(qi)
        Ei[i] = _val(E)
        pairs, gii[i], fown[i] = R.backward(i, fp, B, BS)
        for j, D, G in pairs:
            records[j].append((D, G))
    # F_k = sum_j dE_k/dr_kj - sum_j dE_j/dr_jk, H_k = -dE_k/dS_k - sum_j dE_j/dS_k (no field): one
    # record per ordered pair gathered by its target atom
    F = np.zeros((n, 3))
    H = np.zeros((n, 3))
    for k in range(n):
        f = list(fown[k])
        h = [-gii[k][0], -gii[k][1], -gii[k][2]]
        for D, G in records[k]:
            def one():
                for c in range(3):
                    f[c] = f[c] - D[c]
                    h[c] = h[c] - G[c]
            R._count("gather_pair", one)
        F[k] = [_val(v) for v in f]
        H[k] = [_val(v) for v in h]
    model = O.Model(params)
    box, per = np.array([100.0, 100.0, 100.0]), np.array([0, 0, 0])
    ref = O.evaluate(model, pos, spin, species, box, per)
    qref = O.descriptors(model, pos, spin, species, box, per)
    return dict(R=R, q=q, Ei=Ei, F=F, H=H, ref=ref, qref=qref, params=params)


def test_restatement_is_the_method(counted):
    """The counted code computes the oracle's descriptors, energies, forces and fields."""
    c = counted
    scale = np.maximum(np.abs(c["qref"]).max(0), 1e-12)
    assert (np.abs(c["q"] - c["qref"]) / scale).max() < 1e-10
    assert np.abs(c["Ei"] - c["ref"]["Ei"]).max() < 1e-10 * np.abs(c["ref"]["Ei"]).max()
    assert np.abs(c["F"] - c["ref"]["F"]).max() < 1e-10 * np.abs(c["ref"]["F"]).max()
    assert np.abs(c["H"] - c["ref"]["H"]).max() < 1e-10 * np.abs(c["ref"]["H"]).max()


def test_cluster_exercises_every_kind_of_pair(counted):
    R = counted["R"]
    assert len(R.pairs["fwd_ang_pair"]) >= 40 and len(R.pairs["fwd_rad_pair"]) > len(R.pairs["fwd_ang_pair"])


def test_every_pair_of_a_kind_costs_the_same(counted):
    for kind, counts in counted["R"].pairs.items():
        assert len(set(counts)) == 1, (kind, sorted(set(counts)))


def test_flops_module_equals_the_counts(counted):
    c = {k: v[0] for k, v in counted["R"].pairs.items()}
    assert (flops.FWD_RADIAL_PAIR, flops.FWD_ANGULAR_PAIR) == (c["fwd_rad_pair"], c["fwd_ang_pair"])
    assert (flops.FWD_ATOM_RAD, flops.FWD_ATOM_ANG) == (c["fwd_atom_rad"], c["fwd_atom_ang"])
    assert flops.NETWORK_ATOM == c["network"]
    assert (flops.BWD_ATOM_RAD, flops.BWD_ATOM_ANG) == (c["bwd_atom_rad"], c["bwd_atom_ang"])
    assert (flops.BWD_RADIAL_PAIR, flops.BWD_ANGULAR_PAIR) == (c["bwd_rad_pair"], c["bwd_ang_pair"])
    assert flops.GATHER_PAIR == c["gather_pair"]
    assert flops.FWD_ATOM == flops.FWD_ATOM_RAD + flops.FWD_ATOM_ANG
    assert flops.BWD_ATOM == flops.BWD_ATOM_RAD + flops.BWD_ATOM_ANG


def test_per_atom_totals_follow_the_counts(counted):
    """flops.per_atom at the cluster's own neighbour counts equals the total counted work."""
    R = counted["R"]
    n = R.n
    n_r = len(R.pairs["fwd_rad_pair"]) / n
    n_a = len(R.pairs["fwd_ang_pair"]) / n
    total = sum(sum(v) for v in R.pairs.values()) / n
    assert abs(flops.per_atom(n_r, n_a)["total"] - total) < 1e-9 * total
