"""Partition-of-unity discretisation oracle (Section 4, Examples 5.1 and 5.4).

Test infrastructure only: imported by tests, smoke() and the CPU baseline of
bench.py, never by the CUDA library.

What is computed, in the paper's terms:

* Cover (Section 4, Fig. 4.1): level with m patches per side, cell width h = 1/m;
  patch omega_a is cell a stretched by 1.5 about its centre, i.e. the interval
  ((a - 1/4) h, (a + 5/4) h), clipped to [0, 1].  2-D patches are tensor products,
  block index i = iy * m + ix.
* Partition of unity (Section 4, reading of the construction deferred by the paper
  to its companion work): phi_a = 1 on its own zone, blends to its neighbour across
  the overlap zone of width h/2 with S(t) = 6t^5 - 15t^4 + 10t^3 (C^2), is 1 up to
  the domain boundary on boundary patches; 2-D phi_i = phi_ix(x) phi_iy(y).
  sum_i phi_i = 1 holds exactly.
* Local spaces (Section 5): total degree <= p, written in tensor Legendre
  polynomials P_a(xi) P_b(eta) on the clipped patch box mapped to [-1, 1]^2, ordered
  by total degree a + b and then by b.  dim V_i = (p+1)(p+2)/2.
* Stiffness and load (Section 4 Galerkin system; Nitsche forms of Example 5.1 for
  the biharmonic equation and of Example 5.4 for -Delta^3 u = f):
  A_(i,k),(j,l) = a_n(phi_i theta_i^k, phi_j theta_j^l), b_(i,k) = l_n(phi_i theta_i^k).
  Integrals are tensor Gauss-Legendre rules with q points per direction on every
  sub-cell of the grid of PU breakpoints, so polynomial integrands are exact.
* Prolongation (Section 4): global-to-local L2 projection onto each fine local space
  over omega_i cap Omega; restriction is its transpose; coarse operators are the
  Galerkin products A_{l-1} = P_l^T A_l P_l (Section 5).

The integrals here are evaluated by brute force: every integrand is formed at every
tensor quadrature point of every sub-cell and summed.
"""
from __future__ import annotations

import dataclasses
from math import comb

import numpy as np
from numpy.polynomial import legendre as npleg
from numpy.polynomial import polynomial as nppoly

from . import blocks as bk

# ---------------------------------------------------------------------------
# Cover, partition of unity, local basis
# ---------------------------------------------------------------------------

_SMOOTHSTEP = np.array([0.0, 0.0, 0.0, 10.0, -15.0, 6.0])  # S(t) = 10t^3 - 15t^4 + 6t^5


def local_dim(p: int) -> int:
    """dim V_i = binom(p+2, 2) (Section 5)."""
    return comb(p + 2, 2)


def basis_exponents(p: int) -> list[tuple[int, int]]:
    """Legendre degrees (a, b), a + b <= p, by total degree then by b."""
    return [(s - b, b) for s in range(p + 1) for b in range(s + 1)]


def patch_box_1d(m: int, a: int) -> tuple[float, float]:
    """Clipped 1-D support of patch a: ((a - 1/4) h, (a + 5/4) h) cap [0, 1]."""
    return max((a - 0.25) / m, 0.0), min((a + 1.25) / m, 1.0)


def breakpoints_1d(m: int) -> np.ndarray:
    """All PU breakpoints of a level: 0, (a + 1/4) h, (a + 3/4) h, 1."""
    pts = {0.0, 1.0}
    for a in range(m):
        for fr in (0.25, 0.75):
            x = (a + fr) / m
            if 0.0 < x < 1.0:
                pts.add(x)
    return np.array(sorted(pts))


def smoothstep(t: np.ndarray, r: int) -> np.ndarray:
    """r-th derivative of S(t)."""
    c = _SMOOTHSTEP
    for _ in range(r):
        c = nppoly.polyder(c)
    return nppoly.polyval(t, c)


def pu_1d(m: int, a: int, x: np.ndarray, r: int) -> np.ndarray:
    """r-th derivative of the 1-D PU function phi_a at the points x."""
    x = np.asarray(x, dtype=np.float64)
    h = 1.0 / m
    out = np.zeros_like(x)
    own_lo = (a + 0.25) / m if a > 0 else 0.0
    own_hi = (a + 0.75) / m if a < m - 1 else 1.0
    own = (x >= own_lo) & (x <= own_hi)
    if r == 0:
        out[own] = 1.0
    if a > 0:
        lo = (a - 0.25) / m
        sel = (x >= lo) & (x < own_lo)
        t = np.clip((x[sel] - lo) / (0.5 * h), 0.0, 1.0)
        out[sel] = smoothstep(t, r) * (2.0 / h) ** r
    if a < m - 1:
        lo = (a + 0.75) / m
        hi = (a + 1.25) / m
        sel = (x > own_hi) & (x <= hi)
        t = np.clip((x[sel] - lo) / (0.5 * h), 0.0, 1.0)
        val = smoothstep(t, r) * (2.0 / h) ** r
        out[sel] = (1.0 - val) if r == 0 else -val
    return out


def legendre(j: int, xi: np.ndarray, r: int) -> np.ndarray:
    """r-th derivative of the Legendre polynomial P_j at xi."""
    c = np.zeros(j + 1)
    c[j] = 1.0
    if r:
        c = npleg.legder(c, r)
    return npleg.legval(xi, c)


def local_poly_1d(m: int, a: int, j: int, x: np.ndarray, r: int) -> np.ndarray:
    """r-th derivative of P_j(xi(x)), xi the affine map of patch a's box to [-1, 1]."""
    lo, hi = patch_box_1d(m, a)
    w = hi - lo
    xi = (2.0 * x - lo - hi) / w
    return legendre(j, xi, r) * (2.0 / w) ** r


def factor_1d(m: int, a: int, j: int, x: np.ndarray, n: int) -> np.ndarray:
    """n-th derivative of X(x) = phi_a(x) P_j(xi(x)) by the Leibniz rule."""
    return sum(comb(n, r) * pu_1d(m, a, x, r) * local_poly_1d(m, a, j, x, n - r)
               for r in range(n + 1))


def active_1d(m: int, lo: float, hi: float) -> list[int]:
    """Patches whose clipped support contains the sub-interval (lo, hi)."""
    mid = 0.5 * (lo + hi)
    out = []
    for a in range(m):
        plo, phi = patch_box_1d(m, a)
        if plo < mid < phi:
            out.append(a)
    return out


# ---------------------------------------------------------------------------
# Differential operators as {(alpha, beta): coefficient}  (d^alpha/dx d^beta/dy)
# ---------------------------------------------------------------------------

OP_I = {(0, 0): 1.0}
OP_LAP = {(2, 0): 1.0, (0, 2): 1.0}
OP_BILAP = {(4, 0): 1.0, (2, 2): 2.0, (0, 4): 1.0}


def op_dx(op):
    return {(al + 1, be): c for (al, be), c in op.items()}


def op_dy(op):
    return {(al, be + 1): c for (al, be), c in op.items()}


def op_dn(op, n):
    """Normal derivative n . grad applied after op."""
    out = {}
    for k, c in op_dx(op).items():
        out[k] = out.get(k, 0.0) + n[0] * c
    for k, c in op_dy(op).items():
        out[k] = out.get(k, 0.0) + n[1] * c
    return {k: c for k, c in out.items() if c != 0.0}


def max_order(op) -> int:
    return max(max(al, be) for (al, be) in op)


ISOTROPIC = (1.0, 0.0, 1.0)


def anisotropy(kappa: float, theta: float) -> tuple:
    """(S11, S12, S22) of S = R(theta) diag(kappa, 1) R(theta)^T (Example 5.2)."""
    c, s = np.cos(theta), np.sin(theta)
    return (kappa * c * c + s * s, (kappa - 1.0) * c * s, kappa * s * s + c * c)


def op_aniso_lap(S):
    """tr(S H(w)) = S11 w_xx + 2 S12 w_xy + S22 w_yy, the Laplacian of Example 5.2."""
    ops = {(2, 0): S[0], (1, 1): 2.0 * S[1], (0, 2): S[2]}
    return {k: c for k, c in ops.items() if c != 0.0}


@dataclasses.dataclass(frozen=True)
class Equation:
    """order = 4: Delta^2 u = f (Example 5.1), or with S != I the anisotropic S_ij S_kl u_,ijkl = f
    of Example 5.2 (Delta w replaced by tr(S H(w)), grad w . n by grad w . (S n)); order = 6:
    -Delta^3 u = f (Example 5.4)."""
    order: int
    S: tuple = ISOTROPIC

    def __post_init__(self):
        if self.order != 4 and tuple(self.S) != ISOTROPIC:
            raise ValueError("anisotropy is defined for the biharmonic equation only (Example 5.2)")

    def lap(self):
        return OP_LAP if tuple(self.S) == ISOTROPIC else op_aniso_lap(self.S)

    def conormal(self, n):
        """S n (n itself when isotropic)."""
        if tuple(self.S) == ISOTROPIC:
            return n
        return (self.S[0] * n[0] + self.S[1] * n[1], self.S[1] * n[0] + self.S[2] * n[1])

    def interior_pairs(self):
        """Pairs (op on v, op on u, coefficient) of the domain integral of a_n(v, u)."""
        if self.order == 4:
            L = self.lap()
            return [(L, L, 1.0)]
        gl = (op_dx(OP_LAP), op_dy(OP_LAP))
        return [(gl[0], gl[0], 1.0), (gl[1], gl[1], 1.0)]

    def boundary_pairs(self, n, gamma):
        """Pairs (op on v, op on u, coefficient) of the boundary integrals of a_n(v, u)."""
        if self.order == 4:
            L, sn = self.lap(), self.conormal(n)
            dn = op_dn(OP_I, sn)
            dnlap = op_dn(L, sn)
            return [(OP_I, OP_I, gamma[0]), (OP_I, dnlap, 1.0), (dnlap, OP_I, 1.0),
                    (dn, dn, gamma[1]), (dn, L, -1.0), (L, dn, -1.0)]
        dn = op_dn(OP_I, n)
        dnlap = op_dn(OP_LAP, n)
        dnbil = op_dn(OP_BILAP, n)
        return [(OP_I, OP_I, gamma[0]), (OP_I, dnbil, -1.0), (dnbil, OP_I, -1.0),
                (dn, dn, gamma[1]), (dn, OP_BILAP, 1.0), (OP_BILAP, dn, 1.0),
                (OP_LAP, OP_LAP, gamma[2]), (OP_LAP, dnlap, -1.0), (dnlap, OP_LAP, -1.0)]

    def load_boundary_terms(self, n, gamma):
        """(index of boundary datum g_j, op on v, coefficient) of l_n(v)."""
        if self.order == 4:
            L, sn = self.lap(), self.conormal(n)
            return [(0, OP_I, gamma[0]), (0, op_dn(L, sn), 1.0),
                    (1, op_dn(OP_I, sn), gamma[1]), (1, L, -1.0)]
        dn = op_dn(OP_I, n)
        return [(0, OP_I, gamma[0]), (0, op_dn(OP_BILAP, n), -1.0),
                (1, dn, gamma[1]), (1, OP_BILAP, 1.0),
                (2, OP_LAP, gamma[2]), (2, op_dn(OP_LAP, n), -1.0)]


# Constants C_j of the Nitsche penalties gamma^(j) = C_j (p+1)^2 h^-(order-1-2j).  The paper
# only asks for "large enough" penalties; these are the smallest round values for which
# the assembled matrices are SPD on levels m = 2..16 (checked by dense eigenvalues).
NITSCHE_CONSTANTS = {4: (4.0, 2.0), 6: (1.0e4, 1.0e2, 1.0)}


def nitsche_gamma(order: int, p: int, m: int, constants=None, S=ISOTROPIC) -> list[float]:
    """Penalties gamma^(j) = C_j (p+1)^2 h^-(order-1-2j), j < order/2 (Examples 5.1, 5.4).

    Anisotropic biharmonic (Example 5.2): the consistency terms int v grad(tr(S H u)) . (S n)
    carry |S|^2 against the penalty int gamma^(0) u v, so gamma^(0) is scaled by |S|_2^2 (the
    penalty on grad u . (S n) already carries S)."""
    h = 1.0 / m
    C = NITSCHE_CONSTANTS[order] if constants is None else constants
    g = [C[j] * (p + 1) ** 2 * h ** (-(order - 1 - 2 * j)) for j in range(order // 2)]
    if tuple(S) != ISOTROPIC:
        g[0] *= float(np.max(np.linalg.eigvalsh(np.array([[S[0], S[1]], [S[1], S[2]]])))) ** 2
    return g


# ---------------------------------------------------------------------------
# Basis evaluation on tensor point sets
# ---------------------------------------------------------------------------

class _Tables1D:
    """Cache of X_{a,j}^{(r)} at the Gauss points of each 1-D sub-interval."""

    def __init__(self, m: int, p: int, pts: np.ndarray, rmax: int):
        self.m, self.p, self.rmax = m, p, rmax
        self.pts = pts
        self.cache = {}

    def get(self, a: int) -> np.ndarray:
        if a not in self.cache:
            t = np.empty((self.p + 1, self.rmax + 1, len(self.pts)))
            for j in range(self.p + 1):
                for r in range(self.rmax + 1):
                    t[j, r] = factor_1d(self.m, a, j, self.pts, r)
            self.cache[a] = t
        return self.cache[a]


def _op_values(op, exps, TX: np.ndarray, TY: np.ndarray) -> np.ndarray:
    """(Op psi_k)(x_q, y_r) for every basis k, flattened over the tensor points (q-major)."""
    d = len(exps)
    out = np.zeros((d, TX.shape[2] * TY.shape[2]))
    for k, (ja, jb) in enumerate(exps):
        acc = 0.0
        for (al, be), c in op.items():
            acc = acc + c * np.outer(TX[ja, al], TY[jb, be])
        out[k] = np.ravel(acc)
    return out


def fourier_source(coef: np.ndarray, decay: float):
    """f(x,y) = sum_ab c_ab (a^2 + b^2)^(-decay/2) sin(a pi x) sin(b pi y)."""
    K = coef.shape[0]
    a = np.arange(1, K + 1)
    scale = (a[:, None] ** 2 + a[None, :] ** 2) ** (-decay / 2.0)
    cs = coef * scale

    def f(x, y):
        sx = np.sin(np.pi * np.outer(a, x))  # (K, n)
        sy = np.sin(np.pi * np.outer(a, y))
        return np.einsum("ab,an,bn->n", cs, sx, sy)
    return f


@dataclasses.dataclass
class Assembled:
    A: bk.BlockCSR
    b: np.ndarray
    M: bk.BlockCSR
    gamma: list


def assemble(m: int, p: int, order: int, gamma, f=None, g=None, q: int | None = None,
             with_mass: bool = True, rows=None, S=ISOTROPIC) -> Assembled:
    """Stiffness A, load b and mass matrix M of the PUM space of level m.

    f(x, y) is the source, g = [g0, g1, (g2)] the boundary data (callables of
    x, y on the boundary), both default to zero.  q = Gauss points per
    direction on each sub-cell (default p + 6, exact for the PU-polynomial
    integrands of both equations).  rows: only these block rows are assembled
    (the other rows of A, M and b stay empty / zero).
    """
    keep = None if rows is None else set(int(r) for r in rows)
    eq = Equation(order, tuple(S))
    d = local_dim(p)
    exps = basis_exponents(p)
    q = q or p + 6
    gx, gw = npleg.leggauss(q)
    bp = breakpoints_1d(m)
    n = m * m
    rmax = order - 1  # highest derivative in one direction on the boundary
    ent = {}
    ment = {}
    bvec = np.zeros(n * d)

    def add(store, i, j, blk):
        if (i, j) in store:
            store[(i, j)] += blk
        else:
            store[(i, j)] = blk.copy()

    subs = []
    for s in range(len(bp) - 1):
        lo, hi = bp[s], bp[s + 1]
        pts = 0.5 * (hi - lo) * gx + 0.5 * (hi + lo)
        wts = 0.5 * (hi - lo) * gw
        subs.append((pts, wts, active_1d(m, lo, hi), _Tables1D(m, p, pts, rmax)))

    ipairs = eq.interior_pairs()
    # domain integrals
    for (px, wx, ax_list, tx) in subs:
        for (py, wy, ay_list, ty) in subs:
            W = np.ravel(np.outer(wx, wy))
            X, Y = np.meshgrid(px, py, indexing="ij")
            X, Y = np.ravel(X), np.ravel(Y)
            patches = [(ax, ay) for ay in ay_list for ax in ax_list]
            if keep is not None and not any(pp[1] * m + pp[0] in keep for pp in patches):
                continue
            vals = {}
            for (ax, ay) in patches:
                TX, TY = tx.get(ax), ty.get(ay)
                vals[(ax, ay)] = ([(_op_values(ov, exps, TX, TY), _op_values(ou, exps, TX, TY), c)
                                   for (ov, ou, c) in ipairs],
                                  _op_values(OP_I, exps, TX, TY))
            fv = f(X, Y) if f is not None else None
            for pi in patches:
                i = pi[1] * m + pi[0]
                if keep is not None and i not in keep:
                    continue
                psi_i = vals[pi][1]
                if fv is not None:
                    bvec[i * d:(i + 1) * d] += psi_i @ (W * fv)
                for pj in patches:
                    j = pj[1] * m + pj[0]
                    blk = np.zeros((d, d))
                    for (vi, _, c), (_, uj, _) in zip(vals[pi][0], vals[pj][0]):
                        blk += c * (vi * W) @ uj.T
                    add(ent, i, j, blk)
                    if with_mass:
                        add(ment, i, j, (psi_i * W) @ vals[pj][1].T)

    # boundary integrals: four edges of the unit square
    edges = [((-1.0, 0.0), 0, 0.0), ((1.0, 0.0), 0, 1.0), ((0.0, -1.0), 1, 0.0), ((0.0, 1.0), 1, 1.0)]
    for nvec, axis, val in edges:
        bpairs = eq.boundary_pairs(nvec, gamma)
        lterms = eq.load_boundary_terms(nvec, gamma)
        fixed = [a for a in range(m) if patch_box_1d(m, a)[0] <= val <= patch_box_1d(m, a)[1]]
        pt = np.array([val])
        for (ps, ws, along_list, tab) in subs:
            if keep is not None and not any(((ai * m + af) if axis == 0 else (af * m + ai)) in keep
                                            for ai in along_list for af in fixed):
                continue
            for af in fixed:
                Tfix = np.empty((p + 1, rmax + 3, 1))
                for j in range(p + 1):
                    for r in range(rmax + 3):
                        Tfix[j, r] = factor_1d(m, af, j, pt, r)
                Talong = {}
                for aa in along_list:
                    t = np.empty((p + 1, rmax + 3, len(ps)))
                    for j in range(p + 1):
                        for r in range(rmax + 3):
                            t[j, r] = factor_1d(m, aa, j, ps, r)
                    Talong[aa] = t

                def opv(op, aa):
                    if axis == 0:
                        return _op_values(op, exps, Tfix, Talong[aa])
                    return _op_values(op, exps, Talong[aa], Tfix)

                for ai in along_list:
                    i = (ai * m + af) if axis == 0 else (af * m + ai)
                    if keep is not None and i not in keep:
                        continue
                    if g is not None:
                        xs = np.full_like(ps, val) if axis == 0 else ps
                        ys = ps if axis == 0 else np.full_like(ps, val)
                        for (gi, ov, c) in lterms:
                            gv = g[gi](xs, ys)
                            bvec[i * d:(i + 1) * d] += c * opv(ov, ai) @ (ws * gv)
                    for aj in along_list:
                        j = (aj * m + af) if axis == 0 else (af * m + aj)
                        blk = np.zeros((d, d))
                        for (ov, ou, c) in bpairs:
                            blk += c * (opv(ov, ai) * ws) @ opv(ou, aj).T
                        add(ent, i, j, blk)

    A = bk.from_blocks(n, n, d, ent)
    M = bk.from_blocks(n, n, d, ment) if with_mass else None
    return Assembled(A, bvec, M, list(gamma))


# ---------------------------------------------------------------------------
# Evaluation of PUM functions, interpolation of polynomials
# ---------------------------------------------------------------------------

def evaluate(m: int, p: int, coef: np.ndarray, x: np.ndarray, y: np.ndarray,
             op=OP_I) -> np.ndarray:
    """(Op u)(x, y) for u = sum_i phi_i sum_k coef_(i,k) theta_i^k."""
    exps = basis_exponents(p)
    d = len(exps)
    rmax = max_order(op)
    out = np.zeros(len(x))
    for iy in range(m):
        for ix in range(m):
            i = iy * m + ix
            TX = np.array([[factor_1d(m, ix, j, x, r) for r in range(rmax + 1)] for j in range(p + 1)])
            TY = np.array([[factor_1d(m, iy, j, y, r) for r in range(rmax + 1)] for j in range(p + 1)])
            for k, (ja, jb) in enumerate(exps):
                c = coef[i * d + k]
                if c == 0.0:
                    continue
                for (al, be), cc in op.items():
                    out += c * cc * TX[ja, al] * TY[jb, be]
    return out


def local_projection(m: int, p: int, func, q: int = 12) -> np.ndarray:
    """Coefficients of each patch's L2 projection of func onto V_i over omega_i cap Omega.

    For a polynomial of degree <= p the projection reproduces it exactly.
    """
    exps = basis_exponents(p)
    d = len(exps)
    gx, gw = npleg.leggauss(q)
    out = np.zeros(m * m * d)
    for iy in range(m):
        for ix in range(m):
            x0, x1 = patch_box_1d(m, ix)
            y0, y1 = patch_box_1d(m, iy)
            px = 0.5 * (x1 - x0) * gx + 0.5 * (x1 + x0)
            py = 0.5 * (y1 - y0) * gx + 0.5 * (y1 + y0)
            W = np.ravel(np.outer(0.5 * (x1 - x0) * gw, 0.5 * (y1 - y0) * gw))
            X, Y = np.meshgrid(px, py, indexing="ij")
            X, Y = np.ravel(X), np.ravel(Y)
            th = np.array([np.ravel(np.outer(local_poly_1d(m, ix, a, px, 0), local_poly_1d(m, iy, b, py, 0)))
                           for (a, b) in exps])
            Mi = (th * W) @ th.T
            rhs = th @ (W * func(X, Y))
            i = iy * m + ix
            out[i * d:(i + 1) * d] = np.linalg.solve(Mi, rhs)
    return out


# ---------------------------------------------------------------------------
# Transfers and Galerkin hierarchy
# ---------------------------------------------------------------------------

def prolongation(m_f: int, p: int, q: int | None = None, rows=None) -> bk.BlockCSR:
    """P: V_{l-1} -> V_l by global-to-local L2 projection (Section 4).

    Block (i, j) = M_i^{-1} B_ij with M_i = int_{omega_i cap Omega} theta_i theta_i^T and
    B_ij = int_{omega_i cap Omega} theta_i (phi_j^c theta_j^c)^T, integrated over the
    sub-cells of the fine box cut at all fine and coarse PU breakpoints.
    """
    assert m_f % 2 == 0
    m_c = m_f // 2
    exps = basis_exponents(p)
    d = len(exps)
    q = q or p + 6
    gx, gw = npleg.leggauss(q)
    cuts = np.union1d(breakpoints_1d(m_f), breakpoints_1d(m_c))

    # 1-D pieces of each fine box: points, weights, fine Legendre values, coarse factor values
    def pieces(a):
        lo, hi = patch_box_1d(m_f, a)
        grid = [lo] + [c for c in cuts if lo < c < hi] + [hi]
        out = []
        for u in range(len(grid) - 1):
            pts = 0.5 * (grid[u + 1] - grid[u]) * gx + 0.5 * (grid[u + 1] + grid[u])
            wts = 0.5 * (grid[u + 1] - grid[u]) * gw
            th = np.array([local_poly_1d(m_f, a, j, pts, 0) for j in range(p + 1)])
            co = {c: np.array([factor_1d(m_c, c, j, pts, 0) for j in range(p + 1)])
                  for c in active_1d(m_c, grid[u], grid[u + 1])}
            out.append((wts, th, co))
        return out

    keep = None if rows is None else set(int(r) for r in rows)
    need = range(m_f) if keep is None else sorted({r % m_f for r in keep} | {r // m_f for r in keep})
    pcs = {a: pieces(a) for a in need}
    ent = {}
    for iy in range(m_f):
        for ix in range(m_f):
            i = iy * m_f + ix
            if keep is not None and i not in keep:
                continue
            Mi = np.zeros((d, d))
            Bs = {}
            for (wx, thx, cox) in pcs[ix]:
                for (wy, thy, coy) in pcs[iy]:
                    W = np.ravel(np.outer(wx, wy))
                    th = np.array([np.ravel(np.outer(thx[a], thy[b])) for (a, b) in exps])
                    Mi += (th * W) @ th.T
                    for jy, Ty in coy.items():
                        for jx, Tx in cox.items():
                            j = jy * m_c + jx
                            psi = np.array([np.ravel(np.outer(Tx[a], Ty[b])) for (a, b) in exps])
                            Bs[j] = Bs.get(j, 0.0) + (th * W) @ psi.T
            for j, B in Bs.items():
                ent[(i, j)] = np.linalg.solve(Mi, B)
    return bk.from_blocks(m_f * m_f, m_c * m_c, d, ent)


@dataclasses.dataclass
class Hierarchy:
    """Levels ordered finest first: A[0] finest, P[l] maps level l+1 -> level l."""
    m: list
    A: list
    P: list
    b: np.ndarray
    M: bk.BlockCSR | None
    gamma: list


def build_hierarchy(m: int, p: int, order: int, n_levels: int, f=None, with_mass: bool = False,
                    constants=None, S=ISOTROPIC) -> Hierarchy:
    """Finest-level assembly plus Galerkin coarse operators A_{l-1} = P^T A_l P (Section 5)."""
    gamma = nitsche_gamma(order, p, m, constants, S)
    asm = assemble(m, p, order, gamma, f=f, with_mass=with_mass, S=S)
    ms, As, Ps = [m], [asm.A], []
    for _ in range(n_levels - 1):
        P = prolongation(ms[-1], p)
        Ac = bk.galerkin_product(P.transpose(), As[-1], P)
        Ps.append(P)
        As.append(Ac)
        ms.append(ms[-1] // 2)
    return Hierarchy(ms, As, Ps, asm.b, asm.M, gamma)


def dof_count(level: int, p: int, p_boundary: int | None = None, dim: int = 2) -> int:
    """Number of unknowns of the uniform level-l cover in dimension dim (Example 5.1 / 5.3).

    Patches whose support meets the boundary use degree p_boundary when given.
    """
    m = 2 ** level
    n_total = m ** dim
    n_inner = max(m - 2, 0) ** dim
    pb = p if p_boundary is None else p_boundary
    return (n_total - n_inner) * comb(pb + dim, dim) + n_inner * comb(p + dim, dim)
