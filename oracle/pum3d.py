"""Partition-of-unity discretisation of the biharmonic equation on the unit cube (Example 5.3).

Test infrastructure only: imported by tests, never by the CUDA library.

The cover, partition of unity and local spaces are those of the square (Section 4, module
``oracle.pum``) taken in three directions:

* patch (ix, iy, iz) of a level with m patches per side is the product of the clipped 1-D
  patches, block index i = (iz m + iy) m + ix; its PU function is phi_ix(x) phi_iy(y) phi_iz(z);
* the local space is the polynomials of total degree <= p, written in tensor Legendre
  polynomials P_a P_b P_c on the patch box mapped to [-1, 1]^3, ordered by total degree and then
  by (c, b); dim V_i = binom(p+3, 3), 20 at the paper's p = 3 (Example 5.3);
* the stiffness matrix and load vector are the Nitsche forms of the biharmonic equation of
  Example 5.1 with the boundary integrals over the six faces of the cube:
  a_n(v, u) = int Delta v Delta u
            + sum over faces of int gamma0 v u + v d_n(Delta u) + d_n(Delta v) u
                                 + gamma1 d_n v d_n u - d_n v Delta u - Delta v d_n u,
  l_n(v)    = int f v + sum over faces of int gamma0 g0 v + g0 d_n(Delta v)
                                          + gamma1 g1 d_n v - g1 Delta v,
  with the penalties gamma^(j) = C_j (p+1)^2 h^-(3-2j) of the square.

Integrals are tensor Gauss-Legendre rules with q points per direction on every sub-cell of the
grid of PU breakpoints (brute force, as in the 2-D module).
"""
from __future__ import annotations

import dataclasses
from math import comb

import numpy as np
from numpy.polynomial import legendre as npleg

from . import blocks as bk
from .pum import NITSCHE_CONSTANTS, active_1d, breakpoints_1d, factor_1d, legendre, patch_box_1d

# Differential operators as {(alpha, beta, gamma): coefficient}, d^alpha/dx d^beta/dy d^gamma/dz.
OP_I = {(0, 0, 0): 1.0}
OP_LAP = {(2, 0, 0): 1.0, (0, 2, 0): 1.0, (0, 0, 2): 1.0}


def local_dim(p: int) -> int:
    """dim V_i = binom(p+3, 3) (Example 5.3)."""
    return comb(p + 3, 3)


def basis_exponents(p: int) -> list[tuple[int, int, int]]:
    """Legendre degrees (a, b, c), a + b + c <= p, by total degree, then by c, then by b."""
    return [(s - b - c, b, c) for s in range(p + 1) for c in range(s + 1) for b in range(s - c + 1)]


def op_d(op, axis: int):
    """The derivative along `axis` applied after op."""
    out = {}
    for k, c in op.items():
        kk = list(k)
        kk[axis] += 1
        out[tuple(kk)] = out.get(tuple(kk), 0.0) + c
    return out


def op_dn(op, n):
    """Normal derivative n . grad applied after op."""
    out = {}
    for axis in range(3):
        if n[axis] == 0.0:
            continue
        for k, c in op_d(op, axis).items():
            out[k] = out.get(k, 0.0) + n[axis] * c
    return {k: c for k, c in out.items() if c != 0.0}


def boundary_pairs(n, gamma):
    """(op on v, op on u, coefficient) of the face integrals of a_n(v, u) (Example 5.1's form)."""
    dn = op_dn(OP_I, n)
    dnlap = op_dn(OP_LAP, n)
    return [(OP_I, OP_I, gamma[0]), (OP_I, dnlap, 1.0), (dnlap, OP_I, 1.0),
            (dn, dn, gamma[1]), (dn, OP_LAP, -1.0), (OP_LAP, dn, -1.0)]


def load_boundary_terms(n, gamma):
    """(index of the boundary datum g_j, op on v, coefficient) of the face integrals of l_n(v)."""
    return [(0, OP_I, gamma[0]), (0, op_dn(OP_LAP, n), 1.0),
            (1, op_dn(OP_I, n), gamma[1]), (1, OP_LAP, -1.0)]


def nitsche_gamma(p: int, m: int, constants=None) -> list[float]:
    """gamma^(j) = C_j (p+1)^2 h^-(3-2j), j = 0, 1, with the square's constants by default."""
    h = 1.0 / m
    C = NITSCHE_CONSTANTS[4] if constants is None else constants
    return [C[j] * (p + 1) ** 2 * h ** (-(3 - 2 * j)) for j in range(2)]


def _tables(m: int, p: int, a: int, pts: np.ndarray, rmax: int) -> np.ndarray:
    """[j, r, point]: r-th derivative of phi_a(x) P_j(xi(x)) at the points."""
    t = np.empty((p + 1, rmax + 1, len(pts)))
    for j in range(p + 1):
        for r in range(rmax + 1):
            t[j, r] = factor_1d(m, a, j, pts, r)
    return t


def _op_values(op, exps, TX, TY, TZ) -> np.ndarray:
    """(Op psi_k) at the tensor points (x-major, then y, then z) for every local basis function k."""
    d = len(exps)
    out = np.zeros((d, TX.shape[2] * TY.shape[2] * TZ.shape[2]))
    for k, (ja, jb, jc) in enumerate(exps):
        acc = 0.0
        for (al, be, ga), c in op.items():
            acc = acc + c * np.einsum("i,j,k->ijk", TX[ja, al], TY[jb, be], TZ[jc, ga])
        out[k] = np.ravel(acc)
    return out


@dataclasses.dataclass
class Assembled3:
    A: bk.BlockCSR
    b: np.ndarray
    gamma: list


def assemble(m: int, p: int, gamma, f=None, g=None, q: int | None = None) -> Assembled3:
    """Stiffness A and load b of the PUM space of level m on the unit cube.

    f(x, y, z) is the source, g = [g0, g1] the boundary data (callables of x, y, z on the
    boundary), both default to zero.  q = Gauss points per direction on each sub-cell (default
    p + 6, exact for the PU-polynomial integrands).
    """
    exps = basis_exponents(p)
    d = len(exps)
    q = q or p + 6
    gx, gw = npleg.leggauss(q)
    bp = breakpoints_1d(m)
    n = m ** 3
    rmax = 3  # d_n(Delta u) on the faces
    ent = {}
    bvec = np.zeros(n * d)

    def add(i, j, blk):
        if (i, j) in ent:
            ent[(i, j)] += blk
        else:
            ent[(i, j)] = blk.copy()

    def index(a):
        return (a[2] * m + a[1]) * m + a[0]

    subs = []
    for s in range(len(bp) - 1):
        lo, hi = bp[s], bp[s + 1]
        pts = 0.5 * (hi - lo) * gx + 0.5 * (hi + lo)
        wts = 0.5 * (hi - lo) * gw
        act = active_1d(m, lo, hi)
        subs.append((pts, wts, act, {a: _tables(m, p, a, pts, rmax) for a in act}))

    # domain integrals
    for (px, wx, axl, tx) in subs:
        for (py, wy, ayl, ty) in subs:
            for (pz, wz, azl, tz) in subs:
                W = np.ravel(np.einsum("i,j,k->ijk", wx, wy, wz))
                X, Y, Z = (np.ravel(v) for v in np.meshgrid(px, py, pz, indexing="ij"))
                patches = [(ax, ay, az) for az in azl for ay in ayl for ax in axl]
                vals = {a: (_op_values(OP_LAP, exps, tx[a[0]], ty[a[1]], tz[a[2]]),
                            _op_values(OP_I, exps, tx[a[0]], ty[a[1]], tz[a[2]])) for a in patches}
                fv = f(X, Y, Z) if f is not None else None
                for ai in patches:
                    i = index(ai)
                    if fv is not None:
                        bvec[i * d:(i + 1) * d] += vals[ai][1] @ (W * fv)
                    for aj in patches:
                        add(i, index(aj), (vals[ai][0] * W) @ vals[aj][0].T)

    # face integrals: x = 0, 1; y = 0, 1; z = 0, 1
    for axis in range(3):
        others = [t for t in range(3) if t != axis]
        for val, sign in ((0.0, -1.0), (1.0, 1.0)):
            nvec = [0.0, 0.0, 0.0]
            nvec[axis] = sign
            bpairs = boundary_pairs(nvec, gamma)
            lterms = load_boundary_terms(nvec, gamma)
            fixed = [a for a in range(m) if patch_box_1d(m, a)[0] <= val <= patch_box_1d(m, a)[1]]
            tfix = {a: _tables(m, p, a, np.array([val]), rmax) for a in fixed}
            for (pu, wu, aul, tu) in subs:
                for (pv, wv, avl, tv) in subs:
                    W = np.ravel(np.outer(wu, wv))
                    U, V = (np.ravel(v) for v in np.meshgrid(pu, pv, indexing="ij"))
                    coords = [None, None, None]
                    coords[axis] = np.full_like(U, val)
                    coords[others[0]], coords[others[1]] = U, V
                    patches = []
                    for af in fixed:
                        for au in aul:
                            for av in avl:
                                a = [0, 0, 0]
                                a[axis], a[others[0]], a[others[1]] = af, au, av
                                patches.append(tuple(a))

                    def tabs(a):
                        t = [None, None, None]
                        t[axis] = tfix[a[axis]]
                        t[others[0]] = tu[a[others[0]]]
                        t[others[1]] = tv[a[others[1]]]
                        return t

                    cache = {}

                    def opv(op, a):
                        # tensor order of the points: the fixed axis has one point, so the
                        # flattening follows (others[0], others[1]) as U, V do
                        key = (tuple(sorted(op.items())), a)
                        if key not in cache:
                            cache[key] = _op_values(op, exps, *tabs(a))
                        return cache[key]

                    for ai in patches:
                        i = index(ai)
                        if g is not None:
                            for (gi, ov, c) in lterms:
                                bvec[i * d:(i + 1) * d] += c * opv(ov, ai) @ (W * g[gi](*coords))
                        for aj in patches:
                            blk = np.zeros((d, d))
                            for (ov, ou, c) in bpairs:
                                blk += c * (opv(ov, ai) * W) @ opv(ou, aj).T
                            add(i, index(aj), blk)

    return Assembled3(bk.from_blocks(n, n, d, ent), bvec, list(gamma))


def local_projection(m: int, p: int, func, q: int = 10) -> np.ndarray:
    """Coefficients of each patch's L2 projection of func onto V_i over its box (omega_i cap Omega).

    The tensor Legendre basis is orthogonal on the box, so each coefficient is an integral over
    the box divided by the squared norm; a polynomial of degree <= p is reproduced exactly.
    """
    exps = basis_exponents(p)
    d = len(exps)
    gx, gw = npleg.leggauss(q)
    out = np.zeros(m ** 3 * d)
    XI, ETA, ZETA = (np.ravel(v) for v in np.meshgrid(gx, gx, gx, indexing="ij"))  # reference points
    for iz in range(m):
        for iy in range(m):
            for ix in range(m):
                boxes = [patch_box_1d(m, a) for a in (ix, iy, iz)]
                pts = [0.5 * (hi - lo) * gx + 0.5 * (hi + lo) for lo, hi in boxes]
                X, Y, Z = (np.ravel(v) for v in np.meshgrid(*pts, indexing="ij"))
                W = np.ravel(np.einsum("i,j,k->ijk", *[0.5 * (hi - lo) * gw for lo, hi in boxes]))
                fv = func(X, Y, Z)
                i = (iz * m + iy) * m + ix
                for k, (a, b, c) in enumerate(exps):
                    L = legendre(a, XI, 0) * legendre(b, ETA, 0) * legendre(c, ZETA, 0)
                    norm = np.prod([(hi - lo) / (2 * e + 1) for (lo, hi), e in zip(boxes, (a, b, c))])
                    out[i * d + k] = np.sum(W * fv * L) / norm
    return out


def prolongation(m_f: int, p: int, q: int | None = None) -> bk.BlockCSR:
    """P: V_{l-1} -> V_l by global-to-local L2 projection (Section 4), on the cube.

    Block (i, j) = M_i^{-1} B_ij with M_i = int_{omega_i cap Omega} theta_i theta_i^T and
    B_ij = int_{omega_i cap Omega} theta_i (phi_j^c theta_j^c)^T, integrated over the sub-cells of
    the fine box cut at all fine and coarse PU breakpoints.
    """
    assert m_f % 2 == 0
    m_c = m_f // 2
    exps = basis_exponents(p)
    d = len(exps)
    q = q or p + 6
    gx, gw = npleg.leggauss(q)
    cuts = np.union1d(breakpoints_1d(m_f), breakpoints_1d(m_c))

    def pieces(a):  # 1-D pieces of fine box a: weights, fine Legendre values, coarse factor values
        lo, hi = patch_box_1d(m_f, a)
        grid = [lo] + [c for c in cuts if lo < c < hi] + [hi]
        out = []
        for u in range(len(grid) - 1):
            pts = 0.5 * (grid[u + 1] - grid[u]) * gx + 0.5 * (grid[u + 1] + grid[u])
            wts = 0.5 * (grid[u + 1] - grid[u]) * gw
            xi = (2.0 * pts - lo - hi) / (hi - lo)
            th = np.array([legendre(j, xi, 0) for j in range(p + 1)])
            co = {c: np.array([factor_1d(m_c, c, j, pts, 0) for j in range(p + 1)])
                  for c in active_1d(m_c, grid[u], grid[u + 1])}
            out.append((wts, th, co))
        return out

    pcs = {a: pieces(a) for a in range(m_f)}
    ent = {}
    for iz in range(m_f):
        for iy in range(m_f):
            for ix in range(m_f):
                i = (iz * m_f + iy) * m_f + ix
                Mi = np.zeros((d, d))
                Bs = {}
                for (wx, thx, cox) in pcs[ix]:
                    for (wy, thy, coy) in pcs[iy]:
                        for (wz, thz, coz) in pcs[iz]:
                            W = np.ravel(np.einsum("i,j,k->ijk", wx, wy, wz))
                            th = np.array([np.ravel(np.einsum("i,j,k->ijk", thx[a], thy[b], thz[c]))
                                           for (a, b, c) in exps])
                            Mi += (th * W) @ th.T
                            for jz, Tz in coz.items():
                                for jy, Ty in coy.items():
                                    for jx, Tx in cox.items():
                                        j = (jz * m_c + jy) * m_c + jx
                                        psi = np.array([np.ravel(np.einsum("i,j,k->ijk", Tx[a], Ty[b], Tz[c]))
                                                        for (a, b, c) in exps])
                                        Bs[j] = Bs.get(j, 0.0) + (th * W) @ psi.T
                for j, B in Bs.items():
                    ent[(i, j)] = np.linalg.solve(Mi, B)
    return bk.from_blocks(m_f ** 3, m_c ** 3, d, ent)


@dataclasses.dataclass
class Hierarchy3:
    """Levels ordered finest first: A[0] finest, P[l] maps level l+1 -> level l."""
    m: list
    A: list
    P: list
    b: np.ndarray
    gamma: list


def build_hierarchy(m: int, p: int, n_levels: int, f=None, constants=None) -> Hierarchy3:
    """Finest-level assembly on the cube plus Galerkin coarse operators A_{l-1} = P^T A_l P
    (Section 5)."""
    gamma = nitsche_gamma(p, m, constants)
    asm = assemble(m, p, gamma, f=f)
    ms, As, Ps = [m], [asm.A], []
    for _ in range(n_levels - 1):
        P = prolongation(ms[-1], p)
        As.append(bk.galerkin_product(P.transpose(), As[-1], P))
        Ps.append(P)
        ms.append(ms[-1] // 2)
    return Hierarchy3(ms, As, Ps, asm.b, gamma)
