"""PUM space of the square with the local degree raised on boundary patches (Example 5.1).

Test infrastructure only: imported by tests, never by the CUDA library.

Example 5.1 uses local polynomials of degree p = 2 in the interior and raises them to degree 3 on
the patches whose support meets the boundary.  Everything else is the construction of the
``oracle.pum`` module (cover, partition of unity, tensor Legendre bases on the clipped patch
boxes, Nitsche forms of the biharmonic equation); only the local dimension now varies with the
patch: d_i = binom(p_i + 2, 2) with p_i the raised degree on boundary patches.  The unknowns of
patch i are the d_i consecutive entries starting at offsets[i], patches in the order
i = iy m + ix.  The penalties are those of the raised degree, which is the degree of every
function that has a trace on the boundary.

Matrices are returned as dense block dictionaries {(i, j): d_i x d_j} and as scipy CSR matrices
over the scalar unknowns.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.sparse as sps
from numpy.polynomial import legendre as npleg

from .pum import (OP_I, Equation, _op_values, _Tables1D, active_1d, basis_exponents, breakpoints_1d, factor_1d,
                  local_dim, local_poly_1d, nitsche_gamma, patch_box_1d)


def patch_degrees(m: int, p: int, p_boundary: int) -> list[int]:
    """Local degree of every patch (i = iy m + ix): p_boundary when its support meets the
    boundary (first or last patch in x or y), p otherwise."""
    return [p_boundary if (ix in (0, m - 1) or iy in (0, m - 1)) else p for iy in range(m) for ix in range(m)]


def offsets(degrees: list[int]) -> np.ndarray:
    """Start of each patch's unknowns; the last entry is the number of unknowns."""
    return np.concatenate([[0], np.cumsum([local_dim(q) for q in degrees])]).astype(np.int64)


@dataclasses.dataclass
class AssembledRaised:
    degrees: list
    off: np.ndarray
    blocks: dict  # (i, j) -> d_i x d_j
    A: sps.csr_matrix
    b: np.ndarray
    gamma: list


def _to_csr(blocks: dict, off: np.ndarray) -> sps.csr_matrix:
    rows, cols, vals = [], [], []
    for (i, j), B in blocks.items():
        r, c = np.meshgrid(np.arange(off[i], off[i + 1]), np.arange(off[j], off[j + 1]), indexing="ij")
        rows.append(r.ravel())
        cols.append(c.ravel())
        vals.append(B.ravel())
    n = int(off[-1])
    return sps.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))


def assemble(m: int, p: int, p_boundary: int, f=None, g=None, q: int | None = None,
             constants=None) -> AssembledRaised:
    """Stiffness and load of the biharmonic equation (Example 5.1) in the raised space of level m."""
    eq = Equation(4)
    gamma = nitsche_gamma(4, p_boundary, m, constants)
    degs = patch_degrees(m, p, p_boundary)
    off = offsets(degs)
    pmax = max(p, p_boundary)
    exps = {q_: basis_exponents(q_) for q_ in set(degs)}
    q = q or pmax + 6
    gx, gw = npleg.leggauss(q)
    bp = breakpoints_1d(m)
    rmax = 3
    ent = {}
    bvec = np.zeros(int(off[-1]))

    def add(i, j, blk):
        if (i, j) in ent:
            ent[(i, j)] += blk
        else:
            ent[(i, j)] = blk.copy()

    subs = []
    for s in range(len(bp) - 1):
        lo, hi = bp[s], bp[s + 1]
        pts = 0.5 * (hi - lo) * gx + 0.5 * (hi + lo)
        wts = 0.5 * (hi - lo) * gw
        subs.append((pts, wts, active_1d(m, lo, hi), _Tables1D(m, pmax, pts, rmax)))

    ipairs = eq.interior_pairs()
    for (px, wx, axl, tx) in subs:
        for (py, wy, ayl, ty) in subs:
            W = np.ravel(np.outer(wx, wy))
            X, Y = (np.ravel(v) for v in np.meshgrid(px, py, indexing="ij"))
            patches = [(ax, ay) for ay in ayl for ax in axl]
            vals = {}
            for (ax, ay) in patches:
                e = exps[degs[ay * m + ax]]
                TX, TY = tx.get(ax), ty.get(ay)
                vals[(ax, ay)] = ([(_op_values(ov, e, TX, TY), _op_values(ou, e, TX, TY), c) for (ov, ou, c) in ipairs],
                                  _op_values(OP_I, e, TX, TY))
            fv = f(X, Y) if f is not None else None
            for pi in patches:
                i = pi[1] * m + pi[0]
                if fv is not None:
                    bvec[off[i]:off[i + 1]] += vals[pi][1] @ (W * fv)
                for pj in patches:
                    j = pj[1] * m + pj[0]
                    blk = np.zeros((off[i + 1] - off[i], off[j + 1] - off[j]))
                    for (vi, _, c), (_, uj, _) in zip(vals[pi][0], vals[pj][0]):
                        blk += c * (vi * W) @ uj.T
                    add(i, j, blk)

    edges = [((-1.0, 0.0), 0, 0.0), ((1.0, 0.0), 0, 1.0), ((0.0, -1.0), 1, 0.0), ((0.0, 1.0), 1, 1.0)]
    for nvec, axis, val in edges:
        bpairs = eq.boundary_pairs(nvec, gamma)
        lterms = eq.load_boundary_terms(nvec, gamma)
        fixed = [a for a in range(m) if patch_box_1d(m, a)[0] <= val <= patch_box_1d(m, a)[1]]
        pt = np.array([val])
        for (ps, ws, along, _) in subs:
            for af in fixed:
                Tfix = np.empty((pmax + 1, rmax + 3, 1))
                for j in range(pmax + 1):
                    for r in range(rmax + 3):
                        Tfix[j, r] = factor_1d(m, af, j, pt, r)
                Talong = {}
                for aa in along:
                    t = np.empty((pmax + 1, rmax + 3, len(ps)))
                    for j in range(pmax + 1):
                        for r in range(rmax + 3):
                            t[j, r] = factor_1d(m, aa, j, ps, r)
                    Talong[aa] = t

                def idx(aa):
                    return (aa * m + af) if axis == 0 else (af * m + aa)

                def opv(op, aa):
                    e = exps[degs[idx(aa)]]
                    return _op_values(op, e, Tfix, Talong[aa]) if axis == 0 else _op_values(op, e, Talong[aa], Tfix)

                for ai in along:
                    i = idx(ai)
                    if g is not None:
                        xs = np.full_like(ps, val) if axis == 0 else ps
                        ys = ps if axis == 0 else np.full_like(ps, val)
                        for (gi, ov, c) in lterms:
                            bvec[off[i]:off[i + 1]] += c * opv(ov, ai) @ (ws * g[gi](xs, ys))
                    for aj in along:
                        j = idx(aj)
                        blk = np.zeros((off[i + 1] - off[i], off[j + 1] - off[j]))
                        for (ov, ou, c) in bpairs:
                            blk += c * (opv(ov, ai) * ws) @ opv(ou, aj).T
                        add(i, j, blk)

    return AssembledRaised(degs, off, ent, _to_csr(ent, off), bvec, gamma)


def local_projection(m: int, p: int, p_boundary: int, func, q: int = 12) -> np.ndarray:
    """Each patch's L2 projection of func onto its own local space over its box; a polynomial of
    degree <= min(p, p_boundary) is reproduced exactly on every patch."""
    degs = patch_degrees(m, p, p_boundary)
    off = offsets(degs)
    gx, gw = npleg.leggauss(q)
    out = np.zeros(int(off[-1]))
    for iy in range(m):
        for ix in range(m):
            i = iy * m + ix
            (xl, xh), (yl, yh) = patch_box_1d(m, ix), patch_box_1d(m, iy)
            px, py = 0.5 * (xh - xl) * gx + 0.5 * (xh + xl), 0.5 * (yh - yl) * gx + 0.5 * (yh + yl)
            X, Y = (np.ravel(v) for v in np.meshgrid(px, py, indexing="ij"))
            W = np.ravel(np.outer(0.5 * (xh - xl) * gw, 0.5 * (yh - yl) * gw))
            fv = func(X, Y)
            for k, (a, b) in enumerate(basis_exponents(degs[i])):
                L = np.ravel(np.outer(local_poly_1d(m, ix, a, px, 0), local_poly_1d(m, iy, b, py, 0)))
                norm = (xh - xl) / (2 * a + 1) * (yh - yl) / (2 * b + 1)
                out[off[i] + k] = np.sum(W * fv * L) / norm
    return out


def prolongation(m_f: int, p: int, p_boundary: int, q: int | None = None) -> sps.csr_matrix:
    """P of prolongation_blocks as a CSR matrix over the scalar unknowns."""
    blocks, off_f, off_c = prolongation_blocks(m_f, p, p_boundary, q)
    rows, cols, vals = [], [], []
    for (i, j), B in blocks.items():
        r, c = np.meshgrid(np.arange(off_f[i], off_f[i + 1]), np.arange(off_c[j], off_c[j + 1]), indexing="ij")
        rows.append(r.ravel())
        cols.append(c.ravel())
        vals.append(B.ravel())
    return sps.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(int(off_f[-1]), int(off_c[-1])))


def prolongation_blocks(m_f: int, p: int, p_boundary: int, q: int | None = None):
    """P from the raised space of level m_f / 2 to that of level m_f by global-to-local L2
    projection (Section 4): block (i, j) = M_i^{-1} B_ij with M_i the fine local mass matrix and
    B_ij the integral of fine basis i against coarse basis function j (PU times its local
    polynomial), over the fine box cut at all fine and coarse breakpoints."""
    assert m_f % 2 == 0
    m_c = m_f // 2
    dfine, dcoarse = patch_degrees(m_f, p, p_boundary), patch_degrees(m_c, p, p_boundary)
    off_f, off_c = offsets(dfine), offsets(dcoarse)
    pmax = max(p, p_boundary)
    q = q or pmax + 6
    gx, gw = npleg.leggauss(q)
    cuts = np.union1d(breakpoints_1d(m_f), breakpoints_1d(m_c))

    def pieces(a):
        lo, hi = patch_box_1d(m_f, a)
        grid = [lo] + [c for c in cuts if lo < c < hi] + [hi]
        out = []
        for u in range(len(grid) - 1):
            pts = 0.5 * (grid[u + 1] - grid[u]) * gx + 0.5 * (grid[u + 1] + grid[u])
            wts = 0.5 * (grid[u + 1] - grid[u]) * gw
            th = np.array([local_poly_1d(m_f, a, j, pts, 0) for j in range(pmax + 1)])
            co = {c: np.array([factor_1d(m_c, c, j, pts, 0) for j in range(pmax + 1)])
                  for c in active_1d(m_c, grid[u], grid[u + 1])}
            out.append((wts, th, co))
        return out

    pcs = {a: pieces(a) for a in range(m_f)}
    blocks = {}
    for iy in range(m_f):
        for ix in range(m_f):
            i = iy * m_f + ix
            ei = basis_exponents(dfine[i])
            Mi = np.zeros((len(ei), len(ei)))
            Bs = {}
            for (wx, thx, cox) in pcs[ix]:
                for (wy, thy, coy) in pcs[iy]:
                    W = np.ravel(np.outer(wx, wy))
                    th = np.array([np.ravel(np.outer(thx[a], thy[b])) for (a, b) in ei])
                    Mi += (th * W) @ th.T
                    for jy, Ty in coy.items():
                        for jx, Tx in cox.items():
                            j = jy * m_c + jx
                            psi = np.array([np.ravel(np.outer(Tx[a], Ty[b])) for (a, b) in basis_exponents(dcoarse[j])])
                            Bs[j] = Bs.get(j, 0.0) + (th * W) @ psi.T
            for j, B in Bs.items():
                blocks[(i, j)] = np.linalg.solve(Mi, B)
    return blocks, off_f, off_c


# ---------------------------------------------------------------------------
# The raised space on a uniform block layout (padding)
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class PaddedHierarchy:
    """Levels finest first, every block d_pad x d_pad: A[l] and P[l] as BlockCSR, the load vector
    b on the padded unknowns, and per level the indices of the real (unpadded) unknowns."""
    m: list
    A: list
    P: list
    b: np.ndarray
    real: list
    A_raised: sps.csr_matrix  # the finest raised operator, unpadded
    b_raised: np.ndarray


def _pad_csr(M: sps.csr_matrix, off_r: np.ndarray, off_c: np.ndarray, d: int, identity: bool) -> dict:
    """Blocks of M (variable sizes by offsets) embedded top-left in d x d blocks; with identity,
    the padded diagonal entries of the diagonal blocks are 1 (decoupled padded unknowns)."""
    M = M.tocsr()
    nr, nc = len(off_r) - 1, len(off_c) - 1
    rb = np.searchsorted(off_r, np.arange(off_r[-1]), side="right") - 1
    cb = np.searchsorted(off_c, np.arange(off_c[-1]), side="right") - 1
    coo = M.tocoo()
    out = {}
    for r, c, v in zip(coo.row, coo.col, coo.data):
        i, j = int(rb[r]), int(cb[c])
        if (i, j) not in out:
            out[(i, j)] = np.zeros((d, d))
        out[(i, j)][r - off_r[i], c - off_c[j]] += v
    if identity:
        assert nr == nc
        for i in range(nr):
            B = out.setdefault((i, i), np.zeros((d, d)))
            for t in range(off_r[i + 1] - off_r[i], d):
                B[t, t] = 1.0
    return out


def padded_hierarchy(m: int, p: int, p_boundary: int, n_levels: int, f=None) -> PaddedHierarchy:
    """The raised space's Galerkin hierarchy (finest assembly, L2-projection prolongations,
    A_{l-1} = P^T A_l P on the unpadded unknowns), each level written with uniform blocks of the
    raised dimension: padded unknowns carry an identity diagonal and no coupling, so they stay
    zero in every product and the padded system's solution restricted to the real unknowns is
    the raised one."""
    from . import blocks as bk
    d = local_dim(max(p, p_boundary))
    asm = assemble(m, p, p_boundary, f=f)
    A, off = asm.A, asm.off
    ms, As, Ps, reals = [m], [], [], []
    A_l, off_l, m_l = A, off, m
    for lev in range(n_levels):
        As.append(bk.from_blocks(m_l * m_l, m_l * m_l, d, _pad_csr(A_l, off_l, off_l, d, True)))
        reals.append(np.concatenate([np.arange(i * d, i * d + off_l[i + 1] - off_l[i]) for i in range(m_l * m_l)]))
        if lev == n_levels - 1:
            break
        Pb, off_f, off_c = prolongation_blocks(m_l, p, p_boundary)
        Pm = prolongation(m_l, p, p_boundary)
        Ps.append(bk.from_blocks(m_l * m_l, (m_l // 2) ** 2, d, _pad_csr(Pm, off_f, off_c, d, False)))
        A_l = (Pm.T @ A_l @ Pm).tocsr()
        off_l, m_l = off_c, m_l // 2
        ms.append(m_l)
    b = np.zeros(m * m * d)
    b[reals[0]] = asm.b
    return PaddedHierarchy(ms, As, Ps, b, reals, A, asm.b)
