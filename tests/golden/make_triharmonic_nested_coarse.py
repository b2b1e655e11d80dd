"""Write triharmonic256_nested_coarse.json: the oracle's nested block-FSAI on the coarse levels
of the 256x256-patch triharmonic workload (p = 5, d = 21, 9 levels; Example 5.4 with the nested
FSAI of Section 2.2, Algorithm 1 from the diagonal pattern, t_max = 6, tau = 1).

The coarse Galerkin operators A_l = P^T A_{l-1} P carry the finest level's penalties (order
h^-5), and the inner FSAI of A_1 = F_0 A F_0^T is where that shows: on some of these levels A_1
is no longer numerically SPD and the inner level is block Jacobi.  This script builds the whole
hierarchy with the oracle alone (assembly and prolongation split over row strips in worker
processes, Galerkin products as sparse matrix products) and records, per level from 32x32
patches down to 2x2: the outer pattern P(F_0), whether the inner FSAI was formed, the inner
pattern P(G_1) and sum_k log det S_kk, or that the outer FSAI could not be formed because one
of its local matrices is not numerically SPD.  It takes about 40 minutes and 20 GB of memory.

    python tests/golden/make_triharmonic_nested_coarse.py [--workers 8]
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import pum_inputs as pin  # noqa: E402
from oracle import blocks as bk  # noqa: E402
from oracle import fsai, pum  # noqa: E402

PR = pin.TRIHARMONIC_256
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "triharmonic256_nested_coarse.json")
FIRST_LEVEL = 3          # 32 x 32 patches


def _assemble_strip(args):
    m, rows = args
    f = pum.fourier_source(pin.fourier_coefficients(PR.rhs_seed), PR.rhs_decay)
    g = pum.nitsche_gamma(PR.equation, PR.p, m, PR.nitsche)
    asm = pum.assemble(m, PR.p, PR.equation, g, f=f, with_mass=False, rows=rows)
    return _strip(asm.A, rows)


def _prolong_strip(args):
    m_f, rows = args
    return _strip(pum.prolongation(m_f, PR.p, rows=rows), rows)


def _strip(M: bk.BlockCSR, rows):
    r0, r1 = rows[0], rows[-1] + 1
    lo, hi = int(M.indptr[r0]), int(M.indptr[r1])
    return r0, r1, M.n_rows, M.n_cols, M.d, np.diff(M.indptr[r0:r1 + 1]), M.indices[lo:hi], M.blocks[lo:hi]


def _merge(parts) -> bk.BlockCSR:
    parts = sorted(parts, key=lambda p: p[0])
    n_rows, n_cols, d = parts[0][2], parts[0][3], parts[0][4]
    counts = np.concatenate([p[5] for p in parts])
    assert counts.shape[0] == n_rows
    indptr = np.zeros(n_rows + 1, dtype=np.int64)
    np.cumsum(counts, out=indptr[1:])
    return bk.BlockCSR(n_rows, n_cols, d, indptr, np.concatenate([p[6] for p in parts]),
                       np.concatenate([p[7] for p in parts]))


def _rows_only(M: bk.BlockCSR, rows) -> bk.BlockCSR:
    """M with only the given (contiguous) block rows stored."""
    r0, r1 = rows[0], rows[-1] + 1
    lo, hi = int(M.indptr[r0]), int(M.indptr[r1])
    indptr = np.zeros(M.n_rows + 1, dtype=np.int64)
    indptr[r0 + 1:r1 + 1] = M.indptr[r0 + 1:r1 + 1] - lo
    indptr[r1 + 1:] = hi - lo
    return bk.BlockCSR(M.n_rows, M.n_cols, M.d, indptr, M.indices[lo:hi], M.blocks[lo:hi])


def _strips(n, k):
    edges = np.linspace(0, n, k + 1).astype(int)
    return [list(range(edges[i], edges[i + 1])) for i in range(k) if edges[i + 1] > edges[i]]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workers", type=int, default=os.cpu_count() or 4)
    args = ap.parse_args()
    t0 = time.time()
    m = PR.finest_m
    ctx = mp.get_context("spawn")
    with ctx.Pool(args.workers) as pool:
        A = _merge(pool.map(_assemble_strip, [(m, s) for s in _strips(m * m, 4 * args.workers)]))
    print(f"assembled {m}x{m}: {A.nnzb} blocks, {time.time() - t0:.0f} s", flush=True)
    As, ms = [A], [m]
    for _ in range(PR.n_levels - 1):
        mf = ms[-1]
        with ctx.Pool(args.workers) as pool:
            P = _merge(pool.map(_prolong_strip, [(mf, s) for s in _strips(mf * mf, 4 * args.workers)]))
        R = P.transpose()
        # the Galerkin product by strips of coarse rows (rows of R): each strip's rows of R A P are
        # those of the whole product, and the strips bound the memory of the sparse products
        strips = _strips(R.n_rows, max(1, (R.n_rows * R.d) // 40000))
        As.append(_merge([_strip(bk.galerkin_product(_rows_only(R, s), As[-1], P), s) for s in strips]))
        ms.append(mf // 2)
        del P, R
        if 0 <= len(As) - 3 < FIRST_LEVEL:
            As[len(As) - 3] = None  # only the levels recorded below are kept
        print(f"Galerkin level {len(As) - 1} ({ms[-1]}x{ms[-1]}), {time.time() - t0:.0f} s", flush=True)
    out = {"_about": "Oracle nested block-FSAI (Section 2.2; Algorithm 1 from the diagonal, t_max = 6, tau = 1) "
                     "on the coarse Galerkin levels of the 256x256-patch triharmonic problem (p = 5, Example 5.4, "
                     "seed-2 Fourier right-hand side, Nitsche constants of the workload); written by "
                     "make_triharmonic_nested_coarse.py from the oracle alone.",
           "levels": {}}
    for lev in range(FIRST_LEVEL, PR.n_levels - 1):
        A = As[lev]
        t1 = time.time()
        try:
            nf = fsai.nested_fsai(A, fsai.diag_pattern(A.n_rows), PR.t_max, PR.tau)
        except fsai.NotSPD as e:
            # the outer FSAI itself needs a local matrix that is not numerically SPD in FP64
            out["levels"][str(lev)] = {"m": ms[lev], "n": A.n_rows, "d": A.d, "nnzb_A": A.nnzb,
                                       "outer_not_spd": str(e)}
            print(f"level {lev}: outer FSAI not formed ({e}), {time.time() - t1:.0f} s", flush=True)
            continue
        G1 = nf.inner.G
        out["levels"][str(lev)] = {
            "m": ms[lev], "n": A.n_rows, "d": A.d, "nnzb_A": A.nnzb,
            "nested_inner": int(nf.inner_nested),
            "F0_indptr": nf.F0.indptr.tolist(), "F0_indices": nf.F0.indices.tolist(),
            "G1_indptr": G1.indptr.tolist(), "G1_indices": G1.indices.tolist(),
            "logdet_S": nf.logdet_S(),
            "G1_row_fro": [float(np.sqrt(np.sum(G1.blocks[G1.indptr[i]:G1.indptr[i + 1]] ** 2)))
                           for i in range(A.n_rows)],
        }
        print(f"level {lev}: nested_inner {int(nf.inner_nested)}, {time.time() - t1:.0f} s", flush=True)
    with open(OUT, "w") as f:
        json.dump(out, f, separators=(",", ":"))
    print(f"wrote {OUT} in {time.time() - t0:.0f} s")


if __name__ == "__main__":
    main()
