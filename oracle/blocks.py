"""Block-structured sparse matrices (Definition 2.1) for the oracle.

Test infrastructure only.  A matrix with uniform block size d is held as
block-CSR: ``indptr`` (n_rows+1), ``indices`` (nnzb, sorted within each row)
and ``blocks`` (nnzb, d, d).  The sparsity pattern P(A) is the set of stored
blocks: it is *structural* (a stored block may hold zeros), which is how the
Galerkin and FSAI patterns are defined in the oracle.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.sparse as sp


@dataclasses.dataclass
class BlockCSR:
    n_rows: int
    n_cols: int
    d: int
    indptr: np.ndarray
    indices: np.ndarray
    blocks: np.ndarray

    @property
    def nnzb(self) -> int:
        return int(self.indices.shape[0])

    def row(self, i: int) -> np.ndarray:
        return self.indices[self.indptr[i]:self.indptr[i + 1]]

    def pattern(self) -> list[list[int]]:
        return [list(map(int, self.row(i))) for i in range(self.n_rows)]

    def block(self, i: int, j: int) -> np.ndarray | None:
        """Block (i, j), or None when it is not in the pattern."""
        lookup = self.__dict__.get("_lookup")
        if lookup is None:
            lookup = {}
            for r in range(self.n_rows):
                for p in range(int(self.indptr[r]), int(self.indptr[r + 1])):
                    lookup[(r, int(self.indices[p]))] = p
            self.__dict__["_lookup"] = lookup
        p = lookup.get((i, j))
        return None if p is None else self.blocks[p]

    def to_scipy(self) -> sp.csr_matrix:
        return sp.bsr_matrix((self.blocks, self.indices, self.indptr),
                             shape=(self.n_rows * self.d, self.n_cols * self.d)).tocsr()

    def to_dense(self) -> np.ndarray:
        return self.to_scipy().toarray()

    def matvec(self, x: np.ndarray) -> np.ndarray:
        return self.to_scipy() @ x

    def transpose(self) -> "BlockCSR":
        """Explicit block transpose: block (j, i) of the result is block (i, j)^T."""
        entries = {}
        for i in range(self.n_rows):
            for p in range(self.indptr[i], self.indptr[i + 1]):
                entries[(int(self.indices[p]), i)] = self.blocks[p].T
        return from_blocks(self.n_cols, self.n_rows, self.d, entries)


def from_blocks(n_rows: int, n_cols: int, d: int, entries: dict) -> BlockCSR:
    """Build block-CSR from a dict {(i, j): d x d array}; columns sorted per row."""
    rows = [[] for _ in range(n_rows)]
    for (i, j) in entries:
        rows[i].append(j)
    indptr = np.zeros(n_rows + 1, dtype=np.int64)
    indices = []
    blocks = []
    for i in range(n_rows):
        cols = sorted(rows[i])
        indptr[i + 1] = indptr[i] + len(cols)
        indices.extend(cols)
        blocks.extend(np.asarray(entries[(i, j)], dtype=np.float64) for j in cols)
    blocks = np.array(blocks).reshape(-1, d, d) if blocks else np.zeros((0, d, d))
    return BlockCSR(n_rows, n_cols, d, indptr, np.asarray(indices, dtype=np.int64), blocks)


def from_pattern_and_scalar(pattern: list[list[int]], n_cols: int, d: int, S) -> BlockCSR:
    """Blocks of the scalar matrix S (scipy or dense) on a given block pattern (blocks of the
    pattern that S does not store are zero)."""
    B = sp.csr_matrix(S).tobsr(blocksize=(d, d))
    B.sort_indices()
    entries = {}
    for i, cols in enumerate(pattern):
        lo, hi = int(B.indptr[i]), int(B.indptr[i + 1])
        where = dict(zip(B.indices[lo:hi].tolist(), range(lo, hi)))
        for j in cols:
            q = where.get(j)
            entries[(i, j)] = B.data[q] if q is not None else np.zeros((d, d))
    return from_blocks(len(pattern), n_cols, d, entries)


def product_pattern(P1: list[list[int]], P2: list[list[int]]) -> list[list[int]]:
    """Structural pattern of a product: {(i,k) : exists j, (i,j) in P1 and (j,k) in P2}."""
    out = []
    for cols in P1:
        s = set()
        for j in cols:
            s.update(P2[j])
        out.append(sorted(s))
    return out


def transpose_pattern(P: list[list[int]], n_cols: int) -> list[list[int]]:
    out = [[] for _ in range(n_cols)]
    for i, cols in enumerate(P):
        for j in cols:
            out[j].append(i)
    return [sorted(c) for c in out]


def galerkin_product(R: BlockCSR, A: BlockCSR, P: BlockCSR) -> BlockCSR:
    """R A P on the structural pattern P(R) P(A) P(P) (values by sparse matmul)."""
    pat = product_pattern(product_pattern(R.pattern(), A.pattern()), P.pattern())
    S = R.to_scipy() @ A.to_scipy() @ P.to_scipy()
    return from_pattern_and_scalar(pat, P.n_cols, A.d, S)


def diag_blocks(A: BlockCSR) -> np.ndarray:
    """diag_B(A) as an (n, d, d) array."""
    return np.array([A.block(i, i) for i in range(A.n_rows)])
