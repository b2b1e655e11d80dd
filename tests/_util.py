"""Helpers shared by the GPU parity tests: oracle <-> library marshalling and tolerances.

Tolerances (FP64 path).  Every quantity is computed by the oracle and by the CUDA
library from the same inputs with different summation orders, so they differ by
rounding only.  For a quantity obtained by solving a local SPD system of condition
kappa the relative difference is bounded by about kappa * eps; the local FSAI systems
of these PUM matrices have kappa up to ~1e5, giving the 1e-10 bound used for FSAI
factors; assembled matrices and products (no solves) use 1e-12 of their largest entry.
"""
from __future__ import annotations

import numpy as np

from oracle import blocks as bk

TOL_ASSEMBLY = 1e-12
TOL_FSAI = 1e-10
TOL_VECTOR = 1e-10
TOL_HISTORY = 1e-12   # absolute difference of ||r_j|| / ||b|| histories (FP64)


def to_view(A: bk.BlockCSR):
    return (A.indptr, A.indices, A.blocks)


def to_pview(P: bk.BlockCSR):
    return (P.indptr, P.indices, P.blocks, P.n_cols)


def from_export(exp) -> bk.BlockCSR:
    indptr, indices, blocks, n_cols = exp
    return bk.BlockCSR(len(indptr) - 1, n_cols, blocks.shape[1], indptr.astype(np.int64), indices.astype(np.int64),
                       blocks)


def assert_same_pattern(got: bk.BlockCSR, ref: bk.BlockCSR):
    assert got.n_rows == ref.n_rows and got.n_cols == ref.n_cols
    assert np.array_equal(got.indptr, ref.indptr), "block row pointers differ"
    assert np.array_equal(got.indices, ref.indices), "block column indices differ"


def max_rel(got: np.ndarray, ref: np.ndarray) -> float:
    return float(np.max(np.abs(got - ref)) / max(np.max(np.abs(ref)), 1e-300))


def norm_rel(got: np.ndarray, ref: np.ndarray) -> float:
    return float(np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-300))


def cuda(x):
    import torch
    return torch.as_tensor(np.ascontiguousarray(x, dtype=np.float64)).cuda()


def host(t):
    return t.detach().cpu().numpy()
