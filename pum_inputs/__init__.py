"""Seeded synthetic inputs shared by the oracle and the CUDA library's tests.

This module holds no arithmetic of the solver: it only draws random numbers
and names the workload configurations.  Every random number that the method
itself needs (the Lanczos start vector) is produced independently on each
side from the SplitMix64 counter generator; what lives here are the problem
inputs (right-hand-side Fourier coefficients, test vectors, initial errors).
"""
from __future__ import annotations

import dataclasses

import math

import numpy as np


def fourier_coefficients(seed: int, modes: int = 8) -> np.ndarray:
    """Coefficients c_ab ~ N(0,1), a, b = 1..modes, of the smooth right-hand side.

    The source term is f(x,y) = sum_ab c_ab (a^2+b^2)^(-decay/2) sin(a pi x) sin(b pi y);
    the decay exponent is part of the problem description, not drawn here.
    Returned as a (modes, modes) float64 array indexed [a-1, b-1].
    """
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0x5EED]))
    return rng.standard_normal((modes, modes))


def normal_vector(n: int, seed: int) -> np.ndarray:
    """iid N(0,1) float64 vector of length n."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0xA11CE]))
    return rng.standard_normal(n)


def uniform_vector(n: int, seed: int) -> np.ndarray:
    """iid U(-1,1) float64 vector of length n (initial errors for convergence-factor runs)."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0xE0]))
    return rng.uniform(-1.0, 1.0, n)


def spd_block_matrix(n: int, d: int, seed: int, density: float = 0.5) -> np.ndarray:
    """Small dense SPD matrix of size n*d with a random block sparsity pattern.

    Blocks (i, j), i != j, are kept with probability `density` (symmetrically);
    the result is shifted by its smallest eigenvalue so it is safely SPD.
    Used for the FSAI identities on tiny problems.
    """
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0xB10C]))
    N = n * d
    X = rng.standard_normal((N, N))
    A = X @ X.T
    keep = rng.random((n, n)) < density
    keep = np.triu(keep, 1)
    keep = keep | keep.T | np.eye(n, dtype=bool)
    mask = np.kron(keep, np.ones((d, d), dtype=bool))
    A = np.where(mask, A, 0.0)
    A = 0.5 * (A + A.T)
    lam = np.linalg.eigvalsh(A)[0]
    A += (abs(lam) + 1.0 + 0.1 * N) * np.eye(N)
    return A


@dataclasses.dataclass(frozen=True)
class Problem:
    """Description of one synthetic PUM workload (all sizes explicit)."""
    name: str
    equation: int            # 4 = biharmonic (order 2m = 4), 6 = triharmonic
    p: int                   # local polynomial degree, block size d = (p+1)(p+2)/2
    finest_m: int            # patches per side on the finest level
    n_levels: int
    rhs_seed: int
    rhs_decay: float         # f coefficients scaled by (a^2+b^2)^(-decay/2)
    fsai_p0: str             # "lower" (lower block pattern of A) or "diag"
    adaptive: bool
    t_max: int
    tau: float
    nested: bool
    cheb_k: int
    smooth_dtype: str        # "f64", "f32"
    g_dtype: str             # "f64", "f32", "bf16"
    fp32_levels: int = 64    # FP32 form: levels smoothed in FP32 (the coarser ones in FP64)

    @property
    def nitsche(self) -> tuple:
        """Constants C_j of the Nitsche penalties gamma^(j) = C_j (p+1)^2 h^-(order-1-2j)."""
        return NITSCHE_CONSTANTS[self.equation]

    @property
    def d(self) -> int:
        return (self.p + 1) * (self.p + 2) // 2

    @property
    def n_dofs(self) -> int:
        return self.d * self.finest_m ** 2


# Nitsche penalty constants per equation order: the smallest round values for which the
# assembled stiffness matrices are SPD on 2..16 patches per side.
NITSCHE_CONSTANTS = {4: (4.0, 2.0, 0.0), 6: (1.0e4, 1.0e2, 1.0)}

# The workloads of the benchmark suite, with their sizes.
SMALL_BIHARMONIC = Problem("biharmonic p=3 16x16 patches, 4 levels, static block-FSAI, Chebyshev-4 k=2",
                           4, 3, 16, 4, 0, 2.0, "lower", False, 0, 1.0, False, 2, "f64", "f64")
BIHARMONIC_256 = Problem("biharmonic p=3 256x256 patches, 9 levels, adaptive block-FSAI t_max=6, Chebyshev-4 k=3",
                         4, 3, 256, 9, 1, 2.0, "lower", True, 6, 1.0, False, 3, "f64", "f64")
TRIHARMONIC_256 = Problem("triharmonic p=5 256x256 patches, 9 levels, nested adaptive block-FSAI, Chebyshev-4 k=4",
                          6, 5, 256, 9, 2, 3.0, "diag", True, 6, 1.0, True, 4, "f32", "bf16", 2)


def anisotropy_tensor(kappa: float, theta: float) -> tuple:
    """(S11, S12, S22) of the anisotropic biharmonic workload's tensor S = R diag(kappa, 1) R^T,
    R the rotation by theta (the problem data of Example 5.2, passed to both implementations)."""
    c, s = math.cos(theta), math.sin(theta)
    return (kappa * c * c + s * s, (kappa - 1.0) * c * s, kappa * s * s + c * c)


ANISO_KAPPA, ANISO_THETA = 10.0, math.pi / 3


@dataclasses.dataclass(frozen=True)
class Instance:
    """One problem of the batched uneven workload: biharmonic, m x m patches, degree p, levels
    halving m while it stays even (coarsest 1x1 or an odd side such as 3x3)."""
    m: int
    p: int

    @property
    def n_levels(self) -> int:
        n, m = 1, self.m
        while m % 2 == 0 and m > 1:
            m //= 2
            n += 1
        return n

    @property
    def d(self) -> int:
        return (self.p + 1) * (self.p + 2) // 2

    @property
    def n_dofs(self) -> int:
        return self.d * self.m * self.m


def batch_instances(seed: int = 3, count: int = 64, sides=(32, 64, 96, 128), degrees=(2, 3)) -> list:
    """The batched workload: `count` biharmonic instances with sides and degrees drawn by `seed`."""
    rs = np.random.default_rng(seed)
    return [Instance(int(rs.choice(sides)), int(rs.choice(degrees))) for _ in range(count)]


def splitmix64_reference_values():
    """First outputs of SplitMix64 seeded with 0 (Steele, Lea & Flood 2014), as published
    test values of the generator; both the oracle's and the library's implementations are
    checked against them."""
    return [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
