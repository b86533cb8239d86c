"""Seeded synthetic inputs for CP decomposition problems.

This module only *creates inputs*: factor matrices with prescribed collinearity,
the tensors built from them plus noise, random initial guesses for the boot
factor matrices (BFMs) and the test factor matrices (TFMs).  It contains none of
the decomposition method's arithmetic (no MTTKRP, no ALS, no multigrid), so the
CUDA path and the FP64 oracle can both draw their inputs from it.

Conventions
-----------
* A tensor ``Z`` of size I_1 x ... x I_N is a NumPy array indexed
  ``Z[i_1, ..., i_N]`` and stored column-major (``order='F'``: i_1 varies
  fastest), which is the memory layout the device kernels read.
* A factor matrix is an ``I_n x R`` float64 array, column-major.
* Every random draw is seeded from ``numpy.random.default_rng(seed)``;
  the per-mode seed rules are stated in each function.

Workloads
---------
* collinear-factor tensors: each mode's columns have unit-free norms sqrt(I_n)
  and pairwise cosines exactly ``c``; homoscedastic noise at level eta1 and
  optional heteroscedastic noise (noise scaled elementwise by the signal).
* the paper's dense test tensor z_ijk = (i^2 + j^2 + k^2)^(-1/2)
  (Section 6.3).
"""
from __future__ import annotations

import dataclasses
import numpy as np

__all__ = [
    "CPProblem",
    "collinear_factors",
    "normal_factors",
    "cp_tensor",
    "add_noise",
    "initial_guess",
    "test_blocks",
    "make_problem",
    "ijk_tensor",
    "batch_specs",
]


def _rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(int(seed))


def normal_factors(dims, R, seed):
    """Factor matrices with i.i.d. N(0,1) entries; mode n uses seed ``seed*1000 + n``."""
    out = []
    for n, I in enumerate(dims):
        out.append(np.asfortranarray(_rng(seed * 1000 + n).standard_normal((I, R))))
    return out


def collinear_factors(dims, R, congruence, seed):
    """Factor matrices whose columns have norm sqrt(I_n) and pairwise cosine ``congruence``.

    For mode n: draw G ~ N(0,1)^{I_n x R} (seed ``seed*1000 + n``), take the
    thin QR factor Q (orthonormal columns), form the target Gram
    C = (1-c) I + c 1 1^T and its upper Cholesky factor U (C = U^T U), and set
    A = sqrt(I_n) Q U, so that A^T A = I_n C exactly (up to rounding).
    Requires I_n >= R and 0 <= c < 1.
    """
    c = float(congruence)
    if not (0.0 <= c < 1.0):
        raise ValueError("congruence must lie in [0, 1)")
    C = (1.0 - c) * np.eye(R) + c * np.ones((R, R))
    U = np.linalg.cholesky(C).T  # upper factor, C = U^T U
    out = []
    for n, I in enumerate(dims):
        if I < R:
            raise ValueError(f"mode {n} has I_n={I} < R={R}; collinear factors need I_n >= R")
        G = _rng(seed * 1000 + n).standard_normal((I, R))
        Q, _ = np.linalg.qr(G, mode="reduced")
        out.append(np.asfortranarray(np.sqrt(I) * (Q @ U)))
    return out


def cp_tensor(factors):
    """The full tensor sum_r a_r^(1) o ... o a_r^(N), column-major float64."""
    N = len(factors)
    letters = "abcdefgh"[:N]
    spec = ",".join(f"{l}z" for l in letters) + "->" + letters
    return np.asfortranarray(np.einsum(spec, *factors, optimize=True))


def add_noise(T, eta_homo, eta_hetero, seed):
    """Z = T + eta1 ||T|| E1/||E1||, then optionally Z += eta2 ||Z|| E2/||E2||, E2 = T * N(0,1).

    E1 uses seed ``seed*1000 + 500``, the heteroscedastic draw ``seed*1000 + 501``.
    """
    Z = np.array(T, dtype=np.float64, order="F", copy=True)
    if eta_homo > 0:
        E1 = _rng(seed * 1000 + 500).standard_normal(T.shape)
        Z += eta_homo * np.linalg.norm(T.ravel()) * E1 / np.linalg.norm(E1.ravel())
    if eta_hetero > 0:
        E2 = T * _rng(seed * 1000 + 501).standard_normal(T.shape)
        Z += eta_hetero * np.linalg.norm(Z.ravel()) * E2 / np.linalg.norm(E2.ravel())
    return np.asfortranarray(Z)


def initial_guess(dims, R, seed):
    """Random N(0,1) BFMs (the initial iterate); mode n uses seed ``seed*1000 + 100 + n``."""
    return [np.asfortranarray(_rng(seed * 1000 + 100 + n).standard_normal((I, R)))
            for n, I in enumerate(dims)]


def test_blocks(dims, R, n_t, seed):
    """``n_t`` random N(0,1) test blocks (TFMs); block t, mode n uses seed
    ``seed*1000 + 200 + 10*t + n``.  Returned as ``[block][mode]``."""
    return [[np.asfortranarray(_rng(seed * 1000 + 200 + 10 * t + n).standard_normal((I, R)))
             for n, I in enumerate(dims)] for t in range(n_t)]


@dataclasses.dataclass
class CPProblem:
    """One synthetic decomposition problem."""
    Z: np.ndarray            # column-major tensor (float32 or float64)
    R: int
    truth: list              # exact factors the tensor was built from (float64)
    A0: list                 # initial BFMs
    tfms: list               # [block][mode] initial TFMs
    name: str = ""

    @property
    def dims(self):
        return tuple(self.Z.shape)


def make_problem(dims, R, *, congruence=None, eta_homo=0.0, eta_hetero=0.0,
                 dtype=np.float32, seed=0, n_t=2, name=""):
    """Build a problem: factors (collinear if ``congruence`` is given, else
    N(0,1)), tensor, noise, cast to ``dtype`` (the cast tensor is the ground truth
    for every consumer), initial BFMs and ``n_t`` TFM blocks."""
    dims = tuple(int(d) for d in dims)
    if congruence is None:
        truth = normal_factors(dims, R, seed)
    else:
        truth = collinear_factors(dims, R, congruence, seed)
    T = cp_tensor(truth)
    Z = add_noise(T, eta_homo, eta_hetero, seed)
    Z = np.asfortranarray(Z.astype(dtype))
    return CPProblem(Z=Z, R=R, truth=truth, A0=initial_guess(dims, R, seed),
                     tfms=test_blocks(dims, R, n_t, seed), name=name)


def ijk_tensor(s, dtype=np.float64):
    """The paper's dense test tensor z_ijk = (i^2 + j^2 + k^2)^(-1/2), i,j,k = 1..s (Section 6.3)."""
    i = np.arange(1, s + 1, dtype=np.float64)
    Z = 1.0 / np.sqrt(i[:, None, None] ** 2 + i[None, :, None] ** 2 + i[None, None, :] ** 2)
    return np.asfortranarray(Z.astype(dtype))


def laplacian_tensor(d, s, dtype=np.float64):
    """The paper's sparse test problem (Section 6.2), stored dense: the s^d x s^d finite-difference
    Laplacian sum_{k=1..d} I_{s^(d-k)} (x) D (x) I_{s^(k-1)}, D = tridiag(-1, 2, -1) of size s,
    reshaped column-major into an order-2d tensor of size s x ... x s.  Modes 1..d carry the row
    index of the matrix (first grid dimension fastest), modes d+1..2d the column index, so
    Z[i_1..i_d, j_1..j_d] = sum_k D[i_k, j_k] prod_{m != k} [i_m == j_m].  The entries are small
    integers, exact in float32."""
    D = 2.0 * np.eye(s) - np.eye(s, k=1) - np.eye(s, k=-1)
    n = s ** d
    M = np.zeros((n, n))
    for k in range(1, d + 1):
        M += np.kron(np.kron(np.eye(s ** (d - k)), D), np.eye(s ** (k - 1)))
    return np.asfortranarray(np.reshape(M, (s,) * (2 * d), order="F").astype(dtype))


def uniform_start(dims, R, seed):
    """Factor matrices with i.i.d. uniform [0, 1) entries (the paper's initial guesses, Section 6.1),
    mode n from seed*1000 + 300 + n."""
    return [np.asfortranarray(_rng(seed * 1000 + 300 + n).uniform(size=(I, R))) for n, I in enumerate(dims)]


def batch_specs(count, seed=0):
    """Shapes for the uneven batch workload: N in {3,4} with probability 1/2, I_n ~ U[16,128]
    (U[16,48] when N=4), R ~ U{2..8}, congruence ~ U[0.5,0.95], seeded by ``seed``."""
    rng = _rng(seed * 1000 + 900)
    specs = []
    for k in range(count):
        N = int(rng.integers(3, 5))
        hi = 128 if N == 3 else 48
        dims = tuple(int(v) for v in rng.integers(16, hi + 1, size=N))
        R = int(rng.integers(2, 9))
        c = float(rng.uniform(0.5, 0.95))
        specs.append(dict(dims=dims, R=R, congruence=c, seed=k))
    return specs
