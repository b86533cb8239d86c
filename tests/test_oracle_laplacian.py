"""The paper's Laplacian test tensor (Section 6.2, Table tab:LapParams) as the generator builds it,
pinned against its definition element by element and against the closed-form spectrum of the
finite-difference Laplacian; and the oracle's multilevel solver on test 1 (N = 4, s = 20, R = 4)
against plain ALS, the comparison of Table tab:Laplacian (qualitative: far fewer cycles)."""
import itertools

import numpy as np
import pytest

from oracle import tensor as T, als as ALS, multigrid as MG
from paper_1111_6091_gb300 import synth


@pytest.mark.parametrize("d,s", [(1, 4), (2, 3), (3, 2)])
def test_laplacian_elementwise_definition(d, s):
    Z = synth.laplacian_tensor(d, s)
    assert Z.shape == (s,) * (2 * d)
    D = 2.0 * np.eye(s) - np.eye(s, k=1) - np.eye(s, k=-1)
    for idx in itertools.product(range(s), repeat=2 * d):
        i, j = idx[:d], idx[d:]
        v = sum(D[i[k], j[k]] * np.prod([1.0 if i[m] == j[m] else 0.0 for m in range(d) if m != k])
                for k in range(d))
        assert Z[idx] == v


@pytest.mark.parametrize("d,s", [(2, 5), (3, 4)])
def test_laplacian_spectrum_closed_form(d, s):
    """Unfolding the first d modes against the last d gives back the s^d x s^d matrix; its
    eigenvalues are the sums over grid dimensions of D's eigenvalues 2 - 2 cos(k pi / (s + 1))."""
    Z = synth.laplacian_tensor(d, s)
    M = np.reshape(Z, (s ** d, s ** d), order="F")
    assert np.array_equal(M, M.T)
    lam = 2.0 - 2.0 * np.cos(np.arange(1, s + 1) * np.pi / (s + 1))
    expect = np.sort([sum(c) for c in itertools.product(lam, repeat=d)])
    assert np.allclose(np.linalg.eigvalsh(M), expect, rtol=0, atol=1e-12)


def test_laplacian_exact_in_float32():
    Z = synth.laplacian_tensor(2, 20)
    assert np.array_equal(Z.astype(np.float32).astype(np.float64), Z)


def test_multilevel_beats_als_on_laplacian_test_1():
    """Table tab:LapParams test 1 (N = 4, s = 20, R = 4), uniform [0,1] starts, two levels
    (coarsest 10): the multilevel solver reaches g < 1e-8 in far fewer cycles than ALS needs
    iterations (the paper reports 37 cycles against 1897 iterations at 1e-10; qualitative)."""
    Z = synth.laplacian_tensor(2, 20)
    R = 4
    A0 = synth.uniform_start(Z.shape, R, 0)
    tfms = [synth.uniform_start(Z.shape, R, 1 + t) for t in range(2)]
    r = MG.multilevel(Z, A0, tfms, MG.Options(coarsest=(10,) * 4, tol=1e-8))
    assert r.converged and len(r.levels) == 2
    _, it = ALS.als(Z, A0, 4000, tol=1e-8, g_fn=T.g_value)
    assert 5 * (r.setup_cycles + r.solve_cycles) < it
