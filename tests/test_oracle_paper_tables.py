"""Qualitative pin against the paper's dense-tensor table (Section 6.3, Table tab:IJK)."""
import os

import numpy as np

from oracle import tensor as T, als as ALS, multigrid as MG, align
from paper_1111_6091_gb300 import synth

HERE = os.path.dirname(__file__)


def load_rows():
    rows = []
    with open(os.path.join(HERE, "golden", "tab_ijk.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                rows.append([int(v) for v in line.split()])
    return rows


def test_ijk_multilevel_fmg_beats_als_s50_r3():
    s, R, als_it_paper, ml_it_paper, levs = [r for r in load_rows() if r[:2] == [50, 3]][0]
    Z = synth.ijk_tensor(s)
    rng = np.random.default_rng(0)
    A0 = [rng.uniform(size=(s, R)) for _ in range(3)]
    tf = [[rng.uniform(size=(s, R)) for _ in range(3)] for _ in range(2)]
    Ac0 = [rng.uniform(size=(4, R)) for _ in range(3)]
    opts = MG.Options(coarsest=(4, 4, 4), tol=1e-10)
    r = MG.multilevel_fmg(Z, A0, tf, Ac0, 100, opts)
    assert r.converged
    assert len(r.levels) == levs                      # 50 -> 25 -> 13 -> 7 -> 4
    it_ml = r.setup_cycles + r.solve_cycles
    A, it_als = ALS.als(Z, A0, 10000, tol=1e-10, g_fn=T.g_value)
    assert T.g_value(Z, A) < 1e-10
    # same stationary point, and the paper's qualitative gap (more than 20x fewer iterations)
    assert align.factor_error(A, r.A) < 1e-7
    assert it_ml * 20 < it_als
    assert it_ml < 4 * ml_it_paper and it_als > als_it_paper / 4
