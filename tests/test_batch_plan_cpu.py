"""Host logic of the batched form (no GPU): the MTTKRP work units of every mode cover each
(first-mode row, column) pair of the mode's unfolding exactly once, and each unit writes a
partial-sum slot of its own, so the ordered reduction of the slots is the full sum."""

import numpy as np
import pytest

ROWS = 64   # first-mode rows per unit


def _numel(dims):
    return int(np.prod(dims))


def _check_mode(dims, R, target, mode):
    from paper_1111_6091_gb300 import cpmg
    units, nk, tot = cpmg.batch_plan(dims, R, target, mode)
    I0 = dims[0]
    nrb = -(-I0 // ROWS)
    if mode == 0:
        ncol = _numel(dims) // I0
        cover = np.zeros((nrb, ncol), dtype=np.int64)
        slots = set()
        for rb, k, c0, c1, inx in units:
            assert inx == -1 and 0 <= rb < nrb and 0 <= c0 < c1 <= ncol and 0 <= k < nk
            cover[rb, c0:c1] += 1
            assert (k, rb) not in slots   # slot k holds rows of every row block once
            slots.add((k, rb))
    else:
        In = dims[mode]
        ncol = _numel(dims) // (I0 * In)
        cover = np.zeros((In, nrb, ncol), dtype=np.int64)
        slots = set()
        for rb, k, c0, c1, inx in units:
            assert 0 <= inx < In and 0 <= rb < nrb and 0 <= c0 < c1 <= ncol and 0 <= k < nk
            cover[inx, rb, c0:c1] += 1
            assert (inx, k) not in slots
            slots.add((inx, k))
    assert np.all(cover == 1), (dims, mode)
    # the partial storage holds every slot of every mode: 8 per slot per first-mode row (mode 0)
    # or per output row (later modes)
    return tot


SHAPES = [(1, 1, 1), (64, 3, 2), (65, 17, 16), (63, 64, 65), (129, 16, 20), (16, 48, 17, 18),
          (33, 30), (128, 128, 16), (2, 200, 3), (17, 1, 9, 5)]


@pytest.mark.parametrize("dims", SHAPES)
@pytest.mark.parametrize("target", [1, 2048, 8192, 32768])
def test_units_cover_every_pair_once(dims, target):
    R = 3
    totals = {_check_mode(dims, R, target, n) for n in range(len(dims))}
    assert len(totals) == 1   # the partial storage is the same whichever mode is inspected


def test_random_batch_shapes():
    from paper_1111_6091_gb300 import synth
    for sp in synth.batch_specs(24, seed=5):
        for n in range(len(sp["dims"])):
            _check_mode(sp["dims"], sp["R"], 8192, n)


def test_partial_storage_formula():
    """8 doubles per slot and row: mode 0 has nch slots of I_1 rows, mode n > 0 has In * nk."""
    from paper_1111_6091_gb300 import cpmg
    dims, R, target = (70, 65, 16), 8, 4096
    total = 0
    for n in range(3):
        units, nk, tot = cpmg.batch_plan(dims, R, target, n)
        total += 8 * (nk * dims[0] if n == 0 else dims[n] * nk)
    assert total == tot


def test_invalid_plans_rejected():
    from paper_1111_6091_gb300 import cpmg
    for args in (((4,), 2, 8192, 0), ((4, 4, 4, 4, 4), 2, 8192, 0), ((4, 4), 9, 8192, 0), ((4, 4), 2, 0, 0),
                 ((4, 4), 2, 8192, 2), ((4, 0), 2, 8192, 0), ((1 << 16, 1 << 16), 2, 8192, 0)):
        with pytest.raises(cpmg.CpmgError) as e:
            cpmg.batch_plan(*args)
        assert e.value.status == cpmg.INVALID_ARG
