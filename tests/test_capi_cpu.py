"""CPU-side checks of the C ABI: the library builds, loads without a GPU, exports every
function include/cpmg.h declares, and its host-only calls behave."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1111_6091_gb300 import build, cpmg
    build.build()
    return cpmg.lib()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "cpmg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\**\s+\**([A-Za-z_][A-Za-z0-9_]*)\s*\(",
                       src, flags=re.M)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 20, names
    for n in names:
        assert hasattr(lib, n), f"{n} declared in cpmg.h but not exported"


def test_opts_default_is_the_paper_table(lib):
    from paper_1111_6091_gb300 import cpmg
    o = cpmg.make_opts()
    assert (o.nu1_setup, o.nu2_setup, o.nuc_setup, o.n_t) == (5, 5, 100, 2)
    assert (o.nu1, o.nu2, o.nuc) == (1, 1, 50)
    assert o.gs_sweeps == 10 and o.max_cycles == 500 and o.max_als_iters == 10000
    assert o.max_setup_cycles == 5 and abs(o.stag_eps - 0.1) < 1e-15 and o.tol == 1e-10
    # additions that are not in the paper's table: MIXED policy with switch factor 4, no ALS
    # fallback unless asked for
    assert o.precision == cpmg.PREC_MIXED and o.mixed_switch == 4.0 and o.als_fallback == 0
    assert o.dimension_tree == 1 and o.ttm_tensor_cores == 1


def test_status_strings(lib):
    from paper_1111_6091_gb300 import cpmg
    assert cpmg.status_str(cpmg.OK) == "ok"
    assert "budget" in cpmg.status_str(cpmg.OUT_OF_BUDGET)
    assert cpmg.status_str(99) == "unknown status"


def test_null_arguments_rejected_without_gpu(lib):
    from paper_1111_6091_gb300 import cpmg
    assert lib.cpmg_create(None, 0, 0, None) == cpmg.INVALID_ARG
    r = cpmg.cpmg_result()
    o = cpmg.make_opts()
    assert lib.cp_als_sweep(None, None, 3, None, 1, C.byref(o), C.byref(r)) == cpmg.INVALID_ARG
    assert lib.mg_fas_solve(None, None, None, None, C.byref(o), C.byref(r)) == cpmg.INVALID_ARG
    assert lib.cpmg_hier_levels(None) == 0
    assert lib.cpmg_bytes_in_use(None) == 0
    assert lib.mg_fmg(None, None, None, None, None, 100, C.byref(o), C.byref(r)) == cpmg.INVALID_ARG
    assert lib.cpmg_batch_solve(None, 1, None, None, None, C.byref(o), C.byref(r)) == cpmg.INVALID_ARG
    t = C.c_uint64()
    assert lib.cpmg_server_submit(None, None, 2, None, C.byref(o), C.byref(t)) == cpmg.INVALID_ARG
    assert lib.cpmg_server_poll(None, 1, C.byref(r)) == cpmg.INVALID_ARG
    assert lib.cpmg_server_wait(None, 0.0) == cpmg.INVALID_ARG
    assert lib.cpmg_server_config(None, 0, 0, 0, 0) == cpmg.INVALID_ARG
    assert lib.cpmg_server_stats(None, None, None, None, None) == cpmg.INVALID_ARG
    assert lib.cpmg_server_cancel(None, 1) == cpmg.INVALID_ARG
    assert lib.cpmg_debug_config(None, 1.0, 0) == cpmg.INVALID_ARG


def test_struct_layout_matches_header(lib):
    """ctypes mirrors must match the C structs field by field (sizes checked against the header
    field order: int, int64[8], int, int, pointer)."""
    from paper_1111_6091_gb300 import cpmg
    assert C.sizeof(cpmg.cpmg_tensor) == 4 + 4 + 8 * 8 + 4 + 4 + 8
    assert cpmg.cpmg_result.seconds.offset == C.sizeof(cpmg.cpmg_result) - 8
