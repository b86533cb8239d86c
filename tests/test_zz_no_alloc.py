"""The allocation-free MTTKRP entry point (cpmg_mttkrp_noalloc).

It exists for callers that cannot allocate device memory: their own allocator already owns
the GPU, or they cannot afford the synchronization cudaMalloc and cudaFree may cause.  Its
scratch is a fixed array inside the library.  These tests call it through the C ABI several
times in a row on different shapes (so each call starts from the previous call's leftovers in
the shared array) and check every result against the context-based cpmg_mttkrp and against
the oracle's MTTKRP (Eq. fineeq1), within the kernel tests' tolerance.

The file sorts last so that a run stopping at its first failure has run every other test."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

# relative to sum |z| |Khatri-Rao row| per entry: FP32 products, float-pair products
TOL = {0: 2e-5, 3: 1e-11}


def _fn(lib):
    from paper_1111_6091_gb300 import cpmg
    fn = lib.cpmg_mttkrp_noalloc
    fn.restype = C.c_int
    fn.argtypes = [C.POINTER(cpmg.cpmg_tensor), C.c_int, C.POINTER(C.c_void_p), C.c_int, C.c_int,
                   C.c_void_p, C.c_void_p]
    return fn


def _call_noalloc(lib, Z, A, mode, prec):
    import torch
    from paper_1111_6091_gb300 import cpmg
    d = cpmg.tensor_desc(Z)
    R = A[0].shape[0]
    M = torch.full((R, d.dims[mode]), float("nan"), dtype=torch.float64, device="cuda")
    ptrs = (C.c_void_p * len(A))(*[a.data_ptr() for a in A])
    st = torch.cuda.current_stream().cuda_stream
    s = _fn(lib)(C.byref(d), R, ptrs, mode, prec, C.c_void_p(M.data_ptr()), C.c_void_p(st))
    assert s == cpmg.OK, cpmg.status_str(s)
    torch.cuda.current_stream().synchronize()
    return M


def _scale(Zn, An, mode):
    """sum over the contraction of |z| * |Khatri-Rao row|, per output entry"""
    from oracle import tensor as ot
    return ot.mttkrp(np.abs(Zn.astype(np.float64)), [np.abs(a) for a in An], mode)


def _check(cpmg_ctx, lib, dims, R, seed, modes, prec):
    from oracle import tensor as ot
    from paper_1111_6091_gb300 import cpmg
    rng = np.random.default_rng(seed)
    Zn = np.asfortranarray(rng.standard_normal(dims).astype(np.float32))
    An = [np.asfortranarray(rng.standard_normal((I, R))) for I in dims]
    Z = cpmg.colmajor(Zn)
    A = [cpmg.colmajor(a) for a in An]
    for mode in modes:
        got = cpmg.to_numpy(_call_noalloc(lib, Z, A, mode, prec))
        ref = cpmg.to_numpy(cpmg.cpmg_mttkrp(cpmg_ctx, Z, A, mode, prec))
        exact = ot.mttkrp(Zn.astype(np.float64), An, mode)
        scale = _scale(Zn, An, mode)
        assert np.all(np.isfinite(got)), (dims, mode)
        assert np.all(np.abs(got - ref) <= 2 * TOL[prec] * scale + 1e-300), (dims, mode)
        assert np.all(np.abs(got - exact) <= TOL[prec] * scale + 1e-300), (dims, mode)


@pytest.mark.parametrize("prec", [0, 3])
def test_noalloc_matches_mttkrp_and_oracle_two_calls(cpmg_ctx, prec):
    from paper_1111_6091_gb300 import cpmg
    lib = cpmg.lib()
    for dims, R, seed in [((128, 96, 80), 8, 11), ((63, 41, 37), 5, 12)]:
        _check(cpmg_ctx, lib, dims, R, seed, range(3), prec)


def test_noalloc_fewer_units_when_partials_overflow(cpmg_ctx):
    """Mode 0 of a 32768 x 16 x 4 tensor at R=16 in float pairs: 64 row segments of 512 rows
    leave most of the 152 SMs idle, so the default plan takes at least two chunks per segment,
    whose partial sums (2 x 32768 x 16 x 8 bytes = 8 MiB) plus the tables exceed the array.
    The call succeeds only by halving the chunks; the result must not change."""
    from paper_1111_6091_gb300 import cpmg
    _check(cpmg_ctx, cpmg.lib(), (32768, 16, 4), 16, 21, [0, 0], 3)


def test_noalloc_register_kernel_when_table_overflows(cpmg_ctx):
    """Mode 0 of a 16 x 600 x 600 tensor at R=8: the bulk-copy kernel's full Khatri-Rao row
    table is 360000 x 8 x 4 bytes = 11 MiB, more than the array, so the call falls back to the
    register-load kernel and its two small tables."""
    from paper_1111_6091_gb300 import cpmg
    _check(cpmg_ctx, cpmg.lib(), (16, 600, 600), 8, 22, [0, 1], 0)


def test_noalloc_rejects_too_large_and_bad_args(cpmg_ctx):
    import torch
    from paper_1111_6091_gb300 import cpmg
    fn = _fn(cpmg.lib())
    # a first mode of 2^20 rows: even with one work unit per row segment, the float-pair
    # partial sums need 2^20 x 16 (rank) x 8 bytes = 128 MiB, more than the 8 MiB array
    d = cpmg.cpmg_tensor()
    d.N = 2
    d.dims[0] = 1 << 20
    d.dims[1] = 1
    d.dtype = cpmg.F32
    d.mem = cpmg.MEM_DEVICE
    Z = torch.zeros(1 << 20, dtype=torch.float32, device="cuda")
    d.data = Z.data_ptr()
    A = [torch.zeros((16, 1 << 20), dtype=torch.float64, device="cuda"),
         torch.zeros((16, 1), dtype=torch.float64, device="cuda")]
    M = torch.zeros((16, 1 << 20), dtype=torch.float64, device="cuda")
    ptrs = (C.c_void_p * 2)(A[0].data_ptr(), A[1].data_ptr())
    assert fn(C.byref(d), 16, ptrs, 0, 3, C.c_void_p(M.data_ptr()), None) == cpmg.OUT_OF_BUDGET
    assert fn(None, 16, ptrs, 0, 3, C.c_void_p(M.data_ptr()), None) == cpmg.INVALID_ARG
    d.mem = cpmg.MEM_HOST
    assert fn(C.byref(d), 16, ptrs, 0, 3, C.c_void_p(M.data_ptr()), None) == cpmg.INVALID_ARG
