"""The allocation-free MTTKRP entry point (cpmg_mttkrp_noalloc).

It exists for callers that cannot allocate device memory (their allocator owns the GPU,
or they cannot afford cudaMalloc's synchronization); its scratch is a fixed array inside
the library.  This test calls it through the C ABI twice in a row, on different shapes
(so the second call starts from the first call's leftovers in the shared array), and
checks each result against cpmg_mttkrp within the kernel tests' tolerance."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = {0: 2e-5, 3: 1e-11}


def _call_noalloc(lib, Z, A, mode, prec):
    import torch
    from paper_1111_6091_gb300 import cpmg
    fn = lib.cpmg_mttkrp_noalloc
    fn.restype = C.c_int
    fn.argtypes = [C.POINTER(cpmg.cpmg_tensor), C.c_int, C.POINTER(C.c_void_p), C.c_int, C.c_int,
                   C.c_void_p, C.c_void_p]
    d = cpmg.tensor_desc(Z)
    R = A[0].shape[0]
    M = torch.full((R, d.dims[mode]), float("nan"), dtype=torch.float64, device="cuda")
    ptrs = (C.c_void_p * len(A))(*[a.data_ptr() for a in A])
    st = torch.cuda.current_stream().cuda_stream
    s = fn(C.byref(d), R, ptrs, mode, prec, C.c_void_p(M.data_ptr()), C.c_void_p(st))
    assert s == cpmg.OK, cpmg.status_str(s)
    torch.cuda.current_stream().synchronize()
    return M


@pytest.mark.parametrize("prec", [0, 3])
def test_noalloc_matches_mttkrp_two_calls(cpmg_ctx, prec):
    from paper_1111_6091_gb300 import cpmg
    lib = cpmg.lib()
    cases = [((128, 96, 80), 8, 11), ((63, 41, 37), 5, 12)]
    for dims, R, seed in cases:
        rng = np.random.default_rng(seed)
        Zn = np.asfortranarray(rng.standard_normal(dims).astype(np.float32))
        An = [np.asfortranarray(rng.standard_normal((I, R))) for I in dims]
        Z = cpmg.colmajor(Zn)
        A = [cpmg.colmajor(a) for a in An]
        for mode in range(3):
            got = cpmg.to_numpy(_call_noalloc(lib, Z, A, mode, prec))
            ref = cpmg.to_numpy(cpmg.cpmg_mttkrp(cpmg_ctx, Z, A, mode, prec))
            # scale: sum over the contraction of |z| * |Khatri-Rao row|
            absA = [np.abs(a) for a in An]
            Zabs = np.abs(Zn.astype(np.float64))
            letters = "abc"
            spec = letters + "," + ",".join(f"{l}r" for i, l in enumerate(letters) if i != mode) + "->" + letters[mode] + "r"
            scale = np.einsum(spec, Zabs, *[absA[i] for i in range(3) if i != mode])
            assert np.all(np.isfinite(got))
            assert np.all(np.abs(got - ref) <= 2 * TOL[prec] * scale + 1e-300), (dims, mode)


def test_noalloc_rejects_too_large_and_bad_args(cpmg_ctx):
    import torch
    from paper_1111_6091_gb300 import cpmg
    lib = cpmg.lib()
    fn = lib.cpmg_mttkrp_noalloc
    fn.restype = C.c_int
    fn.argtypes = [C.POINTER(cpmg.cpmg_tensor), C.c_int, C.POINTER(C.c_void_p), C.c_int, C.c_int,
                   C.c_void_p, C.c_void_p]
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
