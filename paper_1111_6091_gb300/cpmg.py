"""Thin ctypes binding over libcpmg (include/cpmg.h): argument marshalling only.

Every numeric step runs in the library's CUDA kernels.  If ``libcpmg.so`` has not
been built, :func:`lib` raises instead of falling back to anything else.

Array conventions (same as the C ABI)
-------------------------------------
* A tensor of sizes (I_1, ..., I_N) is column-major.  As a torch tensor it is a
  C-contiguous tensor of the *reversed* shape (I_N, ..., I_1); :func:`colmajor`
  builds one from a NumPy array and :func:`to_numpy` converts back.
* A factor matrix A^(n) (I_n x R, column-major, float64) is a contiguous torch
  float64 tensor of shape (R, I_n).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

MAX_MODES = 8
MAX_RANK = 16
MAX_TEST_BLOCKS = 4

OK, INVALID_ARG, OUT_OF_BUDGET, NOT_CONVERGED, NUMERIC, TIMEOUT, CUDA_ERROR, PENDING, CANCELLED, UNSUPPORTED = range(10)
F32, F64 = 0, 1
MEM_DEVICE, MEM_HOST = 0, 1
PREC_FP32, PREC_FP64, PREC_MIXED, PREC_DF, PREC_BF16X3, PREC_MIXED_BF16 = 0, 1, 2, 3, 4, 5

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcpmg.so")


class cpmg_tensor(C.Structure):
    _fields_ = [("N", C.c_int), ("dims", C.c_int64 * MAX_MODES), ("dtype", C.c_int), ("mem", C.c_int),
                ("data", C.c_void_p)]


class cpmg_opts(C.Structure):
    _fields_ = [("precision", C.c_int), ("tol", C.c_double), ("max_cycles", C.c_int),
                ("max_als_iters", C.c_int), ("nu1_setup", C.c_int), ("nu2_setup", C.c_int),
                ("nuc_setup", C.c_int), ("nu1", C.c_int), ("nu2", C.c_int), ("nuc", C.c_int),
                ("n_t", C.c_int), ("max_setup_cycles", C.c_int), ("stag_eps", C.c_double),
                ("gs_sweeps", C.c_int), ("coarsest", C.c_int64 * MAX_MODES), ("als_fallback", C.c_int),
                ("mixed_switch", C.c_double), ("check_every", C.c_int), ("use_graphs", C.c_int),
                ("ttm_tensor_cores", C.c_int), ("dimension_tree", C.c_int)]


class cpmg_result(C.Structure):
    _fields_ = [("f", C.c_double), ("g", C.c_double), ("iters_setup", C.c_int), ("iters_solve", C.c_int),
                ("iters_als", C.c_int), ("levels", C.c_int), ("restarted", C.c_int),
                ("refine_sweeps", C.c_int), ("status", C.c_int), ("seconds", C.c_double)]


class CpmgError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {status_str(status)} (status {status})")


_lib = None
_P = C.c_void_p
_PP = C.POINTER(C.c_void_p)

_SIGS = {
    "cpmg_opts_default": (None, [C.POINTER(cpmg_opts)]),
    "cpmg_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_size_t, _P]),
    "cpmg_destroy": (None, [_P]),
    "cpmg_set_stream": (C.c_int, [_P, _P]),
    "cpmg_status_str": (C.c_char_p, [C.c_int]),
    "cpmg_bytes_in_use": (C.c_size_t, [_P]),
    "cpmg_mttkrp": (C.c_int, [_P, C.POINTER(cpmg_tensor), C.c_int, _PP, C.c_int, C.c_int, _P]),
    "cpmg_ttm": (C.c_int, [_P, C.POINTER(cpmg_tensor), _PP, C.POINTER(C.c_int64), C.c_int, _P]),
    "cpmg_eval_fg": (C.c_int, [_P, C.POINTER(cpmg_tensor), C.c_int, _PP, C.POINTER(C.c_double),
                               C.POINTER(C.c_double)]),
    "cp_als_sweep": (C.c_int, [_P, C.POINTER(cpmg_tensor), C.c_int, _PP, C.c_int, C.POINTER(cpmg_opts),
                               C.POINTER(cpmg_result)]),
    "mg_setup": (C.c_int, [_P, C.POINTER(cpmg_tensor), C.c_int, _PP, _PP, C.POINTER(cpmg_opts),
                           C.POINTER(C.c_void_p), C.POINTER(cpmg_result)]),
    "mg_fas_solve": (C.c_int, [_P, _P, C.POINTER(cpmg_tensor), _PP, C.POINTER(cpmg_opts),
                               C.POINTER(cpmg_result)]),
    "mg_fmg": (C.c_int, [_P, _P, C.POINTER(cpmg_tensor), _PP, _PP, C.c_int, C.POINTER(cpmg_opts),
                         C.POINTER(cpmg_result)]),
    "cpmg_batch_plan": (C.c_int, [C.c_int, C.POINTER(C.c_int64), C.c_int, C.c_int64, C.c_int,
                                  C.POINTER(C.c_int64), C.c_int64, C.POINTER(C.c_int64), C.POINTER(C.c_int),
                                  C.POINTER(C.c_int64)]),
    "cpmg_hier_free": (None, [_P]),
    "cpmg_hier_levels": (C.c_int, [_P]),
    "cpmg_hier_level_info": (C.c_int, [_P, C.c_int, C.POINTER(C.c_int64), C.POINTER(C.c_int), _P, _PP]),
    "cpmg_decompose": (C.c_int, [_P, C.POINTER(cpmg_tensor), C.c_int, _PP, _PP, C.POINTER(cpmg_opts),
                                 C.POINTER(cpmg_result)]),
    "cpmg_profile_enable": (C.c_int, [_P, C.c_int]),
    "cpmg_profile_read": (C.c_int, [_P, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_int64),
                                    C.POINTER(C.c_double)]),
    "cpmg_profile_reset": (C.c_int, [_P]),
    "cpmg_launch_count": (C.c_int64, [_P]),
    "cpmg_batch_solve": (C.c_int, [_P, C.c_int, C.POINTER(cpmg_tensor), C.POINTER(C.c_int), _PP,
                                   C.POINTER(cpmg_opts), C.POINTER(cpmg_result)]),
    "cpmg_server_config": (C.c_int, [_P, C.c_size_t, C.c_int, C.c_int, C.c_int64]),
    "cpmg_debug_config": (C.c_int, [_P, C.c_double, C.c_int]),
    "cpmg_server_cancel": (C.c_int, [_P, C.c_uint64]),
    "cpmg_server_submit_multilevel": (C.c_int, [_P, C.POINTER(cpmg_tensor), C.c_int, _PP, _PP,
                                                C.POINTER(cpmg_opts), C.POINTER(C.c_uint64)]),
    "cpmg_server_submit": (C.c_int, [_P, C.POINTER(cpmg_tensor), C.c_int, _PP, C.POINTER(cpmg_opts),
                                     C.POINTER(C.c_uint64)]),
    "cpmg_server_poll": (C.c_int, [_P, C.c_uint64, C.POINTER(cpmg_result)]),
    "cpmg_server_wait": (C.c_int, [_P, C.c_double]),
    "cpmg_server_stats": (C.c_int, [_P, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double),
                                    C.POINTER(C.c_int64)]),
}


def lib():
    """Load libcpmg.so (built by ``__graft_entry__.build()``); raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built; run `python -c 'import __graft_entry__ as g; g.build()'`")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def status_str(s: int) -> str:
    return lib().cpmg_status_str(int(s)).decode()


def _check(s: int, where: str, allow=(OK,)):
    if s not in allow:
        raise CpmgError(s, where)
    return s


# ------------------------------------------------------------------ array helpers
def colmajor(a: np.ndarray, device="cuda", dtype=None, pin=False):
    """Torch tensor holding ``a`` column-major (reversed shape, C-contiguous)."""
    import torch
    arr = np.asarray(a)
    if dtype is not None:
        arr = arr.astype(dtype)
    t = torch.from_numpy(np.ascontiguousarray(arr.T))
    if device == "cpu":
        return t.pin_memory() if pin else t.clone()
    return t.to(device)


def to_numpy(t) -> np.ndarray:
    """Inverse of :func:`colmajor`: a Fortran-ordered NumPy array of the original shape."""
    return t.detach().cpu().numpy().T


def _dims(t):
    return tuple(int(d) for d in reversed(t.shape))


def tensor_desc(Z, dims=None) -> cpmg_tensor:
    """Descriptor of a column-major torch tensor (device or host)."""
    import torch
    dims = dims or _dims(Z)
    d = cpmg_tensor()
    d.N = len(dims)
    for i, v in enumerate(dims):
        d.dims[i] = v
    d.dtype = F64 if Z.dtype == torch.float64 else F32
    if Z.dtype not in (torch.float32, torch.float64):
        raise TypeError("tensor must be float32 or float64")
    if not Z.is_contiguous():
        raise ValueError("tensor must be contiguous (reversed-shape column-major view)")
    d.mem = MEM_DEVICE if Z.is_cuda else MEM_HOST
    d.data = Z.data_ptr()
    return d


def _ptrs(ts):
    arr = (C.c_void_p * max(1, len(ts)))()
    for i, t in enumerate(ts):
        arr[i] = t.data_ptr()
    return arr


def make_opts(**kw) -> cpmg_opts:
    o = cpmg_opts()
    lib().cpmg_opts_default(C.byref(o))
    for k, v in kw.items():
        if k == "coarsest":
            for i, x in enumerate(v):
                o.coarsest[i] = int(x)
        else:
            setattr(o, k, v)
    return o


def result_dict(r: cpmg_result) -> dict:
    return {k: getattr(r, k) for k, _ in cpmg_result._fields_}


# ------------------------------------------------------------------ context
class Context:
    """A libcpmg context on ``device``, issuing work on the current torch stream."""

    def __init__(self, device=0, budget_bytes=0, stream=None):
        import torch
        self.device = device
        if stream is None:
            stream = torch.cuda.current_stream(device).cuda_stream
        h = C.c_void_p()
        _check(lib().cpmg_create(C.byref(h), int(device), C.c_size_t(budget_bytes), C.c_void_p(stream)),
               "cpmg_create")
        self.h = h

    def close(self):
        if self.h:
            lib().cpmg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def bytes_in_use(self):
        return lib().cpmg_bytes_in_use(self.h)

    def launches(self):
        return lib().cpmg_launch_count(self.h)

    def profile(self, enable=True):
        _check(lib().cpmg_profile_enable(self.h, int(enable)), "cpmg_profile_enable")

    def profile_read(self, kind=0):
        ms, n, b = C.c_double(), C.c_int64(), C.c_double()
        _check(lib().cpmg_profile_read(self.h, kind, C.byref(ms), C.byref(n), C.byref(b)), "cpmg_profile_read")
        return ms.value, n.value, b.value

    def profile_reset(self):
        _check(lib().cpmg_profile_reset(self.h), "cpmg_profile_reset")

    def debug_config(self, wait_limit_s=2.0, unreachable_barrier=False):
        """Failure-detection test hook of the batched form (cpmg_debug_config)."""
        _check(lib().cpmg_debug_config(self.h, float(wait_limit_s), int(bool(unreachable_barrier))),
               "cpmg_debug_config")


# ------------------------------------------------------------------ calls (same names as the ABI)
def cpmg_mttkrp(ctx, Z, A, mode, precision=PREC_FP32, M=None):
    import torch
    R = A[0].shape[0]
    d = tensor_desc(Z)
    if M is None:
        M = torch.empty((R, d.dims[mode]), dtype=torch.float64, device=Z.device)
    _check(lib().cpmg_mttkrp(ctx.h, C.byref(d), R, _ptrs(A), mode, precision, C.c_void_p(M.data_ptr())),
           "cpmg_mttkrp")
    return M


def cpmg_ttm(ctx, Z, Rhat, tensor_cores=0):
    """Rhat: list (per mode) of torch float64 (I_n, Ic) tensors = column-major Ic x I_n, or None."""
    import torch
    d = tensor_desc(Z)
    N = d.N
    ic = (C.c_int64 * MAX_MODES)()
    ptrs = (C.c_void_p * MAX_MODES)()
    out_dims = list(_dims(Z))
    for n in range(N):
        if Rhat[n] is not None:
            ic[n] = Rhat[n].shape[1]
            ptrs[n] = Rhat[n].data_ptr()
            out_dims[n] = int(Rhat[n].shape[1])
    Y = torch.empty(tuple(reversed(out_dims)), dtype=Z.dtype, device=Z.device)
    _check(lib().cpmg_ttm(ctx.h, C.byref(d), ptrs, ic, int(tensor_cores), C.c_void_p(Y.data_ptr())), "cpmg_ttm")
    return Y


def cpmg_batch_solve(ctx, Zs, As, opts=None, **kw):
    """Batched CP-ALS on the tensors ``Zs`` with factor lists ``As`` (updated in place): all on the
    device, or all host (CPU, preferably pinned) tensors, which the library copies in and out.
    Returns (status, list of result dicts)."""
    o = opts or make_opts(**kw)
    n = len(Zs)
    descs = (cpmg_tensor * n)()
    ranks = (C.c_int * n)()
    keep = []
    rows = (C.c_void_p * n)()
    for t, (Z, A) in enumerate(zip(Zs, As)):
        descs[t] = tensor_desc(Z)
        ranks[t] = A[0].shape[0]
        p = _ptrs(A)
        keep.append(p)
        rows[t] = C.cast(p, C.c_void_p)
    res = (cpmg_result * n)()
    s = lib().cpmg_batch_solve(ctx.h, n, descs, ranks, C.cast(rows, _PP), C.byref(o), res)
    _check(s, "cpmg_batch_solve", allow=(OK, NOT_CONVERGED, NUMERIC))
    return s, [result_dict(r) for r in res]


class Server:
    """Request server on a context (continuous batching of CP-ALS problems)."""

    def __init__(self, ctx, budget_bytes=0, max_active=0, sweeps_per_launch=0, unit_elements=0):
        self.ctx = ctx
        self._keep = {}
        _check(lib().cpmg_server_config(ctx.h, int(budget_bytes), int(max_active), int(sweeps_per_launch),
                                        int(unit_elements)), "cpmg_server_config")

    def submit(self, Z, A, opts=None, **kw):
        o = opts or make_opts(**kw)
        d = tensor_desc(Z)
        p = _ptrs(A)
        t = C.c_uint64()
        _check(lib().cpmg_server_submit(self.ctx.h, C.byref(d), A[0].shape[0], p, C.byref(o), C.byref(t)),
               "cpmg_server_submit")
        self._keep[t.value] = (Z, A, p)
        return t.value

    def submit_multilevel(self, Z, A, A_test, opts=None, **kw):
        """Queue a request for the multilevel driver (Section 6.1); A_test: n_t blocks of N arrays."""
        o = opts or make_opts(**kw)
        o.n_t = len(A_test)
        d = tensor_desc(Z)
        p = _ptrs(A)
        flat = [a for blk in A_test for a in blk]
        pt = _ptrs(flat)
        t = C.c_uint64()
        _check(lib().cpmg_server_submit_multilevel(self.ctx.h, C.byref(d), A[0].shape[0], C.cast(p, _PP),
                                                   C.cast(pt, _PP), C.byref(o), C.byref(t)),
               "cpmg_server_submit_multilevel")
        self._keep[t.value] = (Z, A, A_test, p, pt)
        return t.value

    def poll(self, ticket):
        """None while pending, else the result dict."""
        r = cpmg_result()
        s = lib().cpmg_server_poll(self.ctx.h, C.c_uint64(ticket), C.byref(r))
        if s == PENDING:
            return None
        _check(s, "cpmg_server_poll")
        self._keep.pop(ticket, None)
        return result_dict(r)

    def cancel(self, ticket):
        _check(lib().cpmg_server_cancel(self.ctx.h, C.c_uint64(ticket)), "cpmg_server_cancel")

    def wait(self, timeout_s=600.0):
        return lib().cpmg_server_wait(self.ctx.h, float(timeout_s))

    def stats(self):
        p50, p99, rps, n = C.c_double(), C.c_double(), C.c_double(), C.c_int64()
        _check(lib().cpmg_server_stats(self.ctx.h, C.byref(p50), C.byref(p99), C.byref(rps), C.byref(n)),
               "cpmg_server_stats")
        return {"p50_s": p50.value, "p99_s": p99.value, "req_per_s": rps.value, "completed": n.value}


def cpmg_eval_fg(ctx, Z, A):
    d = tensor_desc(Z)
    f, g = C.c_double(), C.c_double()
    _check(lib().cpmg_eval_fg(ctx.h, C.byref(d), A[0].shape[0], _ptrs(A), C.byref(f), C.byref(g)), "cpmg_eval_fg")
    return f.value, g.value


def cp_als_sweep(ctx, Z, A, nsweeps, opts=None, **kw):
    o = opts or make_opts(**kw)
    r = cpmg_result()
    d = tensor_desc(Z)
    s = lib().cp_als_sweep(ctx.h, C.byref(d), A[0].shape[0], _ptrs(A), int(nsweeps), C.byref(o), C.byref(r))
    _check(s, "cp_als_sweep", allow=(OK, NOT_CONVERGED))
    return result_dict(r)


class Hierarchy:
    def __init__(self, h):
        self.h = h

    def levels(self):
        return lib().cpmg_hier_levels(self.h)

    def level_info(self, level, with_rhat=False):
        dims = (C.c_int64 * MAX_MODES)()
        co = (C.c_int * MAX_MODES)()
        _check(lib().cpmg_hier_level_info(self.h, level, dims, co, None, None), "cpmg_hier_level_info")
        return dims, co

    def level_tensor(self, level, N, dtype):
        import torch
        dims = (C.c_int64 * MAX_MODES)()
        co = (C.c_int * MAX_MODES)()
        _check(lib().cpmg_hier_level_info(self.h, level, dims, co, None, None), "cpmg_hier_level_info")
        shape = tuple(int(dims[n]) for n in range(N))
        Y = torch.empty(tuple(reversed(shape)), dtype=dtype, device="cuda")
        _check(lib().cpmg_hier_level_info(self.h, level, dims, co, C.c_void_p(Y.data_ptr()), None),
               "cpmg_hier_level_info")
        return Y, shape, [bool(co[n]) for n in range(N)]

    def rhat(self, level, N):
        dims = (C.c_int64 * MAX_MODES)()
        co = (C.c_int * MAX_MODES)()
        _check(lib().cpmg_hier_level_info(self.h, level, dims, co, None, None), "cpmg_hier_level_info")
        bufs, ptrs = [], (C.c_void_p * MAX_MODES)()
        for n in range(N):
            if co[n]:
                I = int(dims[n])
                Ic = (I + 1) // 2
                b = np.zeros((I, Ic), dtype=np.float64)  # C-order (I, Ic) == column-major Ic x I
                bufs.append(b)
                ptrs[n] = b.ctypes.data
            else:
                bufs.append(None)
        _check(lib().cpmg_hier_level_info(self.h, level, dims, co, None, ptrs), "cpmg_hier_level_info")
        return [None if b is None else b.T for b in bufs]

    def free(self):
        if self.h:
            lib().cpmg_hier_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def mg_setup(ctx, Z, A_boot, A_test, opts=None, **kw):
    o = opts or make_opts(**kw)
    r = cpmg_result()
    d = tensor_desc(Z)
    h = C.c_void_p()
    flat = [t for blk in A_test for t in blk]
    s = lib().mg_setup(ctx.h, C.byref(d), A_boot[0].shape[0], _ptrs(A_boot), _ptrs(flat), C.byref(o),
                       C.byref(h), C.byref(r))
    _check(s, "mg_setup")
    return Hierarchy(h), result_dict(r)


def mg_fas_solve(ctx, hier, Z, A, opts=None, **kw):
    o = opts or make_opts(**kw)
    r = cpmg_result()
    d = tensor_desc(Z)
    s = lib().mg_fas_solve(ctx.h, hier.h, C.byref(d), _ptrs(A), C.byref(o), C.byref(r))
    _check(s, "mg_fas_solve", allow=(OK, NOT_CONVERGED))
    return result_dict(r)


def mg_fmg(ctx, hier, Z, A_coarsest, A, nu=100, opts=None, **kw):
    """One FMG-CP-FAS cycle (Algorithm 3) from the coarsest-level start A_coarsest, then the
    down-sweep rebuild of the hierarchy's operators; the finest-level factors go to A."""
    o = opts or make_opts(**kw)
    r = cpmg_result()
    d = tensor_desc(Z)
    s = lib().mg_fmg(ctx.h, hier.h, C.byref(d), _ptrs(A_coarsest), _ptrs(A), int(nu), C.byref(o), C.byref(r))
    _check(s, "mg_fmg")
    return result_dict(r)


def batch_plan(dims, R, unit_elements, mode):
    """The batched form's MTTKRP work units of one mode of one tensor (host only): an int64
    array of rows (rb, k, c0, c1, in_idx), the slot count nk and the partial-sum doubles."""
    N = len(dims)
    d = (C.c_int64 * N)(*[int(v) for v in dims])
    n = C.c_int64()
    _check(lib().cpmg_batch_plan(N, d, int(R), int(unit_elements), int(mode), None, 0, C.byref(n), None, None),
           "cpmg_batch_plan")
    out = np.zeros((max(n.value, 1), 5), dtype=np.int64)
    nk, tot = C.c_int(), C.c_int64()
    _check(lib().cpmg_batch_plan(N, d, int(R), int(unit_elements), int(mode),
                                 out.ctypes.data_as(C.POINTER(C.c_int64)), n.value, C.byref(n), C.byref(nk),
                                 C.byref(tot)), "cpmg_batch_plan")
    return out[:n.value], nk.value, tot.value


def cpmg_decompose(ctx, Z, A, A_test, opts=None, **kw):
    o = opts or make_opts(**kw)
    r = cpmg_result()
    d = tensor_desc(Z)
    flat = [t for blk in A_test for t in blk]
    s = lib().cpmg_decompose(ctx.h, C.byref(d), A[0].shape[0], _ptrs(A), _ptrs(flat), C.byref(o), C.byref(r))
    _check(s, "cpmg_decompose", allow=(OK, NOT_CONVERGED))
    return result_dict(r)
