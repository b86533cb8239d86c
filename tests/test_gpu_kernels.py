"""GPU parity of the single kernels against the FP64 oracle: MTTKRP (all modes, FP32 /
float-pair / FP64 arithmetic, ragged and multi-segment shapes, N = 2..5, R = 1..16), the
TTM restriction, and f / g."""
import numpy as np
import pytest

from oracle import tensor as T, multigrid as MG

pytestmark = pytest.mark.gpu

TOL = {0: 2e-5, 3: 1e-11, 1: 5e-13}   # relative to sum_j |z_j phi_j| per output entry


def rnd(shape, seed, dtype=np.float32):
    return np.asfortranarray(np.random.default_rng(seed).standard_normal(shape).astype(dtype))


def factors(dims, R, seed):
    rng = np.random.default_rng(seed)
    return [np.asfortranarray(rng.standard_normal((I, R))) for I in dims]


def check_mttkrp(ctx, Zn, A, precs):
    from paper_1111_6091_gb300 import cpmg
    Z = cpmg.colmajor(Zn)
    Ad = [cpmg.colmajor(a) for a in A]
    Z64 = Zn.astype(np.float64)
    for n in range(Zn.ndim):
        ref = T.mttkrp(Z64, A, n)
        scale = T.unfold(np.abs(Z64), n) @ np.abs(T.phi(A, n))
        for prec in precs:
            M = cpmg.to_numpy(cpmg.cpmg_mttkrp(ctx, Z, Ad, n, prec))
            err = np.abs(M - ref)
            bound = TOL[prec] * scale + 1e-300
            assert np.all(err <= bound), (n, prec, float(np.max(err / np.maximum(scale, 1e-300))))


CASES = [
    ((64, 40, 36), 10),      # float4 path, several CTAs
    ((63, 41, 37), 5),       # ragged first mode: scalar path
    ((1, 7, 5), 3),          # first mode of size 1
    ((5, 1, 9), 2),          # a middle mode of size 1
    ((2100, 5, 3), 4),       # first mode wider than one CTA: two row segments
    ((2049, 3, 3), 2),       # odd, five row segments
    ((300, 200), 7),         # N = 2
    ((20, 18, 16, 14), 6),   # N = 4
    ((8, 7, 6, 5, 4), 3),    # N = 5
    ((40, 30, 20), 16),      # R = 16
    ((33, 17, 9), 1),        # R = 1
]


@pytest.mark.parametrize("dims,R", CASES)
def test_mttkrp_float_tensor(cpmg_ctx, dims, R):
    check_mttkrp(cpmg_ctx, rnd(dims, 1), factors(dims, R, 2), precs=(0, 3, 1))


@pytest.mark.parametrize("dims,R", [((20, 20, 20), 3), ((21, 19, 17), 4), ((6, 5, 4, 3), 2)])
def test_mttkrp_double_tensor(cpmg_ctx, dims, R):
    check_mttkrp(cpmg_ctx, rnd(dims, 3, np.float64), factors(dims, R, 4), precs=(0, 1))


def test_mttkrp_bitwise_reproducible(cpmg_ctx):
    from paper_1111_6091_gb300 import cpmg
    Zn = rnd((128, 96, 80), 5)
    A = [cpmg.colmajor(a) for a in factors(Zn.shape, 8, 6)]
    Z = cpmg.colmajor(Zn)
    for n in range(3):
        for prec in (0, 3):
            a = cpmg.cpmg_mttkrp(cpmg_ctx, Z, A, n, prec).cpu().numpy()
            b = cpmg.cpmg_mttkrp(cpmg_ctx, Z, A, n, prec).cpu().numpy()
            assert np.array_equal(a, b)


def test_mttkrp_full_size_400cubed(cpmg_ctx):
    """The 400^3 rank-10 float tensor of the bench workload, every mode, every entry."""
    from paper_1111_6091_gb300 import cpmg, synth
    p = synth.make_problem((400, 400, 400), 10, congruence=0.95, eta_homo=0.01, dtype=np.float32, seed=0)
    check_mttkrp(cpmg_ctx, p.Z, p.A0, precs=(0, 3))


def rhat_for(I, R, seed):
    rng = np.random.default_rng(seed)
    P = MG.interpolation(rng.standard_normal((I, 2 * R)), np.ones(2 * R), I)
    return MG.transform(P)[1]


@pytest.mark.parametrize("dims,mask", [((20, 18, 16), (1, 1, 1)), ((33, 7, 65), (1, 0, 1)),
                                       ((9, 8, 7, 6), (1, 1, 1, 1)), ((130, 70), (0, 1))])
def test_ttm_restrict(cpmg_ctx, dims, mask):
    import torch
    from paper_1111_6091_gb300 import cpmg
    Zn = rnd(dims, 7)
    Rh = [rhat_for(I, 2, 8 + i) if m else None for i, (I, m) in enumerate(zip(dims, mask))]
    Y = cpmg.cpmg_ttm(cpmg_ctx, cpmg.colmajor(Zn),
                      [None if r is None else torch.from_numpy(np.ascontiguousarray(r.T)).cuda() for r in Rh])
    modes = [i for i, m in enumerate(mask) if m]
    Z64 = Zn.astype(np.float64)
    ref = T.ttm_modes(Z64, Rh, modes)
    scale = T.ttm_modes(np.abs(Z64), [None if r is None else np.abs(r) for r in Rh], modes)
    err = np.abs(cpmg.to_numpy(Y) - ref)
    assert np.all(err <= 2e-5 * scale + 1e-30)


# split BF16 on tcgen05: x = hi + lo; hi*hi + hi*lo + lo*hi drops lo*lo and the rounding of
# lo, each at most 2^-18 |x||y|, plus FP32 accumulation; bound per entry 1e-4 of sum |R||Z|
# per mode product, the RMS of (error / scale) must stay under 2e-5.
TC_CASES = [
    ((20, 18, 16), (1, 1, 1), "rhat"),      # mode 1 tensor map, later modes direct loads
    ((33, 7, 65), (1, 0, 1), "rhat"),       # ragged: direct loads, tile tails
    ((64, 40, 36), (1, 1, 1), "rhat"),      # tensor maps for every mode, several tiles
    ((9, 8, 7, 6), (1, 1, 1, 1), "rhat"),   # 4-way, direct loads
    ((130, 70), (0, 1), "rhat"),            # last mode only, two 128-row tiles
    ((512, 6, 5), (1, 0, 0), "dense"),      # Ic = 256: the widest accumulator
    ((8, 400, 12), (0, 1, 0), "dense"),     # Ic = 200 (padded to 208), middle mode
    ((200, 300, 4), (0, 1, 0), "dense"),    # Ic = 150, L = 200: tensor map, K tail of 12
]


@pytest.mark.parametrize("dims,mask,kind", TC_CASES)
def test_ttm_tensor_cores(cpmg_ctx, dims, mask, kind):
    import torch
    from paper_1111_6091_gb300 import cpmg
    Zn = rnd(dims, 17)
    rng = np.random.default_rng(18)
    Rh = []
    for i, (I, m) in enumerate(zip(dims, mask)):
        if not m:
            Rh.append(None)
        elif kind == "rhat":
            Rh.append(rhat_for(I, 2, 8 + i))
        else:
            Rh.append(rng.standard_normal(((I + 1) // 2, I)))
    Y = cpmg.cpmg_ttm(cpmg_ctx, cpmg.colmajor(Zn),
                      [None if r is None else torch.from_numpy(np.ascontiguousarray(r.T)).cuda() for r in Rh],
                      tensor_cores=1)
    modes = [i for i, m in enumerate(mask) if m]
    Z64 = Zn.astype(np.float64)
    ref = T.ttm_modes(Z64, Rh, modes)
    scale = T.ttm_modes(np.abs(Z64), [None if r is None else np.abs(r) for r in Rh], modes)
    rel = np.abs(cpmg.to_numpy(Y) - ref) / scale
    assert np.max(rel) <= 1e-4 * len(modes), float(np.max(rel))
    assert np.sqrt(np.mean(rel ** 2)) <= 2e-5, float(np.sqrt(np.mean(rel ** 2)))


def test_ttm_tensor_cores_unsupported(cpmg_ctx):
    """Float64 tensors and Ic > 256 are refused on the tensor-core path, not rerouted."""
    import torch
    from paper_1111_6091_gb300 import cpmg
    Zd = cpmg.colmajor(rnd((8, 6, 4), 1, np.float64))
    R = torch.zeros((8, 4), dtype=torch.float64, device="cuda")
    with pytest.raises(cpmg.CpmgError) as e:
        cpmg.cpmg_ttm(cpmg_ctx, Zd, [R, None, None], tensor_cores=1)
    assert e.value.status == cpmg.UNSUPPORTED
    Zf = cpmg.colmajor(rnd((600, 3, 2), 1))
    R = torch.zeros((600, 300), dtype=torch.float64, device="cuda")
    with pytest.raises(cpmg.CpmgError) as e:
        cpmg.cpmg_ttm(cpmg_ctx, Zf, [R, None, None], tensor_cores=1)
    assert e.value.status == cpmg.UNSUPPORTED


def test_ttm_tensor_cores_400cubed_sampled(cpmg_ctx):
    """The level-0 restriction of the 400^3 workload (three modes 400 -> 200, the sizes the
    solver runs), checked at sampled coarse entries the oracle computes one by one."""
    import torch
    from paper_1111_6091_gb300 import cpmg
    dims = (400, 400, 400)
    Zn = rnd(dims, 23)
    rng = np.random.default_rng(24)
    Rh = [rng.standard_normal((200, 400)) for _ in range(3)]
    Y = cpmg.cpmg_ttm(cpmg_ctx, cpmg.colmajor(Zn),
                      [torch.from_numpy(np.ascontiguousarray(r.T)).cuda() for r in Rh], tensor_cores=1)
    Yh = cpmg.to_numpy(Y)
    assert Yh.shape == (200, 200, 200)
    Z64 = Zn.astype(np.float64)
    Za = np.abs(Z64)
    idx = [(0, 0, 0), (199, 199, 199), (17, 123, 5), (101, 0, 198)] + \
          [tuple(int(v) for v in rng.integers(0, 200, 3)) for _ in range(8)]
    for (a, b, c) in idx:
        want = np.einsum("ijk,i,j,k->", Z64, Rh[0][a], Rh[1][b], Rh[2][c], optimize=True)
        sc = np.einsum("ijk,i,j,k->", Za, np.abs(Rh[0][a]), np.abs(Rh[1][b]), np.abs(Rh[2][c]), optimize=True)
        assert abs(Yh[a, b, c] - want) <= 3e-4 * sc, (a, b, c)


def test_ttm_double_tensor(cpmg_ctx):
    import torch
    from paper_1111_6091_gb300 import cpmg
    dims = (20, 20, 20)
    Zn = rnd(dims, 9, np.float64)
    Rh = [rhat_for(20, 3, 10 + i) for i in range(3)]
    Y = cpmg.cpmg_ttm(cpmg_ctx, cpmg.colmajor(Zn), [torch.from_numpy(np.ascontiguousarray(r.T)).cuda() for r in Rh])
    ref = T.ttm_modes(Zn, Rh, range(3))
    assert np.allclose(cpmg.to_numpy(Y), ref, rtol=1e-12, atol=1e-12 * np.max(np.abs(ref)))


@pytest.mark.parametrize("dims,R,dt", [((20, 20, 20), 3, np.float64), ((48, 40, 36), 5, np.float32),
                                       ((12, 11, 10, 9), 4, np.float32)])
def test_eval_f_g(cpmg_ctx, dims, R, dt):
    from paper_1111_6091_gb300 import cpmg
    Zn = rnd(dims, 11, dt)
    A = factors(dims, R, 12)
    f, g = cpmg.cpmg_eval_fg(cpmg_ctx, cpmg.colmajor(Zn), [cpmg.colmajor(a) for a in A])
    Z64 = Zn.astype(np.float64)
    assert np.isclose(f, T.f_value(Z64, A), rtol=1e-12)
    assert np.isclose(g, T.g_value(Z64, A), rtol=1e-10)
