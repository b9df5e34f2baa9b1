"""GPU parity of the non-symmetric all-pairs path (Section III-B, Eq. (7)-(8)):
r(x_i, y_j) between the rows of two matrices, through the C ABI, against
the FP64 oracle element by element.

Tolerances are those of the triangle (test_gpu_parity.py): FP64 1e-12,
FP32 4e-6, BF16X3 / FP16X3S 1e-5, BF16X1 a sanity bound of 2e-2.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 4e-6, "bf16x3": 1e-5, "fp16x3s": 1e-5,
       "bf16x4": 1e-5, "bf16x1": 2e-2}
SENT = 7.0


def _data(n, l, seed):
    X = synth.counts_log(n, l, seed, dtype=np.float32)
    if n > 4:
        X[n // 3] = 3.25                       # zero variance: NaN row/col
        X[n // 2] = X[n // 2] + np.float32(1e5)  # large offset
    return X


def _cross(pcc, X, Y, prec, ldr=None, ranges=None):
    import torch
    if prec == "fp64":
        X, Y = X.astype(np.float64), Y.astype(np.float64)
    ZX = pcc.pcc_standardize(torch.from_numpy(X).cuda(), prec)
    ZY = pcc.pcc_standardize(torch.from_numpy(Y).cuda(), prec)
    nx, ny = X.shape[0], Y.shape[0]
    ldr = ny if ldr is None else ldr
    dt = torch.float64 if prec == "fp64" else torch.float32
    R = torch.full((nx, ldr), SENT, dtype=dt, device="cuda")
    if ranges is None:
        pcc.pcc_cross_allpairs(ZX, ZY, R, ldr)
    else:
        for a, b in ranges:
            pcc.pcc_cross_allpairs(ZX, ZY, R, ldr, a, b)
    st = pcc.pcc_sync_status(ZX)
    assert st == 0, pcc.pcc_status_string(st)
    return R.cpu().numpy().astype(np.float64), ZX, ZY


def _compare(got, want, tol, what):
    gn, wn = np.isnan(got), np.isnan(want)
    assert np.array_equal(gn, wn), f"{what}: NaN pattern differs"
    assert not np.any(got == SENT), f"{what}: unwritten output"
    err = np.max(np.abs(got[~wn] - want[~wn])) if (~wn).any() else 0.0
    assert err <= tol, f"{what}: max|dr| = {err:.3e} > {tol:.1e}"


SHAPES = [(2, 3, 2), (5, 2, 7), (129, 300, 64), (300, 129, 33),
          (513, 257, 96), (700, 1030, 40)]


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16x3", "fp16x3s",
                                  "bf16x4", "bf16x1"])
@pytest.mark.parametrize("nx,ny,l", SHAPES)
def test_cross_parity(pcc_gpu, prec, nx, ny, l):
    X = _data(nx, l, 3000 + nx + l)
    Y = _data(ny, l, 4000 + ny + l)
    got, _, _ = _cross(pcc_gpu, X, Y, prec)
    _compare(got, oracle.cross_rows(X, Y), TOL[prec],
             f"{prec} {nx}x{ny} l={l}")


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_cross_pitch_leaves_gap_untouched(pcc_gpu, prec):
    X = _data(300, 50, 11)
    Y = _data(270, 50, 12)
    got, _, _ = _cross(pcc_gpu, X, Y, prec, ldr=301)
    assert np.all(got[:, 270:] == SENT)
    _compare(got[:, :270], oracle.cross_rows(X, Y), TOL[prec], prec)


@pytest.mark.parametrize("cluster,pair", [(1, 0), (2, 1)])
def test_cross_self_matches_triangle_bits(pcc_gpu, cluster, pair):
    """cross(Z, Z) is the full square: its strict upper part is the packed
    triangle bit for bit (same operand roles, same K order, same epilogue
    arithmetic), its lower part the transpose within 1e-5, and the diagonal
    1 within BF16X3's worst case at |r| = 1.  That case is a row whose mass
    sits in one sample, so nothing averages out: 2 * 2^-18 for the
    represented z = hi + lo of both operands, 2^-18 for the dropped lo*lo
    term, and the accumulation, which drops up to two FP32 ulps toward zero
    on each of its 30 updates at l = 130: 1.9e-5 (measured: 1.5e-5)."""
    import torch
    pcc = pcc_gpu
    old = pcc.pcc_get_tuning()
    pcc.pcc_set_tuning(cluster=cluster, pair_mma=pair)
    try:
        X = _data(600, 130, 13)
        Xd = torch.from_numpy(X).cuda()
        Z = pcc.pcc_standardize(Xd, "bf16x3")
        n = X.shape[0]
        R = torch.full((n, n), SENT, device="cuda")
        pcc.pcc_cross_allpairs(Z, Z, R)
        P = torch.full((n * (n - 1) // 2,), SENT, device="cuda")
        pcc.pcc_allpairs_upper(Z, P)
        assert pcc.pcc_sync_status(Z) == 0
        R = R.cpu().numpy()
        P = P.cpu().numpy()
    finally:
        pcc.pcc_set_tuning(cluster=old["cluster"], pair_mma=old["pair_mma"])
    I, J = np.triu_indices(n, 1)
    up = R[I, J]
    assert np.array_equal(np.isnan(up), np.isnan(P))
    ok = ~np.isnan(P)
    assert np.array_equal(up[ok].view(np.uint32), P[ok].view(np.uint32))
    lo = R[J, I]
    assert np.nanmax(np.abs(lo - up)) <= 1e-5
    d = np.diag(R)
    good = ~np.isnan(d)
    assert good.sum() == n - 1  # the constant row
    bound = 3 * 2.0 ** -18 + 30 * 2 * 2.0 ** -23
    assert np.max(np.abs(d[good] - 1)) <= bound


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_cross_tile_ranges_union(pcc_gpu, prec):
    X = _data(700, 60, 14)
    Y = _data(530, 60, 15)
    whole, ZX, ZY = _cross(pcc_gpu, X, Y, prec)
    T = pcc_gpu.pcc_cross_num_tiles(ZX, ZY)
    assert T > 2
    for parts in (2, 5):
        cuts = [T * k // parts for k in range(parts + 1)]
        got, _, _ = _cross(pcc_gpu, X, Y, prec,
                           ranges=list(zip(cuts, cuts[1:])))
        assert np.array_equal(np.isnan(got), np.isnan(whole))
        ok = ~np.isnan(whole)
        assert np.array_equal(got[ok], whole[ok])


@pytest.mark.parametrize("prec", ["fp32", "bf16x3", "fp16x3s"])
def test_cross_edges_band_rule(pcc_gpu, prec):
    """Edges with |r| >= tau: every oracle edge farther than the tolerance
    above tau is found, nothing farther than it below tau is, and the fused
    R equals the plain call."""
    import torch
    pcc = pcc_gpu
    l = 64
    X = synth.counts_log(900, l, 16, dtype=np.float32)
    # noisy copies of every third X row (r ~ 0.9-1) and unrelated rows;
    # exact copies are the split forms' worst case, covered in
    # test_gpu_worstcase.py
    rng = np.random.default_rng(17)
    C = X[::3].astype(np.float64)
    C = C + 0.2 * C.std(1, keepdims=True) * rng.standard_normal(C.shape)
    Y = np.vstack([C.astype(np.float32),
                   synth.counts_log(200, l, 17, dtype=np.float32)])
    nx, ny = X.shape[0], Y.shape[0]
    tau = 0.6
    ZX = pcc.pcc_standardize(torch.from_numpy(X).cuda(), prec)
    ZY = pcc.pcc_standardize(torch.from_numpy(Y).cuda(), prec)
    cap = 1 << 20
    E = torch.zeros(cap * 12, dtype=torch.uint8, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    R = torch.full((nx, ny), SENT, device="cuda")
    pcc.pcc_cross_edges(ZX, ZY, tau, E, cap, cnt, R)
    assert pcc.pcc_sync_status(ZX) == 0
    c = int(cnt.item())
    rec = E[:c * 12].cpu().numpy().view(np.uint32).reshape(-1, 3)
    gi, gj = rec[:, 0].astype(np.int64), rec[:, 1].astype(np.int64)
    gr = rec[:, 2].copy().view(np.float32).astype(np.float64)
    want = oracle.cross_rows(X, Y)
    tol = TOL[prec]
    got = set(zip(gi.tolist(), gj.tolist()))
    assert len(got) == c  # no duplicates
    sure = np.argwhere(np.abs(want) >= tau + tol)
    assert {(int(i), int(j)) for i, j in sure} <= got
    for i, j, r in zip(gi, gj, gr):
        assert abs(want[i, j]) >= tau - tol
        assert abs(r - want[i, j]) <= tol
    assert c > 100
    Rf = R.cpu().numpy().astype(np.float64)
    _compare(Rf, want, tol, prec)


def test_cross_invalid_arguments(pcc_gpu):
    import torch
    pcc = pcc_gpu
    X = torch.from_numpy(_data(100, 40, 18)).cuda()
    Y = torch.from_numpy(_data(90, 41, 19)).cuda()
    ZX = pcc.pcc_standardize(X, "bf16x3")
    ZY = pcc.pcc_standardize(Y, "bf16x3")
    ZXf = pcc.pcc_standardize(X, "fp32")
    R = torch.zeros((100, 100), device="cuda")
    with pytest.raises(pcc.PccError):        # different l
        pcc.pcc_cross_allpairs(ZX, ZY, R, 100)
    ZY2 = pcc.pcc_standardize(Y[:, :40].contiguous(), "bf16x3")
    with pytest.raises(pcc.PccError):        # different forms
        pcc.pcc_cross_allpairs(ZXf, ZY2, R, 100)
    with pytest.raises(pcc.PccError):        # ldr < ny
        pcc.pcc_cross_allpairs(ZX, ZY2, R, 89)
    T = pcc.pcc_cross_num_tiles(ZX, ZY2)
    with pytest.raises(pcc.PccError):        # range past the end
        pcc.pcc_cross_allpairs(ZX, ZY2, R, 100, 0, T + 1)
    pcc.pcc_cross_allpairs(ZX, ZY2, R, 100)
    assert pcc.pcc_sync_status(ZX) == 0


def test_cross_full_workload(pcc_gpu):
    """The cross workload at its benchmarked size: X 65,536 x 512 against
    Y 32,768 x 512 (log counts, seeds 6 and 7), dense FP32 R of 8.6 GB, in
    the default form.  10^6 sampled (i, j) against the oracle, and every
    pair against the FP64 CUDA-core cross matrix (itself within 1e-12 of
    the oracle on the samples)."""
    import json

    import torch

    from gpu_compare import max_abs_diff
    pcc = pcc_gpu
    nx, ny, l = 65536, 32768, 512
    X = synth.counts_log(nx, l, 6)
    Y = synth.counts_log(ny, l, 7)
    Xd, Yd = torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()
    ZX, ZY = pcc.pcc_standardize(Xd, "auto"), pcc.pcc_standardize(Yd, "auto")
    R = torch.empty((nx, ny), dtype=torch.float32, device="cuda")
    pcc.pcc_cross_allpairs(ZX, ZY, R)
    assert pcc.pcc_sync_status(ZX) == 0
    rng = np.random.default_rng(106)
    I = rng.integers(0, nx, 1_000_000)
    J = rng.integers(0, ny, 1_000_000)
    want = oracle.cross_pairs(X, Y, I, J)
    ok = ~np.isnan(want)
    idx = torch.from_numpy(I * ny + J).cuda()
    got = R.view(-1)[idx].cpu().numpy().astype(np.float64)
    assert np.array_equal(np.isnan(got), np.isnan(want))
    err = float(np.max(np.abs(got[ok] - want[ok])))
    assert err <= 1e-5
    X64, Y64 = pcc.pcc_standardize(Xd, "fp64"), pcc.pcc_standardize(Yd, "fp64")
    R64 = torch.empty((nx, ny), dtype=torch.float64, device="cuda")
    pcc.pcc_cross_allpairs(X64, Y64, R64)
    assert pcc.pcc_sync_status(X64) == 0
    err64 = float(np.max(np.abs(R64.view(-1)[idx].cpu().numpy()[ok] -
                                want[ok])))
    assert err64 <= 1e-12
    err_all, nan_differs = max_abs_diff(R.view(-1), R64.view(-1))
    assert not nan_differs
    assert err_all <= 1e-5
    print(json.dumps({"cross_workload_max_abs_dr": err,
                      "fp64_path_vs_oracle": err64,
                      "all_pairs_max_abs_dr_vs_fp64_path": err_all}))
